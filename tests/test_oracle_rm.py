"""Pins for the oracle's residual-modulated velocity network (the reading of
the paper's "residual blocks with adaptive modulation conditioned on the
physical context", section "Network Architecture and Inputs") and its CFM
gradient (Eq. 9).

Each forward pin builds a network whose blocks act on one or two hidden
units only, so the velocity has a closed form in scalars: a dropped residual
term, a shift or scale taken from the wrong condition component, a block
applied out of order or a modulation applied after the SiLU all change it.
The reverse pass is pinned against central differences of the loss.
"""
import math

import numpy as np
import pytest

import synth
from oracle import mlp, train


def _silu(v):
    return v / (1.0 + math.exp(-v))


def _zero_rm():
    net = synth.rm_weights(1)
    net["W"] = [np.zeros_like(w) for w in net["W"]]
    return net


def _load(tmp_path, net, name="rm.bin"):
    p = str(tmp_path / name)
    synth.write_weights(p, net)
    return mlp.read_weights(p)


def test_rm_weight_file_round_trip(tmp_path):
    net = synth.rm_weights(3, m_std=0.5, g_std=0.25)
    o = _load(tmp_path, net)
    assert o.rm
    for j in range(3):
        np.testing.assert_array_equal(o.M[j], net["M"][j].astype(np.float64))
        np.testing.assert_array_equal(o.G[j], net["G"][j].astype(np.float64))
    for l in range(5):
        np.testing.assert_array_equal(o.W[l], net["W"][l].astype(np.float64))
    plain = _load(tmp_path, synth.kaiming_weights(3), "plain.bin")
    assert not plain.rm
    # an unknown flag bit, and an RM file cut short, are rejected
    raw = bytearray((tmp_path / "rm.bin").read_bytes())
    raw[48:52] = (3).to_bytes(4, "little")
    (tmp_path / "bad.bin").write_bytes(bytes(raw))
    with pytest.raises(ValueError):
        mlp.read_weights(str(tmp_path / "bad.bin"))
    (tmp_path / "short.bin").write_bytes((tmp_path / "rm.bin").read_bytes()[:-4])
    with pytest.raises(ValueError):
        mlp.read_weights(str(tmp_path / "short.bin"))


def test_rm_single_path(tmp_path):
    # x_0 -> hidden unit 0 (layer 1, weight a); block j maps unit 0 to itself
    # with weight w_j, so a_{j} = a_{j-1} + silu(w_j a_{j-1}) on unit 0 and
    # every other unit stays 0; v_0 = a_4[0]. One Euler step: x_0 + v_0.
    net = _zero_rm()
    a = float(np.float32(0.7))
    w = [float(np.float32(v)) for v in (1.5, -0.75, 0.5)]
    net["W"][0][0, 5] = a
    for j in range(3):
        net["W"][j + 1][0, 0] = w[j]
    net["W"][4][0, 0] = 1.0
    o = _load(tmp_path, net)
    cond, _, _ = synth.sampler_conditions(8, 5)
    z = synth.gaussian_noise(8, 6)
    y = mlp.sample(o, cond, z, 1, "euler")
    for i in range(8):
        x0 = float(z[0, i])
        u = _silu(a * x0)
        for j in range(3):
            u = u + _silu(w[j] * u)
        assert abs(y[0, i] - (x0 + u)) < 1e-14
        np.testing.assert_allclose(y[1:, i], z[1:, i].astype(np.float64), atol=0)


def test_rm_condition_shift_and_scale(tmp_path):
    # Block weights zero: hidden unit 1 gets only the condition shift
    # m_j c_std[3] (standardized ln tau) scaled by 1 + gt_j c_std[3] +
    # gc_j c_std[4]; unit 2 only the bias beta_j, unmodulated. Outputs 2 and 3
    # read units 1 and 2, so over one Euler step
    #   v_2 = sum_j silu((1 + gt_j u3 + gc_j u4) m_j u3),  v_3 = sum_j silu(beta_j).
    net = _zero_rm()
    net["cond_mean"] = np.array([0, 0, 0, 1.5, 0.25], np.float32)
    net["cond_std"] = np.array([1, 1, 1, 2.0, 0.5], np.float32)
    m = [0.8, -1.1, 0.6]
    gt = [0.3, -0.2, 0.45]
    gc = [-0.5, 0.35, 0.1]
    beta = [0.4, -0.9, 1.3]
    for j in range(3):
        net["M"][j][1, 3] = m[j]
        net["G"][j][0, 1] = gt[j]
        net["G"][j][1, 1] = gc[j]
        net["b"][j + 1][2] = beta[j]
    net["W"][4][2, 1] = 1.0
    net["W"][4][3, 2] = 1.0
    o = _load(tmp_path, net)
    cond, _, _ = synth.sampler_conditions(6, 11)
    z = synth.gaussian_noise(6, 12)
    y = mlp.sample(o, cond, z, 1, "euler")
    f = lambda v: float(np.float32(v))
    for i in range(6):
        u3 = (float(cond[3, i]) - 1.5) / 2.0
        u4 = (float(cond[4, i]) - 0.25) / 0.5
        v2 = sum(_silu((1 + f(gt[j]) * u3 + f(gc[j]) * u4) * f(m[j]) * u3) for j in range(3))
        v3 = sum(_silu(f(beta[j])) for j in range(3))
        assert abs(y[2, i] - (float(z[2, i]) + v2)) < 1e-13
        assert abs(y[3, i] - (float(z[3, i]) + v3)) < 1e-13


def test_rm_modulation_scales_the_whole_preactivation(tmp_path):
    # Unit 0 carries x_0 through layer 1 (weight 1) and block 1 maps it to
    # unit 3 with weight w plus bias beta and shift m c_std[0]; G scales the
    # sum: a_2[3] = silu((1 + gt u3) (w silu(x_0) + beta + m u0)); blocks 2-3
    # leave unit 3 unchanged (their rows are zero and silu(0) = 0).
    net = _zero_rm()
    net["W"][0][0, 5] = 1.0
    w, beta, m, gt = 0.9, -0.3, 0.7, 0.6
    net["W"][1][3, 0] = w
    net["b"][1][3] = beta
    net["M"][0][3, 0] = m
    net["G"][0][0, 3] = gt
    net["W"][4][1, 3] = 1.0
    o = _load(tmp_path, net)
    cond, _, _ = synth.sampler_conditions(5, 13)
    z = synth.gaussian_noise(5, 14)
    y = mlp.sample(o, cond, z, 1, "euler")
    f = lambda v: float(np.float32(v))
    for i in range(5):
        u0, u3 = float(cond[0, i]), float(cond[3, i])
        pre = f(w) * _silu(float(z[0, i])) + f(beta) + f(m) * u0
        expect = float(z[1, i]) + _silu((1 + f(gt) * u3) * pre)
        assert abs(y[1, i] - expect) < 1e-13


def _rm_problem(B, seed):
    g = np.random.default_rng(seed)
    net = synth.rm_weights(seed, m_std=0.3, g_std=0.3)
    P = {"W": [np.asarray(w, np.float64) * 0.8 for w in net["W"]],
         "b": [g.standard_normal(len(v)) * 0.2 for v in net["b"]],
         "M": [np.asarray(m, np.float64) for m in net["M"]],
         "G": [np.asarray(q, np.float64) for q in net["G"]]}
    cn = g.standard_normal((B, 5))
    x1 = g.standard_normal((B, 4))
    x0 = g.standard_normal((B, 4))
    t = g.random(B)
    return P, cn, x1, x0, t


def test_rm_loss_matches_sampler_velocity():
    # The training forward pass is the sampler's velocity at x_t.
    P, cn, x1, x0, t = _rm_problem(7, 3)
    net = mlp.Net(P["W"], P["b"], np.zeros(5), np.ones(5), np.zeros(4), np.ones(4), P["M"], P["G"])
    loss, _ = train.cfm_loss_grad_rm(P, cn, x1, x0, t)
    xt = (1 - t)[:, None] * x0 + t[:, None] * x1
    v = mlp.velocity(net, cn, xt, t)
    assert abs(loss - np.mean(np.sum((v - (x1 - x0)) ** 2, axis=1))) < 1e-12


def test_rm_gradient_by_central_differences():
    P, cn, x1, x0, t = _rm_problem(6, 7)
    _, G = train.cfm_loss_grad_rm(P, cn, x1, x0, t)
    g = np.random.default_rng(2)
    h = 1e-6

    def loss_with(key, l, idx, delta):
        Q = {k: [a.copy() for a in v] for k, v in P.items()}
        Q[key][l][idx] += delta
        return train.cfm_loss_grad_rm(Q, cn, x1, x0, t)[0]

    for key, n in (("W", 5), ("b", 5), ("M", 3), ("G", 3)):
        for l in range(n):
            for _ in range(6):
                idx = tuple(int(g.integers(s)) for s in P[key][l].shape)
                fd = (loss_with(key, l, idx, h) - loss_with(key, l, idx, -h)) / (2 * h)
                an = G[key][l][idx]
                assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (key, l, idx, fd, an)


def test_rm_has_no_e4m3_network(tmp_path):
    o = _load(tmp_path, synth.rm_weights(1))
    with pytest.raises(ValueError):
        mlp.quantized_e4m3(o)
