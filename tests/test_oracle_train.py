"""Pins for the oracle's CFM loss and gradient (Eq. 9), AdamW and statistics."""
import math

import numpy as np
import pytest
import torch
from scipy import stats as sstats

import synth
from oracle import mlp, train
from oracle import stats as ostats


def _small_problem(B=8, seed=0, scale=0.5):
    g = np.random.default_rng(seed)
    net = synth.kaiming_weights(seed + 1)
    W = [w.astype(np.float64) * scale for w in net["W"]]
    b = [g.standard_normal(v.shape) * 0.1 for v in net["b"]]
    cn = g.standard_normal((B, 5))
    x1 = g.standard_normal((B, 4))
    x0 = g.standard_normal((B, 4))
    t = g.random(B)
    return W, b, cn, x1, x0, t


def test_loss_matches_definition():
    W, b, cn, x1, x0, t = _small_problem()
    loss, _, _ = train.cfm_loss_grad(W, b, cn, x1, x0, t)
    net = mlp.Net(W, b, np.zeros(5), np.ones(5), np.zeros(4), np.ones(4))
    xt = (1 - t)[:, None] * x0 + t[:, None] * x1
    v = mlp.velocity(net, cn, xt, t)
    assert abs(loss - np.mean(np.sum((v - (x1 - x0)) ** 2, axis=1))) < 1e-12


def test_constant_velocity_loss_and_bias_gradient():
    # v = b5 everywhere: L = mean ||b5 - (x1 - x0)||^2 and dL/db5 = 2 (b5 - mean(x1 - x0)).
    W, b, cn, x1, x0, t = _small_problem(B=16, seed=3)
    W = [np.zeros_like(w) for w in W]
    b = [np.zeros_like(v) for v in b]
    b[4] = np.array([0.3, -0.2, 0.1, 0.5])
    loss, gW, gb = train.cfm_loss_grad(W, b, cn, x1, x0, t)
    u = x1 - x0
    assert abs(loss - np.mean(np.sum((b[4] - u) ** 2, axis=1))) < 1e-13
    np.testing.assert_allclose(gb[4], 2 * (b[4] - u.mean(axis=0)), atol=1e-13)
    for l in range(4):
        assert np.all(gW[l] == 0) and np.all(gb[l] == 0)


def test_gradient_by_central_differences():
    W, b, cn, x1, x0, t = _small_problem(B=6, seed=7)
    _, gW, gb = train.cfm_loss_grad(W, b, cn, x1, x0, t)
    g = np.random.default_rng(1)
    h = 1e-6
    for l in range(5):
        for _ in range(12):
            i = g.integers(W[l].shape[0])
            j = g.integers(W[l].shape[1])
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (train.cfm_loss_grad(Wp, b, cn, x1, x0, t)[0]
                  - train.cfm_loss_grad(Wm, b, cn, x1, x0, t)[0]) / (2 * h)
            assert abs(fd - gW[l][i, j]) < 1e-6 * max(1.0, abs(fd)), (l, i, j, fd, gW[l][i, j])
        i = g.integers(b[l].shape[0])
        bp = [v.copy() for v in b]
        bm = [v.copy() for v in b]
        bp[l][i] += h
        bm[l][i] -= h
        fd = (train.cfm_loss_grad(W, bp, cn, x1, x0, t)[0]
              - train.cfm_loss_grad(W, bm, cn, x1, x0, t)[0]) / (2 * h)
        assert abs(fd - gb[l][i]) < 1e-6 * max(1.0, abs(fd))


def test_adamw_matches_torch():
    g = np.random.default_rng(0)
    p0 = g.standard_normal(50)
    grads = [g.standard_normal(50) for _ in range(6)]
    tp = torch.nn.Parameter(torch.tensor(p0, dtype=torch.float64))
    opt = torch.optim.AdamW([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.01)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, gr in enumerate(grads, start=1):
        tp.grad = torch.tensor(gr, dtype=torch.float64)
        opt.step()
        p, m, v = train.adamw_step(p, gr, m, v, k)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=1e-15)


def test_w1_matches_scipy_and_closed_form():
    g = np.random.default_rng(4)
    a, b = g.standard_normal(1000), g.standard_normal(1000) * 1.3 + 0.2
    assert abs(ostats.w1(a, b) - sstats.wasserstein_distance(a, b)) < 1e-12
    c = g.standard_normal(777)
    assert abs(ostats.w1(a, c) - sstats.wasserstein_distance(a, c)) < 1e-12
    # a pure shift moves every quantile by the same amount
    assert abs(ostats.w1(a, a + 0.7) - 0.7) < 1e-12


def test_moments_and_sigma_bar():
    g = np.random.default_rng(5)
    x = g.standard_normal(5000)
    mu, var, skew = ostats.moments(x)
    assert abs(mu - x.mean()) < 1e-15 and abs(var - x.var()) < 1e-15
    assert abs(skew - sstats.skew(x)) < 1e-12
    runs = g.standard_normal((5, 30))
    expect = np.mean(np.std(runs, axis=0, ddof=1))
    assert abs(ostats.sigma_bar(runs) - expect) < 1e-14


def test_rect_network_gradient_by_central_differences():
    # 6 condition components: W1 has 26 columns, the aspect in column 25
    g = np.random.default_rng(4)
    net = synth.kaiming_weights_rect(3)
    W = [w.astype(np.float64) * 0.5 for w in net["W"]]
    b = [g.standard_normal(v.shape) * 0.1 for v in net["b"]]
    B = 6
    cn = g.standard_normal((B, 6))
    x1, x0, t = g.standard_normal((B, 4)), g.standard_normal((B, 4)), g.random(B)
    _, gW, _ = train.cfm_loss_grad(W, b, cn, x1, x0, t)
    assert gW[0].shape == (256, 26)
    h = 1e-6
    for j in (0, 7, 25):
        for i in g.integers(256, size=4):
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[0][i, j] += h
            Wm[0][i, j] -= h
            fd = (train.cfm_loss_grad(Wp, b, cn, x1, x0, t)[0]
                  - train.cfm_loss_grad(Wm, b, cn, x1, x0, t)[0]) / (2 * h)
            assert abs(fd - gW[0][i, j]) < 1e-6 * max(1.0, abs(fd))
