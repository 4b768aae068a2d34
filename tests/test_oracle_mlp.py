"""Pins for the oracle's velocity network, flow-ODE integrator (Eq. 8) and
exit-state decoding (Eq. 11)."""
import math

import numpy as np
import pytest

import synth
from oracle import mlp


def _zero_net():
    net = synth.kaiming_weights(1)
    net["W"] = [np.zeros_like(w) for w in net["W"]]
    return net


def _load(tmp_path, net, name="w.bin"):
    p = str(tmp_path / name)
    synth.write_weights(p, net)
    return mlp.read_weights(p)


def test_weight_file_round_trip(tmp_path):
    net = synth.kaiming_weights(1)
    net["cond_mean"] = np.arange(5, dtype=np.float32)
    net["y_std"] = np.array([1.5, 2.0, 2.5, 3.0], np.float32)
    o = _load(tmp_path, net)
    for l in range(5):
        np.testing.assert_array_equal(o.W[l], net["W"][l].astype(np.float64))
        np.testing.assert_array_equal(o.b[l], net["b"][l].astype(np.float64))
    np.testing.assert_array_equal(o.cond_mean, np.arange(5))
    np.testing.assert_array_equal(o.y_std, [1.5, 2.0, 2.5, 3.0])
    # Kaiming-normal: per-layer sample std close to sqrt(2 / fan_in)
    for l, fan_in in enumerate(synth.DIMS[:-1]):
        if net["W"][l].size > 10000:
            assert abs(net["W"][l].std() / math.sqrt(2.0 / fan_in) - 1) < 0.02


def test_weight_file_rejects_garbage(tmp_path):
    p = tmp_path / "bad.bin"
    p.write_bytes(b"NOPE" + b"\0" * 64)
    with pytest.raises(ValueError):
        mlp.read_weights(str(p))


def test_time_embedding_values():
    e = mlp.time_embedding(np.array([0.0, 0.25]))
    np.testing.assert_allclose(e[0], [0.0] * 8 + [1.0] * 8, atol=0)
    expect = [math.sin(2 ** j * math.pi * 0.25) for j in range(8)] + \
             [math.cos(2 ** j * math.pi * 0.25) for j in range(8)]
    np.testing.assert_allclose(e[1], expect, atol=1e-15)


@pytest.mark.parametrize("integrator", ["euler", "midpoint"])
@pytest.mark.parametrize("steps", [1, 3, 16])
def test_constant_velocity_is_exact(tmp_path, integrator, steps):
    # All weights zero except the output bias: v = b5, so x(1) = x(0) + b5.
    net = _zero_net()
    net["b"][4] = np.array([0.5, -1.25, 2.0, 0.125], np.float32)
    o = _load(tmp_path, net)
    cond, _, _ = synth.sampler_conditions(64, 3)
    z = synth.gaussian_noise(64, 4)
    y = mlp.sample(o, cond, z, steps, integrator)
    np.testing.assert_allclose(y, z.astype(np.float64) + net["b"][4][:, None].astype(np.float64),
                               rtol=0, atol=1e-14)


def _silu(z):
    return z / (1.0 + math.exp(-z))


def test_single_path_through_the_network(tmp_path):
    # One chain of units: input column 5 (= x_0, after the 5 condition
    # features) -> hidden unit 0 of every layer -> output 0. Then
    # v_0 = silu^4(a x_0) and the other outputs are 0; K = 1 Euler gives
    # x_0(1) = x_0 + silu^4(a x_0).
    net = _zero_net()
    a = float(np.float32(0.7))  # the file stores float32 weights
    net["W"][0][0, 5] = a
    for l in (1, 2, 3):
        net["W"][l][0, 0] = 1.0
    net["W"][4][0, 0] = 1.0
    o = _load(tmp_path, net)
    cond, _, _ = synth.sampler_conditions(8, 5)
    z = synth.gaussian_noise(8, 6)
    y = mlp.sample(o, cond, z, 1, "euler")
    for i in range(8):
        x0 = float(z[0, i])
        expect = x0 + _silu(_silu(_silu(_silu(a * x0))))
        assert abs(y[0, i] - expect) < 1e-14
        np.testing.assert_allclose(y[1:, i], z[1:, i].astype(np.float64), atol=0)


def test_condition_and_time_columns(tmp_path):
    # Input order [cond(5), x(4), emb(16)] and condition standardization:
    # hidden unit 0 reads standardized ln tau (column 3) and unit 1 reads
    # emb column 9 + 2 = sin(4 pi t); the output sums the two chains.
    net = _zero_net()
    net["cond_mean"] = np.array([0, 0, 0, 1.5, 0], np.float32)
    net["cond_std"] = np.array([1, 1, 1, 2.0, 1], np.float32)
    net["W"][0][0, 3] = 1.0
    net["W"][0][1, 9 + 2] = 1.0
    for l in (1, 2, 3):
        net["W"][l][0, 0] = 1.0
        net["W"][l][1, 1] = 1.0
    net["W"][4][2, 0] = 1.0
    net["W"][4][3, 1] = 1.0
    o = _load(tmp_path, net)
    cond, _, _ = synth.sampler_conditions(4, 8)
    z = synth.gaussian_noise(4, 9)
    steps = 4
    y = mlp.sample(o, cond, z, steps, "euler")
    f4 = lambda v: _silu(_silu(_silu(_silu(v))))
    for i in range(4):
        u = (float(cond[3, i]) - 1.5) / 2.0
        e2 = float(z[2, i]) + f4(u)
        e3 = float(z[3, i]) + sum(f4(math.sin(4 * math.pi * k / steps)) for k in range(steps)) / steps
        assert abs(y[2, i] - e2) < 1e-13 and abs(y[3, i] - e3) < 1e-13


@pytest.mark.parametrize("steps", [1, 5, 16])
def test_integrators_on_linear_field(steps):
    # dx/dt = a x: Euler gives (1 + a h)^K x0, the midpoint rule
    # (1 + a h + (a h)^2 / 2)^K x0, classical RK4 the degree-4 Taylor
    # polynomial of exp(a h) to the power K.
    a, h = -0.8, 1.0 / steps
    x0 = np.array([[1.0, -2.0, 0.5, 3.0]])
    ye = mlp.integrate(lambda x, t: a * x, x0, steps, "euler")
    ym = mlp.integrate(lambda x, t: a * x, x0, steps, "midpoint")
    yr = mlp.integrate(lambda x, t: a * x, x0, steps, "rk4")
    z = a * h
    np.testing.assert_allclose(ye, (1 + z) ** steps * x0, rtol=1e-14)
    np.testing.assert_allclose(ym, (1 + z + 0.5 * z ** 2) ** steps * x0, rtol=1e-14)
    np.testing.assert_allclose(yr, (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24) ** steps * x0,
                               rtol=1e-13)


def test_rk4_on_time_field_is_simpson():
    # dx/dt = f(t): RK4 reduces to Simpson's rule per step.
    K = 5
    f = lambda t: np.exp(np.sin(3 * t))
    y = mlp.integrate(lambda x, t: f(t) + 0 * x, np.zeros((1, 1)), K, "rk4")
    h = 1.0 / K
    expect = sum(h / 6 * (f(k * h) + 4 * f(k * h + h / 2) + f(k * h + h)) for k in range(K))
    assert abs(y[0, 0] - expect) < 1e-14


def test_integrators_on_time_field():
    # dx/dt = cos(t): Euler is the left Riemann sum, midpoint the midpoint sum.
    K = 8
    ye = mlp.integrate(lambda x, t: np.cos(t) + 0 * x, np.zeros((1, 1)), K, "euler")
    ym = mlp.integrate(lambda x, t: np.cos(t) + 0 * x, np.zeros((1, 1)), K, "midpoint")
    assert abs(ye[0, 0] - sum(math.cos(k / K) for k in range(K)) / K) < 1e-15
    assert abs(ym[0, 0] - sum(math.cos((k + 0.5) / K) for k in range(K)) / K) < 1e-15


def test_decode_rules(tmp_path):
    net = _zero_net()
    net["y_mean"] = np.array([0, 0, 0, 0], np.float32)
    net["y_std"] = np.array([1, 1, 1, 1], np.float32)
    o = _load(tmp_path, net)
    y = np.array([
        [4.25, 0.0, 0.0, math.log(2.0)],      # wraps to bottom face, q = 0.25
        [-0.5, -0.6, 0.8, 0.0],               # wraps to left face, q = 0.5
        [1.5, -3.0, 4.0, -40.0],              # right face, inward -> reflected
        [2.75, 0.6, -0.8, 1.0],               # top face, inward -> reflected
    ]).T
    d = mlp.decode(o, y)
    np.testing.assert_array_equal(d["face"], [0, 3, 1, 2])
    np.testing.assert_allclose(d["q"], [0.25, 0.5, 0.5, 0.75], atol=1e-15)
    # zero direction -> outward normal of the bottom face
    np.testing.assert_allclose([d["ux"][0], d["uy"][0]], [0.0, -1.0])
    np.testing.assert_allclose([d["ux"][1], d["uy"][1]], [-0.6, 0.8])
    np.testing.assert_allclose([d["ux"][2], d["uy"][2]], [0.6, 0.8])
    np.testing.assert_allclose([d["ux"][3], d["uy"][3]], [0.6, 0.8])
    np.testing.assert_array_equal(d["inward"], [False, False, True, True])
    np.testing.assert_allclose(d["s"], [2.0, 1.0, mlp.S_MIN, math.e])


def test_decode_disk_rules(tmp_path):
    # x-y geometry: the projected direction stays inside the unit disk
    net = _zero_net()
    net["y_mean"] = np.array([0, 0, 0, 0], np.float32)
    net["y_std"] = np.array([1, 1, 1, 1], np.float32)
    o = _load(tmp_path, net)
    y = np.array([
        [1.5, 0.3, 0.4, 0.0],      # right face, inside the disk: kept
        [1.5, 3.0, 4.0, 0.0],      # outside the disk: back onto the circle
        [1.5, -0.3, 0.4, 0.0],     # inward: reflected
        [1.5, 0.0, 0.5, 0.0],      # parallel to the face: outward normal
        [0.25, 0.0, 0.0, 0.0],     # zero on the bottom face: outward normal
        [2.5, -0.6, -0.8, 0.0],    # top face, on the circle, inward: reflected
        [-0.5, -0.28, -0.96, 0.0], # wraps to the left face, unit, outward
    ]).T
    d = mlp.decode_disk(o, y)
    np.testing.assert_array_equal(d["face"], [1, 1, 1, 1, 0, 2, 3])
    ex = np.array([[0.3, 0.4], [0.6, 0.8], [0.3, 0.4], [1.0, 0.0], [0.0, -1.0],
                   [-0.6, 0.8], [-0.28, -0.96]])
    np.testing.assert_allclose(np.stack([d["ux"], d["uy"]], 1), ex, atol=1e-15)
    np.testing.assert_allclose(d["uz"], [math.sqrt(0.75), 0, math.sqrt(0.75), 0, 0, 0, 0],
                               atol=1e-7)
    np.testing.assert_array_equal(d["inward"], [False, False, True, False, False, True, False])
    # on the circle the disk decode is the circle decode
    f = mlp.decode(o, y[:, [1, 5, 6]])
    g = mlp.decode_disk(o, y[:, [1, 5, 6]])
    for k in ("face", "q", "ux", "uy", "s"):
        np.testing.assert_allclose(f[k], g[k], atol=1e-15)


def test_decode_destandardizes(tmp_path):
    net = _zero_net()
    net["y_mean"] = np.array([2.0, 0.0, 0.0, 1.0], np.float32)
    net["y_std"] = np.array([0.5, 2.0, 2.0, 0.25], np.float32)
    o = _load(tmp_path, net)
    d = mlp.decode(o, np.array([[1.0], [0.3], [0.4], [-4.0]]))
    assert d["face"][0] == 2 and abs(d["q"][0] - 0.5) < 1e-15
    np.testing.assert_allclose([d["ux"][0], d["uy"][0]], [0.6, 0.8])
    assert abs(d["s"][0] - 1.0) < 1e-15


def _e4m3_values():
    # every non-negative finite E4M3 value, from the format's definition:
    # zero, subnormals m/8 2^-6, normals (1 + m/8) 2^(e-7) up to 448
    v = [0.0] + [m / 8 * 2.0 ** -6 for m in range(1, 8)]
    v += [(1 + m / 8) * 2.0 ** (e - 7) for e in range(1, 16) for m in range(8)]
    return np.array(v[:-1])  # e = 15, m = 7 is NaN


def test_round_e4m3_format_values():
    v = _e4m3_values()
    assert v.size == 127 and v[-1] == 448.0 and np.all(np.diff(v) > 0)
    np.testing.assert_array_equal(mlp.round_e4m3(v), v)
    np.testing.assert_array_equal(mlp.round_e4m3(-v), -v)
    # midpoints go to the neighbour with the even code (code = index here)
    mid = 0.5 * (v[:-1] + v[1:])
    even = np.where(np.arange(v.size - 1) % 2 == 0, v[:-1], v[1:])
    np.testing.assert_array_equal(mlp.round_e4m3(mid), even)
    # just off the midpoint: nearest
    np.testing.assert_array_equal(mlp.round_e4m3(mid * (1 - 1e-9)), v[:-1])
    np.testing.assert_array_equal(mlp.round_e4m3(mid * (1 + 1e-9)), v[1:])
    # saturation
    np.testing.assert_array_equal(mlp.round_e4m3([449.0, 1e6, -1e30]), [448.0, 448.0, -448.0])


def test_round_e4m3_matches_torch_cast():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn")
    rng = np.random.default_rng(0)
    x = rng.standard_normal(200000) * np.exp(rng.uniform(-14, 7, 200000))
    x = np.clip(x, -448, 448)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.round_e4m3(x), ref)


def test_quantized_e4m3_weights(tmp_path):
    o = _load(tmp_path, synth.kaiming_weights(1))
    q = mlp.quantized_e4m3(o)
    for l in (0, 4):
        np.testing.assert_array_equal(q.W[l], o.W[l])
    for l in (1, 2, 3):
        sc = np.abs(o.W[l]).max(axis=1, keepdims=True) / 448.0
        err = np.abs(q.W[l] - o.W[l])
        # half a spacing: 2^-4 relative in the normal range, 2^-10 s below it
        assert np.all(err <= np.maximum(np.abs(o.W[l]) / 16, sc * 2.0 ** -10) * (1 + 1e-12))
        # each row's largest weight maps to 448 and is kept (up to the
        # rounding of the division and multiplication by s_c)
        i = np.arange(256), np.abs(o.W[l]).argmax(axis=1)
        np.testing.assert_allclose(q.W[l][i], o.W[l][i], rtol=1e-15)


def test_quantized_e4m3_single_path(tmp_path):
    # the chain of test_single_path_through_the_network: its weights are
    # exact in E4M3 after scaling (row max 1 -> 448), so only the inputs of
    # layers 2-4 are rounded: x_0(1) = x_0 + silu(r(silu(r(silu(r(silu(a x_0)))))))
    net = _zero_net()
    a = float(np.float32(0.7))
    net["W"][0][0, 5] = a
    for l in (1, 2, 3):
        net["W"][l][0, 0] = 1.0
    net["W"][4][0, 0] = 1.0
    q = mlp.quantized_e4m3(_load(tmp_path, net))
    cond, _, _ = synth.sampler_conditions(8, 5)
    z = synth.gaussian_noise(8, 6)
    y = mlp.sample(q, cond, z, 1, "euler")
    r = lambda u: float(mlp.round_e4m3(u))
    for i in range(8):
        x0 = float(z[0, i])
        expect = x0 + _silu(r(_silu(r(_silu(r(_silu(a * x0)))))))
        assert abs(y[0, i] - expect) < 1e-14


def test_evaluation_counts_and_times():
    # the paper's timed solver, RK4 with 12 fixed steps, makes 48 network
    # evaluations per sample; Euler K and midpoint 2K; every evaluation time
    # lies in [0, 1] on the step's nodes (t_k, t_k + h/2, t_k + h)
    for integ, steps, count in (("rk4", 12, 48), ("euler", 16, 16), ("midpoint", 8, 16)):
        seen = []

        def v(x, t):
            seen.append(t)
            return 0.0 * x

        mlp.integrate(v, np.zeros((1, 4)), steps, integ)
        assert len(seen) == count, integ
        h = 1.0 / steps
        nodes = {round(k * h / 2, 12) for k in range(2 * steps + 1)}
        assert all(0.0 <= t <= 1.0 and round(t, 12) in nodes for t in seen)


def test_rect_network_reads_the_aspect_as_input_25(tmp_path):
    # a network for rectangular cells: 6 condition components, the aspect
    # ln(tau_y / tau_x) entering as input column 25 (after the embedding).
    # Only W1[0, 25] and the output chain through unit 0 are non-zero, so
    # v_2 = silu^4(a * standardized aspect) and one Euler step adds it.
    net = synth.kaiming_weights_rect(1)
    net["W"] = [np.zeros_like(w) for w in net["W"]]
    net["cond_mean"] = np.array([0, 0, 0, 0, 0, 0.5], np.float32)
    net["cond_std"] = np.array([1, 1, 1, 1, 1, 2.0], np.float32)
    a = float(np.float32(0.8))
    net["W"][0][0, 25] = a
    for l in (1, 2, 3):
        net["W"][l][0, 0] = 1.0
    net["W"][4][2, 0] = 1.0
    o = _load(tmp_path, net, "rect.bin")
    assert o.W[0].shape == (256, 26) and o.cond_mean.shape == (6,)
    cond = synth.rect_conditions(6, 3)
    z = synth.gaussian_noise(6, 4)
    y = mlp.sample(o, cond, z, 1, "euler")
    for i in range(6):
        u = (float(cond[5, i]) - 0.5) / 2.0
        expect = float(z[2, i]) + _silu(_silu(_silu(_silu(a * u))))
        assert abs(y[2, i] - expect) < 1e-13
    # a square-cell file and a rect file of the same first 25 columns agree
    # on squares (aspect 0 with zero mean)
    sq = synth.kaiming_weights(2)
    rc = dict(sq)
    rc["W"] = list(sq["W"])
    rc["W"][0] = np.concatenate([sq["W"][0], np.full((256, 1), 0.3, np.float32)], axis=1)
    rc["cond_mean"] = np.zeros(6, np.float32)
    rc["cond_std"] = np.ones(6, np.float32)
    o_sq, o_rc = _load(tmp_path, sq, "sq.bin"), _load(tmp_path, rc, "rc.bin")
    cond5, _, _ = synth.sampler_conditions(8, 5)
    cond6 = np.concatenate([cond5, np.zeros((1, 8), np.float32)])
    z = synth.gaussian_noise(8, 6)
    np.testing.assert_allclose(mlp.sample(o_rc, cond6, z, 3, "euler"),
                               mlp.sample(o_sq, cond5, z, 3, "euler"), atol=1e-12)
