"""x-y geometry transport solves on the GPU (transport_solve_xy,
transport_solve_wall_xy: cells are cross-sections of infinite prisms,
directions 3-D) against the oracle.

* One pure-absorber cell, surface source and volumetric source: flux and
  leakage against quadrature of the 3-D chord (the closed forms the oracle's
  x-y solve is pinned to).
* Heterogeneous 16 x 16 grids, cell by cell against the oracle's event loop
  (8 seeds per side, |z| <= 4 in 99 % of the cells, <= 6 in all): the random
  walk (GMC_METHOD_ANALOG; walks on the sphere, births on the sphere) and GMC
  with an x-y network (FP32 and BF16; births walked), the oracle driving its
  event loop with the same network and decoding into the unit disk.
* The committed x-y network against the x-y random walk on the solve
  benchmark's materials.
"""
import math
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def xctx(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_13965_gb300 as g
    path = str(tmp_path_factory.mktemp("xy") / "k.bin")
    # the flat solve tests' network (Kaiming seed 1): exits spread over the
    # cell without the heavy track-length tail a random output
    # standardization gives, so the per-cell spread is estimable from 8 runs
    synth.write_weights(path, synth.kaiming_weights(1))
    ctx = g.Context(0)
    g.gmc_load_xy_weights(ctx, path)
    yield {"ctx": ctx, "path": path}
    ctx.close()


def _set(ctx, **kw):
    import paper_2512_13965_gb300 as g
    cfg = g.gmc_get_config(ctx)
    for k, v in kw.items():
        setattr(cfg, k, v)
    g.gmc_set_config(ctx, cfg)


def _solve(ctx, tau, c, src, n, method, seed, wall=None):
    import paper_2512_13965_gb300 as g
    ny, nx = tau.shape
    f = np.zeros(ny * nx)
    args = [np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c)]
    if wall is None:
        st = g.transport_solve_xy(ctx, nx, ny, *args, np.ascontiguousarray(src, np.float32).ravel(),
                                  n, method, seed, f)
    else:
        st = g.transport_solve_wall_xy(ctx, nx, ny, *args, np.ascontiguousarray(wall, np.float32),
                                       n, method, seed, f)
    return f.reshape(ny, nx), st.as_dict()


def _chord(x, y, ux, uy, tau):
    with np.errstate(divide="ignore", invalid="ignore"):
        lx = np.where(ux > 0, (tau - x) / ux, np.where(ux < 0, -x / ux, np.inf))
        ly = np.where(uy > 0, (tau - y) / uy, np.where(uy < 0, -y / uy, np.inf))
    return np.minimum(lx, ly)


def _mid(n, lo=0.0, hi=1.0):
    return lo + (np.arange(n) + 0.5) * (hi - lo) / n


@pytest.mark.parametrize("tau", [0.4, 1.7])
def test_xy_wall_single_cell_quadrature(xctx, tau):
    import paper_2512_13965_gb300 as g
    X, M2, P = np.meshgrid(_mid(160), _mid(160), _mid(160, 0.0, 2.0 * np.pi), indexing="ij")
    l = _chord(np.zeros_like(X), X * tau, np.sqrt(M2), np.sqrt(1.0 - M2) * np.cos(P), tau)
    sc = (1.0 - np.exp(-l)) / tau
    f_q, var, leak_q = sc.mean(), sc.var(), np.exp(-l).mean()
    n = 2_000_000
    f, st = _solve(xctx["ctx"], np.full((1, 1), tau), np.zeros((1, 1)), None, n,
                   g.GMC_METHOD_ANALOG, 3, wall=np.ones(1))
    assert abs(f[0, 0] - f_q) < 4 * math.sqrt(var / n) + 1e-4 * f_q, (f[0, 0], f_q)
    assert abs(st["leaked"] / n - leak_q) < 4 * math.sqrt(leak_q * (1 - leak_q) / n) + 1e-4


@pytest.mark.parametrize("tau", [0.6, 2.5])
def test_xy_volumetric_single_cell_quadrature(xctx, tau):
    import paper_2512_13965_gb300 as g
    xs, mus, phis = _mid(48), _mid(48), _mid(96, 0.0, 2.0 * np.pi)
    acc = acc2 = leak = 0.0
    for x in xs:
        Y, MU, P = np.meshgrid(xs, mus, phis, indexing="ij")
        r = np.sqrt(1.0 - MU * MU)
        l = _chord(np.full_like(Y, x * tau), Y * tau, r * np.cos(P), r * np.sin(P), tau)
        sc = (1.0 - np.exp(-l)) / tau
        acc += sc.mean()
        acc2 += (sc * sc).mean()
        leak += np.exp(-l).mean()
    f_q, f2_q, leak_q = acc / xs.size, acc2 / xs.size, leak / xs.size
    n = 2_000_000
    f, st = _solve(xctx["ctx"], np.full((1, 1), tau), np.zeros((1, 1)), np.ones((1, 1)), n,
                   g.GMC_METHOD_ANALOG, 5)
    assert abs(f[0, 0] - f_q) < 4 * math.sqrt((f2_q - f_q * f_q) / n) + 2e-4 * f_q, (f[0, 0], f_q)
    assert abs(st["leaked"] / n - leak_q) < 4 * math.sqrt(leak_q * (1 - leak_q) / n) + 2e-4


def _percell(ctx, tau, c, src, method, sampler, wall=None, K=8, n_gpu=20000, n_oracle=4000):
    import _oracle_pool as P
    gpu = [_solve(ctx, tau, c, src, n_gpu, method, 1000 + k, wall=wall)[0] for k in range(K)]
    tasks = [{"grid": (tau, c, src), "n": n_oracle, "seed": 2000 + k, "sampler": sampler,
              "internal": None, "wall": wall, "geometry": "xy"} for k in range(K)]
    orc = P.solve_many(tasks)
    P.assert_per_cell(gpu, [f for f, _ in orc])


def _grid16(seed, hi=5.0):
    return synth.grid_problem(n=16, seed=seed, tau_range=(0.1, hi), block=4, source=4)


def test_xy_analog_solve_per_cell(xctx):
    import paper_2512_13965_gb300 as g
    _set(xctx["ctx"], bank_capacity=1 << 16)
    tau, c, src = _grid16(41)
    _percell(xctx["ctx"], tau, c, src, g.GMC_METHOD_ANALOG, ("walk_global_xy",))


def test_xy_wall_analog_solve_per_cell(xctx):
    import paper_2512_13965_gb300 as g
    _set(xctx["ctx"], bank_capacity=1 << 16)
    tau, c, _ = _grid16(43)
    wall = np.linspace(1.0, 2.0, 16)
    _percell(xctx["ctx"], tau, c, None, g.GMC_METHOD_ANALOG, ("walk_global_xy",), wall=wall)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_xy_gmc_solve_per_cell(xctx, prec):
    # cells inside the box (tau >= 0.1, c in [0.5, 0.999]) are all sampled
    import paper_2512_13965_gb300 as g
    _set(xctx["ctx"], precision=g.GMC_FP32 if prec == "fp32" else g.GMC_BF16, steps=4,
         integrator=g.GMC_EULER, bank_capacity=1 << 16, gmc_min_tau=0.0)
    tau, c, src = _grid16(45, hi=20.0)
    _percell(xctx["ctx"], tau, c, src, g.GMC_METHOD_GMC, ("mlp_xy", xctx["path"], 4, "euler"))


def test_xy_gmc_needs_the_xy_network():
    import paper_2512_13965_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, os.path.join(ROOT, "paper_2512_13965_gb300", "weights",
                                             "gmc_boundary.bin"))
        tau, c, src = _grid16(47)
        with pytest.raises(g.GMCError) as e:
            _solve(ctx, tau, c, src, 100, g.GMC_METHOD_GMC, 1)
        assert e.value.status == g.GMC_ENOWEIGHTS
    finally:
        ctx.close()


def test_committed_xy_network_against_the_xy_walk():
    # the committed x-y boundary network (births walked) against the x-y
    # random walk, 32 x 32 grid of the solve benchmark's materials, 4e6
    # histories, BF16 midpoint 8: within 2 %
    import paper_2512_13965_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    ctx = g.Context(0)
    try:
        g.gmc_load_xy_weights(ctx, os.path.join(ROOT, "paper_2512_13965_gb300", "weights",
                                                "gmc_xy.bin"))
        _set(ctx, precision=g.GMC_BF16, steps=8, integrator=g.GMC_MIDPOINT, gmc_min_tau=0.0)
        tau, c, src = synth.grid_problem(n=32, seed=5, tau_range=(0.1, 500.0), block=8, source=4)
        fa, _ = _solve(ctx, tau, c, src, 2_000_000, g.GMC_METHOD_ANALOG, 1)
        fb, _ = _solve(ctx, tau, c, src, 2_000_000, g.GMC_METHOD_ANALOG, 2)
        f_mc = 0.5 * (fa + fb)
        floor = np.linalg.norm(fa - fb) / np.linalg.norm(f_mc) / math.sqrt(2.0)
        f, st = _solve(ctx, tau, c, src, 4_000_000, g.GMC_METHOD_GMC, 3)
        err = np.linalg.norm(f - f_mc) / np.linalg.norm(f_mc)
        assert floor < 0.006 and err < 0.02, (err, floor)
        assert st["transmissions"] > 0
    finally:
        ctx.close()


def _u01_f32(x):
    # the device's float uniform: fma((float)x, 2^-32, 2^-32)
    return (x.astype(np.float32) * np.float32(2.0 ** -32) + np.float32(2.0 ** -32)).astype(np.float32)


def test_xy_internal_training_data_matches_oracle_walk(xctx):
    # the x-y internal model's data: inputs from Philox (i, 0/1, tag 9), the
    # walk on the sphere from the birth point against the oracle's x-y walk
    # on the same counters, sample by sample
    import oracle
    from oracle import transport as OT
    import paper_2512_13965_gb300 as g
    n, seed = 4000, 43
    cond = torch.empty(5, n, device="cuda")
    y = torch.empty(4, n, device="cuda")
    g.gmc_train_data_internal_xy(xctx["ctx"], n, seed, 0.3, 30.0, 0.5, 0.999, cond, y)
    torch.cuda.synchronize()
    c = cond.cpu().numpy()
    yg = y.cpu().numpy().astype(np.float64)
    raw0 = oracle.rng.philox_batch(seed, n, id0=0, event=0, tag=9)
    raw1 = oracle.rng.philox_batch(seed, n, id0=0, event=1, tag=9)
    lo, hi = np.log(np.float32(0.3)), np.log(np.float32(30.0))
    np.testing.assert_allclose(c[2], lo + (hi - lo) * _u01_f32(raw0[:, 0]), rtol=1e-5, atol=1e-5)
    X, Y = _u01_f32(raw0[:, 2]), _u01_f32(raw0[:, 3])
    np.testing.assert_array_equal(c[0], X)
    np.testing.assert_array_equal(c[1], Y)
    phi = 2.0 * np.pi * _u01_f32(raw1[:, 0]).astype(np.float64)
    mu = 2.0 * _u01_f32(raw1[:, 1]).astype(np.float64) - 1.0
    r = np.sqrt(np.maximum(1.0 - mu * mu, 0.0))
    tau = np.exp(c[2].astype(np.float64))
    same = 0
    for i in range(n):
        w = OT.walk_one_xy(tau[i], float(c[3, i]), OT.MODE_IMPLICIT, float(X[i]) * tau[i],
                           float(Y[i]) * tau[i], r[i] * np.cos(phi[i]), r[i] * np.sin(phi[i]),
                           seed, i, 2)
        if int(np.floor(yg[0, i])) == w["face"] and abs(yg[3, i] - np.log(w["s"])) < 1e-3:
            same += 1
            assert abs(yg[0, i] - (w["face"] + w["q"])) < 1e-3
            assert abs(yg[1, i] - w["ux"]) < 1e-4 and abs(yg[2, i] - w["uy"]) < 1e-4
    assert same > 0.99 * n
    assert np.all(yg[1] ** 2 + yg[2] ** 2 <= 1.0 + 1e-6)


def test_xy_gmc_solve_with_internal_births_per_cell(xctx):
    # births sampled by an x-y internal model (the Kaiming test network)
    # against the oracle's event loop with the same network, cell by cell
    import paper_2512_13965_gb300 as g
    ctx = xctx["ctx"]
    # (after this test only tests on contexts of their own follow: the
    # tests above walk their births)
    import _oracle_pool as P
    g.gmc_load_internal_xy_weights(ctx, xctx["path"])
    _set(ctx, precision=g.GMC_FP32, steps=4, integrator=g.GMC_EULER, bank_capacity=1 << 16,
         gmc_min_tau=0.0)
    tau, c, src = _grid16(49, hi=20.0)
    gpu = [_solve(ctx, tau, c, src, 20000, g.GMC_METHOD_GMC, 1000 + k)[0] for k in range(8)]
    tasks = [{"grid": (tau, c, src), "n": 4000, "seed": 2000 + k,
              "sampler": ("mlp_xy", xctx["path"], 4, "euler"),
              "internal": ("mlp_xy", xctx["path"], 4, "euler"), "wall": None, "geometry": "xy"}
             for k in range(8)]
    orc = P.solve_many(tasks)
    P.assert_per_cell(gpu, [f for f, _ in orc])


def test_committed_xy_internal_network():
    # the committed x-y internal model with the x-y boundary network: the
    # x-y solve within 2 % of the x-y walk, and faster than walking births
    import paper_2512_13965_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    w = os.path.join(ROOT, "paper_2512_13965_gb300", "weights")
    ctx = g.Context(0)
    try:
        g.gmc_load_xy_weights(ctx, os.path.join(w, "gmc_xy.bin"))
        _set(ctx, precision=g.GMC_BF16, steps=8, integrator=g.GMC_MIDPOINT, gmc_min_tau=0.0)
        tau, c, src = synth.grid_problem(n=32, seed=5, tau_range=(0.1, 500.0), block=8, source=4)
        fa, _ = _solve(ctx, tau, c, src, 2_000_000, g.GMC_METHOD_ANALOG, 1)
        fb, _ = _solve(ctx, tau, c, src, 2_000_000, g.GMC_METHOD_ANALOG, 2)
        f_mc = 0.5 * (fa + fb)
        _, st_walked = _solve(ctx, tau, c, src, 4_000_000, g.GMC_METHOD_GMC, 3)
        g.gmc_load_internal_xy_weights(ctx, os.path.join(w, "gmc_internal_xy.bin"))
        f, st = _solve(ctx, tau, c, src, 4_000_000, g.GMC_METHOD_GMC, 3)
        err = np.linalg.norm(f - f_mc) / np.linalg.norm(f_mc)
        assert err < 0.02, err
        assert st["collisions"] < 0.1 * st_walked["collisions"], (st, st_walked)
        assert st["seconds"] < st_walked["seconds"], (st["seconds"], st_walked["seconds"])
    finally:
        ctx.close()
