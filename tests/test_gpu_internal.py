"""Internal (volumetric-source) model on the GPU: its training data against
the oracle walk from interior points, its sampler against the FP64 network,
and GMC solves whose births it samples against the oracle's event loop.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import transport as OT

import _oracle_pool as P

pytestmark = pytest.mark.gpu


def _u01_f32(x):
    # the device's float uniform: fma((float)x, 2^-32, 2^-32)
    return (x.astype(np.float32) * np.float32(2.0 ** -32) + np.float32(2.0 ** -32)).astype(np.float32)


@pytest.fixture(scope="module")
def ictx(kaiming_file):
    # its own context: with an internal model loaded, GMC births use it
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    g.gmc_load_weights(ctx, kaiming_file)
    g.gmc_load_internal_weights(ctx, kaiming_file)
    yield ctx
    ctx.close()


def test_internal_training_data_matches_oracle_walk(ictx):
    import paper_2512_13965_gb300 as g
    n, seed = 6000, 41
    cond = torch.empty(5, n, device="cuda")
    y = torch.empty(4, n, device="cuda")
    g.gmc_train_data_internal(ictx, n, seed, 0.3, 30.0, 0.5, 0.999, cond, y)
    torch.cuda.synchronize()
    c = cond.cpu().numpy()
    yg = y.cpu().numpy().astype(np.float64)
    raw0 = oracle.rng.philox_batch(seed, n, id0=0, event=0, tag=7)
    raw1 = oracle.rng.philox_batch(seed, n, id0=0, event=1, tag=7)
    lo, hi = np.log(np.float32(0.3)), np.log(np.float32(30.0))
    np.testing.assert_allclose(c[2], lo + (hi - lo) * _u01_f32(raw0[:, 0]), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(c[3], 0.5 + (0.999 - 0.5) * _u01_f32(raw0[:, 1]), rtol=1e-6)
    X, Y = _u01_f32(raw0[:, 2]), _u01_f32(raw0[:, 3])
    np.testing.assert_array_equal(c[0], X)
    np.testing.assert_array_equal(c[1], Y)
    np.testing.assert_allclose(c[4], np.minimum(np.minimum(X, Y), np.minimum(1 - X, 1 - Y)), atol=1e-7)
    ang = 2.0 * np.pi * _u01_f32(raw1[:, 0]).astype(np.float64)
    tau = np.exp(c[2].astype(np.float64))
    same = 0
    for i in range(n):
        r = OT.walk_one(tau[i], float(c[3, i]), OT.MODE_IMPLICIT, float(X[i]) * tau[i],
                        float(Y[i]) * tau[i], np.cos(ang[i]), np.sin(ang[i]), seed, i, 2)
        if int(np.floor(yg[0, i])) == r["face"] and abs(yg[3, i] - np.log(r["s"])) < 1e-3:
            same += 1
            assert abs(yg[0, i] - (r["face"] + r["q"])) < 1e-3
            assert abs(yg[1, i] - r["ux"]) < 1e-4 and abs(yg[2, i] - r["uy"]) < 1e-4
    assert same > 0.99 * n


def test_internal_sampler_fp32_parity(ictx, kaiming_file):
    import paper_2512_13965_gb300 as g
    net = oracle.mlp.read_weights(kaiming_file)
    n = 3000
    rng = np.random.default_rng(7)
    X, Y = rng.random(n), rng.random(n)
    tau = np.exp(rng.uniform(np.log(0.1), np.log(1000.0), n))
    cc = rng.uniform(0.5, 0.999, n)
    cond = OT.internal_condition(X, Y, tau, cc).astype(np.float32)
    z = synth.gaussian_noise(n, 8)
    y = torch.empty(4, n, device="cuda")
    g.gmc_sample_internal(ictx, n, torch.from_numpy(cond).cuda(), torch.from_numpy(z).cuda(), 0, 0,
                          6, g.GMC_EULER, g.GMC_FP32, y, None)
    torch.cuda.synchronize()
    expect = oracle.mlp.sample(net, cond, z, 6, "euler")
    assert np.abs(y.cpu().numpy() - expect).max() < 1e-4


def _set(ctx, **kw):
    import paper_2512_13965_gb300 as g
    cfg = g.gmc_get_config(ctx)
    for k, v in kw.items():
        setattr(cfg, k, v)
    g.gmc_set_config(ctx, cfg)


def test_gmc_solve_with_internal_births_per_cell(ictx, kaiming_file):
    # births sampled by the internal model, transmissions by the boundary
    # model (both FP32): K independent seeds per side against the oracle's
    # event loop with the same two networks, compared cell by cell
    import paper_2512_13965_gb300 as g
    _set(ictx, precision=g.GMC_FP32, steps=4, integrator=g.GMC_EULER, bank_capacity=1 << 16)
    tau, c, src = synth.grid_problem(n=16, seed=31, tau_range=(0.1, 5.0), block=4, source=4)
    ny, nx = tau.shape
    args = [np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c, src)]
    n_gpu, n_orc, K = 20000, 4000, 8
    gpu = []
    for k in range(K):
        flux = np.zeros(ny * nx)
        st = g.transport_solve(ictx, nx, ny, *args, n_gpu, g.GMC_METHOD_GMC, 1000 + k, flux).as_dict()
        gpu.append((flux.reshape(ny, nx), st))
    spec = ("mlp", kaiming_file, 4, "euler")
    orc = P.solve_many([{"grid": (tau, c, src), "n": n_orc, "seed": 2000 + k, "sampler": spec,
                         "internal": spec} for k in range(K)])
    P.assert_per_cell([f for f, _ in gpu], [f for f, _ in orc])
    z = P.per_cell_z([[st["leaked"] / n_gpu] for _, st in gpu], [[st["leak"] / n_orc] for _, st in orc])
    assert abs(z[0]) <= 4.0
    for _, st in gpu:
        assert abs(st["absorbed"] + st["leaked"] - st["roulette_net"] - n_gpu) < 1e-4 * n_gpu
        assert st["collisions"] == 0  # no birth was walked


def test_internal_births_at_equivalent_conditions_per_cell(ictx, kaiming_file):
    # births in cells outside the training box sampled by the internal model
    # at the scattering-equivalent condition, walked where there is none;
    # against the oracle's event loop with the same reading
    import paper_2512_13965_gb300 as g
    from test_gpu_transport import BOX, _outside_box_grid
    _set(ictx, precision=g.GMC_FP32, steps=4, integrator=g.GMC_EULER, bank_capacity=1 << 16)
    tau, c, _ = _outside_box_grid(seed=41)
    src = np.ones_like(tau) / tau.size  # births everywhere, walked cells included
    ny, nx = tau.shape
    args = [np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c, src)]
    n_gpu, n_orc, K = 20000, 4000, 8
    gpu = []
    for k in range(K):
        flux = np.zeros(ny * nx)
        st = g.transport_solve(ictx, nx, ny, *args, n_gpu, g.GMC_METHOD_GMC, 1000 + k, flux).as_dict()
        gpu.append((flux.reshape(ny, nx), st))
    spec = ("equivalent", kaiming_file, 4, "euler", BOX)
    orc = P.solve_many([{"grid": (tau, c, src), "n": n_orc, "seed": 2000 + k, "sampler": spec,
                         "internal": spec} for k in range(K)])
    P.assert_per_cell([f for f, _ in gpu], [f for f, _ in orc])
    for _, st in gpu:
        assert abs(st["absorbed"] + st["leaked"] - st["roulette_net"] - n_gpu) < 1e-4 * n_gpu
        assert st["collisions"] > 0


def test_hybrid_with_internal_model_all_thin_equals_analog(ictx):
    # with the internal model loaded, births in thin cells are walked too
    import paper_2512_13965_gb300 as g
    tau, c, src = synth.grid_problem(n=12, seed=36, tau_range=(0.1, 120.0), block=4, source=4)
    ny, nx = tau.shape
    args = [np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c, src)]
    out = {}
    for name, method, mt in (("analog", g.GMC_METHOD_ANALOG, 0.0), ("hybrid", g.GMC_METHOD_GMC, 1e30)):
        _set(ictx, bank_capacity=1 << 14, precision=g.GMC_FP32, steps=4, gmc_min_tau=mt)
        f = np.zeros(ny * nx)
        st = g.transport_solve(ictx, nx, ny, *args, 3000, method, 29, f).as_dict()
        out[name] = (f, st)
    _set(ictx, gmc_min_tau=0.0)
    fa, sa = out["analog"]
    fh, sh = out["hybrid"]
    np.testing.assert_allclose(fh, fa, rtol=1e-9, atol=1e-12 * np.abs(fa).max())
    for k in ("transmissions", "collisions", "roulette_kills"):
        assert sh[k] == sa[k], k
