"""The network for rectangular cells on the GPU (weight files with n_cond = 6:
the aspect ln(tau_y / tau_x) as input column 25; section "Network
Architecture and Inputs", whose condition holds both optical dimensions)
against the oracle.

* Training data (gmc_train_data_rect): inputs from Philox (i, 0/1, tag 10),
  the walk in the rectangle against the oracle's on the same counters.
* Sampler: FP32 within 1e-4 of the FP64 network, BF16 within the BF16 bounds;
  a rectangular-cell network whose aspect column is zero gives, bit for bit,
  the square-cell network's samples.
* Training on the FP32 path: the gradient against the oracle's, a short run
  lowering the loss, the committed file (n_cond 6) read back by the oracle,
  a checkpoint that continues the run.
* Paths that take square cells (solves, gmc_transmit_noalloc) and paths the
  network does not have (FP8, the CTA-pair kernel, BF16 training) refuse it.
* Solves on rectangular cells (transport_solve_rect): on squares they are
  the square solve; the random walk and GMC with a rectangular-cell network
  against the oracle's solve on rectangles, cell by cell.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import transport as OT

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
BF16_MAX, BF16_P999 = 0.1, 0.06


def _u01_f32(x):
    return (x.astype(np.float32) * np.float32(2.0 ** -32) + np.float32(2.0 ** -32)).astype(np.float32)


def _rect_net(seed=5):
    net = synth.kaiming_weights_rect(seed)
    g = synth.generator(seed + 77)
    net["b"] = [(g.standard_normal(len(b)) * 0.3).astype(np.float32) for b in net["b"]]
    net["cond_mean"] = g.uniform(-1.0, 1.0, 6).astype(np.float32)
    net["cond_std"] = g.uniform(0.5, 2.0, 6).astype(np.float32)
    return net


@pytest.fixture(scope="module")
def rctx(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_13965_gb300 as g
    d = tmp_path_factory.mktemp("rect")
    path = str(d / "rect.bin")
    synth.write_weights(path, _rect_net())
    ctx = g.Context(0)
    g.gmc_load_weights(ctx, path)
    yield {"ctx": ctx, "path": path, "net": oracle.mlp.read_weights(path), "dir": d}
    ctx.close()


def _run(ctx, cond, noise, steps, integ, prec):
    import paper_2512_13965_gb300 as g
    n = cond.shape[1]
    y = torch.full((4, n), float("nan"), device="cuda")
    g.gmc_transmit(ctx, n, torch.from_numpy(cond).cuda(), torch.from_numpy(noise).cuda(), 0, 0,
                   steps, integ, prec, y, None, n_cond=cond.shape[0])
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def test_rect_training_data_matches_oracle_walk(rctx):
    import paper_2512_13965_gb300 as g
    n, seed = 4000, 17
    cond = torch.empty(6, n, device="cuda")
    y = torch.empty(4, n, device="cuda")
    g.gmc_train_data_rect(rctx["ctx"], n, seed, 0.3, 30.0, 0.25, 4.0, 0.5, 0.999, cond, y)
    torch.cuda.synchronize()
    c = cond.cpu().numpy().astype(np.float64)
    yg = y.cpu().numpy().astype(np.float64)
    raw0 = oracle.rng.philox_batch(seed, n, id0=0, event=0, tag=10)
    raw1 = oracle.rng.philox_batch(seed, n, id0=0, event=1, tag=10)
    lo, hi = np.log(np.float32(0.3)), np.log(np.float32(30.0))
    np.testing.assert_allclose(c[3], lo + (hi - lo) * _u01_f32(raw0[:, 0]), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(c[4], 0.5 + (0.999 - 0.5) * _u01_f32(raw0[:, 1]), rtol=1e-6)
    np.testing.assert_array_equal(c[0], _u01_f32(raw0[:, 2]).astype(np.float64))
    np.testing.assert_allclose(c[2], 2 * _u01_f32(raw0[:, 3]) - 1, atol=1e-7)
    la_lo, la_hi = np.log(np.float32(0.25)), np.log(np.float32(4.0))
    np.testing.assert_allclose(c[5], la_lo + (la_hi - la_lo) * _u01_f32(raw1[:, 0]), atol=1e-5)
    tx, ty = np.exp(c[3]), np.exp(c[3] + c[5])
    r = OT.transmit_rect(c[0], c[1], c[2], tx, ty, c[4], OT.MODE_IMPLICIT, seed,
                         ids=np.arange(n, dtype=np.uint64), events=np.full(n, 2, np.uint32))
    same = (np.floor(yg[0]) == r["face"]) & (np.abs(yg[3] - np.log(r["s"])) < 1e-3)
    assert same.mean() > 0.99
    assert np.abs(yg[0] - (r["face"] + r["q"]))[same].max() < 1e-3


INTEGS = [("euler", 8), ("midpoint", 4), ("rk4", 3)]


@pytest.mark.parametrize("integ,steps", INTEGS)
def test_rect_sampler_matches_oracle(rctx, integ, steps):
    import paper_2512_13965_gb300 as g
    code = {"euler": g.GMC_EULER, "midpoint": g.GMC_MIDPOINT, "rk4": g.GMC_RK4}[integ]
    n = 2 * 256 + 91
    cond = synth.rect_conditions(n, 21 + steps)
    z = synth.gaussian_noise(n, 22 + steps)
    expect = oracle.mlp.sample(rctx["net"], cond, z, steps, integ)
    y32 = _run(rctx["ctx"], cond, z, steps, code, g.GMC_FP32)
    assert np.abs(y32 - expect).max() < FP32_TOL
    y16 = _run(rctx["ctx"], cond, z, steps, code, g.GMC_BF16)
    err = np.abs(y16 - expect)
    assert err.max() < BF16_MAX and np.quantile(err, 0.999) < BF16_P999, (err.max(),)


def test_rect_network_with_zero_aspect_column_is_the_square_network(rctx):
    # same first 25 columns, aspect column zero: every output bit equal to the
    # square-cell network's, FP32 and BF16
    import paper_2512_13965_gb300 as g
    sq = synth.biased_weights(9)
    rc = dict(sq)
    rc["W"] = list(sq["W"])
    rc["W"][0] = np.concatenate([sq["W"][0], np.zeros((256, 1), np.float32)], axis=1)
    rc["cond_mean"] = np.concatenate([sq["cond_mean"], [0.3]]).astype(np.float32)
    rc["cond_std"] = np.concatenate([sq["cond_std"], [1.7]]).astype(np.float32)
    p_sq, p_rc = str(rctx["dir"] / "sq.bin"), str(rctx["dir"] / "rc.bin")
    synth.write_weights(p_sq, sq)
    synth.write_weights(p_rc, rc)
    n = 700
    cond6 = synth.rect_conditions(n, 31)
    z = synth.gaussian_noise(n, 32)
    ctx = g.Context(0)
    try:
        out = {}
        for name, p, cond in (("sq", p_sq, cond6[:5].copy()), ("rc", p_rc, cond6)):
            g.gmc_load_weights(ctx, p)
            out[name] = [_run(ctx, cond, z, 6, g.GMC_EULER, prec) for prec in (g.GMC_FP32, g.GMC_BF16)]
        for a, b in zip(out["sq"], out["rc"]):
            np.testing.assert_array_equal(a, b)
    finally:
        ctx.close()


def test_rect_network_refused_where_cells_are_square(rctx):
    import paper_2512_13965_gb300 as g
    ctx = rctx["ctx"]
    n = 256
    cond = synth.rect_conditions(n, 41)
    z = synth.gaussian_noise(n, 42)
    with pytest.raises(g.GMCError) as e:
        _run(ctx, cond, z, 4, g.GMC_EULER, g.GMC_FP8)
    assert e.value.status == g.GMC_EINVAL
    cfg = g.gmc_get_config(ctx)
    cfg.sampler_kernel = g.GMC_KERNEL_PAIR
    g.gmc_set_config(ctx, cfg)
    try:
        with pytest.raises(g.GMCError) as e:
            _run(ctx, cond, z, 4, g.GMC_EULER, g.GMC_BF16)
        assert e.value.status == g.GMC_EINVAL
    finally:
        cfg.sampler_kernel = g.GMC_KERNEL_TILE
        g.gmc_set_config(ctx, cfg)
    tau, c, src = synth.grid_problem(n=8, seed=3, block=4, source=2)
    f = np.zeros(64)
    with pytest.raises(g.GMCError) as e:
        g.transport_solve(ctx, 8, 8, *(np.ascontiguousarray(a, np.float32).ravel()
                                       for a in (tau, c, src)), 100, g.GMC_METHOD_GMC, 1, f)
    assert e.value.status == g.GMC_EINVAL
    dc = torch.from_numpy(cond[:5].copy()).cuda()
    y = torch.empty(4, n, device="cuda")
    with pytest.raises(g.GMCError) as e:
        g.gmc_transmit_noalloc(ctx, n, dc, None, 1, 0, 4, g.GMC_EULER, y, None)
    assert e.value.status == g.GMC_EINVAL


def _split(flat):
    o = 0
    W, b = [], []
    for r, cdim in [(256, 32), (256, 256), (256, 256), (256, 256), (4, 256)]:
        W.append(flat[o:o + r * cdim].reshape(r, cdim).astype(np.float64))
        o += r * cdim
        b.append(flat[o:o + r].astype(np.float64))
        o += r
    W[0] = W[0][:, :26]
    return W, b


@pytest.fixture(scope="module")
def rtrain(rctx):
    import paper_2512_13965_gb300 as g
    ctx = rctx["ctx"]
    g.gmc_load_weights(ctx, rctx["path"])
    n = 1 << 18
    cond = torch.empty(6, n, device="cuda")
    y = torch.empty(4, n, device="cuda")
    g.gmc_train_data_rect(ctx, n, 7, 0.1, 1000.0, 0.25, 4.0, 0.5, 0.999, cond, y)
    cfg = g.gmc_train_config(batch=4096, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                             weight_decay=0.01, seed=13, precision=g.GMC_FP32)
    g.gmc_train_begin(ctx, n, cond, y, cfg)
    return {"cond": cond, "y": y, "n": n, "cfg": cfg}


def test_rect_bf16_training_is_refused(rctx, rtrain):
    import paper_2512_13965_gb300 as g
    bad = g.gmc_train_config(batch=4096, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                             weight_decay=0.01, seed=13, precision=g.GMC_BF16)
    with pytest.raises(g.GMCError) as e:
        g.gmc_train_begin(rctx["ctx"], rtrain["n"], rtrain["cond"], rtrain["y"], bad)
    assert e.value.status == g.GMC_EINVAL


def test_rect_gradient_matches_oracle(rctx, rtrain):
    import paper_2512_13965_gb300 as g
    ctx = rctx["ctx"]
    g.gmc_train_begin(ctx, rtrain["n"], rtrain["cond"], rtrain["y"], rtrain["cfg"])
    B = 80
    rng = np.random.default_rng(6)
    cn = rng.standard_normal((B, 6)).astype(np.float32)
    x1 = rng.standard_normal((B, 4)).astype(np.float32)
    x0 = rng.standard_normal((B, 4)).astype(np.float32)
    t = rng.random(B).astype(np.float32)
    P = g.gmc_train_param_count_ctx(ctx)
    grad = np.zeros(P, np.float32)
    loss = g.gmc_train_grad(ctx, B, cn, x1, x0, t, grad, n_cond=6)
    params = np.zeros(P, np.float32)
    g.gmc_train_params(ctx, params)
    W, b = _split(params)
    ref_loss, gW, gb = oracle.train.cfm_loss_grad(W, b, cn.astype(np.float64), x1.astype(np.float64),
                                                  x0.astype(np.float64), t.astype(np.float64))
    assert abs(loss - ref_loss) < 1e-4 * max(1.0, abs(ref_loss))
    GW, Gb = _split(grad)
    for l in range(5):
        assert np.abs(GW[l] - gW[l]).max() < 1e-4 * max(np.abs(gW[l]).max(), 1e-12), ("W", l)
        assert np.abs(Gb[l] - gb[l]).max() < 1e-4 * max(np.abs(gb[l]).max(), 1e-12), ("b", l)
    assert np.abs(GW[0][:, 25]).max() > 0  # the aspect column learns
    assert np.all(grad[:256 * 32].reshape(256, 32)[:, 26:] == 0)


def test_rect_training_lowers_loss_commits_and_resumes(rctx, rtrain, tmp_path):
    import paper_2512_13965_gb300 as g
    ctx = rctx["ctx"]
    g.gmc_load_weights(ctx, rctx["path"])
    n, cond, y, cfg = rtrain["n"], rtrain["cond"], rtrain["y"], rtrain["cfg"]
    g.gmc_train_begin(ctx, n, cond, y, cfg)
    losses = np.zeros(300, np.float32)
    g.gmc_train_steps(ctx, 300, losses)
    assert np.all(np.isfinite(losses)) and losses[-50:].mean() < 0.8 * losses[:10].mean()
    blob = g.gmc_train_save_state(ctx)
    a = np.zeros(g.gmc_train_param_count_ctx(ctx), np.float32)
    g.gmc_train_steps(ctx, 5)
    g.gmc_train_params(ctx, a)
    out = str(tmp_path / "rect_trained.bin")
    g.gmc_train_commit(ctx, out)
    net = oracle.mlp.read_weights(out)
    assert net.W[0].shape == (256, 26) and net.cond_mean.shape == (6,)
    np.testing.assert_array_equal(net.W[0], _split(a)[0][0])
    # the committed network samples as the oracle says
    m = 300
    c6 = synth.rect_conditions(m, 51)
    z = synth.gaussian_noise(m, 52)
    assert np.abs(_run(ctx, c6, z, 4, g.GMC_EULER, g.GMC_FP32)
                  - oracle.mlp.sample(net, c6, z, 4, "euler")).max() < FP32_TOL
    # the checkpoint continues the run (5 more steps from the saved state)
    g.gmc_load_weights(ctx, rctx["path"])
    g.gmc_train_begin(ctx, n, cond, y, cfg)
    g.gmc_train_load_state(ctx, blob)
    g.gmc_train_steps(ctx, 5)
    b = np.zeros_like(a)
    g.gmc_train_params(ctx, b)
    assert np.abs(b - a).max() <= 1e-6 * max(1.0, np.abs(a).max())


# ---- rectangular cells in the solve (transport_solve_rect) -----------------

def _solve_rect(ctx, sig, c, src, dx, dy, n, method, seed):
    import paper_2512_13965_gb300 as g
    ny, nx = sig.shape
    f = np.zeros(ny * nx)
    st = g.transport_solve_rect(ctx, nx, ny, *(np.ascontiguousarray(a, np.float32).ravel()
                                               for a in (sig, c, src)), dx, dy, n, method, seed, f)
    return f.reshape(ny, nx), st.as_dict()


def test_rect_solve_on_square_cells_is_the_square_solve(rctx):
    # dx = dy = 1: the walk of the rectangle with equal sides, flux divided by
    # 1: the random-walk solve equals transport_solve on tau = sigma
    import paper_2512_13965_gb300 as g
    ctx = rctx["ctx"]
    tau, c, src = synth.grid_problem(n=16, seed=61, tau_range=(0.1, 5.0), block=4, source=4)
    a, sa = _solve_rect(ctx, tau, c, src, 1.0, 1.0, 20000, g.GMC_METHOD_ANALOG, 5)
    f = np.zeros(256)
    sb = g.transport_solve(ctx, 16, 16, *(np.ascontiguousarray(x, np.float32).ravel()
                                           for x in (tau, c, src)), 20000, g.GMC_METHOD_ANALOG, 5, f)
    # the same histories; FP64 atomic tallies add in any order
    np.testing.assert_allclose(a.ravel(), f, rtol=1e-9, atol=1e-12 * np.abs(f).max())
    assert sa["transmissions"] == sb.transmissions


def _percell_rect(ctx, sig, c, src, dx, dy, method, sampler, K=8, n_gpu=20000, n_oracle=4000):
    import _oracle_pool as P
    gpu = [_solve_rect(ctx, sig, c, src, dx, dy, n_gpu, method, 1000 + k)[0] for k in range(K)]
    tasks = [{"grid": (sig, c, src), "n": n_oracle, "seed": 2000 + k, "sampler": sampler,
              "internal": None, "wall": None, "cell": (dx, dy)} for k in range(K)]
    orc = P.solve_many(tasks)
    P.assert_per_cell(gpu, [f for f, _ in orc])


def test_rect_analog_solve_per_cell(rctx):
    import paper_2512_13965_gb300 as g
    sig, c, src = synth.grid_problem(n=16, seed=63, tau_range=(0.2, 8.0), block=4, source=4)
    _percell_rect(rctx["ctx"], sig, c, src, 0.5, 1.5, g.GMC_METHOD_ANALOG, ("walk_global_rect",))


def test_rect_gmc_solve_per_cell(rctx):
    # GMC with the rectangular-cell test network, FP32, against the oracle's
    # event loop with the same network (canonical sides per entry face)
    # (the Kaiming rectangular-cell network: zero biases and identity
    # standardization keep the track lengths free of a heavy tail, so the
    # per-cell spread is estimable from 8 runs)
    import paper_2512_13965_gb300 as g
    ctx = rctx["ctx"]
    path = str(rctx["dir"] / "rect_kaiming.bin")
    synth.write_weights(path, synth.kaiming_weights_rect(1))
    g.gmc_load_weights(ctx, path)
    cfg = g.gmc_get_config(ctx)
    cfg.precision, cfg.steps, cfg.integrator, cfg.gmc_min_tau = g.GMC_FP32, 4, g.GMC_EULER, 0.0
    cfg.bank_capacity = 1 << 16
    g.gmc_set_config(ctx, cfg)
    # sigma dx and sigma dy inside the networks' box [0.1, 1000], c in [0.5, 0.999]
    sig, c, src = synth.grid_problem(n=16, seed=65, tau_range=(0.4, 8.0), block=4, source=4)
    _percell_rect(ctx, sig, c, src, 0.5, 1.5, g.GMC_METHOD_GMC, ("mlp_rect", path, 4, "euler"))


def test_rect_solve_needs_a_rect_network():
    import os
    import paper_2512_13965_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, os.path.join(root, "paper_2512_13965_gb300", "weights", "gmc_boundary.bin"))
        sig, c, src = synth.grid_problem(n=8, seed=3, block=4, source=2)
        with pytest.raises(g.GMCError) as e:
            _solve_rect(ctx, sig, c, src, 0.5, 1.5, 100, g.GMC_METHOD_GMC, 1)
        assert e.value.status == g.GMC_EINVAL
        # sizes the walk cannot hold in FP32: refused on the host, any method
        for dx, dy, s in ((0.0, 1.0, 1.0), (1.0, float("inf"), 1.0), (1e-30, 1e10, 1.0),
                          (1.0, 1e30, 1e10)):
            with pytest.raises(g.GMCError) as e:
                _solve_rect(ctx, sig * s, c, src, dx, dy, 100, g.GMC_METHOD_ANALOG, 1)
            assert e.value.status == g.GMC_EINVAL, (dx, dy, s)
    finally:
        ctx.close()
