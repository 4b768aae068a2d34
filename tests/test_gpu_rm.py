"""The residual-modulated velocity network (weight-file flag 1; the reading of
the paper's residual blocks with adaptive modulation, section "Network
Architecture and Inputs") on the GPU against the FP64 oracle.

Sampler (Eq. 8): the FP32 path within 1e-4 absolute per output, the BF16
tensor-core tile kernel within the BF16 sampler's bounds (max 0.1, p99.9
0.06 on standardized outputs), at sizes spanning several 128-row tiles with a
ragged tail, for Euler, midpoint and RK4, with non-zero condition shifts and
channel scales and a non-identity standardization. Training (Eq. 9): the FP32
gradient of every tensor, M and G included, within 1e-4 of the oracle's
relative to the tensor's largest entry; a short run lowers the loss; the
committed file carries flag 1 and reads back in the oracle; a checkpoint
continues the run (bit for bit when two uninterrupted runs agree bit for
bit, else within their spread), and an MLP checkpoint is refused. Paths the
network does not have (FP8, the CTA-pair kernel, BF16 training) are refused
with GMC_EINVAL.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
BF16_MAX, BF16_P999 = 0.1, 0.06


def _rm_net(seed=21):
    # biased Kaiming layers with the residual blocks' weights scaled by 0.35:
    # three blocks add to the stream instead of replacing it, and at full
    # Kaiming scale it grows until the outputs reach hundreds; at 0.35 they
    # stay at the plain test network's scale (|y| up to about 6)
    base = synth.biased_weights(seed)
    base["W"] = [w * np.float32(0.35) if l in (1, 2, 3) else w for l, w in enumerate(base["W"])]
    return synth.rm_weights(seed, m_std=0.2, g_std=0.2, base=base)


@pytest.fixture(scope="module")
def rm(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_13965_gb300 as g
    path = str(tmp_path_factory.mktemp("rm") / "rm.bin")
    synth.write_weights(path, _rm_net())
    ctx = g.Context(0)
    g.gmc_load_weights(ctx, path)
    yield {"ctx": ctx, "path": path, "net": oracle.mlp.read_weights(path)}
    ctx.close()


def _run(ctx, cond, noise, steps, integ, prec):
    import paper_2512_13965_gb300 as g
    n = cond.shape[1]
    dc = torch.from_numpy(cond).cuda()
    dz = torch.from_numpy(noise).cuda()
    y = torch.full((4, n), float("nan"), device="cuda")
    g.gmc_transmit(ctx, n, dc, dz, 0, 0, steps, integ, prec, y, None)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


INTEGS = [("euler", 8), ("midpoint", 4), ("rk4", 3)]


@pytest.mark.parametrize("integ,steps", INTEGS)
def test_rm_fp32_sampler_matches_oracle(rm, integ, steps):
    import paper_2512_13965_gb300 as g
    n = 1000
    cond, _, _ = synth.sampler_conditions(n, 31 + steps)
    z = synth.gaussian_noise(n, 32 + steps)
    code = {"euler": g.GMC_EULER, "midpoint": g.GMC_MIDPOINT, "rk4": g.GMC_RK4}[integ]
    y = _run(rm["ctx"], cond, z, steps, code, g.GMC_FP32)
    expect = oracle.mlp.sample(rm["net"], cond, z, steps, integ)
    assert np.abs(y - expect).max() < FP32_TOL


@pytest.mark.parametrize("integ,steps", INTEGS)
def test_rm_bf16_sampler_matches_oracle(rm, integ, steps):
    import paper_2512_13965_gb300 as g
    n = 3 * 256 + 77  # three tile pairs and a ragged tail
    cond, _, _ = synth.sampler_conditions(n, 41 + steps)
    z = synth.gaussian_noise(n, 42 + steps)
    code = {"euler": g.GMC_EULER, "midpoint": g.GMC_MIDPOINT, "rk4": g.GMC_RK4}[integ]
    y = _run(rm["ctx"], cond, z, steps, code, g.GMC_BF16)
    expect = oracle.mlp.sample(rm["net"], cond, z, steps, integ)
    err = np.abs(y - expect)
    assert np.all(np.isfinite(y))
    assert err.max() < BF16_MAX and np.quantile(err, 0.999) < BF16_P999, (err.max(),
                                                                         np.quantile(err, 0.999))


def test_rm_bf16_large_batch_sampled_rows(rm):
    # 2^17 rows (many tile pairs per CTA): rows sampled across the batch
    import paper_2512_13965_gb300 as g
    n = 1 << 17
    cond, _, _ = synth.sampler_conditions(n, 51)
    z = synth.gaussian_noise(n, 52)
    y = _run(rm["ctx"], cond, z, 8, g.GMC_EULER, g.GMC_BF16)
    idx = np.random.default_rng(5).choice(n, 2048, replace=False)
    expect = oracle.mlp.sample(rm["net"], cond[:, idx], z[:, idx], 8, "euler")
    err = np.abs(y[:, idx] - expect)
    assert err.max() < BF16_MAX and np.quantile(err, 0.999) < BF16_P999


def test_rm_refuses_paths_it_does_not_have(rm):
    import paper_2512_13965_gb300 as g
    ctx = rm["ctx"]
    n = 256
    cond, _, _ = synth.sampler_conditions(n, 61)
    z = synth.gaussian_noise(n, 62)
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
    # a GMC solve at FP8 is refused at admission
    cfg.precision = g.GMC_FP8
    g.gmc_set_config(ctx, cfg)
    try:
        tau, c, src = synth.grid_problem(n=8, seed=3, block=4, source=2)
        f = np.zeros(64)
        with pytest.raises(g.GMCError) as e:
            g.transport_solve(ctx, 8, 8, *(np.ascontiguousarray(a, np.float32).ravel()
                                           for a in (tau, c, src)), 100, g.GMC_METHOD_GMC, 1, f)
        assert e.value.status == g.GMC_EINVAL
    finally:
        cfg.precision = g.GMC_BF16
        g.gmc_set_config(ctx, cfg)


def _data(ctx, n, seed):
    import paper_2512_13965_gb300 as g
    cond = torch.empty(5, n, device="cuda")
    y = torch.empty(4, n, device="cuda")
    g.gmc_train_data(ctx, n, seed, 0.1, 1000.0, 0.5, 0.999, cond, y)
    torch.cuda.synchronize()
    return cond, y


def _split(flat):
    # MLP block (W1 [256][32], b1, ..., W5, b5), then M [3][256][5], G [3][2][256]
    o = 0
    W, b = [], []
    for r, cdim in [(256, 32), (256, 256), (256, 256), (256, 256), (4, 256)]:
        W.append(flat[o:o + r * cdim].reshape(r, cdim).astype(np.float64))
        o += r * cdim
        b.append(flat[o:o + r].astype(np.float64))
        o += r
    W[0] = W[0][:, :25]
    M = [flat[o + j * 1280:o + (j + 1) * 1280].reshape(256, 5).astype(np.float64) for j in range(3)]
    o += 3 * 1280
    G = [flat[o + j * 512:o + (j + 1) * 512].reshape(2, 256).astype(np.float64) for j in range(3)]
    o += 3 * 512
    assert o == flat.size
    return {"W": W, "b": b, "M": M, "G": G}


@pytest.fixture(scope="module")
def rm_trainer(rm):
    import paper_2512_13965_gb300 as g
    ctx = rm["ctx"]
    n = 1 << 18
    cond, y = _data(ctx, n, 9)
    cfg = g.gmc_train_config(batch=4096, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                             weight_decay=0.01, seed=13, precision=g.GMC_FP32)
    g.gmc_train_begin(ctx, n, cond, y, cfg)
    return {"cond": cond, "y": y, "n": n, "cfg": cfg}


def test_rm_bf16_training_is_refused(rm, rm_trainer):
    import paper_2512_13965_gb300 as g
    cfg = g.gmc_train_config(batch=4096, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                             weight_decay=0.01, seed=13, precision=g.GMC_BF16)
    with pytest.raises(g.GMCError) as e:
        g.gmc_train_begin(rm["ctx"], rm_trainer["n"], rm_trainer["cond"], rm_trainer["y"], cfg)
    assert e.value.status == g.GMC_EINVAL
    # the refusal came before the FP32 state was touched; begin anew for the
    # tests that follow all the same
    g.gmc_train_begin(rm["ctx"], rm_trainer["n"], rm_trainer["cond"], rm_trainer["y"],
                      rm_trainer["cfg"])


def test_rm_gradient_matches_oracle(rm, rm_trainer):
    import paper_2512_13965_gb300 as g
    ctx = rm["ctx"]
    assert g.gmc_train_param_count_ctx(ctx) == g.gmc_train_param_count() + 5376
    B = 96
    rng = np.random.default_rng(4)
    cn = rng.standard_normal((B, 5)).astype(np.float32)
    x1 = rng.standard_normal((B, 4)).astype(np.float32)
    x0 = rng.standard_normal((B, 4)).astype(np.float32)
    t = rng.random(B).astype(np.float32)
    P = g.gmc_train_param_count_ctx(ctx)
    grad = np.zeros(P, np.float32)
    loss = g.gmc_train_grad(ctx, B, cn, x1, x0, t, grad)
    params = np.zeros(P, np.float32)
    g.gmc_train_params(ctx, params)
    ref_loss, G = oracle.train.cfm_loss_grad_rm(_split(params), cn.astype(np.float64),
                                                x1.astype(np.float64), x0.astype(np.float64),
                                                t.astype(np.float64))
    assert abs(loss - ref_loss) < 1e-4 * max(1.0, abs(ref_loss))
    got = _split(grad)
    for key in ("W", "b", "M", "G"):
        for l, (a, r) in enumerate(zip(got[key], G[key])):
            if key == "W" and l == 0:
                r = r[:, :25]
            scale = max(np.abs(r).max(), 1e-12)
            assert np.abs(a - r).max() < 1e-4 * scale, (key, l, np.abs(a - r).max(), scale)
    assert np.all(grad[:256 * 32].reshape(256, 32)[:, 25:] == 0)


def test_rm_training_lowers_loss_and_commits(rm, rm_trainer, tmp_path):
    import paper_2512_13965_gb300 as g
    ctx = rm["ctx"]
    g.gmc_train_begin(ctx, rm_trainer["n"], rm_trainer["cond"], rm_trainer["y"], rm_trainer["cfg"])
    losses = np.zeros(300, np.float32)
    g.gmc_train_steps(ctx, 300, losses)
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.8 * losses[:10].mean()
    out = str(tmp_path / "rm_trained.bin")
    g.gmc_train_commit(ctx, out)
    net = oracle.mlp.read_weights(out)
    assert net.rm
    P = g.gmc_train_param_count_ctx(ctx)
    params = np.zeros(P, np.float32)
    g.gmc_train_params(ctx, params)
    ref = _split(params)
    for j in range(3):
        np.testing.assert_array_equal(net.M[j], ref["M"][j])
        np.testing.assert_array_equal(net.G[j], ref["G"][j])
    # the committed network is the sampler's: FP32 sampling matches the oracle
    n = 300
    cond, _, _ = synth.sampler_conditions(n, 71)
    z = synth.gaussian_noise(n, 72)
    y = _run(ctx, cond, z, 4, g.GMC_EULER, g.GMC_FP32)
    assert np.abs(y - oracle.mlp.sample(net, cond, z, 4, "euler")).max() < FP32_TOL
    g.gmc_load_weights(ctx, rm["path"])  # back to the module's network


def test_rm_checkpoint_resumes_the_run(rm, rm_trainer, kaiming_file):
    import paper_2512_13965_gb300 as g
    ctx = rm["ctx"]
    g.gmc_load_weights(ctx, rm["path"])
    n, cond, y, cfg = rm_trainer["n"], rm_trainer["cond"], rm_trainer["y"], rm_trainer["cfg"]
    P = g.gmc_train_param_count_ctx(ctx)

    def run(k1, k2, resume):
        g.gmc_train_begin(ctx, n, cond, y, cfg)
        g.gmc_train_steps(ctx, k1)
        if resume:
            blob = g.gmc_train_save_state(ctx)
            g.gmc_train_begin(ctx, n, cond, y, cfg)
            g.gmc_train_load_state(ctx, blob)
        g.gmc_train_steps(ctx, k2)
        p = np.zeros(P, np.float32)
        g.gmc_train_params(ctx, p)
        return p

    a = run(5, 7, False)
    a2 = run(5, 7, False)
    b = run(5, 7, True)
    spread = float(np.abs(a - a2).max())
    if spread == 0.0:
        assert np.array_equal(a, b)
    else:
        assert np.abs(b - a).max() <= 10.0 * spread
    # an MLP checkpoint does not restore into the residual-modulated state
    g.gmc_load_weights(ctx, kaiming_file)
    g.gmc_train_begin(ctx, n, cond, y, cfg)
    mlp_blob = g.gmc_train_save_state(ctx)
    g.gmc_load_weights(ctx, rm["path"])
    g.gmc_train_begin(ctx, n, cond, y, cfg)
    with pytest.raises(g.GMCError) as e:
        g.gmc_train_load_state(ctx, mlp_blob)
    assert e.value.status == g.GMC_EFORMAT


def test_rm_gmc_solve_bf16_per_cell(rm):
    # a GMC solve with the residual-modulated network (BF16 tile kernel)
    # against the oracle's event loop driven by the same network: 8 seeds per
    # side, |z| <= 4 in 99 % of the cells and <= 6 in all
    import _oracle_pool as P
    import paper_2512_13965_gb300 as g
    ctx = rm["ctx"]
    g.gmc_load_weights(ctx, rm["path"])
    cfg = g.gmc_get_config(ctx)
    cfg.precision, cfg.steps, cfg.integrator, cfg.gmc_min_tau = g.GMC_BF16, 4, g.GMC_EULER, 0.0
    cfg.bank_capacity = 1 << 16
    g.gmc_set_config(ctx, cfg)
    tau, c, src = synth.grid_problem(n=16, seed=35, tau_range=(0.1, 20.0), block=4, source=4)
    args = [np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c, src)]
    gpu = []
    for k in range(8):
        f = np.zeros(256)
        g.transport_solve(ctx, 16, 16, *args, 20000, g.GMC_METHOD_GMC, 1000 + k, f)
        gpu.append(f)
    tasks = [{"grid": (tau, c, src), "n": 4000, "seed": 2000 + k, "sampler": ("mlp", rm["path"], 4, "euler"),
              "internal": None, "wall": None} for k in range(8)]
    orc = P.solve_many(tasks)
    P.assert_per_cell(gpu, [f for f, _ in orc])


def test_committed_rm_network_flux_within_bound():
    # the committed residual-modulated boundary network (with the committed
    # internal model) against the GPU walk on a 32 x 32 grid of the solve
    # benchmark's materials, 8e6 histories: within its stated 2 % (1.40 %
    # measured on the 128 x 128 solve at 1e7 histories, floor 0.26 %)
    import os
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2512_13965_gb300 as g
    w = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                     "paper_2512_13965_gb300", "weights")
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, os.path.join(w, "gmc_boundary_rm.bin"))
        g.gmc_load_internal_weights(ctx, os.path.join(w, "gmc_internal.bin"))
        tau, c, src = synth.grid_problem(n=32, seed=5, tau_range=(0.1, 500.0), block=8, source=4)
        args = [np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c, src)]

        def solve(method, seed, n):
            cfg = g.gmc_get_config(ctx)
            cfg.precision, cfg.integrator, cfg.steps, cfg.gmc_min_tau = g.GMC_BF16, g.GMC_MIDPOINT, 8, 0.0
            g.gmc_set_config(ctx, cfg)
            f = np.zeros(1024)
            g.transport_solve(ctx, 32, 32, *args, n, method, seed, f)
            return f

        fa = solve(g.GMC_METHOD_ANALOG, 1, 4_000_000)
        fb = solve(g.GMC_METHOD_ANALOG, 2, 4_000_000)
        f_mc = 0.5 * (fa + fb)
        floor = np.linalg.norm(fa - fb) / np.linalg.norm(f_mc) / np.sqrt(2.0)
        f = solve(g.GMC_METHOD_GMC, 3, 8_000_000)
        err = np.linalg.norm(f - f_mc) / np.linalg.norm(f_mc)
        assert floor < 0.005 and err < 0.02, (err, floor)
    finally:
        ctx.close()
