"""Training on the GPU (gmc_train_*): data from the GPU random walk, the CFM
gradient against the FP64 oracle, AdamW, and the gain of training.
"""
import math

import numpy as np
import pytest
import torch
from scipy import stats as sstats

import oracle
import synth

pytestmark = pytest.mark.gpu


def _u01_f32(x):
    # the device's float uniform: fma((float)x, 2^-32, 2^-32)
    return (x.astype(np.float32) * np.float32(2.0 ** -32) + np.float32(2.0 ** -32)).astype(np.float32)


def _data(ctx, n, seed, tau=(0.1, 1000.0), c=(0.5, 0.999)):
    import paper_2512_13965_gb300 as g
    cond = torch.empty(5, n, device="cuda")
    y = torch.empty(4, n, device="cuda")
    g.gmc_train_data(ctx, n, seed, tau[0], tau[1], c[0], c[1], cond, y)
    torch.cuda.synchronize()
    return cond, y


def test_training_data_inputs_follow_philox(gpu_ctx):
    n, seed = 4096, 17
    cond, _ = _data(gpu_ctx, n, seed)
    c = cond.cpu().numpy()
    raw = oracle.rng.philox_batch(seed, n, id0=0, event=0, tag=5)
    lo, hi = np.log(np.float32(0.1)), np.log(np.float32(1000.0))
    ltau = lo + (hi - lo) * _u01_f32(raw[:, 0])
    np.testing.assert_allclose(c[3], ltau, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(c[4], 0.5 + (0.999 - 0.5) * _u01_f32(raw[:, 1]), rtol=1e-6)
    np.testing.assert_allclose(c[0], _u01_f32(raw[:, 2]), rtol=1e-7)
    sn = 2 * _u01_f32(raw[:, 3]) - 1
    np.testing.assert_allclose(c[2], sn, atol=1e-7)
    np.testing.assert_allclose(c[1] ** 2 + c[2] ** 2, 1.0, atol=1e-6)


def test_training_targets_match_oracle_walk(gpu_ctx):
    # same entries and the same Philox counters (id i, flights from event 1)
    # as the oracle's implicit-capture walk: per-sample agreement
    n, seed = 20000, 23
    cond, y = _data(gpu_ctx, n, seed, tau=(0.3, 30.0))
    c = cond.cpu().numpy().astype(np.float64)
    yg = y.cpu().numpy().astype(np.float64)
    tau = np.exp(c[3])
    r = oracle.transport.transmit(c[0], c[1], c[2], tau, c[4], 1, seed,
                                  ids=np.arange(n, dtype=np.uint64),
                                  events=np.ones(n, dtype=np.uint32))
    p_ref = r["face"] + r["q"]
    same = (np.floor(yg[0]) == r["face"]) & (np.abs(yg[3] - np.log(r["s"])) < 1e-3)
    assert same.mean() > 0.99
    assert np.abs(yg[0] - p_ref)[same].max() < 1e-3
    # the distribution as a whole (all samples, flips included)
    for k, ref in ((0, p_ref), (3, np.log(r["s"]))):
        assert sstats.ks_2samp(yg[k], ref).pvalue > 1e-3


@pytest.fixture(scope="module")
def trainer(gpu_ctx, kaiming_file):
    import paper_2512_13965_gb300 as g
    g.gmc_load_weights(gpu_ctx, kaiming_file)
    n = 1 << 20
    cond, y = _data(gpu_ctx, n, 5)
    cfg = g.gmc_train_config(batch=8192, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                             weight_decay=0.01, seed=11)
    g.gmc_train_begin(gpu_ctx, n, cond, y, cfg)
    return {"cond": cond, "y": y, "n": n, "cfg": cfg}


def _oracle_params(flat):
    # W1 [256][32] (25 real columns), b1, W2, b2, W3, b3, W4, b4, W5, b5
    o = 0
    W, b = [], []
    shapes = [(256, 32), (256, 256), (256, 256), (256, 256), (4, 256)]
    for l, (r, cdim) in enumerate(shapes):
        W.append(flat[o:o + r * cdim].reshape(r, cdim).astype(np.float64))
        o += r * cdim
        b.append(flat[o:o + r].astype(np.float64))
        o += r
    W[0] = W[0][:, :25]
    return W, b


def test_gradient_matches_oracle(gpu_ctx, trainer):
    import paper_2512_13965_gb300 as g
    B = 64
    rng = np.random.default_rng(3)
    cn = rng.standard_normal((B, 5)).astype(np.float32)
    x1 = rng.standard_normal((B, 4)).astype(np.float32)
    x0 = rng.standard_normal((B, 4)).astype(np.float32)
    t = rng.random(B).astype(np.float32)
    P = g.gmc_train_param_count()
    grad = np.zeros(P, np.float32)
    loss = g.gmc_train_grad(gpu_ctx, B, cn, x1, x0, t, grad)
    params = np.zeros(P, np.float32)
    g.gmc_train_params(gpu_ctx, params)
    W, b = _oracle_params(params)
    ref_loss, gW, gb = oracle.train.cfm_loss_grad(W, b, cn.astype(np.float64), x1.astype(np.float64),
                                                  x0.astype(np.float64), t.astype(np.float64))
    assert abs(loss - ref_loss) < 1e-4 * max(1.0, abs(ref_loss))
    GW, Gb = _oracle_params(grad)
    for l in range(5):
        scale = max(np.abs(gW[l]).max(), 1e-12)
        assert np.abs(GW[l] - gW[l]).max() < 1e-4 * scale, ("W", l)
        bs = max(np.abs(gb[l]).max(), 1e-12)
        assert np.abs(Gb[l] - gb[l]).max() < 1e-4 * bs, ("b", l)
    # padding columns of W1 get no gradient
    assert np.all(grad[:256 * 32].reshape(256, 32)[:, 25:] == 0)


def test_adamw_first_step(gpu_ctx, trainer):
    # At step 1 Adam's bias-corrected ratio is g / (|g| + eps), so every
    # parameter with |g| >> eps moves by -lr sign(g) - lr wd p (decoupled decay).
    import paper_2512_13965_gb300 as g
    cfg = trainer["cfg"]
    g.gmc_train_begin(gpu_ctx, trainer["n"], trainer["cond"], trainer["y"], cfg)
    P = g.gmc_train_param_count()
    p0 = np.zeros(P, np.float32)
    g.gmc_train_params(gpu_ctx, p0)
    g.gmc_train_steps(gpu_ctx, 1)
    p1 = np.zeros(P, np.float32)
    g.gmc_train_params(gpu_ctx, p1)
    step = (p1.astype(np.float64) - p0) + cfg.lr * cfg.weight_decay * p0
    # |step| = lr |g| / (|g| + eps) <= lr, equal to lr wherever |g| >> eps
    assert np.all(np.abs(step) <= cfg.lr * (1 + 2e-3))
    moved = np.abs(step) > 0.5 * cfg.lr
    assert moved.mean() > 0.95
    close = np.abs(np.abs(step[moved]) / cfg.lr - 1) < 2e-3
    assert close.mean() > 0.999


def test_training_gain(gpu_ctx, trainer, tmp_path):
    # Train on GPU walk data and compare the exit distributions of the
    # untrained and the trained network with the analog walk at held-out
    # conditions (1-D Wasserstein distance per output).
    import paper_2512_13965_gb300 as g
    g.gmc_train_begin(gpu_ctx, trainer["n"], trainer["cond"], trainer["y"], trainer["cfg"])
    steps = 600
    losses = np.zeros(steps, np.float32)
    g.gmc_train_steps(gpu_ctx, steps, losses)
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.8 * losses[:20].mean()

    def exits(prec_net_loaded, tau, c, n=20000):
        e = synth.cell_entries(n, 77)
        cond = np.stack([e["xi"], e["cos"], e["sin"], np.full(n, np.log(tau), np.float32),
                         np.full(n, c, np.float32)]).astype(np.float32)
        ex = torch.empty(4, n, device="cuda")
        g.gmc_transmit(gpu_ctx, n, torch.from_numpy(cond).cuda(), None, 5, 0, 16, g.GMC_EULER,
                       g.GMC_BF16, None, ex)
        torch.cuda.synchronize()
        return ex.cpu().numpy().astype(np.float64), e

    pairs = [(0.5, 0.9), (3.0, 0.99), (30.0, 0.75)]
    before = {}
    for tau, c in pairs:
        before[(tau, c)] = exits(None, tau, c)[0]
    path = str(tmp_path / "trained.bin")
    g.gmc_train_commit(gpu_ctx, path)
    trained = oracle.mlp.read_weights(path)
    assert trained.y_std.min() > 0
    for tau, c in pairs:
        after, e = exits(None, tau, c)
        n = after.shape[1]
        r = oracle.transport.transmit(e["xi"].astype(np.float64), e["cos"].astype(np.float64),
                                      e["sin"].astype(np.float64), np.full(n, tau), np.full(n, c),
                                      1, 99)
        ref = [r["face"] + r["q"], r["ux"], r["uy"], np.log(r["s"])]
        for k in range(4):
            b = before[(tau, c)][k] if k != 3 else np.log(before[(tau, c)][3])
            a = after[k] if k != 3 else np.log(after[3])
            assert oracle.stats.w1(a, ref[k]) < oracle.stats.w1(b, ref[k]), (tau, c, k)


# BF16 tensor-core training step: the same gradient with BF16 MMA operands
# (FP32 accumulation, FP32 master weights). The bound is stated per layer
# relative to the layer's largest gradient entry, from the arithmetic: one
# BF16 rounding (2^-9 relative) of each operand, accumulated over K terms of
# mixed sign, then carried through four layers of backward.
BF16_GRAD_REL = 3e-2


def _begin_bf16(ctx, trainer):
    import paper_2512_13965_gb300 as g
    c = trainer["cfg"]
    cfg = g.gmc_train_config(batch=c.batch, lr=c.lr, beta1=c.beta1, beta2=c.beta2, eps=c.eps,
                             weight_decay=c.weight_decay, seed=c.seed, precision=g.GMC_BF16)
    g.gmc_train_begin(ctx, trainer["n"], trainer["cond"], trainer["y"], cfg)
    return cfg


@pytest.mark.parametrize("B", [64, 300, 2048])
def test_gradient_bf16_tensor_cores(gpu_ctx, trainer, B):
    import paper_2512_13965_gb300 as g
    _begin_bf16(gpu_ctx, trainer)
    rng = np.random.default_rng(B)
    cn = rng.standard_normal((B, 5)).astype(np.float32)
    x1 = rng.standard_normal((B, 4)).astype(np.float32)
    x0 = rng.standard_normal((B, 4)).astype(np.float32)
    t = rng.random(B).astype(np.float32)
    P = g.gmc_train_param_count()
    grad = np.zeros(P, np.float32)
    loss = g.gmc_train_grad(gpu_ctx, B, cn, x1, x0, t, grad)
    params = np.zeros(P, np.float32)
    g.gmc_train_params(gpu_ctx, params)
    W, b = _oracle_params(params)
    ref_loss, gW, gb = oracle.train.cfm_loss_grad(W, b, cn.astype(np.float64), x1.astype(np.float64),
                                                  x0.astype(np.float64), t.astype(np.float64))
    assert abs(loss - ref_loss) < 1e-2 * max(1.0, abs(ref_loss))
    GW, Gb = _oracle_params(grad)
    for l in range(5):
        scale = max(np.abs(gW[l]).max(), 1e-12)
        assert np.abs(GW[l] - gW[l]).max() < BF16_GRAD_REL * scale, ("W", l)
        bs = max(np.abs(gb[l]).max(), 1e-12)
        assert np.abs(Gb[l] - gb[l]).max() < BF16_GRAD_REL * bs, ("b", l)
        # and far from an unrelated gradient: the error is a small part
        assert np.linalg.norm(GW[l] - gW[l]) < 0.05 * np.linalg.norm(gW[l]), ("W norm", l)
    assert np.all(grad[:256 * 32].reshape(256, 32)[:, 25:] == 0)


def test_training_bf16_reduces_loss(gpu_ctx, trainer, kaiming_file):
    import paper_2512_13965_gb300 as g
    g.gmc_load_weights(gpu_ctx, kaiming_file)  # start untrained (earlier tests commit weights)
    _begin_bf16(gpu_ctx, trainer)
    steps = 400
    losses = np.zeros(steps, np.float32)
    g.gmc_train_steps(gpu_ctx, steps, losses)
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.8 * losses[:20].mean()


def test_bf16_first_step_matches_fp32(gpu_ctx, trainer):
    # One training step of each precision from the same weights on the same
    # batch: the FP32 step draws its rows in a batch kernel, the BF16 step
    # inside its forward kernel, both from the same Philox counters. At step 1
    # AdamW moves every parameter by -lr g / (|g| + eps) - lr wd p, i.e. by
    # -lr sign(g) wherever |g| >> eps, so the two steps move the weights alike
    # except where BF16 arithmetic flips the sign of a near-zero gradient.
    import paper_2512_13965_gb300 as g
    c = trainer["cfg"]
    P = g.gmc_train_param_count()
    res = {}
    for prec in (g.GMC_FP32, g.GMC_BF16):
        cfg = g.gmc_train_config(batch=c.batch, lr=c.lr, beta1=c.beta1, beta2=c.beta2, eps=c.eps,
                                 weight_decay=c.weight_decay, seed=c.seed, precision=prec)
        g.gmc_train_begin(gpu_ctx, trainer["n"], trainer["cond"], trainer["y"], cfg)
        p0 = np.zeros(P, np.float32)
        g.gmc_train_params(gpu_ctx, p0)
        loss = np.zeros(1, np.float32)
        g.gmc_train_steps(gpu_ctx, 1, loss)
        p1 = np.zeros(P, np.float32)
        g.gmc_train_params(gpu_ctx, p1)
        res[prec] = (p0, p1 - p0, float(loss[0]))
    (a0, da, la), (b0, db, lb) = res[g.GMC_FP32], res[g.GMC_BF16]
    assert np.array_equal(a0, b0)
    assert abs(la - lb) < 1e-2 * la, (la, lb)
    moved = np.abs(da) > 0.5 * c.lr
    same = np.abs(da - db) < 0.1 * c.lr
    assert moved.mean() > 0.9
    assert same[moved].mean() > 0.97, same[moved].mean()
