"""The CTA-pair BF16 sampler (GMC_KERNEL_PAIR: M = 256 tiles on two SMs,
tcgen05 cta_group::2, two accumulators per CTA) against the FP64 oracle on
identical weights and noise, with the BF16 bounds of the tile kernel (max
abs error 0.1, p99.9 0.06 on standardized outputs), at sizes that leave
ragged tiles (a 256-row tile split over the pair, pairs of tiles per
cluster, an odd tile count), for every integrator, on a network with nonzero
biases and standardization, with Philox noise drawn in the kernel, and at the
benchmark's full batch (sampled rows). The pair and tile kernels compute the
same BF16 arithmetic, so they also agree closely with each other."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

BF16_MAX, BF16_P999 = 0.1, 0.06


def _set_kernel(ctx, kernel):
    import paper_2512_13965_gb300 as g
    cfg = g.gmc_get_config(ctx)
    cfg.sampler_kernel = kernel
    g.gmc_set_config(ctx, cfg)


@pytest.fixture(scope="module")
def pctx(kaiming_file):
    import paper_2512_13965_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    ctx = g.Context(0)
    g.gmc_load_weights(ctx, kaiming_file)
    yield ctx
    ctx.close()


def _run(ctx, cond, noise, steps, integ, kernel, seed=0, id0=0, want_exit=False):
    import paper_2512_13965_gb300 as g
    _set_kernel(ctx, kernel)
    n = cond.shape[1]
    dc = torch.from_numpy(cond).cuda()
    dz = None if noise is None else torch.from_numpy(noise).cuda()
    y = torch.full((4, n), float("nan"), device="cuda")
    ex = torch.full((4, n), float("nan"), device="cuda") if want_exit else None
    g.gmc_transmit(ctx, n, dc, dz, seed, id0, steps, integ, g.GMC_BF16, y, ex)
    g.gmc_synchronize(ctx)
    return (y.cpu().numpy().astype(np.float64),
            None if ex is None else ex.cpu().numpy().astype(np.float64))


def _check(err):
    a = np.abs(err).ravel()
    assert np.isfinite(a).all()
    assert a.max() < BF16_MAX, a.max()
    assert np.quantile(a, 0.999) < BF16_P999, np.quantile(a, 0.999)


@pytest.mark.parametrize("n", [1, 255, 256, 257, 511, 512 + 13, 8192 + 77])
def test_pair_euler16_against_oracle(pctx, kaiming_file, n):
    import paper_2512_13965_gb300 as g
    net = oracle.mlp.read_weights(kaiming_file)
    cond, _, _ = synth.sampler_conditions(n, 300 + n)
    z = synth.gaussian_noise(n, 400 + n)
    y, _ = _run(pctx, cond, z, 16, g.GMC_EULER, g.GMC_KERNEL_PAIR)
    _check(y - oracle.mlp.sample(net, cond, z, 16, "euler"))


@pytest.mark.parametrize("integ,steps", [("midpoint", 8), ("rk4", 12), ("euler", 1)])
def test_pair_integrators_against_oracle(pctx, kaiming_file, integ, steps):
    import paper_2512_13965_gb300 as g
    net = oracle.mlp.read_weights(kaiming_file)
    n = 4096 + 300
    cond, _, _ = synth.sampler_conditions(n, 17)
    z = synth.gaussian_noise(n, 18)
    code = {"euler": g.GMC_EULER, "midpoint": g.GMC_MIDPOINT, "rk4": g.GMC_RK4}[integ]
    y, _ = _run(pctx, cond, z, steps, code, g.GMC_KERNEL_PAIR)
    _check(y - oracle.mlp.sample(net, cond, z, steps, integ))
    # the tile kernel on the same inputs: the same BF16 arithmetic
    yt, _ = _run(pctx, cond, z, steps, code, g.GMC_KERNEL_TILE)
    assert np.abs(y - yt).max() < 0.05


def test_pair_biased_network_and_decode(tmp_path):
    # nonzero biases in every layer and a random standardization: the bias
    # MMA of layers 2-4, the layer-1 bias of the epilogue, the decode
    import paper_2512_13965_gb300 as g
    p = str(tmp_path / "biased.bin")
    synth.write_weights(p, synth.biased_weights(7))
    net = oracle.mlp.read_weights(p)
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, p)
        n = 3000
        cond, _, _ = synth.sampler_conditions(n, 61)
        z = synth.gaussian_noise(n, 62)
        y, ex = _run(ctx, cond, z, 8, g.GMC_MIDPOINT, g.GMC_KERNEL_PAIR, want_exit=True)
    finally:
        ctx.close()
    ref = oracle.mlp.sample(net, cond, z, 8, "midpoint")
    _check(y - ref)
    # decoded exits of the kernel's own raw outputs: the oracle's decode rules
    d = oracle.mlp.decode(net, y)
    dp = np.abs(ex[0] - (d["face"] + d["q"]))
    assert np.minimum(dp, 4.0 - dp).max() < 1e-3
    assert np.all(np.abs(ex[3] / d["s"] - 1.0) < 1e-3)


def test_pair_philox_noise(pctx, kaiming_file):
    # noise drawn in the kernel equals the same Philox normals passed in
    import paper_2512_13965_gb300 as g
    n = 2000
    cond, _, _ = synth.sampler_conditions(n, 71)
    zt = torch.empty(4, n, device="cuda")
    g.gmc_normals(pctx, n, 9, 500, 0, 2, zt)
    torch.cuda.synchronize()
    y1, _ = _run(pctx, cond, zt.cpu().numpy(), 4, g.GMC_EULER, g.GMC_KERNEL_PAIR)
    y2, _ = _run(pctx, cond, None, 4, g.GMC_EULER, g.GMC_KERNEL_PAIR, seed=9, id0=500)
    np.testing.assert_array_equal(y1, y2)


def test_pair_full_batch_sampled(pctx, kaiming_file):
    # the benchmark's launch (2^20 rows, 16 Euler steps): sampled rows vs the
    # oracle, and the last rows of the last tile
    import paper_2512_13965_gb300 as g
    net = oracle.mlp.read_weights(kaiming_file)
    n = 1 << 20
    cond, _, _ = synth.sampler_conditions(n, 1)
    z = synth.gaussian_noise(n, 3)
    y, _ = _run(pctx, cond, z, 16, g.GMC_EULER, g.GMC_KERNEL_PAIR)
    idx = np.random.default_rng(1).choice(n, 2048, replace=False)
    idx = np.concatenate([idx, np.arange(n - 300, n)])
    _check(y[:, idx] - oracle.mlp.sample(net, cond[:, idx], z[:, idx], 16, "euler"))
    _set_kernel(pctx, g.GMC_KERNEL_TILE)
