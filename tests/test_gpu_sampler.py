"""GPU flow-ODE sampler (gmc_transmit) against the FP64 oracle on identical
weights and noise.

FP32 path: within 1e-4 absolute per output (the contract's FP32 bound).
BF16 path: max abs error 0.1 and p99.9 0.06 on standardized outputs, for
Kaiming random weights (measured on GB300 over 8192 rows: max 0.042-0.048,
p99.9 0.030-0.038 for Euler 16 and 8, midpoint 8 and RK4 12 -- BF16
operands with 8-bit significands, FP32 accumulation).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
BF16_MAX, BF16_P999 = 0.1, 0.06


@pytest.fixture(scope="module")
def net(gpu_ctx, kaiming_file):
    import paper_2512_13965_gb300 as g
    g.gmc_load_weights(gpu_ctx, kaiming_file)
    return oracle.mlp.read_weights(kaiming_file)


def _run(ctx, cond, noise, steps, integ, prec, want_exit=False, seed=0, id0=0):
    import paper_2512_13965_gb300 as g
    n = cond.shape[1]
    dc = torch.from_numpy(cond).cuda()
    dz = None if noise is None else torch.from_numpy(noise).cuda()
    y = torch.full((4, n), float("nan"), device="cuda")
    ex = torch.full((4, n), float("nan"), device="cuda") if want_exit else None
    g.gmc_transmit(ctx, n, dc, dz, seed, id0, steps, integ, prec, y, ex)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64), (None if ex is None else ex.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("n", [1, 63, 64, 65, 4096 + 37])
def test_fp32_euler16_parity(gpu_ctx, net, n):
    import paper_2512_13965_gb300 as g
    cond, _, _ = synth.sampler_conditions(n, 100 + n)
    z = synth.gaussian_noise(n, 200 + n)
    y, _ = _run(gpu_ctx, cond, z, 16, g.GMC_EULER, g.GMC_FP32)
    expect = oracle.mlp.sample(net, cond, z, 16, "euler")
    assert np.abs(y - expect).max() < FP32_TOL


@pytest.mark.parametrize("steps", [1, 3, 8])
def test_fp32_midpoint_parity(gpu_ctx, net, steps):
    import paper_2512_13965_gb300 as g
    n = 777
    cond, _, _ = synth.sampler_conditions(n, 5 + steps)
    z = synth.gaussian_noise(n, 6 + steps)
    y, _ = _run(gpu_ctx, cond, z, steps, g.GMC_MIDPOINT, g.GMC_FP32)
    expect = oracle.mlp.sample(net, cond, z, steps, "midpoint")
    assert np.abs(y - expect).max() < FP32_TOL


def test_fp32_decoded_exit(gpu_ctx, net):
    import paper_2512_13965_gb300 as g
    n = 2000
    cond, _, _ = synth.sampler_conditions(n, 31)
    z = synth.gaussian_noise(n, 32)
    y, ex = _run(gpu_ctx, cond, z, 16, g.GMC_EULER, g.GMC_FP32, want_exit=True)
    d = oracle.mlp.decode(net, oracle.mlp.sample(net, cond, z, 16, "euler"))
    p_ref = d["face"] + d["q"]
    dp = np.abs(ex[0] - p_ref)
    dp = np.minimum(dp, 4.0 - dp)          # the perimeter is periodic
    assert dp.max() < 1e-4
    same_face = np.floor(ex[0]).astype(int) == d["face"]
    assert same_face.mean() > 0.999
    ok = same_face
    assert np.abs(ex[1][ok] - d["ux"][ok]).max() < 1e-3
    assert np.abs(ex[2][ok] - d["uy"][ok]).max() < 1e-3
    assert np.all(np.abs(ex[3] / d["s"] - 1.0) < 1e-3)


def test_internal_noise_is_philox_normals(gpu_ctx, net):
    import paper_2512_13965_gb300 as g
    n = 3000
    cond, _, _ = synth.sampler_conditions(n, 41)
    zt = torch.empty(4, n, device="cuda")
    g.gmc_normals(gpu_ctx, n, 77, 1000, 0, 2, zt)
    torch.cuda.synchronize()
    y1, _ = _run(gpu_ctx, cond, zt.cpu().numpy(), 4, g.GMC_EULER, g.GMC_FP32)
    y2, _ = _run(gpu_ctx, cond, None, 4, g.GMC_EULER, g.GMC_FP32, seed=77, id0=1000)
    np.testing.assert_array_equal(y1, y2)


def test_fp32_full_size_sampled(gpu_ctx, net):
    # the benchmark's batch (2^20, 16 Euler steps): sampled rows vs the oracle
    import paper_2512_13965_gb300 as g
    n = 1 << 20
    cond, _, _ = synth.sampler_conditions(n, 1)
    z = synth.gaussian_noise(n, 3)
    y, _ = _run(gpu_ctx, cond, z, 16, g.GMC_EULER, g.GMC_FP32)
    idx = np.random.default_rng(0).choice(n, 512, replace=False)
    idx = np.concatenate([idx, [0, n - 1]])
    expect = oracle.mlp.sample(net, cond[:, idx], z[:, idx], 16, "euler")
    assert np.abs(y[:, idx] - expect).max() < FP32_TOL


def test_empty_and_errors(gpu_ctx, net):
    import paper_2512_13965_gb300 as g
    y = torch.empty(4, 1, device="cuda")
    c = torch.zeros(5, 1, device="cuda")
    g.gmc_transmit(gpu_ctx, 0, c, None, 0, 0, 16, g.GMC_EULER, g.GMC_FP32, y, None)
    with pytest.raises(g.GMCError) as e:
        g.gmc_transmit(gpu_ctx, 1, c, None, 0, 0, 0, g.GMC_EULER, g.GMC_FP32, y, None)
    assert e.value.status == g.GMC_EINVAL
    with pytest.raises(g.GMCError) as e:
        g.gmc_transmit(gpu_ctx, 1, c, None, 0, 0, 4, g.GMC_EULER, g.GMC_FP32, None, None)
    assert e.value.status == g.GMC_EINVAL


def test_host_buffers_e2e(gpu_ctx, net):
    import paper_2512_13965_gb300 as g
    n = 500
    cond, _, _ = synth.sampler_conditions(n, 51)
    z = synth.gaussian_noise(n, 52)
    y = np.zeros((4, n), np.float32)
    g.gmc_transmit(gpu_ctx, n, cond, z, 0, 0, 8, g.GMC_EULER, g.GMC_FP32, y, None)
    expect = oracle.mlp.sample(net, cond, z, 8, "euler")
    assert np.abs(y - expect).max() < FP32_TOL


@pytest.mark.parametrize("prec_name", ["GMC_FP32", "GMC_BF16"])
def test_pinned_host_buffers_in_place(gpu_ctx, net, prec_name):
    """Page-locked host arrays are read and written by the kernel in place;
    results equal those from device arrays bit for bit (8192 + 77 rows: an
    odd number of 128-row tiles)."""
    import paper_2512_13965_gb300 as g
    prec = getattr(g, prec_name)
    n = 8192 + 77
    cond, _, _ = synth.sampler_conditions(n, 53)
    z = synth.gaussian_noise(n, 54)
    y_dev, ex_dev = _run(gpu_ctx, cond, z, 8, g.GMC_EULER, prec, want_exit=True)
    pc = torch.from_numpy(cond).pin_memory()
    pz = torch.from_numpy(z).pin_memory()
    py = torch.full((4, n), float("nan")).pin_memory()
    pe = torch.full((4, n), float("nan")).pin_memory()
    g.gmc_transmit(gpu_ctx, n, pc, pz, 0, 0, 8, g.GMC_EULER, prec, py, pe)
    # the call returns with the results on the host
    assert np.array_equal(py.numpy().astype(np.float64), y_dev)
    assert np.array_equal(pe.numpy().astype(np.float64), ex_dev)


def _bf16_or_skip(ctx, cond, z, steps, integ=0):
    import paper_2512_13965_gb300 as g
    try:
        return _run(ctx, cond, z, steps, integ, g.GMC_BF16)
    except g.GMCError as e:
        if e.status == g.GMC_ENOTIMPL:
            pytest.skip("BF16 tensor-core path not built")
        raise


@pytest.mark.parametrize("n", [1, 127, 128, 129, 8192 + 77])
def test_bf16_euler16_bound(gpu_ctx, net, n):
    cond, _, _ = synth.sampler_conditions(n, 300 + n)
    z = synth.gaussian_noise(n, 400 + n)
    y, _ = _bf16_or_skip(gpu_ctx, cond, z, 16)
    expect = oracle.mlp.sample(net, cond, z, 16, "euler")
    err = np.abs(y - expect)
    assert np.all(np.isfinite(y))
    assert err.max() < BF16_MAX, err.max()
    if n > 1000:
        assert np.quantile(err, 0.999) < BF16_P999


def test_bf16_midpoint_bound(gpu_ctx, net):
    n = 1000
    cond, _, _ = synth.sampler_conditions(n, 61)
    z = synth.gaussian_noise(n, 62)
    y, _ = _bf16_or_skip(gpu_ctx, cond, z, 8, integ=1)
    expect = oracle.mlp.sample(net, cond, z, 8, "midpoint")
    assert np.abs(y - expect).max() < BF16_MAX


def test_bf16_full_size_sampled(gpu_ctx, net):
    n = 1 << 20
    cond, _, _ = synth.sampler_conditions(n, 1)
    z = synth.gaussian_noise(n, 3)
    y, _ = _bf16_or_skip(gpu_ctx, cond, z, 16)
    idx = np.concatenate([np.random.default_rng(1).choice(n, 1024, replace=False), [0, n - 1]])
    expect = oracle.mlp.sample(net, cond[:, idx], z[:, idx], 16, "euler")
    err = np.abs(y[:, idx] - expect)
    assert err.max() < BF16_MAX
    assert np.all(np.isfinite(y))


@pytest.mark.parametrize("steps", [1, 4, 12])
def test_fp32_rk4_parity(gpu_ctx, net, steps):
    # classical RK4, the fixed-step solver the paper times (12 steps)
    import paper_2512_13965_gb300 as g
    n = 700
    cond, _, _ = synth.sampler_conditions(n, 70 + steps)
    z = synth.gaussian_noise(n, 80 + steps)
    y, _ = _run(gpu_ctx, cond, z, steps, g.GMC_RK4, g.GMC_FP32)
    expect = oracle.mlp.sample(net, cond, z, steps, "rk4")
    assert np.abs(y - expect).max() < FP32_TOL


def test_bf16_rk4_bound(gpu_ctx, net):
    import paper_2512_13965_gb300 as g
    n = 3000
    cond, _, _ = synth.sampler_conditions(n, 91)
    z = synth.gaussian_noise(n, 92)
    y, _ = _bf16_or_skip(gpu_ctx, cond, z, 12, integ=g.GMC_RK4)
    expect = oracle.mlp.sample(net, cond, z, 12, "rk4")
    err = np.abs(y - expect)
    assert err.max() < BF16_MAX and np.quantile(err, 0.999) < BF16_P999


# FP8 path: E4M3 weights (per-output-channel scales) and inputs for layers
# 2-4. Two references: the FP64 network (the size of the 8-bit error, a
# measured bound like BF16's) and the oracle's quantized network
# (oracle.mlp.quantized_e4m3: the same roundings of weights and layer inputs
# in FP64), which the GPU must track much more closely -- what remains is
# accumulation order, the BF16 layers 1 and 5, and E4M3 rounding decisions
# flipped by the FP16 SiLU.
# measured on GB300, 8192 rows, Kaiming weights, Euler 16/8, midpoint 8, RK4 12:
# against FP64 max 0.19-0.26, p99.9 0.15-0.18; against the quantized network
# max 0.07-0.20, p99.9 0.04-0.10 (and the quantized network itself differs from
# FP64 by max 0.21-0.25): the bounds keep a factor of about 2.
FP8_MAX, FP8_P999 = 0.5, 0.3
FP8Q_MAX, FP8Q_P999 = 0.4, 0.2


def _fp8_check(ctx, net, n, steps, integ, iname, seed):
    import paper_2512_13965_gb300 as g
    cond, _, _ = synth.sampler_conditions(n, seed)
    z = synth.gaussian_noise(n, seed + 1)
    y, _ = _run(ctx, cond, z, steps, integ, g.GMC_FP8)
    assert np.all(np.isfinite(y))
    e = np.abs(y - oracle.mlp.sample(net, cond, z, steps, iname))
    eq = np.abs(y - oracle.mlp.sample(oracle.mlp.quantized_e4m3(net), cond, z, steps, iname))
    assert e.max() < FP8_MAX, e.max()
    assert eq.max() < FP8Q_MAX, eq.max()
    if n > 1000:
        assert np.quantile(e, 0.999) < FP8_P999
        assert np.quantile(eq, 0.999) < FP8Q_P999
        # it is the quantized network that the path evaluates
        assert np.median(eq) < 0.5 * np.median(e)
    return e, eq


@pytest.mark.parametrize("n", [1, 129, 8192 + 77])
def test_fp8_euler16_bound(gpu_ctx, net, n):
    _fp8_check(gpu_ctx, net, n, 16, 0, "euler", 500 + n)


def test_fp8_midpoint_and_rk4_bound(gpu_ctx, net):
    import paper_2512_13965_gb300 as g
    _fp8_check(gpu_ctx, net, 2000, 8, g.GMC_MIDPOINT, "midpoint", 71)
    _fp8_check(gpu_ctx, net, 2000, 12, g.GMC_RK4, "rk4", 73)


def test_fp8_full_size_sampled(gpu_ctx, net):
    import paper_2512_13965_gb300 as g
    n = 1 << 20
    cond, _, _ = synth.sampler_conditions(n, 1)
    z = synth.gaussian_noise(n, 3)
    y, _ = _run(gpu_ctx, cond, z, 16, g.GMC_EULER, g.GMC_FP8)
    assert np.all(np.isfinite(y))
    idx = np.concatenate([np.random.default_rng(2).choice(n, 1024, replace=False), [0, n - 1]])
    q = oracle.mlp.quantized_e4m3(net)
    eq = np.abs(y[:, idx] - oracle.mlp.sample(q, cond[:, idx], z[:, idx], 16, "euler"))
    assert eq.max() < FP8Q_MAX
