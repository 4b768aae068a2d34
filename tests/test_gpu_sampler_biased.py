"""GPU samplers against the FP64 oracle on a network with nonzero biases in
every layer and a non-identity standardization (the Kaiming test network has
zero biases): covers the layer-1 bias table, the bias MMA of layers 2-4 (BF16
hi + lo against constant-1 operand columns), the FP8 scale-and-bias epilogue,
the output bias and the condition/exit standardization.

Bounds are those of the Kaiming tests (FP32 1e-4; BF16 max 0.1, p99.9 0.06;
FP8 against the quantized network max 0.4, p99.9 0.2), on standardized ODE
outputs.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
BF16_MAX, BF16_P999 = 0.1, 0.06
FP8Q_MAX, FP8Q_P999 = 0.4, 0.2


@pytest.fixture(scope="module")
def bnet(gpu_ctx, tmp_path_factory):
    import paper_2512_13965_gb300 as g
    path = str(tmp_path_factory.mktemp("wb") / "biased_seed7.bin")
    synth.write_weights(path, synth.biased_weights(7))
    g.gmc_load_weights(gpu_ctx, path)
    yield oracle.mlp.read_weights(path)


def _run(ctx, cond, z, steps, integ, prec, want_exit=False):
    import paper_2512_13965_gb300 as g
    n = cond.shape[1]
    y = torch.full((4, n), float("nan"), device="cuda")
    ex = torch.full((4, n), float("nan"), device="cuda") if want_exit else None
    g.gmc_transmit(ctx, n, torch.from_numpy(cond).cuda(), torch.from_numpy(z).cuda(), 0, 0, steps,
                   integ, prec, y, ex)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64), (None if ex is None else ex.cpu().numpy().astype(np.float64))


def test_biases_are_nonzero(bnet):
    for b in bnet.b:
        assert np.abs(b).max() > 0.1
    assert np.abs(bnet.cond_mean).max() > 0.1 and np.abs(bnet.y_std - 1).max() > 0.1


@pytest.mark.parametrize("integ,iname,steps", [(0, "euler", 16), (1, "midpoint", 8), (2, "rk4", 6)])
def test_fp32_parity(gpu_ctx, bnet, integ, iname, steps):
    import paper_2512_13965_gb300 as g
    n = 2048 + 37
    cond, _, _ = synth.sampler_conditions(n, 700 + integ)
    z = synth.gaussian_noise(n, 710 + integ)
    y, _ = _run(gpu_ctx, cond, z, steps, integ, g.GMC_FP32)
    assert np.abs(y - oracle.mlp.sample(bnet, cond, z, steps, iname)).max() < FP32_TOL


@pytest.mark.parametrize("integ,iname,steps", [(0, "euler", 16), (1, "midpoint", 8), (2, "rk4", 12)])
def test_bf16_bound(gpu_ctx, bnet, integ, iname, steps):
    import paper_2512_13965_gb300 as g
    n = 8192 + 77
    cond, _, _ = synth.sampler_conditions(n, 720 + integ)
    z = synth.gaussian_noise(n, 730 + integ)
    y, _ = _run(gpu_ctx, cond, z, steps, integ, g.GMC_BF16)
    err = np.abs(y - oracle.mlp.sample(bnet, cond, z, steps, iname))
    assert np.all(np.isfinite(y))
    assert err.max() < BF16_MAX, err.max()
    assert np.quantile(err, 0.999) < BF16_P999, np.quantile(err, 0.999)


@pytest.mark.parametrize("integ,iname,steps", [(0, "euler", 16), (2, "rk4", 12)])
def test_fp8_bound(gpu_ctx, bnet, integ, iname, steps):
    import paper_2512_13965_gb300 as g
    n = 4096 + 5
    cond, _, _ = synth.sampler_conditions(n, 740 + integ)
    z = synth.gaussian_noise(n, 750 + integ)
    y, _ = _run(gpu_ctx, cond, z, steps, integ, g.GMC_FP8)
    q = oracle.mlp.quantized_e4m3(bnet)
    eq = np.abs(y - oracle.mlp.sample(q, cond, z, steps, iname))
    assert np.all(np.isfinite(y))
    assert eq.max() < FP8Q_MAX, eq.max()
    assert np.quantile(eq, 0.999) < FP8Q_P999, np.quantile(eq, 0.999)


def test_decoded_exits(gpu_ctx, bnet):
    """Exit decoding with the network's output standardization (FP32 path),
    and valid exits from the BF16 path."""
    import paper_2512_13965_gb300 as g
    n = 3000
    cond, _, _ = synth.sampler_conditions(n, 760)
    z = synth.gaussian_noise(n, 761)
    _, ex = _run(gpu_ctx, cond, z, 16, 0, g.GMC_FP32, want_exit=True)
    d = oracle.mlp.decode(bnet, oracle.mlp.sample(bnet, cond, z, 16, "euler"))
    dp = np.abs(ex[0] - (d["face"] + d["q"]))
    dp = np.minimum(dp, 4.0 - dp)          # the perimeter is periodic
    assert dp.max() < 1e-3
    ok = np.floor(ex[0]).astype(int) == d["face"]
    assert ok.mean() > 0.999
    assert np.abs(ex[1][ok] - d["ux"][ok]).max() < 1e-3
    assert np.abs(ex[2][ok] - d["uy"][ok]).max() < 1e-3
    assert np.all(np.abs(ex[3] / d["s"] - 1.0) < 1e-3)
    _, ex16 = _run(gpu_ctx, cond, z, 16, 0, g.GMC_BF16, want_exit=True)
    assert np.all(np.isfinite(ex16)) and np.all(ex16[3] > 0)
    assert np.all((ex16[0] >= 0) & (ex16[0] < 4))
    assert np.abs(np.hypot(ex16[1], ex16[2]) - 1.0).max() < 1e-5
