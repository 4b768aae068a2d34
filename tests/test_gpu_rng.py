"""GPU Philox4x32-10 and Box-Muller normals against the oracle."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def test_philox_bit_exact(gpu_ctx):
    import paper_2512_13965_gb300 as g
    n = 1 << 20
    for seed, id0, ev, tag in ((0, 0, 0, 0), (0x0123456789ABCDEF, (1 << 32) - 7, 5, 2),
                               (42, 123456789012, 0xFFFFFFFF, 4)):
        out = torch.empty(n, 4, dtype=torch.int32, device="cuda")
        g.gmc_philox(gpu_ctx, n, seed, id0, ev, tag, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        expect = oracle.rng.philox_batch(seed, n, id0=id0, event=ev, tag=tag)
        np.testing.assert_array_equal(got, expect)


def test_philox_host_pointer_path(gpu_ctx):
    import paper_2512_13965_gb300 as g
    out = np.zeros((1000, 4), dtype=np.uint32)
    g.gmc_philox(gpu_ctx, 1000, 7, 3, 1, 1, out)
    np.testing.assert_array_equal(out, oracle.rng.philox_batch(7, 1000, id0=3, event=1, tag=1))


def test_normals_close_to_fp64(gpu_ctx):
    import paper_2512_13965_gb300 as g
    n = 1 << 18
    out = torch.empty(4, n, device="cuda")
    g.gmc_normals(gpu_ctx, n, 9, 100, 3, 2, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    expect = oracle.rng.normal_batch(9, n, id0=100, event=3, tag=2)
    # u = (x+1) 2^-32 rounded to float is off by up to 2^-25 near u = 1, which
    # perturbs sqrt(-2 ln u0) by ~3e-8 / r for small radii r: about 1e-4 of
    # the draws (r < 0.015) exceed 2e-6, none should exceed 1e-3.
    err = np.abs(got - expect) / (1.0 + np.abs(expect))
    assert np.mean(err < 2e-6) > 0.9995
    assert err.max() < 1e-3
