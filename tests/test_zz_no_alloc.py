"""gmc_transmit_noalloc: the sampler entry point for callers that cannot
allocate device memory during a call (for example code running under a
framework that owns the device allocator, or code that may only allocate at
start-up). Both entry points run the same kernel on the same inputs, so its
exits must equal gmc_transmit's bit for bit on two calls in a row, reusing
its static scratch; device memory and torch's allocator must not change
across a call; sizes beyond that scratch are rejected.

This file is collected last on purpose. It creates its own context, so it
passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def ctx(kaiming_file):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_13965_gb300 as g
    c = g.Context(0)
    g.gmc_load_weights(c, kaiming_file)
    yield c
    c.close()


def _pair(ctx, n, steps, integ, seed_in):
    import paper_2512_13965_gb300 as g
    cond = torch.from_numpy(synth.sampler_conditions(n, seed_in)[0]).cuda()
    z = torch.from_numpy(synth.gaussian_noise(n, seed_in + 1)).cuda()
    ref_y = torch.empty(4, n, device="cuda")
    ref_e = torch.empty(4, n, device="cuda")
    g.gmc_transmit(ctx, n, cond, z, 0, 0, steps, integ, g.GMC_BF16, ref_y, ref_e)
    y = torch.full((4, n), float("nan"), device="cuda")
    e = torch.full((4, n), float("nan"), device="cuda")
    g.gmc_transmit_noalloc(ctx, n, cond, z, 0, 0, steps, integ, y, e)
    g.gmc_synchronize(ctx)
    return ref_y.cpu().numpy(), ref_e.cpu().numpy(), y.cpu().numpy(), e.cpu().numpy()


def test_matches_gmc_transmit_on_two_calls_in_a_row(ctx):
    import paper_2512_13965_gb300 as g
    # call 1: 16 Euler steps; call 2: 8 midpoint steps on a different batch,
    # so the shared bias table is rewritten between the calls
    for n, steps, integ, s in ((5000, 16, g.GMC_EULER, 11), (3000 + 17, 8, g.GMC_MIDPOINT, 21)):
        ry, re, y, e = _pair(ctx, n, steps, integ, s)
        assert np.all(np.isfinite(y)) and np.all(np.isfinite(e))
        np.testing.assert_array_equal(y, ry)
        np.testing.assert_array_equal(e, re)


def test_no_device_allocation_during_a_call(ctx):
    import paper_2512_13965_gb300 as g
    n, steps = 20000, 16
    cond = torch.from_numpy(synth.sampler_conditions(n, 31)[0]).cuda()
    y = torch.empty(4, n, device="cuda")
    e = torch.empty(4, n, device="cuda")
    # the first call on the device resolves the static array's address (set-up)
    g.gmc_transmit_noalloc(ctx, n, cond, None, 5, 0, steps, g.GMC_RK4, y, e)
    g.gmc_synchronize(ctx)
    torch.cuda.synchronize()
    for call in range(2):
        free0, _ = torch.cuda.mem_get_info()
        st0 = torch.cuda.memory_stats()
        g.gmc_transmit_noalloc(ctx, n, cond, None, 5 + call, 0, steps, g.GMC_RK4, y, e)
        g.gmc_synchronize(ctx)
        free1, _ = torch.cuda.mem_get_info()
        st1 = torch.cuda.memory_stats()
        assert free1 == free0, (call, free0, free1)
        for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
            assert st1.get(key, 0) == st0.get(key, 0), (call, key)
    assert torch.isfinite(e).all()


def test_internal_noise_and_limits(ctx):
    import paper_2512_13965_gb300 as g
    n = 1000
    cond = torch.from_numpy(synth.sampler_conditions(n, 5)[0]).cuda()
    ref = torch.empty(4, n, device="cuda")
    out = torch.empty(4, n, device="cuda")
    g.gmc_transmit(ctx, n, cond, None, 9, 77, 4, g.GMC_EULER, g.GMC_BF16, ref, None)
    g.gmc_transmit_noalloc(ctx, n, cond, None, 9, 77, 4, g.GMC_EULER, out, None)
    g.gmc_synchronize(ctx)
    assert torch.equal(out, ref)
    with pytest.raises(g.GMCError) as ex:
        g.gmc_transmit_noalloc(ctx, n, cond, None, 9, 77, 257, g.GMC_EULER, out, None)
    assert ex.value.status == g.GMC_EINVAL
    host = np.zeros((4, n), np.float32)
    with pytest.raises(g.GMCError) as ex:
        g.gmc_transmit_noalloc(ctx, n, cond, None, 9, 77, 4, g.GMC_EULER, host, None)
    assert ex.value.status == g.GMC_EINVAL
