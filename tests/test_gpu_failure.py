"""Failure detection on the GPU without faulting it: a bounded device wait on
an mbarrier that nothing arrives at gives up, the host reads GMC_ETIMEOUT
through the device error word, and the context keeps working.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives(kaiming_file):
    import time

    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, kaiming_file)
        t0 = time.perf_counter()
        st = g.gmc_selftest_wait(ctx, 300.0)
        dt = time.perf_counter() - t0
        assert st == g.GMC_ETIMEOUT, g.status_name(st)
        assert "gave up" in g.lib.gmc_last_error(ctx.handle).decode()
        assert 0.25 < dt < 5.0  # it waited about its limit, then returned
        g.gmc_synchronize(ctx)  # the error word was read and cleared
        # the context still computes correctly
        n = 300
        cond, _, _ = synth.sampler_conditions(n, 3)
        z = synth.gaussian_noise(n, 4)
        y = torch.empty(4, n, device="cuda")
        g.gmc_transmit(ctx, n, torch.from_numpy(cond).cuda(), torch.from_numpy(z).cuda(), 0, 0, 4,
                       g.GMC_EULER, g.GMC_FP32, y, None)
        g.gmc_synchronize(ctx)
        expect = oracle.mlp.sample(oracle.mlp.read_weights(kaiming_file), cond, z, 4, "euler")
        assert np.abs(y.cpu().numpy() - expect).max() < 1e-4
    finally:
        ctx.close()


def test_selftest_rejects_bad_limits(gpu_ctx):
    import paper_2512_13965_gb300 as g
    assert g.gmc_selftest_wait(gpu_ctx, 0.0) == g.GMC_EINVAL
    assert g.gmc_selftest_wait(gpu_ctx, 5000.0) == g.GMC_EINVAL
