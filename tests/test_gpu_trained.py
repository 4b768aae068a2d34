"""The trained networks shipped with the package against the analog method.

The scalar flux of a GMC solve with the trained boundary and internal models
must agree with the GPU random walk's flux (the method GMC replaces, itself
pinned to the oracle's walk in test_gpu_transport.py) within the stated
relative L2 error (1 % for the BF16 network, 2 % for FP8), on a
heterogeneous grid with the solve benchmark's materials: tau log-uniform in
[0.1, 500], c in {0.5, 0.999} per block. The
analog reference is two independent half-size runs; their difference gives
the statistical floor. The same solve with the untrained (Kaiming) network
misses the flux by far more: what the training gains.
"""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2512_13965_gb300", "weights")
# stated GMC-vs-analog relative L2 flux errors: BF16 network, and the FP8
# network (E4M3 hidden layers), whose rounding adds a bias of its own
FLUX_ERR_BOUND = {"bf16": 0.01, "fp8": 0.02}
N_HIST = 8_000_000


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def tctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    g.gmc_load_weights(ctx, os.path.join(WEIGHTS, "gmc_boundary.bin"))
    g.gmc_load_internal_weights(ctx, os.path.join(WEIGHTS, "gmc_internal.bin"))
    yield ctx
    ctx.close()


def _grid():
    return synth.grid_problem(n=32, seed=5, tau_range=(0.1, 500.0), block=8, source=4)


def _solve(ctx, method, seed, n, prec=None, integ=None, steps=8):
    import paper_2512_13965_gb300 as g
    tau, c, src = _grid()
    cfg = g.gmc_get_config(ctx)
    cfg.precision = g.GMC_BF16 if prec is None else prec
    cfg.integrator = g.GMC_MIDPOINT if integ is None else integ
    cfg.steps = steps
    cfg.gmc_min_tau = 0.0
    g.gmc_set_config(ctx, cfg)
    f = np.zeros(tau.size)
    st = g.transport_solve(ctx, 32, 32, *(np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c, src)),
                           n, method, seed, f)
    return f, st.as_dict()


@pytest.fixture(scope="module")
def analog(tctx):
    import paper_2512_13965_gb300 as g
    fa, _ = _solve(tctx, g.GMC_METHOD_ANALOG, 1, N_HIST // 2)
    fb, _ = _solve(tctx, g.GMC_METHOD_ANALOG, 2, N_HIST // 2)
    return 0.5 * (fa + fb), _rel(fa, fb) / np.sqrt(2.0)


@pytest.mark.parametrize("prec_name", ["bf16", "fp8"])
def test_trained_gmc_flux_within_bound_of_analog(tctx, analog, prec_name):
    import paper_2512_13965_gb300 as g
    f_mc, floor = analog
    bound = FLUX_ERR_BOUND[prec_name]
    assert floor < 0.4 * FLUX_ERR_BOUND["bf16"]  # enough histories to resolve the bounds
    prec = g.GMC_BF16 if prec_name == "bf16" else g.GMC_FP8
    f, st = _solve(tctx, g.GMC_METHOD_GMC, 3, N_HIST, prec)
    err = _rel(f, f_mc)
    print("flux error %s: %.4f (floor %.4f)" % (prec_name, err, floor))
    assert err <= bound, (prec_name, err, floor)
    assert st["collisions"] == 0  # births sampled by the internal model, no walk
    assert abs(st["absorbed"] + st["leaked"] - st["roulette_net"] - N_HIST) < 1e-4 * N_HIST


def test_untrained_network_misses_the_flux(analog, kaiming_file):
    import paper_2512_13965_gb300 as g
    f_mc, _ = analog
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, kaiming_file)
        f, _ = _solve(ctx, g.GMC_METHOD_GMC, 3, N_HIST // 4)
    finally:
        ctx.close()
    assert _rel(f, f_mc) > 10 * FLUX_ERR_BOUND["bf16"]
