"""The paper's two benchmark problems (Section 5: the lattice and the
linearized hohlraum), 112 x 112 cells with the printed cross sections, solved
by GMC with the wide-range networks shipped with the package (trained on tau
log-uniform in [0.01, 1000]) against the GPU random walk.

Every cell of both problems is optically thin (tau <= 1.16) and most leave
the networks' box in c as well (pure scatterers, strong absorbers): GMC
samples them at their scattering-equivalent condition. With the networks'
box reaching tau = 0.01, every lattice cell has an equivalent condition
inside it, so no lattice cell is walked. The GMC flux (BF16, midpoint 8)
must agree with the walk within 2 % relative L2 at 10^6 histories (the
walk's own run-to-run floor there is 0.5 % on the lattice, 0.9 % on the
hohlraum), and on the lattice it must beat the networks trained on tau in
[0.1, 1000]: under that box the 3072 absorber cells (tau 0.0625, c 0.05)
have no equivalent condition and are walked, and the scatterers are sampled
at the box's edge.
"""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2512_13965_gb300", "weights")
N = 112
N_HIST = 1_000_000
FLUX_ERR_BOUND = 0.02
WIDE_BOX = (0.01, 1000.0, 0.5, 0.999)
NARROW_BOX = (0.1, 1000.0, 0.5, 0.999)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _context(boundary, internal, box):
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    g.gmc_load_weights(ctx, os.path.join(WEIGHTS, boundary))
    g.gmc_load_internal_weights(ctx, os.path.join(WEIGHTS, internal))
    cfg = g.gmc_get_config(ctx)
    cfg.net_tau_lo, cfg.net_tau_hi, cfg.net_c_lo, cfg.net_c_hi = box
    g.gmc_set_config(ctx, cfg)
    return ctx


@pytest.fixture(scope="module")
def contexts():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    wide = _context("gmc_boundary_wide.bin", "gmc_internal_wide.bin", WIDE_BOX)
    narrow = _context("gmc_boundary.bin", "gmc_internal.bin", NARROW_BOX)
    yield {"wide": wide, "narrow": narrow}
    wide.close()
    narrow.close()


def _problem(name):
    import paper_2512_13965_gb300 as g
    if name == "lattice":
        tau, c, src = synth.paper_lattice_problem(N)
        solve = g.transport_solve
    else:
        tau, c, src = synth.paper_hohlraum_problem(N)
        solve = g.transport_solve_wall
    return [np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c, src)], solve


def _solve(ctx, name, method, seed):
    import paper_2512_13965_gb300 as g
    (tau, c, src), solve = _problem(name)
    cfg = g.gmc_get_config(ctx)
    cfg.precision, cfg.integrator, cfg.steps, cfg.gmc_min_tau = g.GMC_BF16, g.GMC_MIDPOINT, 8, 0.0
    g.gmc_set_config(ctx, cfg)
    f = np.zeros(N * N)
    st = solve(ctx, N, N, tau, c, src, N_HIST, method, seed, f)
    return f, st.as_dict()


@pytest.fixture(scope="module")
def walks(contexts):
    import paper_2512_13965_gb300 as g
    out = {}
    for name in ("lattice", "hohlraum"):
        fa, _ = _solve(contexts["wide"], name, g.GMC_METHOD_ANALOG, 11)
        fb, _ = _solve(contexts["wide"], name, g.GMC_METHOD_ANALOG, 12)
        out[name] = (0.5 * (fa + fb), _rel(fa, fb) / np.sqrt(2.0))
    return out


@pytest.mark.parametrize("name", ["lattice", "hohlraum"])
def test_wide_networks_match_the_walk(contexts, walks, name):
    import paper_2512_13965_gb300 as g
    f_mc, floor = walks[name]
    assert floor < 0.012, floor
    f, st = _solve(contexts["wide"], name, g.GMC_METHOD_GMC, 13)
    assert np.all(np.isfinite(f)) and st["transmissions"] > 0
    err = _rel(f, f_mc)
    assert err < FLUX_ERR_BOUND, (name, err, floor)
    if name == "lattice":
        # every lattice cell is sampled (at its equivalent condition): no
        # cell is walked, so the solve makes no collisions
        assert st["collisions"] == 0, st


def test_wide_networks_beat_narrow_on_the_lattice(contexts, walks):
    import paper_2512_13965_gb300 as g
    f_mc, _ = walks["lattice"]
    f_w, _ = _solve(contexts["wide"], "lattice", g.GMC_METHOD_GMC, 13)
    f_n, _ = _solve(contexts["narrow"], "lattice", g.GMC_METHOD_GMC, 13)
    assert _rel(f_w, f_mc) < 0.75 * _rel(f_n, f_mc), (_rel(f_w, f_mc), _rel(f_n, f_mc))


@pytest.mark.parametrize("name", ["lattice", "hohlraum"])
def test_xy_geometry_paper_problems(name):
    # both problems in x-y geometry (3-D directions), the package's x-y
    # network and box [0.1, 1000] x [0.5, 0.999], births walked: GMC BF16
    # midpoint 8 within 2 % of the x-y walk at 10^6 histories (measured
    # 1.19 % and 1.45 %, floors 0.59 % and 0.94 %)
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    try:
        g.gmc_load_xy_weights(ctx, os.path.join(WEIGHTS, "gmc_xy.bin"))
        if name == "lattice":
            tau, c, src = synth.paper_lattice_problem(N)
            solve = g.transport_solve_xy
        else:
            tau, c, src = synth.paper_hohlraum_problem(N)
            solve = g.transport_solve_wall_xy
        args = [np.ascontiguousarray(a, np.float32).ravel() for a in (tau, c, src)]

        def run(method, seed):
            cfg = g.gmc_get_config(ctx)
            cfg.precision, cfg.integrator, cfg.steps, cfg.gmc_min_tau = g.GMC_BF16, g.GMC_MIDPOINT, 8, 0.0
            g.gmc_set_config(ctx, cfg)
            f = np.zeros(N * N)
            solve(ctx, N, N, *args, N_HIST, method, seed, f)
            return f

        fa, fb = run(g.GMC_METHOD_ANALOG, 11), run(g.GMC_METHOD_ANALOG, 12)
        f_mc = 0.5 * (fa + fb)
        floor = _rel(fa, fb) / np.sqrt(2.0)
        err = _rel(run(g.GMC_METHOD_GMC, 13), f_mc)
        assert floor < 0.012 and err < FLUX_ERR_BOUND, (name, err, floor)
    finally:
        ctx.close()
