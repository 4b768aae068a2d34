"""Pins for the oracle's transport solves (Eq. 5-7, Eq. 12 and the four-stage
GMC loop)."""
import math

import numpy as np
import pytest
from scipy import integrate, stats as sstats

import synth
from test_oracle_walk import uncollided_by_face
from oracle import stats as ostats
from oracle import transport as T


def escape_expectation(tau):
    """E[exp(-tau l)] for a uniform point in the unit square and an isotropic
    direction, l the distance to the boundary. By the square's symmetry only
    directions in (0, pi/2) are needed; with a, b the distances to the right
    and top edges, l = min(a / cos, b / sin), and the b-integral is closed."""
    def inner(a, th):
        c, s = math.cos(th), math.sin(th)
        m = a * math.tan(th)
        part1 = (s / tau) * (1.0 - math.exp(-tau * min(m, 1.0) / s))
        part2 = max(1.0 - m, 0.0) * math.exp(-tau * a / c)
        return part1 + part2

    def over_a(th):
        brk = [min(1.0, 1.0 / math.tan(th))] if th > math.pi / 4 else None
        return integrate.quad(inner, 0.0, 1.0, args=(th,), points=brk, epsabs=1e-12, limit=200)[0]
    return (2.0 / math.pi) * integrate.quad(over_a, 1e-12, math.pi / 2 - 1e-12, epsabs=1e-11,
                                            limit=400)[0]


def test_single_cell_pure_absorber_closed_form():
    # c = 0: births fly straight out; the score is (1 - e^{-s}) / tau and the
    # leaked weight e^{-s} with s the optical distance to the boundary.
    tau = 2.0
    e = escape_expectation(tau)
    runs = []
    leaks = []
    for k in range(8):
        flux, st = T.solve_analog(np.full((1, 1), tau), np.zeros((1, 1)), np.ones((1, 1)),
                                  20000, seed=100 + k, w_cut=0.0)
        runs.append(flux[0, 0])
        leaks.append(st["leak"] / 20000)
        assert abs(st["leak"] + st["absorbed"] - 20000) < 1e-8
    runs, leaks = np.array(runs), np.array(leaks)
    se = runs.std(ddof=1) / math.sqrt(len(runs))
    assert abs(runs.mean() - (1.0 - e) / tau) < 4 * se
    assert abs(leaks.mean() - e) < 4 * leaks.std(ddof=1) / math.sqrt(len(leaks))


def test_weight_balance_is_exact():
    # Implicit capture conserves weight exactly: deposited + leaked weight
    # equals the source weight, apart from the roulette's explicit changes.
    tau, c, src = synth.grid_problem(n=8, seed=5, tau_range=(0.1, 5.0), block=4, source=2)
    n = 3000
    flux, st = T.solve_analog(tau, c, src, n, seed=9)
    total = st["absorbed"] + st["leak"] - st["roulette_net"]
    assert abs(total - n) < 1e-8 * n
    # and the flux tally is the deposit divided by sigma_a (Eq. 7)
    sig_a = (1.0 - c.astype(np.float64)) * tau.astype(np.float64)
    assert abs(np.sum(flux * sig_a) * n - st["absorbed"]) < 1e-8 * n


def _zscores(a_runs, b_runs):
    a, b = np.asarray(a_runs), np.asarray(b_runs)
    se = np.sqrt(a.var(axis=0, ddof=1) / a.shape[0] + b.var(axis=0, ddof=1) / b.shape[0])
    d = a.mean(axis=0) - b.mean(axis=0)
    ok = se > 0
    z = np.zeros_like(d)
    z[ok] = d[ok] / se[ok]
    assert np.all(d[~ok] == 0)
    return z


def test_event_loop_with_walk_sampler_matches_mc():
    # Pins the four-stage loop (rotation into the left-entry frame, decoding,
    # rotation back, crossing) independently of the network: with stage 2
    # replaced by the random walk run in the canonical frame, the loop must
    # reproduce the standard MC flux cell by cell.
    tau, c, src = synth.grid_problem(n=6, seed=11, tau_range=(0.1, 4.0), block=3, source=2)
    K, n = 6, 2500
    mc, gm = [], []
    mc_leak, gm_leak = [], []
    for k in range(K):
        f1, s1 = T.solve_analog(tau, c, src, n, seed=200 + k)
        f2, s2 = T.solve_gmc(tau, c, src, n, seed=300 + k, sampler=T.walk_sampler(300 + k))
        mc.append(f1.ravel())
        gm.append(f2.ravel())
        mc_leak.append(s1["leak"] / n)
        gm_leak.append(s2["leak"] / n)
        assert abs(s2["absorbed"] + s2["leak"] - s2["roulette_net"] - n) < 1e-8 * n
    z = _zscores(mc, gm)
    assert np.max(np.abs(z)) < 4.5
    assert np.mean(np.abs(z) > 3) < 0.05
    assert abs(_zscores(np.array(mc_leak)[:, None], np.array(gm_leak)[:, None])[0]) < 4


def test_rotation_rules():
    # Canonical face f maps to global face (f + r) mod 4 with r = (F + 1) mod 4
    # for a particle entering through global face F; directions rotate by r.
    for F in range(4):
        r = (F + 1) % 4
        # the canonical entry direction +x must point into the cell through F
        gx, gy = T.rot(np.array([1.0]), np.array([0.0]), r)
        inward = {0: (0, 1), 1: (-1, 0), 2: (0, -1), 3: (1, 0)}[F]
        assert (round(gx[0]), round(gy[0])) == inward
        assert (3 + r) % 4 == F
    ux, uy = T.rot(np.array([0.6]), np.array([0.8]), 1)
    assert (ux[0], uy[0]) == (-0.8, 0.6)
    bx, by = T.rot(ux, uy, -1)
    assert (bx[0], by[0]) == (0.6, 0.8)


def test_sigma_bar_decays_as_inverse_sqrt_n():
    # Eq. 12 over K = 5 runs: sigma_bar(N) ~ N^{-1/2}.
    tau, c, src = synth.grid_problem(n=8, seed=13, tau_range=(0.1, 3.0), block=4, source=2)
    sb = []
    for n in (1000, 4000, 16000):
        runs = [T.solve_analog(tau, c, src, n, seed=1000 * n + k)[0].ravel() for k in range(5)]
        sb.append(ostats.sigma_bar(runs))
    slope = np.polyfit(np.log([1000, 4000, 16000]), np.log(sb), 1)[0]
    assert -0.62 < slope < -0.38, (slope, sb)


def test_internal_walk_births_reproduce_walked_births():
    # Births through the internal-model path with the exact walk as the
    # "model" (birth direction from the birth draw, walk from event 0) are the
    # walked births history by history: identical flux, leakage, absorption.
    tau, c, src = synth.grid_problem(n=8, seed=21, tau_range=(0.1, 20.0), block=4, source=2)
    a, sa = T.solve_gmc(tau, c, src, 2000, 5, T.walk_sampler(5))
    b, sb = T.solve_gmc(tau, c, src, 2000, 5, T.walk_sampler(5),
                        internal=T.walk_internal_sampler(5))
    np.testing.assert_array_equal(a, b)
    for k in ("leak", "absorbed", "roulette_net", "transmissions", "roulette_kills"):
        assert sa[k] == sb[k], k


def test_internal_condition():
    X = np.array([0.1, 0.9, 0.5, 0.3])
    Y = np.array([0.4, 0.2, 0.5, 0.99])
    cond = T.internal_condition(X, Y, np.array([2.0, 3.0, 4.0, 5.0]), np.array([0.5] * 4))
    np.testing.assert_allclose(cond[0], X)
    np.testing.assert_allclose(cond[1], Y)
    np.testing.assert_allclose(cond[2], np.log([2.0, 3.0, 4.0, 5.0]))
    np.testing.assert_allclose(cond[4], [0.1, 0.1, 0.5, 0.01])


def test_global_frame_walk_sampler_is_the_mc_solve():
    # The event loop with stage 2 replaced by the walk in each cell's own
    # frame (entry point and direction rotated back from the canonical frame,
    # the exit rotated forward) draws exactly what the standard MC solve
    # draws: the same flux to rounding, the same leakage and absorption.
    tau, c, src = synth.grid_problem(n=8, seed=21, tau_range=(0.1, 20.0), block=4, source=2)
    a, sa = T.solve_analog(tau, c, src, 800, 5)
    b, sb = T.solve_gmc(tau, c, src, 800, 5, T.walk_sampler_global(5))
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-15)
    for k in ("leak", "absorbed", "transmissions", "roulette_kills"):
        assert abs(sa[k] - sb[k]) <= 1e-9 * max(1.0, abs(sa[k])), k


# --- surface source on the left boundary ------------------------------------

def _wall_single_cell(tau, c, n, seed):
    """Per-history track lengths of a one-cell problem with the wall source
    (the canonical walk from the births' entry states), and the solve."""
    j, xi, gx, gy = T.wall_births([1.0], n, seed)
    assert np.all(j == 0) and np.all(gx > 0)
    r = T.transmit(xi, gx, gy, np.full(n, tau), np.full(n, c), T.MODE_IMPLICIT, seed,
                   ids=np.arange(n, dtype=np.uint64), events=np.zeros(n, np.uint32))
    flux, st = T.solve_gmc(np.full((1, 1), tau), np.full((1, 1), c), None, n, seed,
                           T.walk_sampler_global(seed), wall=[1.0])
    return r["s"], float(flux[0, 0]), st


def test_wall_source_entry_law():
    # u2 -> sin(theta) uniform in (-1, 1]: the cosine law; u1 -> xi uniform;
    # the row follows the strengths
    j, xi, gx, gy = T.wall_births([1.0, 0.0, 3.0], 40000, 12)
    assert set(np.unique(j)) == {0, 2}
    assert abs(np.mean(j == 2) - 0.75) < 4 * math.sqrt(0.75 * 0.25 / 40000)
    assert np.allclose(gx * gx + gy * gy, 1.0) and np.all(gx >= 0)
    for a in (xi, 0.5 * (gy + 1.0)):
        assert sstats.kstest(a, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("tau", [0.5, 2.0])
def test_wall_source_pure_absorber_closed_form(tau):
    # c = 0 with implicit capture: no collisions, each history crosses the cell
    # on a straight chord of optical length s and deposits 1 - e^{-s}, so the
    # flux is (1 - P_unc) / tau with P_unc the uncollided transmission of the
    # same entry law (the closed form of the walk tests).
    n = 20000
    s, flux, st = _wall_single_cell(tau, 0.0, n, 3)
    per = -np.expm1(-s) / tau
    assert flux == pytest.approx(per.mean(), rel=1e-12)
    expect = (1.0 - uncollided_by_face(tau).sum()) / tau
    assert abs(per.mean() - expect) < 4 * per.std() / math.sqrt(n)
    assert st["transmissions"] == n


def test_wall_source_pure_scatterer_mean_path():
    # c = 1: nothing is absorbed, every history leaks, and the mean track length
    # of a Lambertian inflow is pi tau / 4 for any tau (the path-length
    # invariance), so the flux of the one-cell problem is pi / 4.
    n, tau = 20000, 3.0
    s, flux, st = _wall_single_cell(tau, 1.0, n, 4)
    per = s / tau
    assert flux == pytest.approx(per.mean(), rel=1e-12)
    assert abs(per.mean() - math.pi / 4) < 4 * per.std() / math.sqrt(n)
    assert st["leak"] == pytest.approx(n, rel=1e-12) and st["absorbed"] == 0.0


def test_hohlraum_layout():
    # five material classes where the layout puts them; the source drives the
    # entrance rows, which are window cells on the left boundary
    n = 64
    tau, c, wall = synth.hohlraum_problem(n)
    mats = {m: (t, cc) for m, (t, cc) in synth.HOHLRAUM_MATERIALS.items()}
    assert {(float(a), float(b)) for a, b in zip(tau.ravel(), c.ravel())} == \
        {(float(np.float32(t)), float(np.float32(cc))) for t, cc in mats.values()}
    t_wall, t_win = np.float32(mats["wall"][0]), np.float32(mats["window"][0])
    assert np.all(tau[0, :] == t_wall) and np.all(tau[-1, :] == t_wall) and np.all(tau[:, -1] == t_wall)
    lit = np.flatnonzero(wall > 0)
    assert lit.min() == n // 4 and lit.max() == 3 * n // 4 - 1
    assert np.all(tau[lit, 0] == t_win) and np.all(tau[np.flatnonzero(wall == 0)[4:-4], 0] == t_wall)
    centre = tau[n // 2, n // 2]
    assert centre == np.float32(mats["fuel"][0])
    assert np.allclose(tau, tau[::-1, :])  # mirror symmetry about the horizontal axis
