"""Pins for the oracle's random-walk cell transmission (Eq. 4-6).

Each test checks the oracle against something other than itself: a closed
form computed here by quadrature, an exact invariant of the walk, or a
textbook limit. Statistical checks use 4 standard errors.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import synth
from oracle import transport as T


def _entries(n, seed):
    e = synth.cell_entries(n, seed)
    return (e["xi"].astype(np.float64), e["cos"].astype(np.float64), e["sin"].astype(np.float64))


def _run(n, tau, c, mode, seed=0, eseed=100):
    xi, cs, sn = _entries(n, eseed)
    return T.transmit(xi, cs, sn, np.full(n, tau), np.full(n, c), mode, seed)


def uncollided_by_face(tau):
    """P(exit through face f with no collision) for left-face entry with
    uniform xi and cosine-weighted angle: int_0^1 dxi int (cos th / 2) e^{-d} dth,
    d the chord length to the boundary in optical units."""
    def face_int(face):
        def inner(xi):
            tb, tt = -math.atan(xi), math.atan(1.0 - xi)
            if face == 0:
                f = lambda th: 0.5 * math.cos(th) * math.exp(-xi * tau / -math.sin(th))
                lo, hi = -math.pi / 2, tb
            elif face == 1:
                f = lambda th: 0.5 * math.cos(th) * math.exp(-tau / math.cos(th))
                lo, hi = tb, tt
            else:
                f = lambda th: 0.5 * math.cos(th) * math.exp(-(1.0 - xi) * tau / math.sin(th))
                lo, hi = tt, math.pi / 2
            return integrate.quad(f, lo, hi, epsabs=1e-13, epsrel=1e-11, limit=200)[0]
        return integrate.quad(inner, 0.0, 1.0, epsabs=1e-12, epsrel=1e-10, limit=200)[0]
    return np.array([face_int(0), face_int(1), face_int(2)])


@pytest.mark.parametrize("tau", [0.3, 1.0, 3.0])
def test_pure_absorber_transmission_closed_form(tau):
    # c = 0 analog: every collision absorbs, so transmission through each face
    # is exactly the uncollided probability (the e^{-tau/mu} law on the chord).
    n = 200000
    r = _run(n, tau, 0.0, T.MODE_ANALOG)
    expect = uncollided_by_face(tau)
    for f in range(3):
        p = np.mean((r["status"] == 0) & (r["face"] == f))
        se = math.sqrt(max(expect[f] * (1 - expect[f]), 1e-12) / n)
        assert abs(p - expect[f]) < 4 * se + 1e-12, (f, p, expect[f])
    assert not np.any((r["status"] == 0) & (r["face"] == 3))


def test_uncollided_fraction_with_scattering():
    # With c = 0.9 the particles that exit without any collision still follow
    # the uncollided closed form, face by face.
    n, tau = 200000, 1.0
    r = _run(n, tau, 0.9, T.MODE_ANALOG)
    expect = uncollided_by_face(tau)
    for f in range(3):
        p = np.mean((r["ncoll"] == 0) & (r["face"] == f) & (r["status"] == 0))
        se = math.sqrt(expect[f] * (1 - expect[f]) / n)
        assert abs(p - expect[f]) < 4 * se


def test_outcomes_partition():
    r = _run(50000, 1.0, 0.9, T.MODE_ANALOG)
    exited = r["status"] == 0
    absorbed = r["status"] == 1
    assert np.all(exited ^ absorbed)
    assert np.all(r["face"][absorbed] == -1)
    assert set(np.unique(r["face"][exited])) <= {0, 1, 2, 3}
    # every exited particle points out of its face and q lies in [0, 1]
    f, ux, uy = r["face"][exited], r["ux"][exited], r["uy"][exited]
    out = np.select([f == 0, f == 1, f == 2, f == 3], [-uy, ux, uy, -ux])
    assert np.all(out >= 0)
    assert np.all((r["q"] >= 0) & (r["q"] <= 1))
    assert np.allclose(np.hypot(r["ux"], r["uy"]), 1.0)


def test_mirror_symmetry():
    # y -> tau - y, theta -> -theta maps the problem onto itself, so the
    # bottom and top exit fractions agree and the exit-position histograms on
    # the right face are mirror images.
    n = 200000
    r = _run(n, 2.0, 0.9, T.MODE_ANALOG)
    ex = r["status"] == 0
    pb, pt = np.mean(ex & (r["face"] == 0)), np.mean(ex & (r["face"] == 2))
    se = math.sqrt((pb + pt) / n)
    assert abs(pb - pt) < 4 * se
    right = ex & (r["face"] == 1)
    h, _ = np.histogram(r["q"][right], bins=16, range=(0, 1))
    d = h - h[::-1]
    z = d[:8] / np.sqrt(np.maximum(h[:8] + h[::-1][:8], 1))
    assert np.all(np.abs(z) < 4.5)


@pytest.mark.parametrize("tau,c", [(1.0, 0.9), (5.0, 0.5), (0.3, 0.999), (20.0, 0.999)])
def test_mean_path_length_invariance(tau, c):
    # Mean-path-length invariance (Blanco & Fournier 2003): for a Lambertian
    # entry into a convex 2-D body with any non-absorbing scattering, the mean
    # track length is pi A / P = pi tau / 4 for the square, whatever the
    # scattering rate.
    n = 100000
    r = _run(n, tau, c, T.MODE_IMPLICIT)
    m, se = r["s"].mean(), r["s"].std() / math.sqrt(n)
    assert abs(m - math.pi * tau / 4) < 4 * se
    # and the expected number of collisions is the scattering rate times it
    k = r["ncoll"].astype(np.float64)
    assert abs(k.mean() - c * math.pi * tau / 4) < 4 * k.std() / math.sqrt(n) + 1e-12


@pytest.mark.parametrize("tau,c", [(1.0, 0.9), (4.0, 0.7)])
def test_analog_absorption_identity(tau, c):
    # Collisions are a unit-rate Poisson process along the track, and each one
    # absorbs with probability 1 - c, so P(absorbed) = (1 - c) E[s].
    n = 200000
    r = _run(n, tau, c, T.MODE_ANALOG)
    d = (r["status"] == 1).astype(np.float64) - (1.0 - c) * r["s"]
    assert abs(d.mean()) < 4 * d.std() / math.sqrt(n)


def test_analog_equals_implicit_reweighting():
    # Survival-c analog transport and implicit capture with weight
    # exp(-(1-c) s) give the same expected transmission through every face.
    n, tau, c = 200000, 2.0, 0.8
    ra = _run(n, tau, c, T.MODE_ANALOG, seed=1)
    ri = _run(n, tau, c, T.MODE_IMPLICIT, seed=2, eseed=101)
    wi = np.exp(-(1.0 - c) * ri["s"])
    for f in range(4):
        a = ((ra["status"] == 0) & (ra["face"] == f)).astype(np.float64)
        b = wi * (ri["face"] == f)
        se = math.sqrt(a.var() / n + b.var() / n)
        assert abs(a.mean() - b.mean()) < 4 * se, f


def test_scaling_invariance_in_c_tau():
    # With implicit capture the flights have rate c, so rescaling lengths by
    # c maps (tau, c) onto (c tau, 1): the laws of (c s, p, theta_out) agree.
    n = 40000
    r1 = _run(n, 2.0, 0.5, T.MODE_IMPLICIT, seed=3, eseed=7)
    r2 = _run(n, 1.0, 1.0, T.MODE_IMPLICIT, seed=4, eseed=8)
    assert stats.ks_2samp(0.5 * r1["s"], r2["s"]).pvalue > 1e-3
    assert stats.ks_2samp(r1["face"] + r1["q"], r2["face"] + r2["q"]).pvalue > 1e-3
    assert stats.ks_2samp(r1["ux"], r2["ux"]).pvalue > 1e-3


def test_thin_cell_chords():
    # tau -> 0: every particle streams straight through; the exit point and
    # the track length follow from the chord geometry alone.
    n, tau = 20000, 1e-6
    xi, cs, sn = _entries(n, 55)
    r = T.transmit(xi, cs, sn, np.full(n, tau), np.full(n, 0.9), T.MODE_IMPLICIT, 9)
    assert np.all(r["ncoll"] == 0)
    tn = sn / cs
    right = np.abs(xi + tn - 0.5) <= 0.5
    top = ~right & (sn > 0)
    bot = ~right & (sn < 0)
    assert np.all(r["face"][right] == 1)
    assert np.all(r["face"][top] == 2)
    assert np.all(r["face"][bot] == 0)
    np.testing.assert_allclose(r["q"][right], (xi + tn)[right], atol=1e-9)
    np.testing.assert_allclose(r["q"][top], (1 - (1 - xi) / tn)[top], atol=1e-9)
    np.testing.assert_allclose(r["q"][bot], (xi / np.abs(tn))[bot], atol=1e-9)
    chord = np.where(right, tau / cs, np.where(top, (1 - xi) * tau / sn, xi * tau / np.abs(sn)))
    np.testing.assert_allclose(r["s"], chord, rtol=1e-9)
    np.testing.assert_allclose(r["ux"], cs, rtol=0, atol=0)
