"""Pins for the oracle's random walk in rectangular cells (the geometry
variant with unequal sides): a width tx = height ty reduces it to the square
walk history by history; the uncollided transmission per face and the mean
uncollided chord follow by quadrature; the mean track over the whole boundary
is pi A / P; outcomes partition; top and bottom are mirror images; implicit
capture depends on (c tx, c ty) only; training pairs decode back to the
walk's exits."""
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import transport as T


def _entries(n, seed):
    e = synth.cell_entries(n, seed)
    return (e["xi"].astype(np.float64), e["cos"].astype(np.float64), e["sin"].astype(np.float64))


def _rect(n, tx, ty, c, mode, seed=0, eseed=300):
    xi, cs, sn = _entries(n, eseed)
    return T.transmit_rect(xi, cs, sn, np.full(n, tx), np.full(n, ty), np.full(n, c), mode, seed)


def _faces(tx, ty, xi):
    """Angles of the two right-hand corners seen from (0, xi ty), and the
    chord length to each face as a function of the angle."""
    tb, tt = -math.atan(xi * ty / tx), math.atan((1.0 - xi) * ty / tx)
    chord = {0: lambda th: xi * ty / -math.sin(th), 1: lambda th: tx / math.cos(th),
             2: lambda th: (1.0 - xi) * ty / math.sin(th)}
    span = {0: (-math.pi / 2, tb), 1: (tb, tt), 2: (tt, math.pi / 2)}
    return chord, span


def uncollided_rect(tx, ty):
    """P(exit through face f with no collision), uniform xi and cosine-law
    angle (density cos(th)/2 on (-pi/2, pi/2))."""
    def face_int(f):
        def inner(xi):
            chord, span = _faces(tx, ty, xi)
            g = lambda th: 0.5 * math.cos(th) * math.exp(-chord[f](th))
            return integrate.quad(g, *span[f], epsabs=1e-13, epsrel=1e-11, limit=200)[0]
        return integrate.quad(inner, 0.0, 1.0, epsabs=1e-12, epsrel=1e-10, limit=200)[0]
    return np.array([face_int(0), face_int(1), face_int(2)])


def mean_chord_rect(tx, ty):
    def inner(xi):
        chord, span = _faces(tx, ty, xi)
        return sum(integrate.quad(lambda th: 0.5 * math.cos(th) * chord[f](th), *span[f],
                                  epsabs=1e-13, epsrel=1e-11, limit=200)[0] for f in range(3))
    return integrate.quad(inner, 0.0, 1.0, epsabs=1e-12, epsrel=1e-10, limit=200)[0]


@pytest.mark.parametrize("tau,c,mode", [(0.7, 0.9, T.MODE_IMPLICIT), (3.0, 0.6, T.MODE_ANALOG)])
def test_equal_sides_is_the_square_walk(tau, c, mode):
    n = 5000
    xi, cs, sn = _entries(n, 301)
    ids = np.arange(n, dtype=np.uint64) + 17
    ev = np.full(n, 3, np.uint32)
    a = T.transmit(xi, cs, sn, np.full(n, tau), np.full(n, c), mode, 9, ids=ids, events=ev)
    b = T.transmit_rect(xi, cs, sn, np.full(n, tau), np.full(n, tau), np.full(n, c), mode, 9,
                        ids=ids, events=ev)
    for k in ("status", "face", "ncoll", "events"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("q", "ux", "uy", "s"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("tx,ty", [(2.0, 0.5), (0.5, 3.0)])
def test_uncollided_transmission_closed_form(tx, ty):
    # c = 0 analog: every collision absorbs, so each face's exit fraction is
    # its uncollided probability
    n = 200000
    r = _rect(n, tx, ty, 0.0, T.MODE_ANALOG)
    expect = uncollided_rect(tx, ty)
    for f in range(3):
        p = np.mean((r["status"] == 0) & (r["face"] == f))
        se = math.sqrt(max(expect[f] * (1 - expect[f]), 1e-12) / n)
        assert abs(p - expect[f]) < 4 * se + 1e-12, (f, p, expect[f])
    assert not np.any((r["status"] == 0) & (r["face"] == 3))


@pytest.mark.parametrize("tx,ty", [(2.0, 0.5), (0.5, 3.0)])
def test_mean_uncollided_chord(tx, ty):
    # implicit capture with c = 0: no flights, s is the straight chord
    n = 100000
    r = _rect(n, tx, ty, 0.0, T.MODE_IMPLICIT)
    assert np.all(r["ncoll"] == 0)
    expect = mean_chord_rect(tx, ty)
    assert abs(r["s"].mean() - expect) < 4 * r["s"].std() / math.sqrt(n)


def test_outcomes_partition_and_mirror_symmetry():
    n, tx, ty = 100000, 1.5, 0.8
    r = _rect(n, tx, ty, 0.9, T.MODE_ANALOG)
    out = r["status"] == 0
    assert np.all((r["status"] == 0) | (r["status"] == 1))
    assert np.all(r["face"][out] >= 0) and np.all(r["face"][~out] == -1)
    bottom, top = np.mean(out & (r["face"] == 0)), np.mean(out & (r["face"] == 2))
    assert abs(bottom - top) < 4 * math.sqrt((bottom + top) / n)
    assert np.all((r["q"][out] >= 0) & (r["q"][out] <= 1))


def test_implicit_law_depends_on_c_times_sides():
    # rate c in (tx, ty) is rate 1 in (c tx, c ty) with every length scaled by c
    n, c = 20000, 0.7
    xi, cs, sn = _entries(n, 302)
    a = T.transmit_rect(xi, cs, sn, np.full(n, 2.0), np.full(n, 1.2), np.full(n, c),
                        T.MODE_IMPLICIT, 4)
    b = T.transmit_rect(xi, cs, sn, np.full(n, 2.0 * c), np.full(n, 1.2 * c), np.full(n, 1.0),
                        T.MODE_IMPLICIT, 4)
    same = np.array_equal(a["face"], b["face"]) and np.array_equal(a["ncoll"], b["ncoll"])
    assert same
    assert np.allclose(b["s"], c * a["s"], rtol=1e-9, atol=1e-12)
    assert np.allclose(a["q"], b["q"], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("c", [0.0, 0.5, 0.99])
def test_mean_path_invariance_whole_boundary(c):
    # isotropic inflow over the whole boundary (each face in proportion to its
    # length, cosine law): the mean track length is pi A / P = pi tx ty / (2
    # (tx + ty)) for any scattering rate (implicit capture; Blanco-Fournier).
    # Entering a horizontal face is entering the left face of the cell turned
    # by a quarter, tx <-> ty.
    n, tx, ty = 200000, 2.5, 0.8
    xi, cs, sn = _entries(n, 305)
    vertical = np.random.default_rng(5).random(n) < ty / (tx + ty)
    w = np.where(vertical, tx, ty)
    h = np.where(vertical, ty, tx)
    r = T.transmit_rect(xi, cs, sn, w, h, np.full(n, c), T.MODE_IMPLICIT, 7)
    expect = math.pi * tx * ty / (2.0 * (tx + ty))
    assert abs(r["s"].mean() - expect) < 4 * r["s"].std() / math.sqrt(n), (r["s"].mean(), expect)


def test_training_pairs_round_trip_through_the_decode(tmp_path):
    # the aspect ratio is the sixth condition; targets decode back to the
    # rectangle walk's exits; equal sides give aspect 0 and the square walk
    from oracle import mlp
    n = 20000
    xi, cs, sn = _entries(n, 307)
    tx, c = synth.materials(n, 308)
    ty = tx * np.exp(np.random.default_rng(9).uniform(-2.0, 2.0, n))
    cond, y = T.training_pairs_rect(xi, cs, sn, tx, ty, c, 4)
    assert cond.shape == (6, n) and y.shape == (4, n)
    assert np.allclose(np.exp(cond[5]) * np.exp(cond[3]), ty.astype(np.float64), rtol=1e-6)
    r = T.transmit_rect(xi, cs, sn, tx, ty, c, T.MODE_IMPLICIT, 4)
    p = str(tmp_path / "w.bin")
    synth.write_weights(p, synth.kaiming_weights(1))
    d = mlp.decode(mlp.read_weights(p), y)
    assert np.array_equal(d["face"], r["face"])
    assert np.allclose(d["q"], r["q"], atol=1e-12)
    assert np.allclose(d["ux"], r["ux"], atol=1e-12) and np.allclose(d["uy"], r["uy"], atol=1e-12)
    assert np.allclose(d["s"], r["s"], rtol=1e-12)
    c2, y2 = T.training_pairs_rect(xi, cs, sn, tx, tx, c, 4)
    sq = T.transmit(xi, cs, sn, tx, c, T.MODE_IMPLICIT, 4)
    assert not c2[5].any()
    assert np.array_equal(y2[0], sq["face"] + sq["q"]) and np.array_equal(y2[3], np.log(sq["s"]))
