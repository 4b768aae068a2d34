"""Pins for the oracle's random walk in x-y geometry (the geometry variant in
which a cell is the cross-section of an infinite prism and directions are 3-D
unit vectors; the paper encodes a direction by its projection on the unit
disk). Kept on the circle, the walk is the rectangle walk draw for draw; the
mean 3-D track length of a cosine-law inflow is Cauchy's 4A/P at any
scattering ratio; a thin slab's uncollided transmission is 2 E3(tau) with mean
exit cosine E4/E3; the slab's rotation symmetry about its normal makes the
exit y and z direction components equally distributed (isotropy on the
sphere); collisions average c times the track length; implicit capture
depends on (c tx, c ty) only; training pairs decode back to the walk's
exits."""
import math

import numpy as np
import pytest
from scipy import special

import synth
from oracle import transport as T


def _xy(n, tx, ty, c, mode, seed=3, eseed=400, sphere=True):
    e = synth.cell_entries_xy(n, eseed)
    return T.transmit_xy(e["xi"], e["ux"], e["uy"], e["uz"], np.full(n, tx), np.full(n, ty),
                         np.full(n, c), mode, seed, sphere=sphere)


def _close(a, b, se, k=4.0):
    assert abs(a - b) < k * se + 1e-12, (a, b, se)


@pytest.mark.parametrize("tx,ty,c,mode", [(0.7, 0.7, 0.9, T.MODE_IMPLICIT),
                                          (3.0, 1.2, 0.6, T.MODE_ANALOG)])
def test_on_the_circle_is_the_rectangle_walk(tx, ty, c, mode):
    n = 5000
    e = synth.cell_entries(n, 401)
    xi, cs, sn = (e[k].astype(np.float64) for k in ("xi", "cos", "sin"))
    ids = np.arange(n, dtype=np.uint64) + 5
    ev = np.full(n, 2, np.uint32)
    a = T.transmit_rect(xi, cs, sn, np.full(n, tx), np.full(n, ty), np.full(n, c), mode, 11,
                        ids=ids, events=ev)
    b = T.transmit_xy(xi, cs, sn, np.zeros(n), np.full(n, tx), np.full(n, ty), np.full(n, c),
                      mode, 11, ids=ids, events=ev, sphere=False)
    for k in ("status", "face", "ncoll", "events", "q", "ux", "uy", "s"):
        assert np.array_equal(a[k], b[k]), k
    assert not b["uz"].any()


@pytest.mark.parametrize("tau", [0.5, 4.0])
@pytest.mark.parametrize("c", [0.0, 0.9])
def test_mean_track_length_square_prism(tau, c):
    # Cauchy (c = 0) and its extension to scattering walks: mean 3-D track of a
    # cosine-law inflow is 4 A / P; the four faces of the square are
    # equivalent, so entry through one of them gives tau.
    n = 200000
    r = _xy(n, tau, tau, c, T.MODE_IMPLICIT)
    _close(r["s"].mean(), tau, r["s"].std() / math.sqrt(n))


@pytest.mark.parametrize("c", [0.0, 0.95])
def test_mean_track_length_whole_boundary(c):
    # inflow over the whole boundary, each face in proportion to its length:
    # 4 A / P = 2 tx ty / (tx + ty); a horizontal face is the left face of the
    # cell turned by a quarter (tx <-> ty)
    n, tx, ty = 200000, 2.5, 0.8
    e = synth.cell_entries_xy(n, 402)
    vertical = np.random.default_rng(6).random(n) < ty / (tx + ty)
    w = np.where(vertical, tx, ty)
    h = np.where(vertical, ty, tx)
    r = T.transmit_xy(e["xi"], e["ux"], e["uy"], e["uz"], w, h, np.full(n, c),
                      T.MODE_IMPLICIT, 8)
    _close(r["s"].mean(), 2.0 * tx * ty / (tx + ty), r["s"].std() / math.sqrt(n))


@pytest.mark.parametrize("tx", [0.3, 1.5])
def test_slab_uncollided_transmission(tx):
    # a cell far taller than wide is a slab: with every collision absorbing
    # (c = 0, analog), the fraction leaving through the right face is
    # int_0^1 2 mu exp(-tx / mu) dmu = 2 E3(tx), and the exit cosine of those
    # particles averages E4(tx) / E3(tx)
    n = 400000
    r = _xy(n, tx, 1e6 * tx, 0.0, T.MODE_ANALOG)
    out = (r["status"] == 0) & (r["face"] == 1)
    p = out.mean()
    expect = 2.0 * special.expn(3, tx)
    _close(p, expect, math.sqrt(expect * (1 - expect) / n))
    mu = r["ux"][out]
    _close(mu.mean(), special.expn(4, tx) / special.expn(3, tx), mu.std() / math.sqrt(mu.size))
    # an uncollided exit keeps its entry length: tx / mu
    assert np.allclose(r["s"][out], tx / r["ux"][out], rtol=1e-12)


@pytest.mark.parametrize("tx", [2.0])
def test_slab_mean_track_and_rotation_symmetry(tx):
    # in a slab the inflow and the walk are symmetric under rotations about
    # the normal (x axis), so the exit y and z components share a law; the
    # mean track is 4 V / S = 2 tx per unit area; collisions average c s
    n, c = 200000, 0.95
    r = _xy(n, tx, 1e6 * tx, c, T.MODE_IMPLICIT)
    _close(r["s"].mean(), 2.0 * tx, r["s"].std() / math.sqrt(n))
    ok = r["status"] == 0
    assert ok.all()
    for f in (1, 3):
        m = r["face"] == f
        y2, z2 = r["uy"][m] ** 2, r["uz"][m] ** 2
        d = y2 - z2
        _close(d.mean(), 0.0, d.std() / math.sqrt(d.size))
        d4 = y2 * y2 - z2 * z2
        _close(d4.mean(), 0.0, d4.std() / math.sqrt(d4.size))
    k = r["ncoll"] - c * r["s"]
    _close(k.mean(), 0.0, k.std() / math.sqrt(n))


def test_exit_directions_unit_and_outward():
    n = 50000
    r = _xy(n, 1.7, 0.9, 0.8, T.MODE_IMPLICIT)
    norm = r["ux"] ** 2 + r["uy"] ** 2 + r["uz"] ** 2
    assert np.allclose(norm, 1.0, atol=1e-12)
    assert (np.hypot(r["ux"], r["uy"]) <= 1.0 + 1e-12).all()
    outward = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])[r["face"]]
    assert (r["ux"] * outward[:, 0] + r["uy"] * outward[:, 1] > 0.0).all()
    assert ((r["q"] >= 0.0) & (r["q"] <= 1.0)).all()


def test_top_bottom_mirror():
    n = 200000
    r = _xy(n, 1.3, 1.0, 0.9, T.MODE_IMPLICIT)
    pb, pt = np.mean(r["face"] == 0), np.mean(r["face"] == 2)
    _close(pb - pt, 0.0, math.sqrt((pb + pt) / n))


def test_implicit_law_depends_on_c_times_sides():
    # flights at rate c in a cell of sides (tx, ty) are flights at rate 1 in
    # one of sides (c tx, c ty): exits and c s agree
    n = 100000
    a = _xy(n, 2.0, 1.0, 0.9, T.MODE_IMPLICIT, seed=4, eseed=403)
    b = _xy(n, 1.8, 0.9, 1.0, T.MODE_IMPLICIT, seed=4, eseed=403)
    assert np.array_equal(a["face"], b["face"])
    assert np.array_equal(a["ncoll"], b["ncoll"])
    assert np.allclose(a["q"], b["q"], atol=1e-9)
    assert np.allclose(0.9 * a["s"], b["s"], rtol=1e-9)
    for k in ("ux", "uy", "uz"):
        assert np.allclose(a[k], b[k], atol=1e-12)


def test_training_pairs_round_trip_through_the_disk_decode(tmp_path):
    # targets encode the walk's exit; decoding them with identity statistics
    # gives the exit back (face, q, projected direction, s, |uz|)
    from oracle import mlp
    n = 20000
    e = synth.cell_entries_xy(n, 405)
    tau, c = synth.materials(n, 406)
    cond, y = T.training_pairs_xy(e["xi"], e["ux"], e["uy"], tau, c, 9)
    assert cond.shape == (5, n) and y.shape == (4, n)
    assert np.allclose(cond[3], np.log(tau.astype(np.float64)))
    r = T.transmit_xy(e["xi"], e["ux"], e["uy"], e["uz"], tau, tau, c, T.MODE_IMPLICIT, 9)
    p = str(tmp_path / "w.bin")
    synth.write_weights(p, synth.kaiming_weights(1))
    net = mlp.read_weights(p)
    d = mlp.decode_disk(net, y)
    assert np.array_equal(d["face"], r["face"])
    assert np.allclose(d["q"], r["q"], atol=1e-12)
    assert np.allclose(d["ux"], r["ux"], atol=1e-12) and np.allclose(d["uy"], r["uy"], atol=1e-12)
    assert np.allclose(d["uz"], np.abs(r["uz"]), atol=1e-6)
    assert np.allclose(d["s"], r["s"], rtol=1e-12)
    assert not d["inward"].any()
