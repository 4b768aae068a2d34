"""Pins for the scattering-equivalent condition (cells outside the network's
training box are sampled at the in-box condition with the same scattering
thickness c tau, track lengths scaled by c' / c) and for the generators of the
paper's two benchmark problems (printed cross sections, stand-in layouts).

The map is exact for the implicit-capture walk: run at the equivalent
condition on the same counters it takes the same flights in a scaled cell, so
a solve whose stage 2 is the walk at equivalent conditions reproduces the
walk solve history by history."""
import numpy as np
import pytest

import synth
from oracle import transport as T

BOX = ((0.1, 1000.0), (0.5, 0.999))


def test_identity_inside_the_box():
    g = np.random.default_rng(1)
    tau = np.exp(g.uniform(np.log(0.1), np.log(1000.0), 1000))
    c = g.uniform(0.5, 0.999, 1000)
    tp, cp, ok = T.equivalent_condition(tau, c, *BOX)
    assert ok.all()
    assert np.array_equal(tp, tau) and np.array_equal(cp, c)


def test_same_scattering_thickness_inside_the_box():
    g = np.random.default_rng(2)
    tau = np.exp(g.uniform(np.log(1e-3), np.log(1e5), 20000))
    c = np.where(g.random(20000) < 0.05, 0.0, g.uniform(0.0, 1.0, 20000))
    tp, cp, ok = T.equivalent_condition(tau, c, *BOX)
    w = c * tau
    expect_ok = (w >= 0.5 * 0.1) & (w <= 0.999 * 1000.0) & (c > 0.0)
    # at the two ends of the range the test is decided by one rounding
    edge = np.isclose(w, 0.05, rtol=1e-12) | np.isclose(w, 999.0, rtol=1e-12)
    assert np.array_equal(ok[~edge], expect_ok[~edge])
    assert np.allclose(cp[ok] * tp[ok], w[ok], rtol=1e-14, atol=0.0)
    assert (tp[ok] >= 0.1).all() and (tp[ok] <= 1000.0).all()
    assert (cp[ok] >= 0.5).all() and (cp[ok] <= 0.999).all()
    # cells without an equivalent keep their own values
    assert np.array_equal(tp[~ok], tau[~ok]) and np.array_equal(cp[~ok], c[~ok])


@pytest.mark.parametrize("tau,c", [(0.058, 1.0), (1.16, 0.05), (0.0625, 1.0), (5000.0, 0.1)])
def test_walk_at_the_equivalent_condition(tau, c):
    # same counters: same exits, track length scaled by c' / c
    n = 20000
    e = synth.cell_entries(n, 601)
    xi, cs, sn = (e[k].astype(np.float64) for k in ("xi", "cos", "sin"))
    tp, cp, ok = T.equivalent_condition(np.full(n, tau), np.full(n, c), *BOX)
    assert ok.all() and (tp != tau).all()
    a = T.transmit(xi, cs, sn, np.full(n, tau), np.full(n, c), T.MODE_IMPLICIT, 5)
    b = T.transmit(xi, cs, sn, tp, cp, T.MODE_IMPLICIT, 5)
    assert np.array_equal(a["face"], b["face"])
    assert np.array_equal(a["ncoll"], b["ncoll"])
    assert np.allclose(a["q"], b["q"], atol=1e-9)
    assert np.allclose(a["ux"], b["ux"], atol=1e-12) and np.allclose(a["uy"], b["uy"], atol=1e-12)
    assert np.allclose(a["s"], b["s"] * cp / c, rtol=1e-9)


def test_sampler_routes_cells_without_an_equivalent_to_the_fallback():
    n = 400
    e = synth.cell_entries(n, 602)
    xi, cs, sn = (e[k].astype(np.float64) for k in ("xi", "cos", "sin"))
    tau = np.where(np.arange(n) % 2 == 0, 0.625, 3.0)
    c = np.where(np.arange(n) % 2 == 0, 0.05, 0.7)  # c tau = 0.031 has no equivalent
    ids = np.arange(n, dtype=np.uint64)
    ev = np.zeros(n, np.uint32)
    calls = []

    def tagged(tag):
        def f(xi, cos_c, sin_c, tau, c, ids, events, rot=None):
            calls.append((tag, tau.copy(), c.copy()))
            return (np.zeros(len(xi), np.int64), xi, cos_c, sin_c, np.ones(len(xi)),
                    events + 1)
        return f

    f = T.equivalent_sampler(tagged("net"), tagged("walk"), *BOX)
    face, q, ux, uy, s, out_ev = f(xi, cs, sn, tau, c, ids, ev)
    by = {t: (a, b) for t, a, b in calls}
    assert np.allclose(by["walk"][0], 0.625) and np.allclose(by["walk"][1], 0.05)
    assert np.allclose(by["net"][0], 3.0) and np.allclose(by["net"][1], 0.7)
    assert np.array_equal(q, xi) and np.array_equal(out_ev, ev + 1)


def test_walk_solve_at_equivalent_conditions_is_the_walk_solve_hohlraum():
    tau, c, wall = synth.paper_hohlraum_problem(16)
    assert (c < 0.5).any() and (tau * c < 1.0).any()
    w = T.walk_sampler(7)
    a, sa = T.solve_gmc(tau, c, None, 600, 7, w, wall=wall)
    b, sb = T.solve_gmc(tau, c, None, 600, 7, T.equivalent_sampler(w, w, *BOX), wall=wall)
    np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-15)
    assert sa["transmissions"] == sb["transmissions"]


def test_walk_solve_at_equivalent_conditions_is_the_walk_solve_lattice():
    tau, c, src = synth.paper_lattice_problem(14)
    w = T.walk_sampler(8)
    a, sa = T.solve_gmc(tau, c, src, 600, 8, w)
    b, sb = T.solve_gmc(tau, c, src, 600, 8, T.equivalent_sampler(w, w, *BOX))
    np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-15)
    assert sa["transmissions"] == sb["transmissions"]


def test_paper_lattice_layout():
    n = 112
    tau, c, src = synth.paper_lattice_problem(n)
    h = 7.0 / n
    ab = c < 0.5
    # printed cross sections: background sigma_t 1, c 1; absorbers sigma_t 10, c 0.05
    assert np.allclose(tau[~ab], 1.0 * h) and np.allclose(c[~ab], 1.0)
    assert np.allclose(tau[ab], 10.0 * h) and np.allclose(c[ab], 0.05)
    assert ab.sum() == 12 * 16 * 16
    assert abs(src.sum() - 1.0) < 1e-6 and (src > 0).sum() == 16 * 16
    assert not (ab & (src > 0)).any()
    for k in range(4):
        r = np.rot90(ab, k)
        assert np.array_equal(r, ab) and np.array_equal(r.T, ab)
    with pytest.raises(ValueError):
        synth.paper_lattice_problem(100)


def test_paper_hohlraum_layout():
    n = 112
    tau, c, wall = synth.paper_hohlraum_problem(n)
    h = 1.3 / n
    assert len(synth.PAPER_HOHLRAUM_XS) == 5
    for name, (sa, ss) in synth.PAPER_HOHLRAUM_XS.items():
        m = np.isclose(c, ss / (sa + ss))
        assert m.any(), name
        assert np.allclose(tau[m], (sa + ss) * h), name
    assert np.array_equal(c, c[::-1]) and np.array_equal(tau, tau[::-1])
    assert wall.shape == (n,) and (wall == 1.0).all()


def test_generators_carry_the_printed_cross_sections():
    # tests/golden/paper_benchmark_cross_sections.txt holds the printed values
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_benchmark_cross_sections.txt")
    rows = []
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            prob, region, sa, ss, side, mesh = line.split()
            rows.append((prob, region, float(sa), float(ss), float(side), int(mesh)))
    assert len(rows) == 7
    tables = {"lattice": synth.LATTICE_XS, "hohlraum": synth.PAPER_HOHLRAUM_XS}
    gens = {"lattice": synth.paper_lattice_problem, "hohlraum": synth.paper_hohlraum_problem}
    for prob, region, sa, ss, side, mesh in rows:
        assert tables[prob][region] == (sa, ss), (prob, region)
        tau, c = gens[prob](mesh)[:2]
        st = sa + ss
        m = np.isclose(tau, st * side / mesh, rtol=1e-6) & np.isclose(c, ss / st, rtol=1e-6)
        assert m.any(), (prob, region)
    for prob, table in tables.items():
        assert set(table) == {r for p, r, *_ in rows if p == prob}


def test_network_solve_at_equivalent_conditions_balances_weight(tmp_path):
    # the network (FP64 oracle, random weights) at equivalent conditions, the
    # walk where none exists: implicit capture keeps the weight balance exact
    # (deposited + leaked - roulette changes = histories) and the Eq. 7
    # tally equals the deposit over sigma_a, whatever the sampler returns
    from oracle import mlp
    p = str(tmp_path / "w.bin")
    synth.write_weights(p, synth.biased_weights(7))
    net = mlp.read_weights(p)
    tau, c, src = synth.paper_lattice_problem(7)  # absorbers c tau = 0.5
    tau[0, :3] = 0.02  # c tau = 0.02: no equivalent, walked
    n = 200
    f = T.equivalent_sampler(T.mlp_sampler(net, 2, "euler", 3), T.walk_sampler(3), *BOX)
    flux, st = T.solve_gmc(tau, c, src, n, 3, f, max_waves=5000)
    assert abs(st["absorbed"] + st["leak"] - st["roulette_net"] - n) < 1e-8 * n
    sig_a = (1.0 - c.astype(np.float64)) * tau.astype(np.float64)
    assert abs(np.sum(flux * sig_a) * n - st["absorbed"]) < 1e-8 * n
    assert st["transmissions"] > n


def test_births_at_equivalent_conditions_are_the_walked_births():
    # births walked from their birth point at the equivalent condition, on
    # the same counters, equal the births walked at the cell's own condition
    # (same exits, track lengths scaled by c' / c): a solve with them equals
    # the walk solve history by history; cells without an equivalent (c tau
    # below 0.05) take the fallback
    tau, c, src = synth.paper_lattice_problem(14)
    src = np.where(c < 0.5, 1.0, src).astype(np.float32)  # births in absorbers too
    src /= src.sum()
    tau[0, 0] = 0.02
    src[0, 0] = 0.05
    w = T.walk_sampler(9)
    wi = T.walk_internal_sampler(9)
    a, sa = T.solve_gmc(tau, c, src, 800, 9, w, internal=wi)
    b, sb = T.solve_gmc(tau, c, src, 800, 9, T.equivalent_sampler(w, w, *BOX),
                        internal=T.equivalent_internal_sampler(wi, wi, *BOX))
    np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-15)
    assert sa["transmissions"] == sb["transmissions"]


def test_internal_sampler_routes_cells_without_an_equivalent_to_the_fallback():
    n = 300
    X = np.linspace(0.1, 0.9, n)
    Y = X[::-1].copy()
    tau = np.where(np.arange(n) % 3 == 0, 0.2, 40.0)
    c = np.where(np.arange(n) % 3 == 0, 0.1, 1.0)   # c tau = 0.02 (none) and 40 (c' 0.999)
    calls = []

    def tagged(tag):
        def f(X, Y, tau, c, ids, u):
            calls.append((tag, tau.copy(), c.copy()))
            return (np.zeros(len(X), np.int64), X, Y, Y, np.ones(len(X)), np.ones(len(X), np.uint32))
        return f

    f = T.equivalent_internal_sampler(tagged("net"), tagged("walk"), *BOX)
    face, q, ux, uy, s, ev = f(X, Y, tau, c, np.arange(n, dtype=np.uint64), np.zeros(n))
    by = {t: (a, b) for t, a, b in calls}
    assert np.allclose(by["walk"][0], 0.2) and np.allclose(by["walk"][1], 0.1)
    assert np.allclose(by["net"][1], 0.999) and np.allclose(by["net"][0] * 0.999, 40.0)
    net_rows = np.arange(n) % 3 != 0
    assert np.allclose(s[net_rows], 0.999) and np.allclose(s[~net_rows], 1.0)
    assert np.array_equal(q, X)
