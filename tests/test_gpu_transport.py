"""GPU transport_solve against the oracle solves.

Both sides draw every random number from the same Philox counters, so most
histories follow the same path; float-versus-double rounding can still flip
a decision. The GMC solves are compared cell by cell: K independent seeds on
each side, the GPU solve against the oracle's event loop driven by the same
network (the E4M3-quantized network for the FP8 path), a two-sample z per
cell from the run-to-run spread, |z| <= 4 in at least 99 % of the cells and
<= 6 in all; the analog solves also against the oracle's closed forms.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import transport as OT

import _oracle_pool as P

pytestmark = pytest.mark.gpu


def _solve(ctx, tau, c, src, n, method, seed):
    import paper_2512_13965_gb300 as g
    ny, nx = tau.shape
    flux = np.zeros(ny * nx, dtype=np.float64)
    st = g.transport_solve(ctx, nx, ny, np.ascontiguousarray(tau, np.float32).ravel(),
                           np.ascontiguousarray(c, np.float32).ravel(),
                           np.ascontiguousarray(src, np.float32).ravel(), n, method, seed, flux)
    return flux.reshape(ny, nx), st.as_dict()


def _set(ctx, **kw):
    import paper_2512_13965_gb300 as g
    cfg = g.gmc_get_config(ctx)
    for k, v in kw.items():
        setattr(cfg, k, v)
    g.gmc_set_config(ctx, cfg)


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_analog_solve_matches_oracle(gpu_ctx):
    import paper_2512_13965_gb300 as g
    _set(gpu_ctx, bank_capacity=1 << 14)
    tau, c, src = synth.grid_problem(n=16, seed=21, tau_range=(0.1, 20.0), block=4, source=4)
    n = 20000
    fg, sg = _solve(gpu_ctx, tau, c, src, n, g.GMC_METHOD_ANALOG, 5)
    fo, so = OT.solve_analog(tau, c, src, n, 5)
    assert _rel_l2(fg, fo) < 0.02
    assert abs(sg["leaked"] - so["leak"]) < 0.01 * n
    assert abs(sg["absorbed"] - so["absorbed"]) < 0.01 * n
    # implicit capture conserves weight up to the roulette's explicit changes
    assert abs(sg["absorbed"] + sg["leaked"] - sg["roulette_net"] - n) < 1e-4 * n
    assert sg["transmissions"] > n and sg["collisions"] > 0


def test_analog_solve_statistical(gpu_ctx):
    # independent seeds: the GPU mean over runs agrees with the oracle mean
    import paper_2512_13965_gb300 as g
    tau, c, src = synth.grid_problem(n=8, seed=23, tau_range=(0.1, 5.0), block=4, source=2)
    K, n = 6, 20000
    a = np.array([_solve(gpu_ctx, tau, c, src, n, g.GMC_METHOD_ANALOG, 100 + k)[0].ravel() for k in range(K)])
    b = np.array([OT.solve_analog(tau, c, src, n, 200 + k)[0].ravel() for k in range(K)])
    se = np.sqrt(a.var(0, ddof=1) / K + b.var(0, ddof=1) / K)
    z = (a.mean(0) - b.mean(0)) / np.where(se > 0, se, 1.0)
    assert np.max(np.abs(z)) < 4.5


def test_single_cell_pure_absorber(gpu_ctx):
    import paper_2512_13965_gb300 as g
    from tests.test_oracle_solve import escape_expectation
    _set(gpu_ctx, w_cut=0.0)
    tau = 2.0
    runs = [_solve(gpu_ctx, np.full((1, 1), tau), np.zeros((1, 1)), np.ones((1, 1)), 50000,
                   g.GMC_METHOD_ANALOG, 300 + k)[0][0, 0] for k in range(8)]
    _set(gpu_ctx, w_cut=1e-4)
    e = escape_expectation(tau)
    runs = np.array(runs)
    assert abs(runs.mean() - (1 - e) / tau) < 4 * runs.std(ddof=1) / math.sqrt(len(runs))


@pytest.fixture(scope="module")
def kaiming_net(gpu_ctx, kaiming_file):
    import paper_2512_13965_gb300 as g
    g.gmc_load_weights(gpu_ctx, kaiming_file)
    return oracle.mlp.read_weights(kaiming_file)


K_RUNS = 8          # independent seeds per side
N_GPU = 20000       # histories per GPU run
N_ORACLE = 4000     # histories per oracle run


def _percell(ctx, tau, c, src, sampler, internal=None, wall=None, n_gpu=N_GPU, n_oracle=N_ORACLE):
    """K GPU solves and K oracle solves on independent seeds; per-cell check,
    then the per-history leakage and transmissions compared the same way."""
    import paper_2512_13965_gb300 as g
    gpu = []
    for k in range(K_RUNS):
        if wall is None:
            gpu.append(_solve(ctx, tau, c, src, n_gpu, g.GMC_METHOD_GMC, 1000 + k))
        else:
            gpu.append(_solve_wall(ctx, tau, c, wall, n_gpu, g.GMC_METHOD_GMC, 1000 + k))
    tasks = [{"grid": (tau, c, src), "n": n_oracle, "seed": 2000 + k, "sampler": sampler,
              "internal": internal, "wall": wall} for k in range(K_RUNS)]
    orc = P.solve_many(tasks)
    z = P.assert_per_cell([f for f, _ in gpu], [f for f, _ in orc])
    for kg, ko, n_o in (("leaked", "leak", n_oracle), ("transmissions", "transmissions", n_oracle)):
        a = [[st[kg] / n_gpu] for _, st in gpu]
        b = [[st[ko] / n_o] for _, st in orc]
        assert abs(P.per_cell_z(a, b)[0]) <= 4.0, kg
    for _, st in gpu:
        # implicit capture conserves weight up to the roulette's explicit changes
        assert abs(st["absorbed"] + st["leaked"] - st["roulette_net"] - n_gpu) < 1e-4 * n_gpu
    return z, gpu, orc


def _grid16(seed, hi=5.0):
    return synth.grid_problem(n=16, seed=seed, tau_range=(0.1, hi), block=4, source=4)


def test_gmc_solve_fp32_per_cell(gpu_ctx, kaiming_net, kaiming_file):
    import paper_2512_13965_gb300 as g
    _set(gpu_ctx, precision=g.GMC_FP32, steps=4, integrator=g.GMC_EULER, bank_capacity=1 << 16)
    tau, c, src = _grid16(31)
    _percell(gpu_ctx, tau, c, src, ("mlp", kaiming_file, 4, "euler"))
    # on the same counters the FP32 solve follows the oracle's histories
    # nearly one for one: the flux maps agree closely as a whole too
    fg, _ = _solve(gpu_ctx, tau, c, src, 3000, g.GMC_METHOD_GMC, 9)
    fo, _ = OT.solve_gmc(tau, c, src, 3000, 9, OT.mlp_sampler(kaiming_net, 4, "euler", 9))
    assert _rel_l2(fg, fo) < 0.03


def test_gmc_solve_bf16_per_cell(gpu_ctx, kaiming_net, kaiming_file):
    # the BF16 tensor-core sampler against the FP64 network's event loop
    import paper_2512_13965_gb300 as g
    _set(gpu_ctx, precision=g.GMC_BF16, steps=4, integrator=g.GMC_EULER, bank_capacity=1 << 16)
    tau, c, src = _grid16(33, hi=20.0)
    _percell(gpu_ctx, tau, c, src, ("mlp", kaiming_file, 4, "euler"))


def test_gmc_solve_fp8_per_cell(gpu_ctx, kaiming_net, kaiming_file):
    # the FP8 sampler against the event loop of the E4M3-quantized network
    import paper_2512_13965_gb300 as g
    _set(gpu_ctx, precision=g.GMC_FP8, steps=4, integrator=g.GMC_MIDPOINT, bank_capacity=1 << 16)
    tau, c, src = _grid16(35, hi=20.0)
    _percell(gpu_ctx, tau, c, src, ("mlp_e4m3", kaiming_file, 4, "midpoint"))
    _set(gpu_ctx, integrator=g.GMC_EULER)


BOX = ((0.1, 1000.0), (0.5, 0.999))


def _outside_box_grid(n=16, seed=39):
    # cells on both sides of the training box: thin and thick, c from pure
    # scatterers (c = 1) to strong absorbers (c = 0.05), and a few cells whose
    # scattering thickness c tau has no equivalent (walked)
    g = synth.generator(seed)
    tau = np.exp(g.uniform(np.log(0.02), np.log(30.0), (n, n)))
    c = g.choice([0.05, 0.3, 0.7, 0.95, 1.0], size=(n, n))
    src = np.zeros((n, n))
    src[n // 2 - 2:n // 2 + 2, n // 2 - 2:n // 2 + 2] = 1.0
    src /= src.sum()
    return tau.astype(np.float32), c.astype(np.float32), src.astype(np.float32)


def test_equivalent_condition_solve_per_cell(gpu_ctx, kaiming_net, kaiming_file):
    # cells outside the training box sampled at their scattering-equivalent
    # condition (track length times c'/c), cells without one walked: against
    # the oracle's event loop with the same reading (oracle.transport
    # .equivalent_sampler, the walk in the cell's own frame as fallback)
    import paper_2512_13965_gb300 as g
    tau, c, src = _outside_box_grid()
    tp, cp, ok = OT.equivalent_condition(tau, c, *BOX)
    inside = (tau >= 0.1) & (tau <= 1000.0) & (c >= 0.5) & (c <= 0.999)
    assert (~ok).sum() >= 3 and (ok & ~inside).sum() > 0.3 * tau.size
    _set(gpu_ctx, precision=g.GMC_FP32, steps=4, integrator=g.GMC_EULER, bank_capacity=1 << 16)
    _, gpu, _ = _percell(gpu_ctx, tau, c, src, ("equivalent", kaiming_file, 4, "euler", BOX))
    assert all(st["collisions"] > 0 for _, st in gpu)  # the cells without an equivalent were walked


def test_solve_edge_cases(gpu_ctx, kaiming_net):
    import paper_2512_13965_gb300 as g
    tau, c, src = synth.grid_problem(n=4, seed=41, tau_range=(0.5, 2.0), block=2, source=2)
    f, st = _solve(gpu_ctx, tau, c, src, 0, g.GMC_METHOD_ANALOG, 1)
    assert np.all(f == 0) and st["transmissions"] == 0
    with pytest.raises(g.GMCError) as e:
        _solve(gpu_ctx, tau, c, np.zeros_like(src), 10, g.GMC_METHOD_ANALOG, 1)
    assert e.value.status == g.GMC_EINVAL
    bad = tau.copy()
    bad[0, 0] = -1.0
    with pytest.raises(g.GMCError):
        _solve(gpu_ctx, bad, c, src, 10, g.GMC_METHOD_ANALOG, 1)
    fresh = g.Context(0)
    with pytest.raises(g.GMCError) as e:
        _solve(fresh, tau, c, src, 10, g.GMC_METHOD_GMC, 1)
    assert e.value.status == g.GMC_ENOWEIGHTS
    fresh.close()
    # a particle bank smaller than the history count refills across waves
    _set(gpu_ctx, bank_capacity=1024, precision=g.GMC_BF16, steps=4)
    f1, s1 = _solve(gpu_ctx, tau, c, src, 5000, g.GMC_METHOD_GMC, 3)
    _set(gpu_ctx, bank_capacity=1 << 16)
    f2, s2 = _solve(gpu_ctx, tau, c, src, 5000, g.GMC_METHOD_GMC, 3)
    # per-history results do not depend on the bank size (counter-based RNG;
    # BF16 rows are independent) up to FP64 summation order
    np.testing.assert_allclose(f1, f2, rtol=1e-9, atol=1e-12)
    assert s1["transmissions"] == s2["transmissions"]


@pytest.mark.parametrize("method", ["analog", "gmc"])
def test_flight_cap_changes_no_result(gpu_ctx, kaiming_net, method):
    # Walks cut at flights_per_wave resume with the same random numbers, so the
    # flux is the same for any cap up to the order of the FP64 tally additions;
    # thick cells (FP64 positions) and thin ones both appear.
    import paper_2512_13965_gb300 as g
    m = g.GMC_METHOD_ANALOG if method == "analog" else g.GMC_METHOD_GMC
    tau, c, src = synth.grid_problem(n=12, seed=33, tau_range=(0.1, 300.0), block=4, source=4)
    out = []
    for cap in (1 << 20, 512, 3):
        _set(gpu_ctx, bank_capacity=1 << 14, flights_per_wave=cap, precision=g.GMC_FP32, steps=4)
        f, st = _solve(gpu_ctx, tau, c, src, 3000, m, 17)
        out.append((f, st))
    _set(gpu_ctx, flights_per_wave=512)
    f0, s0 = out[0]
    for f, st in out[1:]:
        np.testing.assert_allclose(f, f0, rtol=1e-9, atol=1e-12 * np.abs(f0).max())
        assert st["transmissions"] == s0["transmissions"]
        assert st["collisions"] == s0["collisions"]
        assert st["roulette_kills"] == s0["roulette_kills"]
    assert out[2][1]["waves"] > out[0][1]["waves"]  # the cap did cut walks


def test_hybrid_all_thin_equals_analog(gpu_ctx, kaiming_net):
    # gmc_min_tau above every cell: a GMC solve walks every cell, drawing the
    # same random numbers as the analog solve, so the two agree history by
    # history (up to the order of the FP64 tally additions)
    import paper_2512_13965_gb300 as g
    tau, c, src = synth.grid_problem(n=12, seed=35, tau_range=(0.1, 120.0), block=4, source=4)
    _set(gpu_ctx, bank_capacity=1 << 14, precision=g.GMC_FP32, steps=4, gmc_min_tau=0.0)
    fa, sa = _solve(gpu_ctx, tau, c, src, 4000, g.GMC_METHOD_ANALOG, 23)
    _set(gpu_ctx, gmc_min_tau=1e30)
    fh, sh = _solve(gpu_ctx, tau, c, src, 4000, g.GMC_METHOD_GMC, 23)
    _set(gpu_ctx, gmc_min_tau=0.0)
    np.testing.assert_allclose(fh, fa, rtol=1e-9, atol=1e-12 * np.abs(fa).max())
    for k in ("transmissions", "collisions", "roulette_kills"):
        assert sh[k] == sa[k], k


def test_hybrid_solve_per_cell(gpu_ctx, kaiming_net, kaiming_file):
    # cells thinner than 2 walked, thicker ones sampled (FP32 network)
    import paper_2512_13965_gb300 as g
    _set(gpu_ctx, precision=g.GMC_FP32, steps=4, integrator=g.GMC_EULER, bank_capacity=1 << 16,
         gmc_min_tau=2.0)
    tau, c, src = _grid16(37, hi=8.0)
    try:
        _, gpu, _ = _percell(gpu_ctx, tau, c, src, ("hybrid", kaiming_file, 4, 2.0))
    finally:
        _set(gpu_ctx, gmc_min_tau=0.0)
    assert all(st["collisions"] > 0 for _, st in gpu)


# --- surface source on the left boundary (transport_solve_wall) --------------

def _solve_wall(ctx, tau, c, wall, n, method, seed):
    import paper_2512_13965_gb300 as g
    ny, nx = tau.shape
    flux = np.zeros(ny * nx, dtype=np.float64)
    st = g.transport_solve_wall(ctx, nx, ny, np.ascontiguousarray(tau, np.float32).ravel(),
                                np.ascontiguousarray(c, np.float32).ravel(),
                                np.ascontiguousarray(wall, np.float32), n, method, seed, flux)
    return flux.reshape(ny, nx), st.as_dict()


def _wall_strengths(ny, seed):
    w = synth.generator(seed).uniform(0.0, 1.0, ny).astype(np.float32)
    w[: ny // 4] = 0.0  # part of the wall does not emit
    return w


def test_wall_analog_solve_matches_oracle(gpu_ctx):
    import paper_2512_13965_gb300 as g
    _set(gpu_ctx, bank_capacity=1 << 14)
    tau, c, _ = synth.grid_problem(n=8, seed=41, tau_range=(0.1, 5.0), block=4, source=2)
    wall = _wall_strengths(8, 42)
    n = 8000
    fg, sg = _solve_wall(gpu_ctx, tau, c, wall, n, g.GMC_METHOD_ANALOG, 6)
    fo, so = OT.solve_gmc(tau, c, None, n, 6, OT.walk_sampler_global(6), wall=wall)
    assert _rel_l2(fg, fo) < 0.02
    assert abs(sg["leaked"] - so["leak"]) < 0.01 * n
    assert abs(sg["transmissions"] - so["transmissions"]) < 0.01 * so["transmissions"]
    assert abs(sg["absorbed"] + sg["leaked"] - sg["roulette_net"] - n) < 1e-4 * n
    # rows of the first column that do not emit still see flux from their neighbours,
    # and the flux falls away from the wall on average
    assert fg[:, 0].mean() > fg[:, -1].mean()


def test_wall_gmc_solve_fp32_per_cell(gpu_ctx, kaiming_net, kaiming_file):
    import paper_2512_13965_gb300 as g
    _set(gpu_ctx, precision=g.GMC_FP32, steps=4, integrator=g.GMC_EULER, bank_capacity=1 << 16)
    tau, c, _ = _grid16(43)
    wall = _wall_strengths(16, 44)
    _percell(gpu_ctx, tau, c, None, ("mlp", kaiming_file, 4, "euler"), wall=wall)


@pytest.mark.parametrize("tau,c", [(0.5, 0.0), (2.0, 0.0), (3.0, 1.0)])
def test_wall_single_cell_closed_forms(gpu_ctx, tau, c):
    # one cell lit from the left: pure absorber (c = 0) -> (1 - P_unc) / tau,
    # pure scatterer (c = 1) -> pi / 4 (mean path pi tau / 4 of a Lambertian
    # inflow); the spread per history comes from the oracle's walks
    import paper_2512_13965_gb300 as g
    from test_oracle_walk import uncollided_by_face
    _set(gpu_ctx, bank_capacity=1 << 16)
    n = 1 << 18
    f, st = _solve_wall(gpu_ctx, np.full((1, 1), tau), np.full((1, 1), c), [1.0], n,
                        g.GMC_METHOD_ANALOG, 8)
    j, xi, gx, gy = OT.wall_births([1.0], 4000, 9)
    r = OT.transmit(xi, gx, gy, np.full(4000, tau), np.full(4000, c), OT.MODE_IMPLICIT, 9,
                    ids=np.arange(4000, dtype=np.uint64), events=np.zeros(4000, np.uint32))
    per = (r["s"] / tau) if c == 1.0 else (-np.expm1(-r["s"]) / tau)
    expect = math.pi / 4 if c == 1.0 else (1.0 - uncollided_by_face(tau).sum()) / tau
    assert abs(f[0, 0] - expect) < 4 * per.std() / math.sqrt(n) + 1e-6
    if c == 1.0:
        assert st["absorbed"] == 0.0 and abs(st["leaked"] - n) < 1e-6 * n


def test_wall_source_errors(gpu_ctx):
    import paper_2512_13965_gb300 as g
    tau = np.ones((2, 2), np.float32)
    with pytest.raises(g.GMCError) as e:
        _solve_wall(gpu_ctx, tau, np.full((2, 2), 0.9, np.float32), [0.0, 0.0], 10,
                    g.GMC_METHOD_ANALOG, 1)
    assert e.value.status == g.GMC_EINVAL
    with pytest.raises(g.GMCError) as e:
        _solve_wall(gpu_ctx, tau, np.full((2, 2), 0.9, np.float32), [1.0, float("nan")], 10,
                    g.GMC_METHOD_ANALOG, 1)
    assert e.value.status == g.GMC_EINVAL
