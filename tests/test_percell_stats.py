"""The per-cell statistical comparison used by the GPU solve tests
(tests/_oracle_pool.py), checked on the CPU with oracle solves on both
sides: independent seeds of the same solve pass; the same runs with one
cell's tally scaled by 1.2, or a transposed flux map, fail; the spawned
pool returns exactly what a direct call returns."""
import numpy as np
import pytest

import synth
from oracle import transport as OT
import _oracle_pool as P


def _grid():
    return synth.grid_problem(n=8, seed=31, tau_range=(0.1, 5.0), block=4, source=2)


@pytest.fixture(scope="module")
def runs():
    tau, c, src = _grid()
    tasks = [{"grid": (tau, c, src), "n": 3000, "seed": s, "sampler": ("walk_global",)}
             for s in range(100, 116)]
    return P.solve_many(tasks)


def test_pool_equals_direct_call(runs):
    tau, c, src = _grid()
    f, st = OT.solve_gmc(tau, c, src, 3000, 100, OT.walk_sampler_global(100))
    np.testing.assert_array_equal(runs[0][0], f)
    assert runs[0][1]["transmissions"] == st["transmissions"]


def test_same_law_passes_and_planted_errors_fail(runs):
    a = [f for f, _ in runs[:8]]
    b = [f for f, _ in runs[8:]]
    z = P.assert_per_cell(a, b)
    assert np.isfinite(z).all()
    # a wrong tally in one reached cell
    k = int(np.argmax(np.mean(b, 0)))
    bad = [f.copy() for f in b]
    for f in bad:
        f.flat[k] *= 1.2
    with pytest.raises(AssertionError):
        P.assert_per_cell(a, bad)
    # a transposed map (a swapped index) fails in many cells
    with pytest.raises(AssertionError):
        P.assert_per_cell(a, [f.T.copy() for f in b])


def test_unreached_cells():
    z = P.per_cell_z(np.zeros((3, 4)), np.zeros((3, 4)))
    assert np.all(z == 0)
    b = np.zeros((3, 4))
    b[:, 1] = 1.0
    z = P.per_cell_z(np.zeros((3, 4)), b)
    assert np.isinf(z[1]) and z[0] == 0
