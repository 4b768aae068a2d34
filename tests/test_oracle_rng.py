"""Pins for the oracle's Philox4x32-10, uniforms and normals."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("|")
        a = [int(x, 16) for x in lhs.split()]
        rows.append((a[:4], a[4:6], [int(x, 16) for x in rhs.split()]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(rng.philox4x32_10(ctr, key)) == expect


def test_counter_convention():
    # ctr = (id_lo, id_hi, event, tag), key = (seed_lo, seed_hi)
    seed, pid, ev, tag = 0x0123456789ABCDEF, 0xFEDCBA9876543210, 7, 3
    a = rng.philox_batch(seed, 1, id0=pid, event=ev, tag=tag)[0]
    b = rng.philox4x32_10([pid & 0xFFFFFFFF, pid >> 32, ev, tag], [seed & 0xFFFFFFFF, seed >> 32])
    assert list(a) == list(b)


def test_uniform_range_and_chi2():
    raw = rng.philox_batch(5, 1 << 16)
    u = rng.u01(raw).ravel()
    assert u.min() > 0.0 and u.max() <= 1.0
    assert rng.u01(np.uint32(0xFFFFFFFF)) == 1.0
    assert rng.u01(np.uint32(0)) == 2.0 ** -32
    counts, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = stats.chisquare(counts)
    assert chi2.pvalue > 1e-4


def test_normals_gaussian():
    z = rng.normal_batch(11, 1 << 15)
    for k in range(4):
        assert stats.kstest(z[k], "norm").pvalue > 1e-4
    # the pair (z0, z1) from one Box-Muller draw is uncorrelated
    assert abs(np.corrcoef(z[0], z[1])[0, 1]) < 4.0 / np.sqrt(z.shape[1])


def test_normals_for_matches_batch():
    ids = np.arange(100, 140, dtype=np.uint64)
    ev = np.full(40, 9, dtype=np.uint32)
    a = rng.normals_for(3, ids, ev, rng.TAG_NOISE)
    b = rng.normal_batch(3, 40, id0=100, event=9, tag=rng.TAG_NOISE)
    np.testing.assert_array_equal(a, b)
