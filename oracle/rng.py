"""Oracle wrappers over the C Philox4x32-10 (test infrastructure only).

Counter convention: ctr = (id_lo, id_hi, event, tag), key = (seed_lo, seed_hi);
uniform u = (x + 1) 2^-32 in (0, 1] as Eq. 4 requires; normals by Box-Muller
in FP64 (the Gaussian seeds z of Eq. 8).
"""
import numpy as np

from ._clib import lib

TAG_WALK = 1
TAG_NOISE = 2
TAG_ROULETTE = 3
TAG_BIRTH = 4


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr = 4 x u32, key = 2 x u32 -> 4 x u32."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def philox_batch(seed, n, id0=0, event=0, tag=0):
    """Raw u32 draws for ids id0..id0+n-1 at one (event, tag): array [n, 4]."""
    out = np.zeros((n, 4), dtype=np.uint32)
    lib().orc_philox_batch(seed, n, id0, event, tag, out.ctypes.data)
    return out


def u01(x):
    """(x + 1) / 2^32 in FP64."""
    return (np.asarray(x, dtype=np.float64) + 1.0) * (1.0 / 4294967296.0)


def normal_batch(seed, n, id0=0, event=0, tag=TAG_NOISE):
    """Four Box-Muller normals per id: array [4, n] (FP64)."""
    out = np.zeros((4, n), dtype=np.float64)
    lib().orc_normal_batch(seed, n, id0, event, tag, out.ctypes.data)
    return out


def normals_for(seed, ids, events, tag=TAG_NOISE):
    """Normals at per-particle (id, event) counters: array [4, n] (FP64)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    events = np.ascontiguousarray(events, dtype=np.uint32)
    out = np.zeros((4, ids.shape[0]), dtype=np.float64)
    lib().orc_normal_ids(seed, ids.shape[0], ids.ctypes.data, events.ctypes.data, tag,
                         out.ctypes.data)
    return out


def uniforms_for(seed, ids, events, tag):
    """Four uniforms per particle at (id, event, tag): array [4, n] (FP64)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    events = np.ascontiguousarray(events, dtype=np.uint32)
    out = np.zeros((4, ids.shape[0]), dtype=np.float64)
    lib().orc_uniform_ids(seed, ids.shape[0], ids.ctypes.data, events.ctypes.data, tag,
                          out.ctypes.data)
    return out
