"""Build and load the oracle's C part (``liboracle.so``) with gcc.

Test infrastructure only. The C sources under ``oracle/`` are plain C99 with
no architecture-specific flags, so they build the same on x86-64 and Arm.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["philox.c", "walk.c", "solve.c"]
_lock = threading.Lock()
_lib = None


def _stale():
    if not os.path.exists(_SO):
        return True
    t = os.path.getmtime(_SO)
    deps = _SOURCES + ["oracle.h"]
    return any(os.path.getmtime(os.path.join(_HERE, s)) > t for s in deps)


def build(force=False):
    """Compile liboracle.so if missing or older than its sources."""
    if not force and not _stale():
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-o", tmp]
    cmd += [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u64, i64, u32, i32, dbl = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_int32, ctypes.c_double)
            P = ctypes.c_void_p
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_philox_batch.argtypes = [u64, i64, u64, u32, u32, P]
            L.orc_normal_batch.argtypes = [u64, i64, u64, u32, u32, P]
            L.orc_normal_ids.argtypes = [u64, i64, P, P, u32, P]
            L.orc_uniform_ids.argtypes = [u64, i64, P, P, u32, P]
            L.orc_transmit_ids.argtypes = [i64, P, P, P, P, P, i32, u64, P, P,
                                           P, P, P, P, P, P, P, P]
            L.orc_transmit_batch.argtypes = [i64, P, P, P, P, P, i32, u64, u64, u32,
                                             P, P, P, P, P, P, P]
            L.orc_walk_one.argtypes = [dbl, dbl, i32, dbl, dbl, dbl, dbl, u64, u64, u32,
                                       P, P, P, P, P]
            L.orc_walk_one_rect.argtypes = [dbl, dbl, dbl, i32, dbl, dbl, dbl, dbl, u64, u64,
                                            u32, P, P, P, P, P]
            L.orc_walk_one_xy.argtypes = [dbl, dbl, i32, dbl, dbl, dbl, dbl, u64, u64, u32,
                                          P, P, P, P, P]
            L.orc_transmit_rect_ids.argtypes = [i64, P, P, P, P, P, P, i32, u64, P, P,
                                                P, P, P, P, P, P, P, P]
            L.orc_transmit_xy_ids.argtypes = [i64, P, P, P, P, P, P, P, i32, i32, u64, P, P,
                                              P, P, P, P, P, P, P, P, P]
            L.orc_solve_analog.argtypes = [i32, i32, P, P, P, i64, u64, dbl, dbl, P, P]
            L.orc_solve_analog.restype = i32
            _lib = L
    return _lib
