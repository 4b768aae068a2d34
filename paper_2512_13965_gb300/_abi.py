"""ctypes binding of libgmc.so (include/gmc.h): argument marshalling only.

Every function has the C name and argument order. Array arguments may be
torch tensors (CUDA tensors pass device pointers, CPU tensors host pointers)
or numpy arrays (host pointers); they must be contiguous and of the C type
the header names. Nothing here computes any step of the method: when the
library is missing the import fails, there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgmc.so")

GMC_OK, GMC_EINVAL, GMC_ENOMEM, GMC_ECUDA, GMC_ETIMEOUT = 0, -1, -2, -3, -4
GMC_EFORMAT, GMC_ENOTIMPL, GMC_EBUSY, GMC_ENOWEIGHTS, GMC_EIO = -5, -6, -7, -8, -9
GMC_FP32, GMC_BF16, GMC_FP8 = 0, 1, 2
GMC_EULER, GMC_MIDPOINT, GMC_RK4 = 0, 1, 2
GMC_ABSORB_ANALOG, GMC_ABSORB_IMPLICIT = 0, 1
GMC_METHOD_ANALOG, GMC_METHOD_GMC = 0, 1


class gmc_config(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("integrator", ctypes.c_int), ("precision", ctypes.c_int),
                ("w_cut", ctypes.c_double), ("p_survive", ctypes.c_double),
                ("bank_capacity", ctypes.c_int64), ("flights_per_wave", ctypes.c_int),
                ("gmc_min_tau", ctypes.c_double)]


class gmc_solve_stats(ctypes.Structure):
    _fields_ = [("leaked", ctypes.c_double), ("absorbed", ctypes.c_double),
                ("roulette_net", ctypes.c_double), ("transmissions", ctypes.c_int64),
                ("collisions", ctypes.c_int64), ("roulette_kills", ctypes.c_int64),
                ("waves", ctypes.c_int64), ("inward_fixes", ctypes.c_int64),
                ("seconds", ctypes.c_double), ("latency", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gmc_solve_req(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("source", ctypes.c_void_p),
                ("n_histories", ctypes.c_int64), ("seed", ctypes.c_uint64)]


class gmc_serve_config(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("memory_budget", ctypes.c_size_t)]


class gmc_train_config(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("weight_decay", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int)]


class GMCError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (status_name(status), message))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgmc.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, i64, u64, u32, i32, sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t)
    sig = {
        "gmc_create": [ctypes.POINTER(ctypes.c_void_p), i32],
        "gmc_destroy": [P],
        "gmc_set_stream": [P, P],
        "gmc_synchronize": [P],
        "gmc_get_config": [P, ctypes.POINTER(gmc_config)],
        "gmc_set_config": [P, ctypes.POINTER(gmc_config)],
        "gmc_philox": [P, i64, u64, u64, u32, u32, P],
        "gmc_normals": [P, i64, u64, u64, u32, u32, P],
        "gmc_load_weights": [P, ctypes.c_char_p],
        "gmc_load_weights_buffer": [P, P, sz],
        "gmc_load_internal_weights": [P, ctypes.c_char_p],
        "gmc_load_internal_weights_buffer": [P, P, sz],
        "gmc_sample_internal": [P, i64, P, P, u64, u64, i32, i32, i32, P, P],
        "gmc_transmit": [P, i64, P, P, u64, u64, i32, i32, i32, P, P],
        "gmc_transmit_noalloc": [P, i64, P, P, u64, u64, i32, i32, P, P],
        "analog_transmit": [P, i64, P, P, P, P, P, i32, u64, u64, u32, P, P, P],
        "analog_transmit_rect": [P, i64, P, P, P, P, P, P, i32, u64, u64, u32, P, P, P],
        "analog_transmit_xy": [P, i64, P, P, P, P, P, P, i32, u64, u64, u32, P, P, P],
        "transport_solve": [P, i32, i32, P, P, P, i64, i32, u64, P,
                            ctypes.POINTER(gmc_solve_stats)],
        "transport_solve_wall": [P, i32, i32, P, P, P, i64, i32, u64, P,
                                 ctypes.POINTER(gmc_solve_stats)],
        "gmc_serve_start": [P, ctypes.POINTER(gmc_serve_config)],
        "gmc_submit": [P, ctypes.POINTER(gmc_solve_req), ctypes.POINTER(ctypes.c_uint64)],
        "gmc_poll": [P, u64, P, ctypes.POINTER(gmc_solve_stats)],
        "gmc_wait": [P, u64, ctypes.c_double, P, ctypes.POINTER(gmc_solve_stats)],
        "gmc_serve_stop": [P],
        "gmc_train_data": [P, i64, u64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, P, P],
        "gmc_train_data_internal": [P, i64, u64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, P, P],
        "gmc_train_begin": [P, i64, P, P, ctypes.POINTER(gmc_train_config)],
        "gmc_train_steps": [P, i64, P],
        "gmc_train_set_lr": [P, ctypes.c_double],
        "gmc_train_grad": [P, i64, P, P, P, P, P, P],
        "gmc_train_params": [P, P],
        "gmc_train_commit": [P, ctypes.c_char_p],
        "gmc_selftest_wait": [P, ctypes.c_double],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.gmc_train_param_count.argtypes = []
    L.gmc_train_param_count.restype = ctypes.c_int64
    L.gmc_status_str.argtypes = [ctypes.c_int]
    L.gmc_status_str.restype = ctypes.c_char_p
    L.gmc_last_error.argtypes = [P]
    L.gmc_last_error.restype = ctypes.c_char_p
    return L


lib = _load()


def status_name(s):
    return lib.gmc_status_str(int(s)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array arguments must be C-contiguous")
        return x.ctypes.data
    raise TypeError("unsupported array argument %r" % type(x))


class Context:
    """Owns one gmc_ctx* (gmc_create / gmc_destroy)."""

    def __init__(self, device=0):
        h = ctypes.c_void_p()
        s = lib.gmc_create(ctypes.byref(h), int(device))
        if s != GMC_OK:
            raise GMCError(s, "gmc_create(device=%d) failed" % device)
        self.handle = h

    def check(self, s):
        if s != GMC_OK:
            raise GMCError(s, lib.gmc_last_error(self.handle).decode())
        return s

    def close(self):
        if self.handle:
            lib.gmc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.handle


def gmc_create(device=0):
    return Context(device)


def gmc_destroy(ctx):
    ctx.close()


def gmc_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    return ctx.check(lib.gmc_set_stream(ctx.handle, raw))


def gmc_synchronize(ctx):
    return ctx.check(lib.gmc_synchronize(ctx.handle))


def gmc_get_config(ctx):
    c = gmc_config()
    ctx.check(lib.gmc_get_config(ctx.handle, ctypes.byref(c)))
    return c


def gmc_set_config(ctx, cfg):
    return ctx.check(lib.gmc_set_config(ctx.handle, ctypes.byref(cfg)))


def gmc_philox(ctx, n, seed, id0, event, tag, out):
    return ctx.check(lib.gmc_philox(ctx.handle, n, seed, id0, event, tag, _ptr(out)))


def gmc_normals(ctx, n, seed, id0, event, tag, out):
    return ctx.check(lib.gmc_normals(ctx.handle, n, seed, id0, event, tag, _ptr(out)))


def gmc_load_weights(ctx, path):
    return ctx.check(lib.gmc_load_weights(ctx.handle, os.fsencode(path)))


def gmc_load_weights_buffer(ctx, blob):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    return ctx.check(lib.gmc_load_weights_buffer(ctx.handle, ctypes.addressof(buf), len(blob)))


def gmc_load_internal_weights(ctx, path):
    return ctx.check(lib.gmc_load_internal_weights(ctx.handle, os.fsencode(path)))


def gmc_load_internal_weights_buffer(ctx, blob):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    return ctx.check(lib.gmc_load_internal_weights_buffer(ctx.handle, ctypes.addressof(buf),
                                                          len(blob)))


def gmc_sample_internal(ctx, n, cond, noise, seed, id0, steps, integrator, precision, y_raw, exit):
    return ctx.check(lib.gmc_sample_internal(ctx.handle, n, _ptr(cond), _ptr(noise), seed, id0,
                                             steps, integrator, precision, _ptr(y_raw),
                                             _ptr(exit)))


def gmc_transmit(ctx, n, cond, noise, seed, id0, steps, integrator, precision, y_raw, exit):
    return ctx.check(lib.gmc_transmit(ctx.handle, n, _ptr(cond), _ptr(noise), seed, id0, steps,
                                      integrator, precision, _ptr(y_raw), _ptr(exit)))


def gmc_transmit_noalloc(ctx, n, cond, noise, seed, id0, steps, integrator, y_raw, exit):
    return ctx.check(lib.gmc_transmit_noalloc(ctx.handle, n, _ptr(cond), _ptr(noise), seed, id0,
                                              steps, integrator, _ptr(y_raw), _ptr(exit)))


def analog_transmit(ctx, n, xi, cos_in, sin_in, tau, c, mode, seed, id0, event0, status, exit,
                    ncoll=None):
    return ctx.check(lib.analog_transmit(ctx.handle, n, _ptr(xi), _ptr(cos_in), _ptr(sin_in),
                                         _ptr(tau), _ptr(c), mode, seed, id0, event0,
                                         _ptr(status), _ptr(exit), _ptr(ncoll)))


def analog_transmit_rect(ctx, n, xi, cos_in, sin_in, tau_x, tau_y, c, mode, seed, id0, event0,
                         status, exit, ncoll=None):
    return ctx.check(lib.analog_transmit_rect(ctx.handle, n, _ptr(xi), _ptr(cos_in), _ptr(sin_in),
                                              _ptr(tau_x), _ptr(tau_y), _ptr(c), mode, seed, id0,
                                              event0, _ptr(status), _ptr(exit), _ptr(ncoll)))


def analog_transmit_xy(ctx, n, xi, ux_in, uy_in, tau_x, tau_y, c, mode, seed, id0, event0,
                       status, exit, ncoll=None):
    return ctx.check(lib.analog_transmit_xy(ctx.handle, n, _ptr(xi), _ptr(ux_in), _ptr(uy_in),
                                            _ptr(tau_x), _ptr(tau_y), _ptr(c), mode, seed, id0,
                                            event0, _ptr(status), _ptr(exit), _ptr(ncoll)))


def transport_solve(ctx, nx, ny, tau, c, source, n_histories, method, seed, flux, stats=None):
    st = stats if stats is not None else gmc_solve_stats()
    ctx.check(lib.transport_solve(ctx.handle, nx, ny, _ptr(tau), _ptr(c), _ptr(source),
                                  n_histories, method, seed, _ptr(flux), ctypes.byref(st)))
    return st


def transport_solve_wall(ctx, nx, ny, tau, c, wall, n_histories, method, seed, flux, stats=None):
    st = stats if stats is not None else gmc_solve_stats()
    ctx.check(lib.transport_solve_wall(ctx.handle, nx, ny, _ptr(tau), _ptr(c), _ptr(wall),
                                       n_histories, method, seed, _ptr(flux), ctypes.byref(st)))
    return st


def gmc_train_data(ctx, n, seed, tau_lo, tau_hi, c_lo, c_hi, cond, y):
    return ctx.check(lib.gmc_train_data(ctx.handle, n, seed, tau_lo, tau_hi, c_lo, c_hi,
                                        _ptr(cond), _ptr(y)))


def gmc_train_data_internal(ctx, n, seed, tau_lo, tau_hi, c_lo, c_hi, cond, y):
    return ctx.check(lib.gmc_train_data_internal(ctx.handle, n, seed, tau_lo, tau_hi, c_lo, c_hi,
                                                 _ptr(cond), _ptr(y)))


def gmc_train_begin(ctx, n, cond, y, cfg):
    return ctx.check(lib.gmc_train_begin(ctx.handle, n, _ptr(cond), _ptr(y), ctypes.byref(cfg)))


def gmc_train_steps(ctx, n_steps, losses=None):
    return ctx.check(lib.gmc_train_steps(ctx.handle, n_steps, _ptr(losses)))


def gmc_train_set_lr(ctx, lr):
    return ctx.check(lib.gmc_train_set_lr(ctx.handle, lr))


def gmc_train_grad(ctx, B, cn, x1, x0, t, grad):
    loss = ctypes.c_double()
    ctx.check(lib.gmc_train_grad(ctx.handle, B, _ptr(cn), _ptr(x1), _ptr(x0), _ptr(t),
                                 ctypes.byref(loss), _ptr(grad)))
    return loss.value


def gmc_train_params(ctx, out):
    return ctx.check(lib.gmc_train_params(ctx.handle, _ptr(out)))


def gmc_train_param_count():
    return int(lib.gmc_train_param_count())


def gmc_train_commit(ctx, path=None):
    return ctx.check(lib.gmc_train_commit(ctx.handle, None if path is None else os.fsencode(path)))


def gmc_serve_start(ctx, method, memory_budget):
    cfg = gmc_serve_config(method=method, memory_budget=memory_budget)
    return ctx.check(lib.gmc_serve_start(ctx.handle, ctypes.byref(cfg)))


def gmc_submit(ctx, nx, ny, tau, c, source, n_histories, seed):
    """tau, c, source: host float32 arrays of ny*nx cells; returns the ticket."""
    req = gmc_solve_req(nx=nx, ny=ny, tau=_ptr(tau), c=_ptr(c), source=_ptr(source),
                        n_histories=n_histories, seed=seed)
    t = ctypes.c_uint64()
    ctx.check(lib.gmc_submit(ctx.handle, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def gmc_poll(ctx, ticket, flux):
    """Returns stats when done, None while the request runs."""
    st = gmc_solve_stats()
    s = lib.gmc_poll(ctx.handle, ticket, _ptr(flux), ctypes.byref(st))
    if s == GMC_EBUSY:
        return None
    ctx.check(s)
    return st


def gmc_wait(ctx, ticket, timeout_s, flux):
    st = gmc_solve_stats()
    ctx.check(lib.gmc_wait(ctx.handle, ticket, timeout_s, _ptr(flux), ctypes.byref(st)))
    return st


def gmc_serve_stop(ctx):
    return ctx.check(lib.gmc_serve_stop(ctx.handle))


def gmc_selftest_wait(ctx, limit_ms):
    """Returns the status of the bounded-wait self-test (GMC_ETIMEOUT expected)."""
    return lib.gmc_selftest_wait(ctx.handle, float(limit_ms))
