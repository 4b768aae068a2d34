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
GMC_KERNEL_TILE, GMC_KERNEL_PAIR = 0, 1


class gmc_config(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("integrator", ctypes.c_int), ("precision", ctypes.c_int),
                ("w_cut", ctypes.c_double), ("p_survive", ctypes.c_double),
                ("bank_capacity", ctypes.c_int64), ("flights_per_wave", ctypes.c_int),
                ("gmc_min_tau", ctypes.c_double),
                ("net_tau_lo", ctypes.c_double), ("net_tau_hi", ctypes.c_double),
                ("net_c_lo", ctypes.c_double), ("net_c_hi", ctypes.c_double),
                ("sampler_kernel", ctypes.c_int)]


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
        "gmc_load_internal_xy_weights": [P, ctypes.c_char_p],
        "gmc_load_internal_xy_weights_buffer": [P, P, sz],
        "gmc_sample_internal_xy": [P, i64, P, P, u64, u64, i32, i32, i32, P, P],
        "gmc_load_xy_weights": [P, ctypes.c_char_p],
        "gmc_load_xy_weights_buffer": [P, P, sz],
        "gmc_sample_internal": [P, i64, P, P, u64, u64, i32, i32, i32, P, P],
        "gmc_transmit_xy": [P, i64, P, P, u64, u64, i32, i32, i32, P, P],
        "gmc_transmit": [P, i64, P, P, u64, u64, i32, i32, i32, P, P],
        "gmc_transmit_noalloc": [P, i64, P, P, u64, u64, i32, i32, P, P],
        "analog_transmit": [P, i64, P, P, P, P, P, i32, u64, u64, u32, P, P, P],
        "analog_transmit_rect": [P, i64, P, P, P, P, P, P, i32, u64, u64, u32, P, P, P],
        "analog_transmit_xy": [P, i64, P, P, P, P, P, P, i32, u64, u64, u32, P, P, P],
        "transport_solve": [P, i32, i32, P, P, P, i64, i32, u64, P,
                            ctypes.POINTER(gmc_solve_stats)],
        "transport_solve_wall": [P, i32, i32, P, P, P, i64, i32, u64, P,
                                 ctypes.POINTER(gmc_solve_stats)],
        "transport_solve_xy": [P, i32, i32, P, P, P, i64, i32, u64, P,
                               ctypes.POINTER(gmc_solve_stats)],
        "transport_solve_rect": [P, i32, i32, P, P, P, ctypes.c_float, ctypes.c_float, i64, i32,
                                 u64, P, ctypes.POINTER(gmc_solve_stats)],
        "transport_solve_wall_xy": [P, i32, i32, P, P, P, i64, i32, u64, P,
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
        "gmc_train_data_xy": [P, i64, u64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, P, P],
        "gmc_train_data_internal_xy": [P, i64, u64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, P, P],
        "gmc_train_data_rect": [P, i64, u64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P],
        "gmc_train_begin": [P, i64, P, P, ctypes.POINTER(gmc_train_config)],
        "gmc_train_steps": [P, i64, P],
        "gmc_train_set_lr": [P, ctypes.c_double],
        "gmc_train_grad": [P, i64, P, P, P, P, P, P],
        "gmc_train_params": [P, P],
        "gmc_train_param_count_ctx": [P, ctypes.POINTER(ctypes.c_int64)],
        "gmc_train_commit": [P, ctypes.c_char_p],
        "gmc_train_state_size": [P, ctypes.POINTER(ctypes.c_size_t)],
        "gmc_train_save_state": [P, P, sz],
        "gmc_train_load_state": [P, P, sz],
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


def _arr(x, itemsize, count, name):
    """_ptr after checking what the call will touch: `count` elements of
    `itemsize` bytes (the header's layout for that argument). A mismatch
    raises GMCError(GMC_EINVAL) before anything runs: the library itself
    cannot see a buffer's size, and a short or wider-typed buffer would be
    read or written past its end. None and raw integer addresses pass as
    they are (the library rejects a null array it needs)."""
    if x is None or isinstance(x, int):
        return _ptr(x)
    if hasattr(x, "data_ptr"):
        size, have = x.element_size(), x.numel()
    elif isinstance(x, np.ndarray):
        size, have = x.itemsize, x.size
    else:
        return _ptr(x)
    if size != itemsize:
        raise GMCError(GMC_EINVAL, "%s: elements of %d bytes expected, got %d"
                       % (name, itemsize, size))
    if count > 0 and have < count:
        raise GMCError(GMC_EINVAL, "%s: %d elements needed, buffer has %d" % (name, count, have))
    return _ptr(x)


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
        self.cells = {}  # grid size of each queued serving ticket

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


def _sampler_args(n, cond, noise, n_cond=5):
    return _arr(cond, 4, n_cond * n, "cond"), _arr(noise, 4, 4 * n, "noise")


def _sampler_out(n, y_raw, exit):
    return _arr(y_raw, 4, 4 * n, "y_raw"), _arr(exit, 4, 4 * n, "exit")


def _walk_in(n, **arrays):
    return [_arr(v, 4, n, k) for k, v in arrays.items()]


def _walk_out(n, status, exit, ncoll):
    return _arr(status, 4, n, "status"), _arr(exit, 4, 4 * n, "exit"), _arr(ncoll, 4, n, "ncoll")


def _grid(m, tau, c):
    return _arr(tau, 4, m, "tau"), _arr(c, 4, m, "c")


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
    return ctx.check(lib.gmc_philox(ctx.handle, n, seed, id0, event, tag,
                                    _arr(out, 4, 4 * n, "out")))


def gmc_normals(ctx, n, seed, id0, event, tag, out):
    return ctx.check(lib.gmc_normals(ctx.handle, n, seed, id0, event, tag,
                                     _arr(out, 4, 4 * n, "out")))


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


def gmc_load_internal_xy_weights(ctx, path):
    return ctx.check(lib.gmc_load_internal_xy_weights(ctx.handle, os.fsencode(path)))


def gmc_load_internal_xy_weights_buffer(ctx, blob):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    return ctx.check(lib.gmc_load_internal_xy_weights_buffer(ctx.handle, ctypes.addressof(buf),
                                                             len(blob)))


def gmc_load_xy_weights(ctx, path):
    return ctx.check(lib.gmc_load_xy_weights(ctx.handle, os.fsencode(path)))


def gmc_load_xy_weights_buffer(ctx, blob):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    return ctx.check(lib.gmc_load_xy_weights_buffer(ctx.handle, ctypes.addressof(buf), len(blob)))


def gmc_transmit_xy(ctx, n, cond, noise, seed, id0, steps, integrator, precision, y_raw, exit):
    return ctx.check(lib.gmc_transmit_xy(ctx.handle, n, *_sampler_args(n, cond, noise), seed, id0,
                                         steps, integrator, precision,
                                         *_sampler_out(n, y_raw, exit)))


def gmc_sample_internal(ctx, n, cond, noise, seed, id0, steps, integrator, precision, y_raw, exit):
    return ctx.check(lib.gmc_sample_internal(ctx.handle, n, *_sampler_args(n, cond, noise),
                                             seed, id0, steps, integrator, precision,
                                             *_sampler_out(n, y_raw, exit)))


def gmc_sample_internal_xy(ctx, n, cond, noise, seed, id0, steps, integrator, precision, y_raw,
                           exit):
    return ctx.check(lib.gmc_sample_internal_xy(ctx.handle, n, *_sampler_args(n, cond, noise),
                                                seed, id0, steps, integrator, precision,
                                                *_sampler_out(n, y_raw, exit)))


def gmc_transmit(ctx, n, cond, noise, seed, id0, steps, integrator, precision, y_raw, exit,
                 n_cond=5):
    """n_cond: rows of cond, 5, or 6 for a network of rectangular cells."""
    return ctx.check(lib.gmc_transmit(ctx.handle, n, *_sampler_args(n, cond, noise, n_cond), seed, id0,
                                      steps, integrator, precision,
                                      *_sampler_out(n, y_raw, exit)))


def gmc_transmit_noalloc(ctx, n, cond, noise, seed, id0, steps, integrator, y_raw, exit):
    return ctx.check(lib.gmc_transmit_noalloc(ctx.handle, n, *_sampler_args(n, cond, noise),
                                              seed, id0, steps, integrator,
                                              *_sampler_out(n, y_raw, exit)))


def analog_transmit(ctx, n, xi, cos_in, sin_in, tau, c, mode, seed, id0, event0, status, exit,
                    ncoll=None):
    ins = _walk_in(n, xi=xi, cos_in=cos_in, sin_in=sin_in, tau=tau, c=c)
    return ctx.check(lib.analog_transmit(ctx.handle, n, *ins, mode, seed, id0, event0,
                                         *_walk_out(n, status, exit, ncoll)))


def analog_transmit_rect(ctx, n, xi, cos_in, sin_in, tau_x, tau_y, c, mode, seed, id0, event0,
                         status, exit, ncoll=None):
    ins = _walk_in(n, xi=xi, cos_in=cos_in, sin_in=sin_in, tau_x=tau_x, tau_y=tau_y, c=c)
    return ctx.check(lib.analog_transmit_rect(ctx.handle, n, *ins, mode, seed, id0, event0,
                                              *_walk_out(n, status, exit, ncoll)))


def analog_transmit_xy(ctx, n, xi, ux_in, uy_in, tau_x, tau_y, c, mode, seed, id0, event0,
                       status, exit, ncoll=None):
    ins = _walk_in(n, xi=xi, ux_in=ux_in, uy_in=uy_in, tau_x=tau_x, tau_y=tau_y, c=c)
    return ctx.check(lib.analog_transmit_xy(ctx.handle, n, *ins, mode, seed, id0, event0,
                                            *_walk_out(n, status, exit, ncoll)))


def transport_solve(ctx, nx, ny, tau, c, source, n_histories, method, seed, flux, stats=None):
    st = stats if stats is not None else gmc_solve_stats()
    m = max(nx, 0) * max(ny, 0)
    ctx.check(lib.transport_solve(ctx.handle, nx, ny, *_grid(m, tau, c), _arr(source, 4, m, "source"),
                                  n_histories, method, seed, _arr(flux, 8, m, "flux"),
                                  ctypes.byref(st)))
    return st


def transport_solve_wall(ctx, nx, ny, tau, c, wall, n_histories, method, seed, flux, stats=None):
    st = stats if stats is not None else gmc_solve_stats()
    m = max(nx, 0) * max(ny, 0)
    ctx.check(lib.transport_solve_wall(ctx.handle, nx, ny, *_grid(m, tau, c),
                                       _arr(wall, 4, max(ny, 0), "wall"), n_histories, method,
                                       seed, _arr(flux, 8, m, "flux"), ctypes.byref(st)))
    return st


def transport_solve_xy(ctx, nx, ny, tau, c, source, n_histories, method, seed, flux, stats=None):
    st = stats if stats is not None else gmc_solve_stats()
    m = max(nx, 0) * max(ny, 0)
    ctx.check(lib.transport_solve_xy(ctx.handle, nx, ny, *_grid(m, tau, c),
                                     _arr(source, 4, m, "source"), n_histories, method, seed,
                                     _arr(flux, 8, m, "flux"), ctypes.byref(st)))
    return st


def transport_solve_rect(ctx, nx, ny, sigma, c, source, dx, dy, n_histories, method, seed, flux,
                         stats=None):
    st = stats if stats is not None else gmc_solve_stats()
    m = max(nx, 0) * max(ny, 0)
    ctx.check(lib.transport_solve_rect(ctx.handle, nx, ny, *_grid(m, sigma, c),
                                       _arr(source, 4, m, "source"), dx, dy, n_histories, method,
                                       seed, _arr(flux, 8, m, "flux"), ctypes.byref(st)))
    return st


def transport_solve_wall_xy(ctx, nx, ny, tau, c, wall, n_histories, method, seed, flux,
                            stats=None):
    st = stats if stats is not None else gmc_solve_stats()
    m = max(nx, 0) * max(ny, 0)
    ctx.check(lib.transport_solve_wall_xy(ctx.handle, nx, ny, *_grid(m, tau, c),
                                          _arr(wall, 4, max(ny, 0), "wall"), n_histories, method,
                                          seed, _arr(flux, 8, m, "flux"), ctypes.byref(st)))
    return st


def gmc_train_data(ctx, n, seed, tau_lo, tau_hi, c_lo, c_hi, cond, y):
    return ctx.check(lib.gmc_train_data(ctx.handle, n, seed, tau_lo, tau_hi, c_lo, c_hi,
                                        _arr(cond, 4, 5 * n, "cond"), _arr(y, 4, 4 * n, "y")))


def gmc_train_data_internal(ctx, n, seed, tau_lo, tau_hi, c_lo, c_hi, cond, y):
    return ctx.check(lib.gmc_train_data_internal(ctx.handle, n, seed, tau_lo, tau_hi, c_lo, c_hi,
                                                 _arr(cond, 4, 5 * n, "cond"),
                                                 _arr(y, 4, 4 * n, "y")))


def gmc_train_data_xy(ctx, n, seed, tau_lo, tau_hi, c_lo, c_hi, cond, y):
    return ctx.check(lib.gmc_train_data_xy(ctx.handle, n, seed, tau_lo, tau_hi, c_lo, c_hi,
                                           _arr(cond, 4, 5 * n, "cond"), _arr(y, 4, 4 * n, "y")))


def gmc_train_data_rect(ctx, n, seed, tau_lo, tau_hi, aspect_lo, aspect_hi, c_lo, c_hi, cond, y):
    return ctx.check(lib.gmc_train_data_rect(ctx.handle, n, seed, tau_lo, tau_hi, aspect_lo,
                                             aspect_hi, c_lo, c_hi, _arr(cond, 4, 6 * n, "cond"),
                                             _arr(y, 4, 4 * n, "y")))


def gmc_train_data_internal_xy(ctx, n, seed, tau_lo, tau_hi, c_lo, c_hi, cond, y):
    return ctx.check(lib.gmc_train_data_internal_xy(ctx.handle, n, seed, tau_lo, tau_hi, c_lo, c_hi,
                                                    _arr(cond, 4, 5 * n, "cond"),
                                                    _arr(y, 4, 4 * n, "y")))


def gmc_train_begin(ctx, n, cond, y, cfg):
    return ctx.check(lib.gmc_train_begin(ctx.handle, n, _arr(cond, 4, 5 * n, "cond"),
                                         _arr(y, 4, 4 * n, "y"), ctypes.byref(cfg)))


def gmc_train_steps(ctx, n_steps, losses=None):
    return ctx.check(lib.gmc_train_steps(ctx.handle, n_steps, _arr(losses, 4, n_steps, "losses")))


def gmc_train_set_lr(ctx, lr):
    return ctx.check(lib.gmc_train_set_lr(ctx.handle, lr))


def gmc_train_grad(ctx, B, cn, x1, x0, t, grad, n_cond=5):
    """n_cond: columns of cn, 5, or 6 for a network of rectangular cells."""
    loss = ctypes.c_double()
    P = gmc_train_param_count_ctx(ctx)
    ctx.check(lib.gmc_train_grad(ctx.handle, B, _arr(cn, 4, n_cond * B, "cn"), _arr(x1, 4, 4 * B, "x1"),
                                 _arr(x0, 4, 4 * B, "x0"), _arr(t, 4, B, "t"),
                                 ctypes.byref(loss), _arr(grad, 4, P, "grad")))
    return loss.value


def gmc_train_params(ctx, out):
    return ctx.check(lib.gmc_train_params(ctx.handle,
                                          _arr(out, 4, gmc_train_param_count_ctx(ctx), "out")))


def gmc_train_param_count():
    return int(lib.gmc_train_param_count())


def gmc_train_param_count_ctx(ctx):
    n = ctypes.c_int64()
    ctx.check(lib.gmc_train_param_count_ctx(ctx.handle, ctypes.byref(n)))
    return n.value


def gmc_train_state_size(ctx):
    n = ctypes.c_size_t()
    ctx.check(lib.gmc_train_state_size(ctx.handle, ctypes.byref(n)))
    return n.value


def gmc_train_save_state(ctx):
    """Returns the training checkpoint as bytes."""
    n = gmc_train_state_size(ctx)
    buf = ctypes.create_string_buffer(n)
    ctx.check(lib.gmc_train_save_state(ctx.handle, ctypes.addressof(buf), n))
    return buf.raw


def gmc_train_load_state(ctx, blob):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    return ctx.check(lib.gmc_train_load_state(ctx.handle, ctypes.addressof(buf), len(blob)))


def gmc_train_commit(ctx, path=None):
    return ctx.check(lib.gmc_train_commit(ctx.handle, None if path is None else os.fsencode(path)))


def gmc_serve_start(ctx, method, memory_budget):
    cfg = gmc_serve_config(method=method, memory_budget=memory_budget)
    return ctx.check(lib.gmc_serve_start(ctx.handle, ctypes.byref(cfg)))


def gmc_submit(ctx, nx, ny, tau, c, source, n_histories, seed):
    """tau, c, source: host float32 arrays of ny*nx cells; returns the ticket."""
    m = max(nx, 0) * max(ny, 0)
    gt, gc = _grid(m, tau, c)
    req = gmc_solve_req(nx=nx, ny=ny, tau=gt, c=gc, source=_arr(source, 4, m, "source"),
                        n_histories=n_histories, seed=seed)
    t = ctypes.c_uint64()
    ctx.check(lib.gmc_submit(ctx.handle, ctypes.byref(req), ctypes.byref(t)))
    ctx.cells[t.value] = m
    return t.value


def gmc_poll(ctx, ticket, flux):
    """Returns stats when done, None while the request runs."""
    st = gmc_solve_stats()
    s = lib.gmc_poll(ctx.handle, ticket, _arr(flux, 8, ctx.cells.get(ticket, 0), "flux"),
                     ctypes.byref(st))
    if s == GMC_EBUSY:
        return None
    ctx.check(s)
    ctx.cells.pop(ticket, None)
    return st


def gmc_wait(ctx, ticket, timeout_s, flux):
    st = gmc_solve_stats()
    ctx.check(lib.gmc_wait(ctx.handle, ticket, timeout_s,
                           _arr(flux, 8, ctx.cells.get(ticket, 0), "flux"), ctypes.byref(st)))
    ctx.cells.pop(ticket, None)
    return st


def gmc_serve_stop(ctx):
    return ctx.check(lib.gmc_serve_stop(ctx.handle))


def gmc_selftest_wait(ctx, limit_ms):
    """Returns the status of the bounded-wait self-test (GMC_ETIMEOUT expected)."""
    return lib.gmc_selftest_wait(ctx.handle, float(limit_ms))
