"""The solve engine's host-side rules (csrc/host_rules.h), compiled into a
host-only library with no GPU and checked against the oracle: each cell's
scattering-equivalent condition and routing (the values stage 1 and stage 3
of a GMC solve read), and the sizes a solve on rectangular cells accepts;
and the serving pool's free list (admission by memory) against a model of
the pool's bytes.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import transport as OT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_13965_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

WRAPPER = r'''
#include <cstring>
#include "ckpt.h"
#include "host_rules.h"
using namespace gmc;
extern "C" {
void hr_equivalent(long n, const double *tau, const double *c, double t_lo, double t_hi,
                   double c_lo, double c_hi, double *tau_n, double *c_n, int *ok) {
  for (long k = 0; k < n; ++k)
    ok[k] = equivalent_condition(tau[k], c[k], t_lo, t_hi, c_lo, c_hi, &tau_n[k], &c_n[k]);
}
void hr_equivalent_rect(long n, const double *tx, const double *ty, const double *c, double t_lo,
                        double t_hi, double c_lo, double c_hi, double *tx_n, double *c_n, int *ok) {
  for (long k = 0; k < n; ++k)
    ok[k] = equivalent_condition_rect(tx[k], ty[k], c[k], t_lo, t_hi, c_lo, c_hi, &tx_n[k], &c_n[k]);
}
void hr_cell_condition_rect(long n, const float *tau, const float *c, double aspect, double t_lo,
                            double t_hi, double c_lo, double c_hi, float *ltau_n, float *c_n,
                            float *s_scale, unsigned char *walk) {
  for (long k = 0; k < n; ++k) {
    const CellCondition r = cell_condition((double)tau[k], (double)c[k], t_lo, t_hi, c_lo, c_hi,
                                           0.0, (double)tau[k] * aspect);
    ltau_n[k] = r.ltau_n;
    c_n[k] = r.c_n;
    s_scale[k] = r.s_scale;
    walk[k] = r.walk;
  }
}
void hr_cell_condition(long n, const float *tau, const float *c, double t_lo, double t_hi,
                       double c_lo, double c_hi, double min_tau, float *ltau_n, float *c_n,
                       float *s_scale, unsigned char *walk) {
  for (long k = 0; k < n; ++k) {
    const CellCondition r = cell_condition((double)tau[k], (double)c[k], t_lo, t_hi, c_lo, c_hi,
                                           min_tau);
    ltau_n[k] = r.ltau_n;
    c_n[k] = r.c_n;
    s_scale[k] = r.s_scale;
    walk[k] = r.walk;
  }
}
void *fl_new(size_t bytes) {
  FreeList *f = new FreeList();
  f->reset(bytes);
  return f;
}
void fl_delete(void *h) { delete (FreeList *)h; }
int fl_alloc(void *h, size_t bytes, size_t *off) { return ((FreeList *)h)->alloc(bytes, off); }
void fl_release(void *h, size_t off, size_t bytes) { ((FreeList *)h)->release(off, bytes); }
long fl_regions(void *h, size_t *offs, size_t *lens, long cap) {
  long k = 0;
  for (const auto &r : ((FreeList *)h)->regions()) {
    if (k < cap) { offs[k] = r.first; lens[k] = r.second; }
    ++k;
  }
  return k;
}
int hr_config(int steps, int integ, int prec, double w_cut, double p_survive, long long cap,
              int fpw, double min_tau, double t_lo, double t_hi, double c_lo, double c_hi,
              int kernel) {
  gmc_config c;
  c.steps = steps;
  c.integrator = integ;
  c.precision = prec;
  c.w_cut = w_cut;
  c.p_survive = p_survive;
  c.bank_capacity = cap;
  c.flights_per_wave = fpw;
  c.gmc_min_tau = min_tau;
  c.net_tau_lo = t_lo;
  c.net_tau_hi = t_hi;
  c.net_c_lo = c_lo;
  c.net_c_hi = c_hi;
  c.sampler_kernel = kernel;
  return config_check(c);
}
int hr_data_ranges(float tl, float th, float cl, float ch, float al, float ah) {
  return data_ranges_ok(tl, th, cl, ch, al, ah);
}
int hr_train_config(int batch, double lr, double b1, double b2, double eps, double wd, int prec) {
  gmc_train_config c;
  std::memset(&c, 0, sizeof(c));
  c.batch = batch;
  c.lr = lr;
  c.beta1 = b1;
  c.beta2 = b2;
  c.eps = eps;
  c.weight_decay = wd;
  c.precision = prec;
  return train_config_check(c);
}
// a checkpoint header that is valid but for the given hyperparameters
int hr_ckpt_hyper(double lr, double b1, double b2, double eps, double wd) {
  float st[20] = {0};
  for (int k = 5; k < 10; ++k) st[k] = 1.0f;
  for (int k = 14; k < 18; ++k) st[k] = 1.0f;
  TrainCkpt h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "GMCT", 4);
  h.version = kCkptVersion;
  h.params = 10;
  h.batch = 16;
  h.n = 100;
  h.precision = 1;
  h.lr = lr;
  h.beta1 = b1;
  h.beta2 = b2;
  h.eps = eps;
  h.weight_decay = wd;
  std::memcpy(h.stats, st, sizeof(st));
  const CkptTarget t{10, 16, 100, 1, 0, 5, st};
  return ckpt_check(h, t);
}
int hr_grid(long ncell, int ny, const float *tau, const float *c, const float *src, int wall,
            double *cdf, double *total, long *bad) {
  int64_t b = -1;
  const int r = grid_source_check(ncell, ny, tau, c, src, wall != 0, cdf, total, &b);
  *bad = (long)b;
  return r;
}
int hr_rect_sizes_check(const float *sigma, long n, float dx, float dy, long *bad) {
  size_t b = (size_t)-1;
  const int r = rect_sizes_check(sigma, (size_t)n, dx, dy, &b);
  *bad = r == 3 ? (long)b : -1;
  return r;
}
}
'''

BOX = (0.1, 1000.0, 0.5, 0.999)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("needs g++")
    d = tmp_path_factory.mktemp("host_rules")
    src, so = d / "w.cpp", d / "libhr.so"
    src.write_text(WRAPPER)
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC, "-I", INCLUDE,
                        str(src), "-o", str(so)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(str(so))
    P, D, F, LG = ctypes.c_void_p, ctypes.c_double, ctypes.c_float, ctypes.c_long
    L.hr_equivalent.argtypes = [LG, P, P, D, D, D, D, P, P, P]
    L.hr_cell_condition.argtypes = [LG, P, P, D, D, D, D, D, P, P, P, P]
    L.hr_equivalent_rect.argtypes = [LG, P, P, P, D, D, D, D, P, P, P]
    L.hr_cell_condition_rect.argtypes = [LG, P, P, D, D, D, D, D, P, P, P, P]
    L.hr_rect_sizes_check.argtypes = [P, LG, F, F, P]
    L.hr_rect_sizes_check.restype = ctypes.c_int
    I = ctypes.c_int
    L.hr_config.argtypes = [I, I, I, D, D, ctypes.c_longlong, I, D, D, D, D, D, I]
    L.hr_config.restype = I
    L.hr_data_ranges.argtypes = [F] * 6
    L.hr_data_ranges.restype = I
    L.hr_train_config.argtypes = [I, D, D, D, D, D, I]
    L.hr_train_config.restype = I
    L.hr_ckpt_hyper.argtypes = [D] * 5
    L.hr_ckpt_hyper.restype = I
    L.hr_grid.argtypes = [LG, ctypes.c_int, P, P, P, ctypes.c_int, P, P, P]
    L.hr_grid.restype = ctypes.c_int
    S = ctypes.c_size_t
    L.fl_new.argtypes, L.fl_new.restype = [S], P
    L.fl_delete.argtypes = [P]
    L.fl_alloc.argtypes, L.fl_alloc.restype = [P, S, P], ctypes.c_int
    L.fl_release.argtypes = [P, S, S]
    L.fl_regions.argtypes, L.fl_regions.restype = [P, P, P, LG], LG
    return L


def _cells(n, seed):
    # tau log-uniform over [1e-4, 1e5], c uniform in [0, 1], plus the edges:
    # c = 0 and 1, the box's corners and sides, c tau at both ends of the
    # range that has an equivalent (c_lo tau_lo, c_hi tau_hi), just inside
    # and outside it
    g = np.random.default_rng(seed)
    tau = np.exp(g.uniform(np.log(1e-4), np.log(1e5), n))
    c = g.uniform(0.0, 1.0, n)
    t_lo, t_hi, c_lo, c_hi = BOX
    edge_t = [t_lo, t_hi, 1.0, 0.05, 2000.0, t_lo * c_lo / 0.2, np.nextafter(t_lo, 0)]
    edge_c = [0.0, 1.0, c_lo, c_hi, 0.2, np.nextafter(c_lo, 0), np.nextafter(c_hi, 2)]
    et, ec = np.meshgrid(edge_t, edge_c)
    lo_w, hi_w = c_lo * t_lo, c_hi * t_hi
    wt = np.array([lo_w, hi_w, lo_w * (1 - 1e-12), hi_w * (1 + 1e-12), lo_w * (1 + 1e-12)])
    return np.concatenate([tau, et.ravel(), wt / 0.3]), np.concatenate([c, ec.ravel(), np.full(5, 0.3)])


def test_equivalent_condition_is_the_oracles(lib):
    tau, c = _cells(20000, 3)
    n = tau.size
    tn, cn, ok = np.zeros(n), np.zeros(n), np.zeros(n, np.int32)
    lib.hr_equivalent(n, tau.ctypes.data, c.ctypes.data, *BOX, tn.ctypes.data, cn.ctypes.data,
                      ok.ctypes.data)
    tp, cp, okp = OT.equivalent_condition(tau, c, BOX[:2], BOX[2:])
    np.testing.assert_array_equal(ok.astype(bool), okp)
    np.testing.assert_array_equal(tn, tp)
    np.testing.assert_array_equal(cn, cp)
    # what the map promises where it applies: c' tau' = c tau (to rounding)
    # and (tau', c') inside the box
    m = okp
    np.testing.assert_allclose(cn[m] * tn[m], c[m] * tau[m], rtol=1e-14)
    assert np.all((tn[m] >= BOX[0]) & (tn[m] <= BOX[1]) & (cn[m] >= BOX[2]) & (cn[m] <= BOX[3]))
    # both sides of the reachable band, and c = 0, occur in the sample
    assert okp.sum() > 1000 and (~okp).sum() > 1000 and not okp[c == 0].any()


@pytest.mark.parametrize("min_tau", [0.0, 0.5])
def test_cell_condition_is_what_the_kernels_read(lib, min_tau):
    tau, c = _cells(20000, 5)
    tau32, c32 = tau.astype(np.float32), c.astype(np.float32)
    n = tau.size
    lt, cn, ss = (np.zeros(n, np.float32) for _ in range(3))
    walk = np.zeros(n, np.uint8)
    lib.hr_cell_condition(n, tau32.ctypes.data, c32.ctypes.data, *BOX, min_tau, lt.ctypes.data,
                          cn.ctypes.data, ss.ctypes.data, walk.ctypes.data)
    t64, c64 = tau32.astype(np.float64), c32.astype(np.float64)
    tp, cp, ok = OT.equivalent_condition(t64, c64, BOX[:2], BOX[2:])
    np.testing.assert_array_equal(lt, np.log(tp).astype(np.float32))
    np.testing.assert_array_equal(cn, cp.astype(np.float32))
    with np.errstate(divide="ignore", invalid="ignore"):
        expect_s = np.where(ok, cp / c64, 1.0).astype(np.float32)
    np.testing.assert_array_equal(ss, expect_s)
    expect_walk = ~ok | ((min_tau > 0.0) & (t64 < min_tau))
    np.testing.assert_array_equal(walk.astype(bool), expect_walk)
    if min_tau > 0.0:
        assert (walk.astype(bool) & ok).any()  # thin cells with an equivalent are walked too


def test_rect_equivalent_condition_is_the_oracles(lib):
    g = np.random.default_rng(6)
    tau, c = _cells(20000, 7)
    n = tau.size
    ty = tau * np.exp(g.uniform(np.log(1 / 60), np.log(60), n))
    ty[:500] = tau[:500]  # square cells among them
    tn, cn, ok = np.zeros(n), np.zeros(n), np.zeros(n, np.int32)
    lib.hr_equivalent_rect(n, tau.ctypes.data, ty.ctypes.data, c.ctypes.data, *BOX, tn.ctypes.data,
                           cn.ctypes.data, ok.ctypes.data)
    tp, cp, okp = OT.equivalent_condition_rect(tau, ty, c, BOX[:2], BOX[2:])
    np.testing.assert_array_equal(ok.astype(bool), okp)
    np.testing.assert_array_equal(tn, tp)
    np.testing.assert_array_equal(cn, cp)
    assert okp.sum() > 1000 and (~okp).sum() > 1000


@pytest.mark.parametrize("aspect", [0.2, 1.0, 7.5])
def test_rect_cell_condition_is_what_the_kernels_read(lib, aspect):
    tau, c = _cells(20000, 9)
    tau32, c32 = tau.astype(np.float32), c.astype(np.float32)
    n = tau.size
    lt, cn, ss = (np.zeros(n, np.float32) for _ in range(3))
    walk = np.zeros(n, np.uint8)
    lib.hr_cell_condition_rect(n, tau32.ctypes.data, c32.ctypes.data, aspect, *BOX, lt.ctypes.data,
                               cn.ctypes.data, ss.ctypes.data, walk.ctypes.data)
    t64, c64 = tau32.astype(np.float64), c32.astype(np.float64)
    tp, cp, ok = OT.equivalent_condition_rect(t64, t64 * aspect, c64, BOX[:2], BOX[2:])
    np.testing.assert_array_equal(lt, np.log(tp).astype(np.float32))
    np.testing.assert_array_equal(cn, cp.astype(np.float32))
    with np.errstate(divide="ignore", invalid="ignore"):
        np.testing.assert_array_equal(ss, np.where(ok, cp / c64, 1.0).astype(np.float32))
    np.testing.assert_array_equal(walk.astype(bool), ~ok)


def _rect(lib, sigma, dx, dy):
    s = np.ascontiguousarray(sigma, np.float32)
    bad = ctypes.c_long(0)
    r = lib.hr_rect_sizes_check(s.ctypes.data, s.size, dx, dy, ctypes.byref(bad))
    return r, bad.value


def test_rect_sizes_accepted_and_refused(lib):
    sig = np.array([0.5, 3.0, 1e-3, 200.0])
    assert _rect(lib, sig, 0.5, 1.5) == (0, -1)
    assert _rect(lib, sig, 1.0, 1.0) == (0, -1)
    for dx, dy in ((0.0, 1.0), (1.0, -1.0), (float("inf"), 1.0), (1.0, float("nan"))):
        assert _rect(lib, sig, dx, dy)[0] == 1, (dx, dy)
    assert _rect(lib, sig, 1e-30, 1e10)[0] == 2  # dy / dx = 1e40
    assert _rect(lib, sig, 1e10, 1e-30)[0] == 2
    assert _rect(lib, sig, 1e-20, 1e15)[0] == 0  # dy / dx = 1e35 with small heights
    assert _rect(lib, [0.5, 1e10, 1.0], 1.0, 1e30) == (3, 1)  # sigma dy = 1e40
    assert _rect(lib, [0.5, 0.0, 1.0], 1.0, 1.0) == (3, 1)
    assert _rect(lib, [0.5, 1.0, -2.0], 1.0, 1.0) == (3, 2)
    assert _rect(lib, [0.5, 1.0, float("nan")], 1.0, 1.0) == (3, 2)


def _regions(lib, h):
    offs, lens = np.zeros(4096, np.uintp), np.zeros(4096, np.uintp)
    k = lib.fl_regions(h, offs.ctypes.data, lens.ctypes.data, 4096)
    assert k <= 4096
    return [(int(o), int(n)) for o, n in zip(offs[:k], lens[:k])]


def _free_runs(used, cap):
    # maximal free intervals of a byte map, in address order
    runs, k = [], 0
    while k < cap:
        if used[k]:
            k += 1
            continue
        j = k
        while j < cap and not used[j]:
            j += 1
        runs.append((k, j - k))
        k = j
    return runs


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pool_free_list_against_a_byte_map(lib, seed):
    # random admissions and completions in units of 256 B (footprints are
    # sums of 256-byte-aligned arrays): every grant is the lowest-addressed
    # free run that holds it, no two grants overlap, a refusal means no run
    # is large enough, the free list is exactly the maximal free runs after
    # every step, and releasing everything leaves the whole pool free
    cap = 2048  # in 256-byte units
    g = np.random.default_rng(seed)
    h = lib.fl_new(cap * 256)
    try:
        used = np.zeros(cap, bool)
        live = []
        refused = 0
        for _ in range(2000):
            if live and (g.random() < 0.45 or len(live) > 60):
                off, n = live.pop(int(g.integers(len(live))))
                lib.fl_release(h, off * 256, n * 256)
                assert used[off:off + n].all()
                used[off:off + n] = False
            else:
                n = int(min(cap, np.ceil(g.lognormal(3.0, 1.2))))
                o = ctypes.c_size_t(0)
                runs = _free_runs(used, cap)
                fits = [r for r in runs if r[1] >= n]
                if lib.fl_alloc(h, n * 256, ctypes.byref(o)):
                    assert o.value % 256 == 0
                    off = o.value // 256
                    assert fits and off == fits[0][0], (off, fits[:2])
                    assert not used[off:off + n].any() and off + n <= cap
                    used[off:off + n] = True
                    live.append((off, n))
                else:
                    assert not fits
                    refused += 1
            assert _regions(lib, h) == [(o * 256, n * 256) for o, n in _free_runs(used, cap)]
        assert refused > 0 and len(live) > 10
        for off, n in reversed(live):
            lib.fl_release(h, off * 256, n * 256)
        assert _regions(lib, h) == [(0, cap * 256)]
    finally:
        lib.fl_delete(h)


def _grid(lib, tau, c, src, wall, ny):
    tau, c, src = (np.ascontiguousarray(a, np.float32) for a in (tau, c, src))
    n = tau.size
    cdf = np.full(n, -1.0)
    tot, bad = ctypes.c_double(-1.0), ctypes.c_long(-2)
    r = lib.hr_grid(n, ny, tau.ctypes.data, c.ctypes.data, src.ctypes.data, int(wall),
                    cdf.ctypes.data, ctypes.byref(tot), ctypes.byref(bad))
    return r, bad.value, cdf, tot.value


def test_grid_checks_and_source_cdf(lib):
    g = np.random.default_rng(8)
    ny, nx = 24, 40
    tau = np.exp(g.uniform(np.log(0.01), np.log(1e4), ny * nx)).astype(np.float32)
    c = g.uniform(0.0, 1.0, ny * nx).astype(np.float32)
    c[:5] = [0.0, 1.0, 0.5, 0.0, 1.0]
    src = np.where(g.random(ny * nx) < 0.3, g.exponential(1.0, ny * nx), 0.0).astype(np.float32)
    # volumetric: the CDF the births search is the running FP64 sum
    r, _, cdf, tot = _grid(lib, tau, c, src, False, ny)
    assert r == 0
    np.testing.assert_array_equal(cdf, np.cumsum(src.astype(np.float64)))
    assert tot == cdf[-1]
    # wall: ny strengths (the rest of the array is not read)
    wall = np.concatenate([g.exponential(1.0, ny), np.full(ny * nx - ny, np.nan)]).astype(np.float32)
    r, _, cdfw, totw = _grid(lib, tau, c, wall, True, ny)
    assert r == 0
    np.testing.assert_array_equal(cdfw[:ny], np.cumsum(wall[:ny].astype(np.float64)))
    assert totw == cdfw[ny - 1] and np.all(cdfw[ny:] == -1.0)
    # refusals, each with the first defect in cell order
    for k, field, v, code in ((17, "tau", 0.0, 1), (3, "tau", -1.0, 1), (90, "tau", np.inf, 1),
                              (5, "tau", np.nan, 1), (60, "c", -1e-7, 1), (61, "c", 1.0001, 1),
                              (62, "c", np.nan, 1), (33, "src", -1.0, 2), (34, "src", np.inf, 2),
                              (35, "src", np.nan, 2)):
        a = {"tau": tau.copy(), "c": c.copy(), "src": src.copy()}
        a[field][k] = v
        assert _grid(lib, a["tau"], a["c"], a["src"], False, ny)[:2] == (code, k), (field, k)
    # a cell's tau before its own source, an earlier source before a later tau
    t2, s2 = tau.copy(), src.copy()
    t2[40], s2[40] = 0.0, -1.0
    assert _grid(lib, t2, c, s2, False, ny)[:2] == (1, 40)
    t2[40], s2[20] = tau[40], -1.0
    assert _grid(lib, t2, c, s2, False, ny)[:2] == (2, 20)
    w2 = wall.copy()
    w2[7] = -2.0
    assert _grid(lib, tau, c, w2, True, ny)[:2] == (3, 7)
    t3 = tau.copy()
    t3[ny * nx - 1] = np.nan  # every cell is checked before the wall strengths
    assert _grid(lib, t3, c, w2, True, ny)[:2] == (1, ny * nx - 1)


CONFIG = dict(steps=16, integ=0, prec=1, w_cut=1e-4, p_survive=0.1, cap=1 << 21, fpw=512,
              min_tau=0.0, t_lo=0.1, t_hi=1000.0, c_lo=0.5, c_hi=0.999, kernel=0)


def _config(lib, **kw):
    c = dict(CONFIG)
    c.update(kw)
    return lib.hr_config(*c.values())


def test_config_ranges(lib):
    inf, nan = float("inf"), float("nan")
    assert _config(lib) == 0
    # the edges of every range are accepted
    for kw in (dict(steps=1), dict(steps=256), dict(integ=2), dict(prec=0), dict(prec=2),
               dict(w_cut=0.0), dict(p_survive=1.0), dict(cap=1024), dict(cap=1 << 28),
               dict(fpw=1), dict(min_tau=inf), dict(t_lo=5.0, t_hi=5.0), dict(c_lo=1.0, c_hi=1.0),
               dict(kernel=1)):
        assert _config(lib, **kw) == 0, kw
    for kw, code in ((dict(steps=0), 1), (dict(steps=257), 1), (dict(integ=3), 2),
                     (dict(integ=-1), 2), (dict(prec=3), 3), (dict(prec=-1), 3),
                     (dict(w_cut=-1e-9), 4), (dict(w_cut=nan), 4), (dict(p_survive=0.0), 4),
                     (dict(p_survive=1.5), 4), (dict(p_survive=nan), 4), (dict(cap=1023), 5),
                     (dict(cap=(1 << 28) + 1), 5), (dict(fpw=0), 6), (dict(min_tau=-1.0), 7),
                     (dict(min_tau=nan), 7), (dict(t_lo=0.0), 8), (dict(t_hi=0.05), 8),
                     (dict(t_hi=inf), 8), (dict(t_lo=nan), 8), (dict(c_lo=0.0), 8),
                     (dict(c_hi=1.01), 8), (dict(c_lo=0.9, c_hi=0.8), 8), (dict(kernel=2), 9)):
        assert _config(lib, **kw) == code, (kw, code)
    # the first field out of range is the one reported
    assert _config(lib, steps=0, kernel=7, cap=1) == 1
    assert _config(lib, fpw=0, kernel=7) == 6


def test_training_data_ranges(lib):
    inf, nan = float("inf"), float("nan")
    ok = (0.1, 1000.0, 0.5, 0.999, 1.0, 1.0)
    assert lib.hr_data_ranges(*ok) == 1
    for args in ((1.0, 1.0, 0.0, 1.0, 1.0, 1.0), (0.1, 1000.0, 0.5, 0.5, 0.25, 4.0),
                 (1e-30, 1e30, 0.0, 0.0, 1.0, 1.0)):
        assert lib.hr_data_ranges(*args) == 1, args
    for k, v in ((0, 0.0), (0, -1.0), (0, nan), (1, 0.05), (1, inf), (1, nan), (2, -0.1),
                 (2, nan), (3, 0.4), (3, 1.01), (3, nan), (4, 0.0), (4, nan), (5, 0.5),
                 (5, inf)):
        a = list(ok)
        a[k] = v
        assert lib.hr_data_ranges(*a) == 0, (k, v)


def test_training_config_ranges_match_the_checkpoints(lib):
    inf, nan = float("inf"), float("nan")
    base = dict(batch=16384, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=0.01, prec=1)

    def chk(**kw):
        c = dict(base)
        c.update(kw)
        return lib.hr_train_config(*c.values())
    assert chk() == 0 and chk(batch=1) == 0 and chk(batch=1 << 20) == 0 and chk(prec=0) == 0
    assert chk(b1=0.0, b2=0.0, wd=0.0) == 0
    for kw, code in ((dict(batch=0), 1), (dict(batch=(1 << 20) + 1), 1), (dict(lr=0.0), 2),
                     (dict(lr=inf), 2), (dict(lr=nan), 2), (dict(prec=2), 3), (dict(prec=-1), 3),
                     (dict(b1=1.0), 4), (dict(b2=-1e-9), 4), (dict(eps=0.0), 4), (dict(eps=inf), 4),
                     (dict(wd=-1.0), 4), (dict(wd=nan), 4)):
        assert chk(**kw) == code, kw
    # a configuration gmc_train_begin accepts writes a checkpoint whose
    # hyperparameters a restore accepts, and the other way round
    g = np.random.default_rng(3)
    vals = [0.0, 1e-12, 0.5, 0.999, 1.0, 1.5, -1e-9, inf, nan]
    seen = set()
    for _ in range(600):
        lr, b1, b2, eps, wd = (float(g.choice(vals)) for _ in range(5))
        begin_ok = chk(lr=lr, b1=b1, b2=b2, eps=eps, wd=wd) == 0
        restore_ok = lib.hr_ckpt_hyper(lr, b1, b2, eps, wd) == 0
        assert begin_ok == restore_ok, (lr, b1, b2, eps, wd)
        seen.add(begin_ok)
    assert seen == {True, False}
