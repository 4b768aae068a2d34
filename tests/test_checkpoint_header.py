"""The training checkpoint's header and the checks a restore applies to it
(csrc/ckpt.h), compiled into a host-only library with no GPU: a header
written for a training state is accepted by that state, and every defect is
refused with its own code, the first one in check order when there are
several (the library maps them to GMC_EFORMAT for a checkpoint that is not
this network's or is damaged, GMC_EINVAL for one of another run or data).
"""
import ctypes
import shutil
import struct
import subprocess
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_13965_gb300", "csrc")

WRAPPER = r'''
#include <cstddef>
#include "ckpt.h"
using namespace gmc;
extern "C" {
size_t ck_size() { return sizeof(TrainCkpt); }
void ck_offsets(size_t *o) {
  o[0] = offsetof(TrainCkpt, magic); o[1] = offsetof(TrainCkpt, version);
  o[2] = offsetof(TrainCkpt, params); o[3] = offsetof(TrainCkpt, step);
  o[4] = offsetof(TrainCkpt, batch); o[5] = offsetof(TrainCkpt, n);
  o[6] = offsetof(TrainCkpt, precision); o[7] = offsetof(TrainCkpt, arch);
  o[8] = offsetof(TrainCkpt, lr); o[9] = offsetof(TrainCkpt, beta1);
  o[10] = offsetof(TrainCkpt, beta2); o[11] = offsetof(TrainCkpt, eps);
  o[12] = offsetof(TrainCkpt, weight_decay); o[13] = offsetof(TrainCkpt, seed);
  o[14] = offsetof(TrainCkpt, stats);
}
int ck_arch(int rm, int ncond) { return ckpt_arch_bits(rm != 0, ncond); }
int ck_check(const void *blob, long long params, long long batch, long long n, int precision,
             int arch, int ncond, const float *stats) {
  TrainCkpt h;
  std::memcpy(&h, blob, sizeof(h));
  const CkptTarget t{params, batch, n, precision, arch, ncond, stats};
  return ckpt_check(h, t);
}
}
'''

OK, NOT_THIS_NETWORK, BAD_STATS, BAD_HYPER, OTHER_RUN, OTHER_DATA = range(6)
FIELDS = ["magic", "version", "params", "step", "batch", "n", "precision", "arch", "lr", "beta1",
          "beta2", "eps", "weight_decay", "seed", "stats"]
FMT = {"version": "<I", "params": "<q", "step": "<q", "batch": "<q", "n": "<q", "precision": "<i",
       "arch": "<i", "lr": "<d", "beta1": "<d", "beta2": "<d", "eps": "<d", "weight_decay": "<d",
       "seed": "<Q"}


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("needs g++")
    d = tmp_path_factory.mktemp("ckpt")
    src, so = d / "w.cpp", d / "libck.so"
    src.write_text(WRAPPER)
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC, str(src), "-o",
                        str(so)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(str(so))
    L.ck_size.restype = ctypes.c_size_t
    L.ck_offsets.argtypes = [ctypes.c_void_p]
    L.ck_check.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
                           ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    L.ck_check.restype = ctypes.c_int
    off = np.zeros(15, np.uintp)
    L.ck_offsets(off.ctypes.data)
    L.off = dict(zip(FIELDS, (int(v) for v in off)))
    return L


class Run:
    """A training state and the header its save writes."""

    def __init__(self, lib, ncond=5, rm=False):
        self.lib = lib
        self.ncond, self.params, self.batch, self.n, self.precision = ncond, 283_652, 16384, 1 << 20, 1
        self.arch = lib.ck_arch(int(rm), ncond)
        g = np.random.default_rng(ncond)
        st = np.zeros(20, np.float32)
        st[:ncond] = g.standard_normal(ncond)
        st[ncond:2 * ncond] = g.uniform(0.5, 2.0, ncond)
        st[2 * ncond:2 * ncond + 4] = g.standard_normal(4)
        st[2 * ncond + 4:2 * ncond + 8] = g.uniform(0.5, 2.0, 4)
        self.stats = st
        h = bytearray(lib.ck_size())
        h[0:4] = b"GMCT"
        vals = {"version": 3, "params": self.params, "step": 1234, "batch": self.batch, "n": self.n,
                "precision": self.precision, "arch": self.arch, "lr": 1e-3, "beta1": 0.9,
                "beta2": 0.999, "eps": 1e-8, "weight_decay": 0.0, "seed": 7}
        for k, v in vals.items():
            struct.pack_into(FMT[k], h, lib.off[k], v)
        h[lib.off["stats"]:lib.off["stats"] + 80] = st.tobytes()
        self.header = bytes(h)

    def check(self, header=None, **target):
        t = dict(params=self.params, batch=self.batch, n=self.n, precision=self.precision,
                 arch=self.arch, ncond=self.ncond, stats=self.stats)
        t.update(target)
        buf = ctypes.create_string_buffer(header if header is not None else self.header,
                                          self.lib.ck_size())
        st = np.ascontiguousarray(t["stats"], np.float32)
        return self.lib.ck_check(buf, t["params"], t["batch"], t["n"], t["precision"], t["arch"],
                                 t["ncond"], st.ctypes.data)

    def patched(self, **fields):
        h = bytearray(self.header)
        for k, v in fields.items():
            if k == "magic":
                h[0:4] = v
            elif k.startswith("stat"):
                struct.pack_into("<f", h, self.lib.off["stats"] + 4 * int(k[4:]), v)
            else:
                struct.pack_into(FMT[k], h, self.lib.off[k], v)
        return bytes(h)


@pytest.mark.parametrize("ncond,rm", [(5, False), (5, True), (6, False)])
def test_a_run_restores_its_own_header(lib, ncond, rm):
    r = Run(lib, ncond, rm)
    assert r.check() == OK
    # means may take any finite value (here one the data has too), beta1 = 0
    # and no weight decay are valid
    st = r.stats.copy()
    st[0] = -3.0
    assert r.check(r.patched(stat0=-3.0, beta1=0.0, weight_decay=0.0), stats=st) == OK


def test_arch_bits(lib):
    assert [lib.ck_arch(0, 5), lib.ck_arch(1, 5), lib.ck_arch(0, 6)] == [0, 1, 2]


@pytest.mark.parametrize("ncond", [5, 6])
def test_each_defect_has_its_code(lib, ncond):
    r = Run(lib, ncond)
    P = r.patched
    cases = [
        (P(magic=b"GMCW"), NOT_THIS_NETWORK), (P(version=2), NOT_THIS_NETWORK),
        (P(params=r.params + 1), NOT_THIS_NETWORK), (P(arch=r.arch ^ 1), NOT_THIS_NETWORK),
        (P(arch=r.arch ^ 2), NOT_THIS_NETWORK),
        (P(lr=0.0), BAD_HYPER), (P(lr=float("inf")), BAD_HYPER), (P(lr=float("nan")), BAD_HYPER),
        (P(beta1=1.0), BAD_HYPER), (P(beta1=-0.1), BAD_HYPER), (P(beta2=1.0), BAD_HYPER),
        (P(eps=0.0), BAD_HYPER), (P(eps=float("nan")), BAD_HYPER),
        (P(weight_decay=-1e-9), BAD_HYPER), (P(weight_decay=float("inf")), BAD_HYPER),
        (P(batch=r.batch + 1), OTHER_RUN), (P(precision=0), OTHER_RUN), (P(step=-1), OTHER_RUN),
        (P(n=r.n - 1), OTHER_DATA),
    ]
    # statistics: every used slot refuses a non-finite value; the standard
    # deviations (cond_std, y_std) refuse zero and negatives too
    nc = ncond
    for k in range(2 * nc + 8):
        cases.append((P(**{"stat%d" % k: float("nan")}), BAD_STATS))
        cases.append((P(**{"stat%d" % k: float("-inf")}), BAD_STATS))
        is_std = nc <= k < 2 * nc or k >= 2 * nc + 4
        cases.append((P(**{"stat%d" % k: 0.0}), BAD_STATS if is_std else OTHER_DATA))
        cases.append((P(**{"stat%d" % k: -0.5}), BAD_STATS if is_std else OTHER_DATA))
    # one bit of one statistic differs from the data's: other data
    s = r.stats.copy()
    s[1] = np.nextafter(s[1], np.float32(10))
    cases.append((P(stat1=float(s[1])), OTHER_DATA))
    # a slot past the used ones is compared, not range-checked
    if 2 * nc + 8 < 20:
        cases.append((P(**{"stat%d" % (2 * nc + 8): float("nan")}), OTHER_DATA))
    for h, code in cases:
        assert r.check(h) == code, code
    # the target side: another training state refuses the header
    assert r.check(params=r.params - 1) == NOT_THIS_NETWORK
    assert r.check(batch=8192) == OTHER_RUN
    assert r.check(n=r.n + 1) == OTHER_DATA


def test_the_first_defect_in_check_order_is_reported(lib):
    r = Run(lib)
    assert r.check(r.patched(version=1, stat0=float("nan"), lr=0.0, batch=1, n=1)) == NOT_THIS_NETWORK
    assert r.check(r.patched(stat5=0.0, lr=0.0, batch=1, n=1)) == BAD_STATS
    assert r.check(r.patched(lr=0.0, batch=1, n=1)) == BAD_HYPER
    assert r.check(r.patched(batch=1, n=1)) == OTHER_RUN
