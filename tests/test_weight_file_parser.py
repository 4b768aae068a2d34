"""The library's GMCW weight-file parser (csrc/gmcw.h), compiled into a
host-only library with no GPU: every committed network and every network
variant (MLP, residual-modulated, rectangular cells) parses to exactly the
arrays the oracle's reader returns, and damaged files are refused with the
status of their first defect.
"""
import ctypes
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import synth
from oracle import mlp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_13965_gb300", "csrc")
WEIGHTS = os.path.join(ROOT, "paper_2512_13965_gb300", "weights")

WRAPPER = r'''
#include "gmcw.h"
using namespace gmc;
extern "C" {
// Parses blob; on success copies the arrays out: stats [2 ncond + 8], then
// W_l and b_l of the five layers back to back, then M and G (rm only).
int gw_parse(const void *blob, size_t n, int *ncond, int *rm, int *layer, float *out,
             size_t out_floats) {
  GmcwNet P;
  *layer = -1;
  const int s = gmcw_parse(blob, n, &P, layer);
  if (s != kGmcwOk) return s;
  *ncond = P.ncond;
  *rm = P.rm ? 1 : 0;
  size_t k = 0;
  auto put = [&](const std::vector<float> &v) {
    for (float x : v) if (k < out_floats) out[k++] = x;
  };
  put(P.stats);
  for (int l = 0; l < 5; ++l) { put(P.w[l]); put(P.b[l]); }
  put(P.m);
  put(P.g);
  return k <= out_floats ? 0 : -1;
}
}
'''

OK, MAGIC, HEADER, UNSUPPORTED, DIMS, STATS, LAYER, MODULATION, TRAILING, STD, NONFINITE = range(11)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("needs g++")
    d = tmp_path_factory.mktemp("gmcw")
    src, so = d / "w.cpp", d / "libgw.so"
    src.write_text(WRAPPER)
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC, str(src), "-o",
                        str(so)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    L.gw_parse.argtypes = [P, ctypes.c_size_t, P, P, P, P, ctypes.c_size_t]
    L.gw_parse.restype = ctypes.c_int
    return L


MAX_FLOATS = 20 + 256 * 26 + 256 + 3 * (256 * 256 + 256) + 4 * 256 + 4 + 3 * 256 * 5 + 3 * 512


def _parse(lib, blob):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    out = np.zeros(MAX_FLOATS, np.float32)
    nc, rm, layer = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    s = lib.gw_parse(buf, len(blob), ctypes.byref(nc), ctypes.byref(rm), ctypes.byref(layer),
                     out.ctypes.data, MAX_FLOATS)
    return s, nc.value, bool(rm.value), layer.value, out


def _expected(net):
    parts = [net.cond_mean, net.cond_std, net.y_mean, net.y_std]
    for W, b in zip(net.W, net.b):
        parts += [W.ravel(), b]
    if net.rm:
        parts += [m.ravel() for m in net.M] + [g.ravel() for g in net.G]
    return np.concatenate(parts)


def _files(tmp_path):
    out = sorted(os.path.join(WEIGHTS, f) for f in os.listdir(WEIGHTS) if f.endswith(".bin"))
    for name, net in (("kaiming", synth.kaiming_weights(1)), ("biased", synth.biased_weights()),
                      ("rm", synth.rm_weights(1, 0.2, 0.2)), ("rect", synth.kaiming_weights_rect(2))):
        p = str(tmp_path / (name + ".bin"))
        synth.write_weights(p, net)
        out.append(p)
    return out


def test_every_network_parses_to_the_oracles_arrays(lib, tmp_path):
    files = _files(tmp_path)
    kinds = set()
    for path in files:
        blob = open(path, "rb").read()
        s, nc, rm, _, out = _parse(lib, blob)
        assert s == OK, (path, s)
        net = mlp.read_weights(path)
        assert nc == net.cond_mean.size and rm == net.rm, path
        exp = _expected(net).astype(np.float32)
        np.testing.assert_array_equal(out[:exp.size], exp, err_msg=path)
        kinds.add((nc, rm))
    assert kinds >= {(5, False), (5, True), (6, False)}


def _header(blob):
    return list(struct.unpack_from("<13I", blob, 0)[1:])  # after the magic


def _with_header(blob, fields):
    return blob[:4] + struct.pack("<12I", *fields) + blob[52:]


@pytest.mark.parametrize("name", ["kaiming", "rm", "rect"])
def test_damaged_files_are_refused(lib, tmp_path, name):
    net = {"kaiming": synth.kaiming_weights(1), "rm": synth.rm_weights(1, 0.2, 0.2),
           "rect": synth.kaiming_weights_rect(2)}[name]
    p = str(tmp_path / "w.bin")
    synth.write_weights(p, net)
    blob = open(p, "rb").read()
    assert _parse(lib, blob)[0] == OK
    h = _header(blob)
    nc = h[8]
    # section boundaries: header, statistics, each layer's W and b, M and G
    off = 52 + 4 * (2 * nc + 8)
    bounds = [(4, HEADER), (51, HEADER), (52, STATS), (off - 4, STATS)]
    dims = h[2:8]
    for l in range(5):
        bounds.append((off + 4, LAYER))
        off += 4 * dims[l + 1] * dims[l] + 4 * dims[l + 1]
        bounds.append((off - 2, LAYER))
    if h[11] & 1:
        bounds += [(off + 100, MODULATION), (len(blob) - 4, MODULATION)]
    assert off + (4 * (3 * 256 * 5 + 3 * 512) if h[11] & 1 else 0) == len(blob)
    for cut, status in bounds:
        assert _parse(lib, blob[:cut])[0] == status, (cut, status)
    s, _, _, layer, _ = _parse(lib, blob[:52 + 4 * (2 * nc + 8) + 4 * 256 * dims[0] + 8])
    assert (s, layer) == (LAYER, 0)  # layer 0's weights complete, its biases cut
    assert _parse(lib, blob[:3])[0] == MAGIC
    assert _parse(lib, b"GMCX" + blob[4:])[0] == MAGIC
    assert _parse(lib, blob + b"\0")[0] == TRAILING
    assert _parse(lib, blob + b"\0\0\0\0")[0] == TRAILING
    # header fields: version, layer count, n_cond, n_state, n_emb, flags, dims
    for i, v in ((0, 2), (1, 4), (8, 7), (8, 4), (9, 3), (10, 8), (11, 2), (11, 5)):
        f = list(h)
        f[i] = v
        assert _parse(lib, _with_header(blob, f))[0] == UNSUPPORTED, (i, v)
    if nc == 6:
        f = list(h)
        f[11] = 1  # the residual-modulated form has no rectangular-cell variant
        assert _parse(lib, _with_header(blob, f))[0] == UNSUPPORTED
    for i, v in ((2, 25 if nc == 6 else 26), (3, 128), (7, 3)):
        f = list(h)
        f[i] = v
        assert _parse(lib, _with_header(blob, f))[0] == DIMS, (i, v)
    # statistics: a zero or negative cond_std, a non-finite entry anywhere
    sbase = 52
    for k, v, status in ((nc, 0.0, STD), (nc + nc - 1, -1.0, STD), (0, np.nan, NONFINITE),
                         (2 * nc + 5, np.inf, NONFINITE), (nc, np.nan, STD)):
        b = bytearray(blob)
        struct.pack_into("<f", b, sbase + 4 * k, v)
        assert _parse(lib, bytes(b))[0] == status, (k, v)
    # the oracle's reader refuses the same layouts and truncations
    for cut, _ in bounds[:3]:
        with pytest.raises(Exception):
            q = tmp_path / "cut.bin"
            q.write_bytes(blob[:cut])
            mlp.read_weights(str(q))
