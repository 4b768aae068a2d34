"""The host-side packing of a network into the tensor-core samplers' byte
images (csrc/tc_pack.h), compiled into a host-only library with no GPU.

The images are decoded here from the swizzle's definition (a 16-byte unit's
index within its 128-byte row XOR the row's index within its 8-row group:
bits 7-9 of the byte address into bits 4-6 for the 128-byte swizzle, bit 7
into bit 4 for the 32-byte one) and compared bit for bit with the weights
rounded by torch's bfloat16 cast and the oracle's E4M3 rounding (itself
pinned to torch's float8_e4m3fn).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import synth
from oracle import mlp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_13965_gb300", "csrc")

WRAPPER = r'''
#include "tc_pack.h"
using namespace gmc::pack;
static float W[5][256 * 256], B[5][256], M[3][256 * 5];
extern "C" {
size_t tp_bytes(int fp8) { return fp8 ? Packed<true>::BYTES : Packed<false>::BYTES; }
void tp_layout(int fp8, size_t *out) {
  out[0] = fp8 ? Packed<true>::OFF_HID : Packed<false>::OFF_HID;
  out[1] = fp8 ? Packed<true>::OFF_B1 : Packed<false>::OFF_B1;
  out[2] = fp8 ? Packed<true>::OFF_B5 : Packed<false>::OFF_B5;
  out[3] = fp8 ? Packed<true>::OFF_BIAS : Packed<false>::OFF_BIAS;
  out[4] = fp8 ? Packed<true>::NCH : Packed<false>::NCH;
}
// w: the five layers back to back as [out][in]; b: [5][256] zero-padded;
// m: [3][256][5] or null
void tp_pack(const float *w, const float *b, const float *m, int nin, int fp8, void *out,
             float *bias, float *scale) {
  size_t k = 0;
  const int dims[6] = {nin, 256, 256, 256, 256, 4};
  for (int l = 0; l < 5; ++l) {
    for (size_t i = 0; i < 256 * 256; ++i) W[l][i] = 0.0f;
    for (int i = 0; i < dims[l + 1] * dims[l]; ++i) W[l][i] = w[k++];
    for (int i = 0; i < 256; ++i) B[l][i] = b[l * 256 + i];
  }
  if (m) for (int j = 0; j < 3; ++j) for (int i = 0; i < 256 * 5; ++i) M[j][i] = m[j * 1280 + i];
  if (fp8) tc_pack_host_fp8(W, B, out, bias, scale, nin);
  else tc_pack_host(W, B, out, bias, m ? M : nullptr, nin);
}
void tp_bf16(long n, const float *x, uint16_t *out) {
  for (long i = 0; i < n; ++i) out[i] = bf16_bits(x[i]);
}
void tp_e4m3(long n, const double *x, uint8_t *out) {
  for (long i = 0; i < n; ++i) out[i] = e4m3_bits(x[i]);
}
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("needs g++")
    d = tmp_path_factory.mktemp("tc_pack")
    src, so = d / "w.cpp", d / "libtp.so"
    src.write_text(WRAPPER)
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC, str(src), "-o",
                        str(so)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    L.tp_bytes.argtypes, L.tp_bytes.restype = [ctypes.c_int], ctypes.c_size_t
    L.tp_layout.argtypes = [ctypes.c_int, P]
    L.tp_pack.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, P, P]
    L.tp_bf16.argtypes = [ctypes.c_long, P, P]
    L.tp_e4m3.argtypes = [ctypes.c_long, P, P]
    return L


def _bf16_torch(x):
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


def _bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32)


def _e4m3_value(code):
    code = np.asarray(code, np.int64)
    mag = code & 0x7F
    e, m = mag >> 3, mag & 7
    v = np.where(e == 0, np.ldexp(m / 8.0, -6), np.ldexp(1.0 + m / 8.0, e - 7))
    return np.where(code & 0x80, -v, v)


def _swz(addr, mask):
    # the byte address inside a swizzled block -> where the byte lies
    addr = np.asarray(addr, np.int64)
    return addr ^ (((addr >> 7) & mask) << 4)


def test_bf16_rounding_is_torchs(lib):
    g = np.random.default_rng(1)
    x = np.concatenate([g.standard_normal(100000).astype(np.float32) * 10.0 ** g.integers(-30, 30, 100000),
                        np.array([0.0, -0.0, 1.0, -2.5, 3e38, -3e38, 1e-40, -1e-42, np.inf, -np.inf],
                                 np.float32)]).astype(np.float32)
    # exact ties: the dropped 16 bits are 0x8000, above an even and an odd value
    ties = (g.integers(0x3F00, 0x4300, 2000, dtype=np.uint32) << 16) | 0x8000
    x = np.concatenate([x, ties.view(np.float32)])
    out = np.zeros(x.size, np.uint16)
    lib.tp_bf16(x.size, x.ctypes.data, out.ctypes.data)
    np.testing.assert_array_equal(out, _bf16_torch(x))


def test_e4m3_rounding_is_the_oracles(lib):
    g = np.random.default_rng(2)
    # every code's value and the midpoints between neighbours (ties), the
    # saturation at 448, and random values over the whole range
    vals = _e4m3_value(np.arange(127))
    mids = 0.5 * (vals[1:] + vals[:-1])
    x = np.concatenate([vals, mids, -mids, [448.0, 460.0, 1e6, -1e6, 0.0, -0.0, 2.0 ** -10],
                        g.uniform(-500, 500, 20000), g.standard_normal(20000) * 0.01])
    out = np.zeros(x.size, np.uint8)
    lib.tp_e4m3(x.size, x.ctypes.data, out.ctypes.data)
    np.testing.assert_array_equal(_e4m3_value(out), mlp.round_e4m3(x))
    assert np.all(out[x < 0] & 0x80) and not np.any(out[x > 0] & 0x80)


def _pack(lib, net, nin, fp8, with_m):
    w = np.concatenate([np.asarray(W, np.float32).ravel() for W in net["W"]])
    b = np.zeros((5, 256), np.float32)
    for l, v in enumerate(net["b"]):
        b[l, :len(v)] = v
    m = np.ascontiguousarray(np.stack(net["M"]), np.float32) if with_m else None
    nb = lib.tp_bytes(int(fp8))
    img = np.zeros(nb, np.uint8)
    bias = np.zeros(1280, np.float32)
    scale = np.zeros(768, np.float32)
    lib.tp_pack(w.ctypes.data, b.ctypes.data, None if m is None else m.ctypes.data, nin, int(fp8),
                img.ctypes.data, bias.ctypes.data, scale.ctypes.data)
    lay = np.zeros(5, np.uintp)
    lib.tp_layout(int(fp8), lay.ctypes.data)
    return img, bias, scale, [int(v) for v in lay]


def _u16(img, byte_off):
    byte_off = np.asarray(byte_off, np.int64)
    return img[byte_off].astype(np.uint16) | (img[byte_off + 1].astype(np.uint16) << 8)


def _common_checks(img, bias, net, nin, lay, b1_ref_scale=0.5):
    W, bvec = [np.asarray(x, np.float32) for x in net["W"]], [np.asarray(x, np.float32) for x in net["b"]]
    _, off_b1, off_b5, _, _ = lay
    rows = np.arange(256)[:, None]
    # layer 1: 256 rows x 16 BF16 (32-byte rows, 32-byte swizzle)
    k = np.arange(16)[None, :]
    got = _u16(img, off_b1 + _swz(rows * 32 + k * 2, 1))
    W1 = W[0].reshape(256, nin)
    cols = np.zeros((256, 16), np.float32)
    cols[:, 0:4] = W1[:, 5:9]
    cols[:, 4:8] = W1[:, 5:9]
    cols[:, 8:13] = W1[:, 0:5]
    if nin == 26:
        cols[:, 15] = W1[:, 25]
    np.testing.assert_array_equal(got, _bf16_torch(np.float32(0.5) * cols))
    # output layer: four K-blocks of 16 rows x 128 B, rows 0..3 real
    d, kk = np.arange(16)[:, None], np.arange(256)[None, :]
    addr = off_b5 + (kk >> 6) * 2048 + _swz(d * 128 + (kk & 63) * 2, 7)
    W5 = np.zeros((16, 256), np.float32)
    W5[:4] = W[4].reshape(4, 256)
    np.testing.assert_array_equal(_u16(img, addr), _bf16_torch(W5))
    # FP32 biases: rows 1..3 = b/2 of layers 2-4, row 4 = b5
    expect = np.zeros((5, 256), np.float32)
    for L in range(1, 4):
        expect[L] = np.float32(0.5) * bvec[L]
    expect[4, :4] = bvec[4]
    np.testing.assert_array_equal(bias.reshape(5, 256), expect)


@pytest.mark.parametrize("kind", ["biased", "rm", "rect"])
def test_bf16_image_decodes_to_the_rounded_network(lib, kind):
    net = {"biased": synth.biased_weights(), "rm": synth.rm_weights(3, 0.3, 0.2),
           "rect": synth.kaiming_weights_rect(4)}[kind]
    nin = 26 if kind == "rect" else 25
    img, bias, _, lay = _pack(lib, net, nin, False, kind == "rm")
    off_hid, _, _, off_bias, nch = lay
    assert nch == 4 and img.size == lib.tp_bytes(0)
    W = [np.asarray(x, np.float32) for x in net["W"]]
    rows, j = np.arange(256)[:, None], np.arange(64)[None, :]
    for L in range(3):
        Wl = W[L + 1].reshape(256, 256)
        for ch in range(nch):
            addr = off_hid + (L * nch + ch) * 32768 + _swz(rows * 128 + j * 2, 7)
            np.testing.assert_array_equal(_u16(img, addr),
                                          _bf16_torch(np.float32(0.5) * Wl[:, 64 * ch:64 * ch + 64]))
    # bias blocks: b/2 as BF16 hi (column 13) + lo (column 14), the
    # residual-modulated shift M c / 2 in columns 8..12, the rest zero
    k = np.arange(16)[None, :]
    for L in range(3):
        blk = _u16(img, off_bias + L * 8192 + _swz(rows * 32 + k * 2, 1))
        half = np.float32(0.5) * np.asarray(net["b"][L + 1], np.float32)
        hi = _bf16_torch(half)
        lo = _bf16_torch(half - _bf16_value(hi))
        np.testing.assert_array_equal(blk[:, 13], hi)
        np.testing.assert_array_equal(blk[:, 14], lo)
        if kind == "rm":
            Mj = np.asarray(net["M"][L], np.float32).reshape(256, 5)
            np.testing.assert_array_equal(blk[:, 8:13], _bf16_torch(np.float32(0.5) * Mj))
            other = [0, 1, 2, 3, 4, 5, 6, 7, 15]
        else:
            other = [c for c in range(16) if c not in (13, 14)]
        assert not blk[:, other].any()
        # hi + lo carries b/2 to about 2^-16 relative
        np.testing.assert_allclose(_bf16_value(hi).astype(np.float64) + _bf16_value(lo), half,
                                   rtol=2.0 ** -15, atol=1e-30)
    _common_checks(img, bias, net, nin, lay)


def test_fp8_image_decodes_to_the_quantized_network(lib):
    net = synth.biased_weights()
    img, bias, scale, lay = _pack(lib, net, 25, True, False)
    off_hid, _, _, off_bias, nch = lay
    assert nch == 2 and img.size == lib.tp_bytes(1)
    rows, j = np.arange(256)[:, None], np.arange(128)[None, :]
    for L in range(3):
        Wl = np.asarray(net["W"][L + 1], np.float32).reshape(256, 256).astype(np.float64)
        sc = np.abs(Wl).max(axis=1)
        sc = np.where(sc > 0, sc / 448.0, 1.0)
        # per-output-channel scales, halved for the SiLU's h = z / 2
        np.testing.assert_array_equal(scale[L * 256:(L + 1) * 256], (0.5 * sc).astype(np.float32))
        codes = np.concatenate([img[off_hid + (L * nch + ch) * 32768 + _swz(rows * 128 + j, 7)]
                                for ch in range(nch)], axis=1)
        np.testing.assert_array_equal(_e4m3_value(codes), mlp.round_e4m3(Wl / sc[:, None]))
        # the bias block holds b / s_c as BF16 hi + lo
        blk = _u16(img, off_bias + L * 8192 + _swz(np.arange(256)[:, None] * 32 +
                                                    np.arange(16)[None, :] * 2, 1))
        v = (np.asarray(net["b"][L + 1], np.float64) / sc).astype(np.float32)
        hi = _bf16_torch(v)
        np.testing.assert_array_equal(blk[:, 13], hi)
        np.testing.assert_array_equal(blk[:, 14], _bf16_torch(v - _bf16_value(hi)))
    _common_checks(img, bias, net, 25, lay)
