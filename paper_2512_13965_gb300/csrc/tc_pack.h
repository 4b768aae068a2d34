// Host-side packing of a velocity network into the byte images the
// tensor-core samplers copy into shared memory (BF16, or E4M3 hidden layers
// with per-output-channel scales), and the layout of the packed buffer.
// Plain C++ with no CUDA headers, so a host-only unit test checks the images
// against the swizzle definition and the oracle's rounding without a GPU.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>

namespace gmc {
namespace pack {

constexpr int kPackCond = 5;   // condition columns of the square-cell network
constexpr int kPackIn = 25;    // its layer-1 inputs; input 25 is a rectangular cell's aspect

// Weight chunk: all 256 output rows x 128 bytes of K (64 BF16 or 128 E4M3
// inputs), K-major, 128-byte swizzle; 32 KB.
constexpr uint32_t CHUNK = 256u * 128u;

// packed global operand buffer (bytes): hidden-layer chunks, then the BF16
// operands of layers 1 and 5
template <bool FP8>
struct Packed {
  static constexpr int NCH = 256 * (FP8 ? 1 : 2) / 128;  // chunks per hidden layer
  static constexpr size_t OFF_HID = 0;                  // [layer 0..2][chunk] x CHUNK
  static constexpr size_t OFF_B1 = 3 * (size_t)NCH * CHUNK;  // 256 rows x 32 B, 32-byte swizzle
  static constexpr size_t OFF_B5 = OFF_B1 + 8192;       // 4 K-blocks x 16 rows x 128 B
  // biases of layers 2-4 as one block per layer of 256 rows x 32 B (32-byte
  // swizzle), K = 16 with the bias in columns 13 (BF16 value) and 14 (BF16
  // remainder), the others zero: b/2 (BF16 variant) or b/s_c (FP8 variant,
  // whose epilogue multiplies the accumulator by s_c/2)
  static constexpr size_t OFF_BIAS = OFF_B5 + 8192;
  static constexpr size_t BYTES = OFF_BIAS + 24576;
};

inline uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
  return (uint16_t)(u >> 16);
}

// element (row, k) of a 128-byte-swizzled K-major block whose rows are 128 B
inline size_t sw128_off(int row, int k) {
  const int c = k >> 3, e = k & 7;
  return (size_t)((row >> 3) * 1024 + (row & 7) * 128 + ((c ^ (row & 7)) << 4) + e * 2);
}

inline size_t sw32_off(int row, int k) {
  const int c = k >> 3, e = k & 7;
  return (size_t)((row >> 3) * 256 + (row & 7) * 32 + ((c ^ ((row >> 2) & 1)) << 4) + e * 2);
}

// byte b (0..127) of row `row` (0..255) in a weight chunk: 128-byte rows,
// 128-byte swizzle
inline size_t chunk_byte_off(int row, int b) {
  const int c = b >> 4, e = b & 15;
  return (size_t)((row >> 3) * 1024 + (row & 7) * 128 + ((c ^ (row & 7)) << 4) + e);
}

// Value of the E4M3 code k (0..126, sign clear): subnormal k/8 2^-6 for an
// exponent field of 0, else (1 + m/8) 2^(e-7); 126 is the largest, 448.
inline double e4m3_value(int k) {
  const int e = k >> 3, m = k & 7;
  return e == 0 ? std::ldexp(m / 8.0, -6) : std::ldexp(1.0 + m / 8.0, e - 7);
}

// Round to the nearest E4M3 value, ties to the even code, saturating at 448.
inline uint8_t e4m3_bits(double x) {
  const uint8_t sign = std::signbit(x) ? 0x80 : 0x00;
  const double a = std::fabs(x);
  if (!(a < 448.0)) return (uint8_t)(sign | 126);
  int lo = 0, hi = 126;  // e4m3_value(lo) <= a < e4m3_value(hi)
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (e4m3_value(mid) <= a) lo = mid;
    else hi = mid;
  }
  const double dl = a - e4m3_value(lo), dh = e4m3_value(hi) - a;
  const int k = dl < dh ? lo : (dh < dl ? hi : ((lo & 1) ? hi : lo));
  return (uint8_t)(sign | k);
}

// Layers 1 and 5 (BF16 in both variants) and the per-layer bias vectors.
inline void pack_b1_b5_bias(const float (*W)[256 * 256], const float (*b)[256], unsigned char *P,
                     size_t off_b1, size_t off_b5, float *bias_host, int nin) {
  auto put = [&](size_t off, float v) {
    const uint16_t u = bf16_bits(v);
    std::memcpy(P + off, &u, 2);
  };
  // layer 1: [x (4) for x_hi, x (4) again for x_lo, cond (5), 0 0, aspect]
  // (the aspect weight, input column 25, only for rectangular cells)
  for (int nrow = 0; nrow < 256; ++nrow) {
    const float *w = &W[0][nrow * nin];
    for (int k = 0; k < 4; ++k) {
      put(off_b1 + sw32_off(nrow, k), 0.5f * w[5 + k]);
      put(off_b1 + sw32_off(nrow, 4 + k), 0.5f * w[5 + k]);
    }
    for (int k = 0; k < 5; ++k) put(off_b1 + sw32_off(nrow, 8 + k), 0.5f * w[k]);
    if (nin > kPackIn) put(off_b1 + sw32_off(nrow, 15), 0.5f * w[kPackIn]);
  }
  // output layer: 16 rows (4 real) x 256 K in four 128-byte-swizzled K-blocks
  for (int d = 0; d < 4; ++d)
    for (int k = 0; k < 256; ++k)
      put(off_b5 + (size_t)(k >> 6) * 2048 + sw128_off(d, k & 63), W[4][d * 256 + k]);
  for (int i = 0; i < 5 * 256; ++i) bias_host[i] = 0.0f;
  for (int L = 1; L < 4; ++L)
    for (int c = 0; c < 256; ++c) bias_host[L * 256 + c] = 0.5f * b[L][c];
  for (int d = 0; d < 4; ++d) bias_host[4 * 256 + d] = b[4][d];
}

// W[l] = W_{l+1} [out][in] as in the weight file, b[l] its bias; M (the
// residual-modulated network only, else null) M_j[256][5]; nin = 25, or 26
// for a network of rectangular cells. Writes Packed<false>::BYTES bytes to
// packed_host and the FP32 biases [5][256] (rows 1..3 halved, row 4 = b5).
inline void tc_pack_host(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                  float *bias_host, const float (*M)[256 * kPackCond], int nin) {
  using PK = Packed<false>;
  unsigned char *P = (unsigned char *)packed_host;
  std::memset(P, 0, PK::BYTES);
  // hidden layers W2..W4: chunk ch holds all 256 output rows and inputs
  // 64 ch .. 64 ch + 63
  for (int L = 0; L < 3; ++L)
    for (int ch = 0; ch < PK::NCH; ++ch) {
      const size_t base = PK::OFF_HID + (size_t)(L * PK::NCH + ch) * CHUNK;
      for (int i = 0; i < 256; ++i)
        for (int j = 0; j < 64; ++j) {
          const uint16_t u = bf16_bits(0.5f * W[L + 1][i * 256 + 64 * ch + j]);
          std::memcpy(P + base + chunk_byte_off(i, 2 * j), &u, 2);
        }
    }
  pack_b1_b5_bias(W, b, P, PK::OFF_B1, PK::OFF_B5, bias_host, nin);
  // bias blocks of layers 2-4: b/2 = hi + lo, both BF16, against the two
  // constant-1 columns of the layer-1 operand
  for (int L = 0; L < 3; ++L)
    for (int c = 0; c < 256; ++c) {
      const float v = 0.5f * b[L + 1][c];
      const uint16_t hi = bf16_bits(v);
      float hif;
      const uint32_t hb = (uint32_t)hi << 16;
      std::memcpy(&hif, &hb, 4);
      const uint16_t lo = bf16_bits(v - hif);
      const size_t base = PK::OFF_BIAS + (size_t)L * 8192;
      std::memcpy(P + base + sw32_off(c, 13), &hi, 2);
      std::memcpy(P + base + sw32_off(c, 14), &lo, 2);
      // residual-modulated network: the condition shift M_l c / 2 against the
      // condition columns 8..12 of the layer-1 operand
      if (M)
        for (int k = 0; k < kPackCond; ++k) {
          const uint16_t u = bf16_bits(0.5f * M[L][c * kPackCond + k]);
          std::memcpy(P + base + sw32_off(c, 8 + k), &u, 2);
        }
    }
}

inline void tc_pack_host_fp8(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                      float *bias_host, float *scale_host, int nin) {
  using PK = Packed<true>;
  unsigned char *P = (unsigned char *)packed_host;
  std::memset(P, 0, PK::BYTES);
  // hidden layers W2..W4: row c as E4M3 codes of W[c][:] / s_c, s_c = amax / 448;
  // chunk ch holds all 256 output rows and inputs 128 ch ..
  for (int L = 0; L < 3; ++L)
    for (int i = 0; i < 256; ++i) {
      const float *w = &W[L + 1][i * 256];
      double amax = 0.0;
      for (int k = 0; k < 256; ++k) amax = std::fmax(amax, std::fabs((double)w[k]));
      const double sc = amax > 0.0 ? amax / 448.0 : 1.0;
      scale_host[L * 256 + i] = (float)(0.5 * sc);  // layers 2-4 carry a factor 1/2
      for (int k = 0; k < 256; ++k) {
        const int ch = k >> 7, j = k & 127;
        P[PK::OFF_HID + (size_t)(L * PK::NCH + ch) * CHUNK + chunk_byte_off(i, j)] =
            e4m3_bits((double)w[k] / sc);
      }
      // bias block: b / s_c as BF16 hi + lo (the epilogue scales by s_c / 2)
      const float v = (float)((double)b[L + 1][i] / sc);
      const uint16_t hi = bf16_bits(v);
      float hif;
      const uint32_t hb = (uint32_t)hi << 16;
      std::memcpy(&hif, &hb, 4);
      const uint16_t lo = bf16_bits(v - hif);
      std::memcpy(P + PK::OFF_BIAS + (size_t)L * 8192 + sw32_off(i, 13), &hi, 2);
      std::memcpy(P + PK::OFF_BIAS + (size_t)L * 8192 + sw32_off(i, 14), &lo, 2);
    }
  pack_b1_b5_bias(W, b, P, PK::OFF_B1, PK::OFF_B5, bias_host, nin);
}

}  // namespace pack
}  // namespace gmc
