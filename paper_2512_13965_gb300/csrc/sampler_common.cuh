// Device helpers and layouts shared by the tensor-core samplers of Eq. 8
// (sampler_tc.cu: one CTA per tile pair; sampler_pair.cu: a CTA pair per
// M = 256 tile): the packed weight buffer, the kernel parameters, the SiLU of
// the epilogue and the layer-1 operand row.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstring>

#include "gmc_internal.cuh"
#include "tc_pack.h"

namespace gmc {
namespace smp {

// the packed weight buffer's layout (tc_pack.h)
constexpr uint32_t CHUNK = pack::CHUNK;
template <bool FP8>
using Packed = pack::Packed<FP8>;

struct Params {
  const unsigned char *packed;
  const float *bias;    // [5][256]: rows 1..3 = b2..b4, row 4 = b5
  const float *bias1;   // [n_eval][256]: W1[:, emb] emb(t_e) + b1
  const float *scale;   // FP8 only: [3][256] per-output-channel scales of W2..W4, halved
  const float *rmg;     // residual-modulated network only: channel scales G [3][2][256]
  NetStats st;
  int64_t n;
  const float *cond;
  const float *noise;
  uint64_t seed, id0;
  int steps, integrator, n_eval;
  float *y_raw, *exitp;
  int *err;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &v, 4);
  return u;
}

// SiLU on two pre-activations already halved (the packed weights and biases
// of layers 1-4 carry a factor 1/2, exact in BF16): with h = z/2,
// SiLU(z) = z sigmoid(z) = h + h tanh(h). Packed BF16x2: one MUFU op and one
// FMA for two outputs, already in the operand format of the next layer.
__device__ __forceinline__ uint32_t silu2_halved(float h0, float h1) {
  uint32_t h, t, o;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(h1), "f"(h0));
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
  asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(o) : "r"(h), "r"(t));
  return o;
}

// As silu2_halved, rounded to two E4M3 codes (low byte from h0): the SiLU in
// packed FP16 (11-bit significand, so the E4M3 rounding sees an accurate
// value), then one saturating conversion.
__device__ __forceinline__ uint32_t silu2_halved_e4m3(float h0, float h1) {
  const __half2 hh = __floats2half2_rn(h0, h1);
  uint32_t h, t, o;
  memcpy(&h, &hh, 4);
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(h));
  asm("fma.rn.f16x2 %0, %1, %2, %1;" : "=r"(o) : "r"(h), "r"(t));
  __half2_raw raw;
  raw.x = (unsigned short)(o & 0xFFFFu);
  raw.y = (unsigned short)(o >> 16);
  return (uint32_t)__nv_cvt_halfraw2_to_fp8x2(raw, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

// 16 B chunk `c` (0..1) of row `r` in a 32-byte-swizzled block.
__device__ __forceinline__ uint32_t sw32(uint32_t base, int r, int c) {
  return base + (uint32_t)((r >> 3) * 256 + (r & 7) * 32 + ((c ^ ((r >> 2) & 1)) << 4));
}

// Layer-1 operand row: [x_hi0..3, x_lo0..3 | cn0..cn4, 1, 1, cn5] in BF16
// (cn5: the aspect of a rectangular cell, 0 for square-cell networks). The
// normalized condition (second 16 bytes) is written once per tile; every
// evaluation rewrites only the ODE state (first 16 bytes). Layer 1's weights
// are zero in columns 13-14; the bias blocks of layers 2-4 use them (and
// have zero in column 15).
__device__ __forceinline__ void write_a1_cond(uint32_t a_base, int r, const float (&cn)[kCondRect]) {
  st_shared_v4(sw32(a_base, r, 1), pack_bf16x2(cn[0], cn[1]), pack_bf16x2(cn[2], cn[3]),
               pack_bf16x2(cn[4], 1.0f), pack_bf16x2(1.0f, cn[5]));
}

// Standardized condition of row gi (< n) into cn (zeros past st.ncond and
// for rows past n).
__device__ __forceinline__ void load_cond(const float *cond, const NetStats &st, int64_t n,
                                          int64_t gi, bool valid, float (&cn)[kCondRect]) {
#pragma unroll
  for (int k = 0; k < kCondRect; ++k)
    cn[k] = valid && k < st.ncond ? (cond[k * n + gi] - st.cond_mean[k]) * st.cond_inv_std[k] : 0.0f;
}

__device__ __forceinline__ void write_a1_x(uint32_t a_base, int r, const float (&x)[4]) {
  float hi[4], lo[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    hi[d] = __bfloat162float(__float2bfloat16_rn(x[d]));
    lo[d] = x[d] - hi[d];
  }
  st_shared_v4(sw32(a_base, r, 0), pack_bf16x2(hi[0], hi[1]), pack_bf16x2(hi[2], hi[3]),
               pack_bf16x2(lo[0], lo[1]), pack_bf16x2(lo[2], lo[3]));
}

// Halved pre-activations of 4 accumulator columns: acc + bias.
__device__ __forceinline__ float4 pre4(const uint32_t *p, const float4 *b4, int q) {
  const float4 b = __ldg(b4 + q);
  return make_float4(__uint_as_float(p[0]) + b.x, __uint_as_float(p[1]) + b.y,
                     __uint_as_float(p[2]) + b.z, __uint_as_float(p[3]) + b.w);
}


// Epilogue pre-activation modes: the bias already in the accumulator (layers
// 2-4, whose biases enter through the MMA), bias added here (layer 1, whose
// bias depends on t), or a per-channel scale (FP8 layers 2-4, bias already in
// the accumulator in units of that scale).
enum : int { kPreNone = 0, kPreBias = 1, kPreScale = 2 };

// SiLU of one thread's 16 accumulator columns starting at col0, packed as the
// next layer's operand: 8 BF16x2 words or, with OUT8, 4 words of four E4M3
// codes (low byte first).
template <int MODE, bool OUT8>
__device__ __forceinline__ void silu16(const uint32_t *v, const float *__restrict__ bias,
                                       const float *__restrict__ scale, int col0, uint32_t (&w)[8]) {
  const float4 *b4 = reinterpret_cast<const float4 *>(bias + col0);
  const float4 *s4 = reinterpret_cast<const float4 *>(scale + col0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float4 z;
    if constexpr (MODE == kPreNone) {
      z = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                      __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
    } else {
      if constexpr (MODE == kPreScale) {
        const float4 sc = __ldg(s4 + q);
        z = make_float4(__uint_as_float(v[4 * q]) * sc.x, __uint_as_float(v[4 * q + 1]) * sc.y,
                        __uint_as_float(v[4 * q + 2]) * sc.z, __uint_as_float(v[4 * q + 3]) * sc.w);
      } else {
        z = pre4(v + 4 * q, b4, q);
      }
    }
    if constexpr (OUT8) {
      w[q] = silu2_halved_e4m3(z.x, z.y) | (silu2_halved_e4m3(z.z, z.w) << 16);
    } else {
      w[2 * q] = silu2_halved(z.x, z.y);
      w[2 * q + 1] = silu2_halved(z.z, z.w);
    }
  }
}

}  // namespace smp

// The CTA-pair BF16 sampler (sampler_pair.cu) for the arguments of one
// launch; `sms` is the device's SM count.
cudaError_t launch_sampler_pair(cudaStream_t stream, const smp::Params &p, int sms);

}  // namespace gmc
