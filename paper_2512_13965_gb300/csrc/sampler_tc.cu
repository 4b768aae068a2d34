// BF16 tensor-core flow-ODE sampler (Eq. 8) for sm_103a: tcgen05 MMA with
// FP32 accumulators in tensor memory, weights streamed by bulk async copies.
//
// Work unit: a tile of 128 particles. One persistent CTA per SM owns two
// tiles (X, Y) at a time and runs all K steps of both, ping-ponging them so
// that the tensor core computes one tile's layer while the epilogue warps
// turn the other tile's accumulator into the next layer's operand:
//
//   MMA warp:      L1(X) L1(Y) L2(X) L2(Y) ... L5(X) L5(Y) | next evaluation
//   epilogue warps:       E1(X) E1(Y) E2(X) ...              (bias, SiLU, BF16)
//
// Per evaluation of v_theta and tile (M = 128 rows):
//   L1: [cn | x_hi | x_lo] (K = 16, BF16) x B1 (N = 256)       -> TMEM
//       (the time-embedding columns of layer 1 are the same for every row,
//        so W1[:, emb] emb(t) + b1 is folded into an FP32 per-evaluation bias)
//   L2..L4: A (128 x 256 BF16, shared memory, 128-byte swizzle) x W
//       (256 x 256, streamed in chunks of all 256 output rows x CHUNK_K)
//       -> TMEM, N = 256 per MMA
//   L5: A x W5 (N = 16, rows 4..15 zero) -> TMEM columns 0..3
// Epilogue: SiLU(z) = h + h tanh(h) with h = z/2 (layers 1-4 are packed with
// weights and biases halved, so the accumulator holds h), in packed BF16x2,
// written back as the next layer's BF16 operand in the 128-byte-swizzled
// K-major layout. The ODE state x stays in FP32 registers of the row's
// epilogue thread.
//
// Roles: warp 0 streams weights, warp 1 owns tensor memory and issues MMAs,
// warps 2.. are the epilogue (EPI_WARPS / 4 threads per row).
// CTAs run in clusters of two that consume the same weight chunks in the
// same order: each CTA copies half of every chunk from L2 and multicasts it
// into both CTAs' stage, so L2 serves each chunk once per pair; a stage is
// refilled only after both CTAs' MMAs have released it.
// Every wait is bounded; a timeout sets *err and the CTA drains and exits.
//
// FP8 variant (template argument FP8): the three 256 x 256 layers (97% of the
// FLOPs) run as kind::f8f6f4 MMAs on E4M3 operands. Each output row c of
// W2..W4 is stored as E4M3 codes of W[c][:] / s_c with s_c = max_k |W[c][k]| / 448
// (per-output-channel scale, FP32), and the epilogue applies h = acc s_c / 2
// + b_c / 2 in one FMA. Activations entering layers 2-4 are E4M3 with unit
// scale (SiLU outputs are >= -0.279 and far below E4M3's 448). Layer 1 keeps
// BF16 operands (the ODE state enters through them) and layer 4's epilogue
// writes BF16, so layer 5 (the velocity) is the same BF16 MMA as above.
// A 16 KB weight chunk then holds 64 inputs instead of 32; byte offsets in
// the operand rows are the same, so descriptors advance identically.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstring>

#include "decode.cuh"
#include "gmc_internal.cuh"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace gmc {
namespace {

using namespace ptx;

constexpr int TM = 128;
#ifndef GMC_TC_CHUNK_K
#define GMC_TC_CHUNK_K 32
#endif
#ifndef GMC_TC_EPI_WARPS
#define GMC_TC_EPI_WARPS 16
#endif
// Weight chunk: all 256 output rows x CHUNK_K inputs, K-major; 32 -> 64-byte
// swizzle (16 KB), 64 -> 128-byte swizzle (32 KB).
constexpr int CHUNK_K = GMC_TC_CHUNK_K;
constexpr uint32_t CHUNK = 256u * CHUNK_K * 2u;
constexpr int MMAS_PER_CHUNK = CHUNK_K / 16;
constexpr uint32_t CHUNK_SWIZZLE = CHUNK_K == 32 ? 4u /* 64B */ : 2u /* 128B */;
constexpr uint32_t CHUNK_SBO = CHUNK_K == 32 ? 512u : 1024u;
constexpr int NST = (81920 / CHUNK) > 5 ? 5 : (int)(81920 / CHUNK);  // stages in 80 KB
#ifndef GMC_TC_SPLIT_TILES
#define GMC_TC_SPLIT_TILES 0  // measured on GB300: 1 is 8 % slower (6.65 vs 6.13 ms per 2^20 x 16 steps)
#endif
constexpr int EPI_WARPS = GMC_TC_EPI_WARPS;      // a multiple of 8 (2 groups x TMEM lane quadrants)
constexpr bool SPLIT_TILES = GMC_TC_SPLIT_TILES != 0;  // one epilogue group per tile
constexpr int TPW = SPLIT_TILES ? 1 : 2;          // tiles served by each epilogue warp
constexpr int GROUP_WARPS = SPLIT_TILES ? EPI_WARPS / 2 : EPI_WARPS;  // warps per tile
constexpr int EPI_COLS = 256 / (GROUP_WARPS / 4);  // accumulator columns per epilogue thread
#ifndef GMC_TC_EPI_CW
#define GMC_TC_EPI_CW 32
#endif
#ifndef GMC_TC_EPI_CW8
#define GMC_TC_EPI_CW8 16
#endif
constexpr int EPI_CW = GMC_TC_EPI_CW;    // accumulator columns per TMEM load, BF16 variant
constexpr int EPI_CW8 = GMC_TC_EPI_CW8;  // the same for the FP8 variant (more live registers)
static_assert((EPI_CW == 16 || EPI_CW == 32) && (EPI_CW8 == 16 || EPI_CW8 == 32), "TMEM load width");
constexpr int THREADS = 32 * (2 + EPI_WARPS);
static_assert(CHUNK_K == 32 || CHUNK_K == 64, "chunk K");
static_assert(EPI_WARPS == 8 || EPI_WARPS == 16, "epilogue warps");
constexpr int CLUSTER = 2;               // CTAs sharing each weight chunk by multicast
constexpr uint32_t SLICE = CHUNK / CLUSTER;
constexpr uint32_t TMEM_COLS = 512;     // two 128 x 256 FP32 accumulators
constexpr int ROW_BYTES = CHUNK_K * 2;  // bytes of one output row in a weight chunk

// packed global operand buffer (bytes): hidden-layer chunks, then the BF16
// operands of layers 1 and 5
template <bool FP8>
struct Packed {
  static constexpr int NCH = 256 * (FP8 ? 1 : 2) / ROW_BYTES;  // chunks per hidden layer
  static constexpr size_t OFF_HID = 0;                  // [layer 0..2][chunk] x CHUNK
  static constexpr size_t OFF_B1 = 3 * (size_t)NCH * CHUNK;  // 256 rows x 32 B, 32-byte swizzle
  static constexpr size_t OFF_B5 = OFF_B1 + 8192;      // 4 K-blocks x 16 rows x 128 B
  static constexpr size_t BYTES = OFF_B5 + 8192;
};

// shared memory (offsets from a 1024-byte aligned base)
constexpr uint32_t S_A0 = 0;                     // tile X operand, 64 KB
constexpr uint32_t S_A1 = 65536;                 // tile Y operand, 64 KB
constexpr uint32_t S_B1 = 131072;                // 8 KB
constexpr uint32_t S_B5 = 139264;                // 8 KB
constexpr uint32_t S_ST = 147456;                // NST weight stages
constexpr uint32_t S_BAR = S_ST + NST * CHUNK;   // barriers and flags
constexpr uint32_t S_TOTAL = S_BAR + 256;
constexpr uint32_t SMEM_BYTES = S_TOTAL + 1024;  // + alignment slack

struct Bars {
  uint64_t full[NST];
  uint64_t empty[NST];
  uint64_t res_full;
  uint64_t a_ready[2];
  uint64_t mma_done[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(Bars) <= 256, "barrier block");

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

// 16 B chunk `c` (0..7) of row `r` in a 128-byte-swizzled K-block.
__device__ __forceinline__ uint32_t sw128(uint32_t base, int r, int c) {
  return base + (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// 16 B chunk `c` (0..1) of row `r` in a 32-byte-swizzled block.
__device__ __forceinline__ uint32_t sw32(uint32_t base, int r, int c) {
  return base + (uint32_t)((r >> 3) * 256 + (r & 7) * 32 + ((c ^ ((r >> 2) & 1)) << 4));
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  // not .aligned: producer and MMA lanes reach this point after divergent loops
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Bulk copy global -> the same shared-memory offset of every CTA in `mask`,
// completing `bytes` on the barrier at the same offset in each of them.
__device__ __forceinline__ void bulk_g2s_multicast(void *dst, const void *src, uint32_t bytes,
                                                   uint64_t *bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// Arrive on the barrier at the same offset in every CTA of `mask` once this
// thread's tcgen05 operations have completed.
__device__ __forceinline__ void mma_commit_multicast(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
      "[%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__device__ void fail(Bars &b, int *err, int code) {
  b.abort = 1;
  atomicExch(err, code);
}

// Layer-1 operand row: [cn0..cn4, x_hi0..3, x_lo0..3, 0, 0, 0] in BF16.
__device__ __forceinline__ void write_a1(uint32_t a_base, int r, const float (&cn)[kCond],
                                        const float (&x)[4]) {
  float hi[4], lo[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    hi[d] = __bfloat162float(__float2bfloat16_rn(x[d]));
    lo[d] = x[d] - hi[d];
  }
  st_shared_v4(sw32(a_base, r, 0), pack_bf16x2(cn[0], cn[1]), pack_bf16x2(cn[2], cn[3]),
               pack_bf16x2(cn[4], hi[0]), pack_bf16x2(hi[1], hi[2]));
  st_shared_v4(sw32(a_base, r, 1), pack_bf16x2(hi[3], lo[0]), pack_bf16x2(lo[1], lo[2]),
               pack_bf16x2(lo[3], 0.0f), pack_bf16x2(0.0f, 0.0f));
}

// Halved pre-activations of 4 accumulator columns: acc + bias, or with
// SCALED (an FP8 layer) acc * scale + bias.
template <bool SCALED>
__device__ __forceinline__ float4 pre4(const uint32_t *p, const float4 *b4, const float4 *s4, int q) {
  const float4 b = __ldg(b4 + q);
  float4 z;
  if constexpr (SCALED) {
    const float4 sc = __ldg(s4 + q);
    z.x = fmaf(__uint_as_float(p[0]), sc.x, b.x);
    z.y = fmaf(__uint_as_float(p[1]), sc.y, b.y);
    z.z = fmaf(__uint_as_float(p[2]), sc.z, b.z);
    z.w = fmaf(__uint_as_float(p[3]), sc.w, b.w);
  } else {
    z.x = __uint_as_float(p[0]) + b.x;
    z.y = __uint_as_float(p[1]) + b.y;
    z.z = __uint_as_float(p[2]) + b.z;
    z.w = __uint_as_float(p[3]) + b.w;
  }
  return z;
}

// bias (and scale) + SiLU on 32 accumulator columns starting at col0,
// stored into the next layer's operand row r: BF16 (four 16-byte chunks of
// a 64-column K-block) or, with OUT8, E4M3 (two 16-byte chunks of a
// 128-column K-block). Both K-blocks have 128-byte rows, 128-byte swizzle.
template <bool SCALED, bool OUT8>
__device__ __forceinline__ void epi32(const uint32_t (&v)[32], const float *__restrict__ bias,
                                      const float *__restrict__ scale, int col0, uint32_t a_base,
                                      int r) {
  const float4 *b4 = reinterpret_cast<const float4 *>(bias + col0);
  const float4 *s4 = SCALED ? reinterpret_cast<const float4 *>(scale + col0) : nullptr;
  if constexpr (OUT8) {
    const uint32_t kb_base = a_base + (uint32_t)(col0 >> 7) * 16384u;
    const int c0 = (col0 & 127) >> 4;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = 4 * j + i;
        const float4 z = pre4<SCALED>(v + 4 * q, b4, s4, q);
        w[i] = silu2_halved_e4m3(z.x, z.y) | (silu2_halved_e4m3(z.z, z.w) << 16);
      }
      st_shared_v4(sw128(kb_base, r, c0 + j), w[0], w[1], w[2], w[3]);
    }
  } else {
    const uint32_t kb_base = a_base + (uint32_t)(col0 >> 6) * 16384u;
    const int c0 = (col0 & 63) >> 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 za = pre4<SCALED>(v + 8 * j, b4, s4, 2 * j);
      const float4 zb = pre4<SCALED>(v + 8 * j + 4, b4, s4, 2 * j + 1);
      st_shared_v4(sw128(kb_base, r, c0 + j), silu2_halved(za.x, za.y), silu2_halved(za.z, za.w),
                   silu2_halved(zb.x, zb.y), silu2_halved(zb.z, zb.w));
    }
  }
}

// bias (and scale) + SiLU on 16 accumulator columns starting at col0 (a
// multiple of 16): one 16-byte E4M3 chunk, or with !OUT8 two BF16 chunks.
template <bool SCALED, bool OUT8>
__device__ __forceinline__ void epi16(const uint32_t (&v)[16], const float *__restrict__ bias,
                                      const float *__restrict__ scale, int col0, uint32_t a_base,
                                      int r) {
  const float4 *b4 = reinterpret_cast<const float4 *>(bias + col0);
  const float4 *s4 = SCALED ? reinterpret_cast<const float4 *>(scale + col0) : nullptr;
  if constexpr (OUT8) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 z = pre4<SCALED>(v + 4 * q, b4, s4, q);
      w[q] = silu2_halved_e4m3(z.x, z.y) | (silu2_halved_e4m3(z.z, z.w) << 16);
    }
    st_shared_v4(sw128(a_base + (uint32_t)(col0 >> 7) * 16384u, r, (col0 & 127) >> 4), w[0], w[1],
                 w[2], w[3]);
  } else {
    const uint32_t kb_base = a_base + (uint32_t)(col0 >> 6) * 16384u;
    const int c0 = (col0 & 63) >> 3;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float4 za = pre4<SCALED>(v + 8 * j, b4, s4, 2 * j);
      const float4 zb = pre4<SCALED>(v + 8 * j + 4, b4, s4, 2 * j + 1);
      st_shared_v4(sw128(kb_base, r, c0 + j), silu2_halved(za.x, za.y), silu2_halved(za.z, za.w),
                   silu2_halved(zb.x, zb.y), silu2_halved(zb.z, zb.w));
    }
  }
}

// One epilogue thread's EPI_COLS columns of a 128 x 256 accumulator: the
// load of the next 32 (CW = 32) or 16 (CW = 16, fewer live registers)
// columns is in flight while the current ones are converted and stored.
template <bool SCALED, bool OUT8, int CW = 32>
__device__ __forceinline__ void epi_layer(uint32_t tcol, const float *__restrict__ bias,
                                          const float *__restrict__ scale, int col0,
                                          uint32_t a_base, int r) {
  constexpr int NCH = EPI_COLS / CW;
  uint32_t buf[2][CW];
  if constexpr (CW == 32) {
    tmem_ld32_raw(tcol, buf[0]);
    tmem_wait_ld_regs(buf[0]);
  } else {
    tmem_ld16_raw(tcol, buf[0]);
    tmem_wait_ld_regs16(buf[0]);
  }
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    if constexpr (CW == 32) {
      if (j + 1 < NCH) tmem_ld32_raw(tcol + 32u * (uint32_t)(j + 1), buf[(j + 1) & 1]);
      epi32<SCALED, OUT8>(buf[j & 1], bias, scale, col0 + 32 * j, a_base, r);
      if (j + 1 < NCH) tmem_wait_ld_regs(buf[(j + 1) & 1]);
    } else {
      if (j + 1 < NCH) tmem_ld16_raw(tcol + 16u * (uint32_t)(j + 1), buf[(j + 1) & 1]);
      epi16<SCALED, OUT8>(buf[j & 1], bias, scale, col0 + 16 * j, a_base, r);
      if (j + 1 < NCH) tmem_wait_ld_regs16(buf[(j + 1) & 1]);
    }
  }
}

struct Params {
  const unsigned char *packed;
  const float *bias;    // [5][256]: rows 1..3 = b2..b4, row 4 = b5
  const float *bias1;   // [n_eval][256]: W1[:, emb] emb(t_e) + b1
  const float *scale;   // FP8 only: [3][256] per-output-channel scales of W2..W4, halved
  NetStats st;
  int64_t n;
  const float *cond;
  const float *noise;
  uint64_t seed, id0;
  int steps, integrator, n_eval;
  float *y_raw, *exitp;
  int *err;
};

// INTEG: the integrator (GMC_EULER, GMC_MIDPOINT, GMC_RK4) as a compile-time
// choice, so an Euler kernel holds no midpoint or RK4 state in registers.
template <bool FP8, int INTEG>
__global__ void __launch_bounds__(THREADS, 1) sampler_tc_kernel(Params P) {
  using PK = Packed<FP8>;
  constexpr int NCH = PK::NCH;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw_addr & 1023u)) & 1023u;
  unsigned char *sm = smem_raw + pad;
  const uint32_t sbase = raw_addr + pad;
  Bars &B = *reinterpret_cast<Bars *>(sm + S_BAR);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&B.full[s], 1);
      mbar_init(&B.empty[s], CLUSTER);
    }
    mbar_init(&B.res_full, 1);
    for (int t = 0; t < 2; ++t) {
      mbar_init(&B.a_ready[t], GROUP_WARPS);
      mbar_init(&B.mma_done[t], 1);
    }
    mbar_init(&B.drain, 1);
    B.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&B.tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // peers multicast into this CTA's barriers only after they exist
  tc_fence_after();
  const uint32_t tmem = B.tmem_base;
  volatile int *abort = &B.abort;
  const uint32_t rank = cluster_rank();
  const uint16_t all_ctas = (uint16_t)((1u << CLUSTER) - 1u);

  const int64_t ntiles = (P.n + TM - 1) / TM;
  const int64_t npairs = (ntiles + 1) / 2;
  // every CTA of a cluster runs the same number of pairs (the chunk stream is
  // shared); pairs past the end have no valid rows
  const int64_t n_iter = (npairs + gridDim.x - 1) / gridDim.x;
  const float h = 1.0f / (float)P.steps;

  if (warp == 0) {
    // ---------------- weight producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      mbar_arrive_expect_tx(&B.res_full, 16384);
      bulk_g2s(sm + S_B1, P.packed + PK::OFF_B1, 8192, &B.res_full);
      bulk_g2s(sm + S_B5, P.packed + PK::OFF_B5, 8192, &B.res_full);
      for (int64_t ip = 0; ip < n_iter && ok; ++ip)
        for (int e = 0; e < P.n_eval && ok; ++e)
          for (int L = 0; L < 3 && ok; ++L)
            for (int T = 0; T < 2 && ok; ++T)
              for (int ch = 0; ch < NCH; ++ch) {
                const int s = it % NST;
                const uint32_t round = it / NST;
                if (!mbar_wait(&B.empty[s], (round & 1u) ^ 1u, abort)) {
                  fail(B, P.err, 1);
                  ok = false;
                  break;
                }
                mbar_arrive_expect_tx(&B.full[s], CHUNK);
                bulk_g2s_multicast(sm + S_ST + s * CHUNK + rank * SLICE,
                                   P.packed + PK::OFF_HID + (size_t)(L * NCH + ch) * CHUNK + rank * SLICE,
                                   SLICE, &B.full[s], all_ctas);
                ++it;
              }
      if (!ok) {
        // drain: every issued copy lands before the CTA exits
        int never = 0;
        for (uint32_t k = (it > NST ? it - NST : 0); k < it; ++k)
          mbar_wait(&B.full[k % NST], (k / NST) & 1u, &never, 1000000000ull);
        mbar_wait(&B.res_full, 0, &never, 1000000000ull);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // The issuing thread shares its scheduler with busy epilogue warps, so the
    // loop is kept lean: descriptors are built once and advanced by constant
    // offsets (the start-address field counts 16-byte units), the chunk loop
    // is unrolled, and a stage that has already landed costs one try_wait.
    if (lane == 0) {
      bool ok = mbar_wait(&B.res_full, 0, abort);
      if (!ok) fail(B, P.err, 2);
      uint32_t aph[2] = {0, 0};
      uint32_t stage = 0, sph = 0;  // next weight stage and its phase parity
      const uint32_t id256 = idesc_bf16_m128(256), id16 = idesc_bf16_m128(16);
      const uint32_t idh = FP8 ? idesc_e4m3_m128(256) : id256;  // hidden layers
      const uint64_t dA[2] = {smem_desc(sbase + S_A0, 1024, kSwizzle128B),
                              smem_desc(sbase + S_A1, 1024, kSwizzle128B)};
      const uint64_t dA1[2] = {smem_desc(sbase + S_A0, 256, kSwizzle32B),
                               smem_desc(sbase + S_A1, 256, kSwizzle32B)};
      const uint64_t dB1 = smem_desc(sbase + S_B1, 256, kSwizzle32B);
      const uint64_t dB5 = smem_desc(sbase + S_B5, 1024, kSwizzle128B);
      const uint64_t dST = smem_desc(sbase + S_ST, CHUNK_SBO, CHUNK_SWIZZLE);
      for (int64_t ip = 0; ip < n_iter && ok; ++ip)
        for (int e = 0; e < P.n_eval && ok; ++e)
          for (int L = 0; L < 5 && ok; ++L)
            for (int T = 0; T < 2 && ok; ++T) {
              if (!mbar_try_wait(&B.a_ready[T], aph[T] & 1u) &&
                  !mbar_wait(&B.a_ready[T], aph[T] & 1u, abort)) {
                fail(B, P.err, 3);
                ok = false;
                break;
              }
              ++aph[T];
              tc_fence_after();
              const uint32_t d = tmem + (uint32_t)T * 256u;
              if (L == 0) {
                mma_f16(d, dA1[T], dB1, id256, 0);
              } else if (L < 4) {
                const uint64_t a0 = dA[T];
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                  if (!mbar_try_wait(&B.full[stage], sph) && !mbar_wait(&B.full[stage], sph, abort)) {
                    fail(B, P.err, 4);
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                  // chunk ch = operand bytes ROW_BYTES ch .. of all 256 output
                  // rows (CHUNK_K BF16 or 2 CHUNK_K E4M3 inputs): A at K-block
                  // (ROW_BYTES ch)/128, byte (ROW_BYTES ch) % 128 of its rows;
                  // each MMA takes 32 bytes of K
                  const int kb = ch * ROW_BYTES;
                  const uint64_t a_ch = a0 + (uint64_t)((kb >> 7) * 1024 + ((kb & 127) >> 4));
                  const uint64_t b_ch = dST + (uint64_t)(stage * (CHUNK >> 4));
#pragma unroll
                  for (int k = 0; k < MMAS_PER_CHUNK; ++k) {
                    if constexpr (FP8)
                      mma_f8(d, a_ch + (uint64_t)(2 * k), b_ch + (uint64_t)(2 * k), idh,
                             (ch | k) != 0);
                    else
                      mma_f16(d, a_ch + (uint64_t)(2 * k), b_ch + (uint64_t)(2 * k), idh,
                              (ch | k) != 0);
                  }
                  mma_commit_multicast(&B.empty[stage], all_ctas);
                  if (++stage == NST) {
                    stage = 0;
                    sph ^= 1u;
                  }
                }
                if (!ok) break;
              } else {
                const uint64_t a0 = dA[T];
#pragma unroll
                for (int kb = 0; kb < 4; ++kb)
#pragma unroll
                  for (int k = 0; k < 4; ++k)
                    mma_f16(d, a0 + (uint64_t)(kb * 1024 + k * 2), dB5 + (uint64_t)(kb * 128 + k * 2),
                            id16, (kb | k) != 0);
              }
              mma_commit(&B.mma_done[T]);
            }
      // all issued MMAs complete before tensor memory is released
      mma_commit(&B.drain);
      int never = 0;
      mbar_wait(&B.drain, 0, &never, 1000000000ull);
    }
  } else {
    // ---------------- epilogue ----------------
    // SPLIT_TILES: warps 2 .. 2+GROUP-1 serve tile X and the rest tile Y, so
    // one group converts its accumulator while the other waits for its MMA;
    // otherwise every epilogue warp serves both tiles in turn.
    const int ew = warp - 2;
    const int t0 = SPLIT_TILES ? ew / GROUP_WARPS : 0;  // first tile of this warp
    const int q = warp & 3;                             // TMEM lane quadrant of the warp
    const int hf = (ew % GROUP_WARPS) >> 2;             // column part within the group
    const int r = 32 * q + lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    float cn[TPW][kCond], x[TPW][4], xm[TPW][4], ka[TPW][4];
    uint32_t dph[TPW];
#pragma unroll
    for (int tt = 0; tt < TPW; ++tt) dph[tt] = 0;
    bool ok = true;
    for (int64_t ip = 0; ip < n_iter && ok; ++ip) {
      const int64_t pr = blockIdx.x + ip * gridDim.x;
#pragma unroll
      for (int tt = 0; tt < TPW; ++tt) {
        const int T = t0 + tt;
        const int64_t g = (2 * pr + T) * TM + r;
        const bool valid = g < P.n;
        if (hf == 0) {
#pragma unroll
          for (int k = 0; k < kCond; ++k)
            cn[tt][k] = valid ? (P.cond[k * P.n + g] - P.st.cond_mean[k]) * P.st.cond_inv_std[k] : 0.0f;
          if (!valid) {
#pragma unroll
            for (int d = 0; d < 4; ++d) x[tt][d] = 0.0f;
          } else if (P.noise) {
#pragma unroll
            for (int d = 0; d < 4; ++d) x[tt][d] = P.noise[d * P.n + g];
          } else {
            const float4 z = box_muller4(philox_draw(P.seed, P.id0 + (uint64_t)g, 0u, kTagNoise));
            x[tt][0] = z.x;
            x[tt][1] = z.y;
            x[tt][2] = z.z;
            x[tt][3] = z.w;
          }
          write_a1(sbase + (T ? S_A1 : S_A0), r, cn[tt], x[tt]);
          fence_proxy_async_smem();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.a_ready[T]);
      }
      for (int e = 0; e < P.n_eval && ok; ++e) {
        for (int L = 0; L < 4 && ok; ++L)
#pragma unroll
          for (int tt = 0; tt < TPW; ++tt) {
            const int T = t0 + tt;
            if (!mbar_wait(&B.mma_done[T], dph[tt] & 1u, abort)) {
              fail(B, P.err, 5);
              ok = false;
              break;
            }
            ++dph[tt];
            tc_fence_after();
            const float *bias = L == 0 ? P.bias1 + (size_t)e * 256 : P.bias + L * 256;
            const uint32_t a_base = sbase + (T ? S_A1 : S_A0);
            const uint32_t tcol = tmem + lane_off + (uint32_t)T * 256u + (uint32_t)(hf * EPI_COLS);
            const int col0 = hf * EPI_COLS;
            if constexpr (FP8) {
              // layer 1 (BF16 MMA) and layers 2-3 feed E4M3 operands; layer 4
              // feeds the BF16 operand of layer 5
              if (L == 0)
                epi_layer<false, true, EPI_CW8>(tcol, bias, nullptr, col0, a_base, r);
              else if (L < 3)
                epi_layer<true, true, EPI_CW8>(tcol, bias, P.scale + (L - 1) * 256, col0, a_base, r);
              else
                epi_layer<true, false, EPI_CW8>(tcol, bias, P.scale + 2 * 256, col0, a_base, r);
            } else {
              epi_layer<false, false, EPI_CW>(tcol, bias, nullptr, col0, a_base, r);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.a_ready[T]);
          }
        if (!ok) break;
        const bool last = e == P.n_eval - 1;
#pragma unroll
        for (int tt = 0; tt < TPW; ++tt) {
          const int T = t0 + tt;
          if (!mbar_wait(&B.mma_done[T], dph[tt] & 1u, abort)) {
            fail(B, P.err, 6);
            ok = false;
            break;
          }
          ++dph[tt];
          tc_fence_after();
          if (hf == 0) {
            float v[4];
            tmem_ld4(tmem + lane_off + (uint32_t)T * 256u, v);
            tmem_wait_ld_regs4(v);
#pragma unroll
            for (int d = 0; d < 4; ++d) v[d] += __ldg(P.bias + 4 * 256 + d);
            float *xin = x[tt];
            if (INTEG == GMC_MIDPOINT && (e & 1) == 0) {
#pragma unroll
              for (int d = 0; d < 4; ++d) xm[tt][d] = fmaf(0.5f * h, v[d], x[tt][d]);
              xin = xm[tt];
            } else if (INTEG == GMC_RK4) {
              // evaluation e % 4 = i gives k_{i+1}; ka = k1 + 2 k2 + 2 k3 + k4
              const int i = e & 3;
              if (i == 3) {
#pragma unroll
                for (int d = 0; d < 4; ++d) x[tt][d] = fmaf(h * (1.0f / 6.0f), ka[tt][d] + v[d], x[tt][d]);
              } else {
                const float wgt = i == 0 ? 1.0f : 2.0f, hs = i == 2 ? h : 0.5f * h;
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                  ka[tt][d] = i == 0 ? v[d] : fmaf(wgt, v[d], ka[tt][d]);
                  xm[tt][d] = fmaf(hs, v[d], x[tt][d]);
                }
                xin = xm[tt];
              }
            } else {
#pragma unroll
              for (int d = 0; d < 4; ++d) x[tt][d] = fmaf(h, v[d], x[tt][d]);
            }
            if (!last) {
              float xi[4] = {xin[0], xin[1], xin[2], xin[3]};
              write_a1(sbase + (T ? S_A1 : S_A0), r, cn[tt], xi);
              fence_proxy_async_smem();
            }
          }
          tc_fence_before();
          __syncwarp();
          if (!last && lane == 0) mbar_arrive(&B.a_ready[T]);
          if (last && hf == 0) {
            const int64_t g = (2 * pr + T) * TM + r;
            if (g < P.n) {
              if (P.y_raw) {
#pragma unroll
                for (int d = 0; d < 4; ++d) P.y_raw[d * P.n + g] = x[tt][d];
              }
              if (P.exitp) {
                bool inward;
                const float4 o = decode_exit(x[tt][0], x[tt][1], x[tt][2], x[tt][3], P.st, &inward);
                P.exitp[g] = o.x;
                P.exitp[P.n + g] = o.y;
                P.exitp[2 * P.n + g] = o.z;
                P.exitp[3 * P.n + g] = o.w;
              }
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();  // no peer multicasts into this CTA's barriers after it exits
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// bias1[e][c] = b1[c] + sum_j W1[c][9 + j] emb_j(t_e), FP32.
__global__ void layer1_bias_kernel(const float *__restrict__ w1t, const float *__restrict__ b1,
                                   int steps, int integrator, int n_eval, float *__restrict__ out) {
  const int e = blockIdx.x, c = threadIdx.x;
  if (e >= n_eval) return;
  const float h = 1.0f / (float)steps;
  float t;
  if (integrator == GMC_MIDPOINT) {
    t = (float)(e >> 1) * h + (float)(e & 1) * 0.5f * h;
  } else if (integrator == GMC_RK4) {
    const int i = e & 3;  // stage times t_k, t_k + h/2, t_k + h/2, t_k + h
    t = (float)(e >> 2) * h + (i == 0 ? 0.0f : (i == 3 ? h : 0.5f * h));
  } else {
    t = (float)e * h;
  }
  float acc = b1[c];
  for (int j = 0; j < kEmb; ++j) acc = fmaf(w1t[(kCond + kState + j) * kHidden + c], time_embedding(j, t), acc);
  out[(size_t)e * kHidden + c] = 0.5f * acc;  // layers 1-4 carry a factor 1/2
}

uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
  return (uint16_t)(u >> 16);
}

// element (row, k) of a 128-byte-swizzled K-major block whose rows are 128 B
size_t sw128_off(int row, int k) {
  const int c = k >> 3, e = k & 7;
  return (size_t)((row >> 3) * 1024 + (row & 7) * 128 + ((c ^ (row & 7)) << 4) + e * 2);
}

size_t sw32_off(int row, int k) {
  const int c = k >> 3, e = k & 7;
  return (size_t)((row >> 3) * 256 + (row & 7) * 32 + ((c ^ ((row >> 2) & 1)) << 4) + e * 2);
}

// byte b of row `row` in a weight chunk (ROW_BYTES-byte rows: 64-byte swizzle
// for 64, 128-byte swizzle for 128)
size_t chunk_byte_off(int row, int b) {
  const int c = b >> 4, e = b & 15;
  if (ROW_BYTES == 64)
    return (size_t)((row >> 3) * 512 + (row & 7) * 64 + ((c ^ ((row >> 1) & 3)) << 4) + e);
  return (size_t)((row >> 3) * 1024 + (row & 7) * 128 + ((c ^ (row & 7)) << 4) + e);
}

// Value of the E4M3 code k (0..126, sign clear): subnormal k/8 2^-6 for an
// exponent field of 0, else (1 + m/8) 2^(e-7); 126 is the largest, 448.
double e4m3_value(int k) {
  const int e = k >> 3, m = k & 7;
  return e == 0 ? std::ldexp(m / 8.0, -6) : std::ldexp(1.0 + m / 8.0, e - 7);
}

// Round to the nearest E4M3 value, ties to the even code, saturating at 448.
uint8_t e4m3_bits(double x) {
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
void pack_b1_b5_bias(const float (*W)[256 * 256], const float (*b)[256], unsigned char *P,
                     size_t off_b1, size_t off_b5, float *bias_host) {
  auto put = [&](size_t off, float v) {
    const uint16_t u = bf16_bits(v);
    std::memcpy(P + off, &u, 2);
  };
  // layer 1: [cond (5), x (4) for x_hi, x (4) again for x_lo, 0 0 0]
  for (int nrow = 0; nrow < 256; ++nrow) {
    const float *w = &W[0][nrow * 25];
    for (int k = 0; k < 5; ++k) put(off_b1 + sw32_off(nrow, k), 0.5f * w[k]);
    for (int k = 0; k < 4; ++k) {
      put(off_b1 + sw32_off(nrow, 5 + k), 0.5f * w[5 + k]);
      put(off_b1 + sw32_off(nrow, 9 + k), 0.5f * w[5 + k]);
    }
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

}  // namespace

size_t tc_packed_bytes(bool fp8) { return fp8 ? Packed<true>::BYTES : Packed<false>::BYTES; }

void tc_pack_host(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                  float *bias_host) {
  using PK = Packed<false>;
  unsigned char *P = (unsigned char *)packed_host;
  std::memset(P, 0, PK::BYTES);
  // hidden layers W2..W4: chunk ch holds all 256 output rows and K CHUNK_K ch ..
  for (int L = 0; L < 3; ++L)
    for (int ch = 0; ch < PK::NCH; ++ch) {
      const size_t base = PK::OFF_HID + (size_t)(L * PK::NCH + ch) * CHUNK;
      for (int i = 0; i < 256; ++i)
        for (int j = 0; j < CHUNK_K; ++j) {
          const uint16_t u = bf16_bits(0.5f * W[L + 1][i * 256 + ch * CHUNK_K + j]);
          std::memcpy(P + base + chunk_byte_off(i, 2 * j), &u, 2);
        }
    }
  pack_b1_b5_bias(W, b, P, PK::OFF_B1, PK::OFF_B5, bias_host);
}

void tc_pack_host_fp8(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                      float *bias_host, float *scale_host) {
  using PK = Packed<true>;
  unsigned char *P = (unsigned char *)packed_host;
  std::memset(P, 0, PK::BYTES);
  // hidden layers W2..W4: row c as E4M3 codes of W[c][:] / s_c, s_c = amax / 448;
  // chunk ch holds all 256 output rows and K ROW_BYTES ch ..
  for (int L = 0; L < 3; ++L)
    for (int i = 0; i < 256; ++i) {
      const float *w = &W[L + 1][i * 256];
      double amax = 0.0;
      for (int k = 0; k < 256; ++k) amax = std::fmax(amax, std::fabs((double)w[k]));
      const double sc = amax > 0.0 ? amax / 448.0 : 1.0;
      scale_host[L * 256 + i] = (float)(0.5 * sc);  // layers 2-4 carry a factor 1/2
      for (int k = 0; k < 256; ++k) {
        const int ch = k / ROW_BYTES, j = k % ROW_BYTES;
        P[PK::OFF_HID + (size_t)(L * PK::NCH + ch) * CHUNK + chunk_byte_off(i, j)] =
            e4m3_bits((double)w[k] / sc);
      }
    }
  pack_b1_b5_bias(W, b, P, PK::OFF_B1, PK::OFF_B5, bias_host);
}

namespace {
template <bool FP8, int INTEG>
cudaError_t launch_tc(cudaStream_t stream, const Params &p, int sms) {
  auto kernel = sampler_tc_kernel<FP8, INTEG>;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.n + TM - 1) / TM, npairs = (ntiles + 1) / 2;
  int64_t g = npairs < sms ? npairs : sms;
  g = (g + CLUSTER - 1) / CLUSTER * CLUSTER;
  if (g > sms / CLUSTER * CLUSTER) g = sms / CLUSTER * CLUSTER;
  const int grid = (int)g;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  lc.blockDim = dim3(THREADS);
  lc.dynamicSmemBytes = SMEM_BYTES;
  lc.stream = stream;
  // a persistent grid must be co-resident: at most the clusters that fit
  static int max_clusters = -1;
  if (max_clusters < 0) {
    lc.gridDim = dim3((unsigned)(sms / CLUSTER * CLUSTER));
    int mc = 0;
    if (cudaOccupancyMaxActiveClusters(&mc, kernel, &lc) != cudaSuccess || mc < 1) {
      cudaGetLastError();
      mc = sms / CLUSTER;
    }
    max_clusters = mc;
  }
  const int grid_fit = grid < max_clusters * CLUSTER ? grid : max_clusters * CLUSTER;
  lc.gridDim = dim3((unsigned)grid_fit);
  e = cudaLaunchKernelEx(&lc, kernel, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_sampler_tc(cudaStream_t stream, const void *packed, const float *bias,
                              const NetF32 &f32, const NetStats &st, int64_t n, const float *cond,
                              const float *noise, uint64_t seed, uint64_t id0, int steps,
                              int integrator, float *y_raw, float *exit, int *err,
                              float *bias1_scratch, const float *fp8_scale) {
  if (n <= 0) return cudaSuccess;
  const int n_eval = integrator == GMC_RK4 ? 4 * steps : (integrator == GMC_MIDPOINT ? 2 * steps : steps);
  layer1_bias_kernel<<<n_eval, kHidden, 0, stream>>>(f32.w1t, f32.b1, steps, integrator, n_eval,
                                                     bias1_scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  Params p;
  p.packed = (const unsigned char *)packed;
  p.bias = bias;
  p.bias1 = bias1_scratch;
  p.scale = fp8_scale;
  p.st = st;
  p.n = n;
  p.cond = cond;
  p.noise = noise;
  p.seed = seed;
  p.id0 = id0;
  p.steps = steps;
  p.integrator = integrator;
  p.n_eval = n_eval;
  p.y_raw = y_raw;
  p.exitp = exit;
  p.err = err;
  if (fp8_scale) {
    if (integrator == GMC_RK4) return launch_tc<true, GMC_RK4>(stream, p, sms);
    if (integrator == GMC_MIDPOINT) return launch_tc<true, GMC_MIDPOINT>(stream, p, sms);
    return launch_tc<true, GMC_EULER>(stream, p, sms);
  }
  if (integrator == GMC_RK4) return launch_tc<false, GMC_RK4>(stream, p, sms);
  if (integrator == GMC_MIDPOINT) return launch_tc<false, GMC_MIDPOINT>(stream, p, sms);
  return launch_tc<false, GMC_EULER>(stream, p, sms);
}

}  // namespace gmc
