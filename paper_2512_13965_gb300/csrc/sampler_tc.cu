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
#include <cuda_bf16.h>

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
constexpr int CHUNKS = 256 / CHUNK_K;             // per hidden layer
constexpr int MMAS_PER_CHUNK = CHUNK_K / 16;
constexpr uint32_t CHUNK_SWIZZLE = CHUNK_K == 32 ? 4u /* 64B */ : 2u /* 128B */;
constexpr uint32_t CHUNK_SBO = CHUNK_K == 32 ? 512u : 1024u;
constexpr int NST = (81920 / CHUNK) > 5 ? 5 : (int)(81920 / CHUNK);  // stages in 80 KB
constexpr int EPI_WARPS = GMC_TC_EPI_WARPS;      // a multiple of 4 (TMEM lane quadrants)
constexpr int EPI_COLS = 256 / (EPI_WARPS / 4);   // accumulator columns per epilogue thread
constexpr int EPI_CH = EPI_COLS / 32;             // 32-column TMEM loads per thread
constexpr int THREADS = 32 * (2 + EPI_WARPS);
static_assert(CHUNK_K == 32 || CHUNK_K == 64, "chunk K");
static_assert(EPI_WARPS == 8 || EPI_WARPS == 16, "epilogue warps");
constexpr int CLUSTER = 2;               // CTAs sharing each weight chunk by multicast
constexpr uint32_t SLICE = CHUNK / CLUSTER;
constexpr uint32_t TMEM_COLS = 512;     // two 128 x 256 FP32 accumulators

// packed global operand buffer (bytes)
constexpr size_t OFF_HID = 0;                    // [layer 0..2][chunk 0..7] x 16 KB
constexpr size_t OFF_B1 = 3 * CHUNKS * CHUNK;    // 256 rows x 32 B, 32-byte swizzle
constexpr size_t OFF_B5 = OFF_B1 + 8192;         // 4 K-blocks x 16 rows x 128 B
constexpr size_t PACKED = OFF_B5 + 8192;

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

// bias + SiLU on 32 accumulator columns starting at col0, stored as four
// 16-byte chunks of the next layer's operand row r.
__device__ __forceinline__ void epi32(const uint32_t (&v)[32], const float *__restrict__ bias,
                                      int col0, uint32_t a_base, int r) {
  const float4 *b4 = reinterpret_cast<const float4 *>(bias + col0);
  const uint32_t kb_base = a_base + (uint32_t)(col0 >> 6) * 16384u;
  const int c0 = (col0 & 63) >> 3;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 ba = __ldg(b4 + 2 * j), bb = __ldg(b4 + 2 * j + 1);
    const uint32_t *p = v + 8 * j;
    st_shared_v4(sw128(kb_base, r, c0 + j),
                 silu2_halved(__uint_as_float(p[0]) + ba.x, __uint_as_float(p[1]) + ba.y),
                 silu2_halved(__uint_as_float(p[2]) + ba.z, __uint_as_float(p[3]) + ba.w),
                 silu2_halved(__uint_as_float(p[4]) + bb.x, __uint_as_float(p[5]) + bb.y),
                 silu2_halved(__uint_as_float(p[6]) + bb.z, __uint_as_float(p[7]) + bb.w));
  }
}

struct Params {
  const unsigned char *packed;
  const float *bias;    // [5][256]: rows 1..3 = b2..b4, row 4 = b5
  const float *bias1;   // [n_eval][256]: W1[:, emb] emb(t_e) + b1
  NetStats st;
  int64_t n;
  const float *cond;
  const float *noise;
  uint64_t seed, id0;
  int steps, integrator, n_eval;
  float *y_raw, *exitp;
  int *err;
};

__global__ void __launch_bounds__(THREADS, 1) sampler_tc_kernel(Params P) {
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
      mbar_init(&B.a_ready[t], EPI_WARPS);
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
      bulk_g2s(sm + S_B1, P.packed + OFF_B1, 8192, &B.res_full);
      bulk_g2s(sm + S_B5, P.packed + OFF_B5, 8192, &B.res_full);
      for (int64_t ip = 0; ip < n_iter && ok; ++ip)
        for (int e = 0; e < P.n_eval && ok; ++e)
          for (int L = 0; L < 3 && ok; ++L)
            for (int T = 0; T < 2 && ok; ++T)
              for (int ch = 0; ch < CHUNKS; ++ch) {
                const int s = it % NST;
                const uint32_t round = it / NST;
                if (!mbar_wait(&B.empty[s], (round & 1u) ^ 1u, abort)) {
                  fail(B, P.err, 1);
                  ok = false;
                  break;
                }
                mbar_arrive_expect_tx(&B.full[s], CHUNK);
                bulk_g2s_multicast(sm + S_ST + s * CHUNK + rank * SLICE,
                                   P.packed + OFF_HID + (size_t)(L * CHUNKS + ch) * CHUNK + rank * SLICE,
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
                for (int ch = 0; ch < CHUNKS; ++ch) {
                  if (!mbar_try_wait(&B.full[stage], sph) && !mbar_wait(&B.full[stage], sph, abort)) {
                    fail(B, P.err, 4);
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                  // chunk ch = K columns CHUNK_K ch .. of all 256 output rows: A at
                  // K-block (CHUNK_K ch)/64, byte 2 (CHUNK_K ch % 64) of its rows
                  const int k0 = ch * CHUNK_K;
                  const uint64_t a_ch = a0 + (uint64_t)((k0 >> 6) * 1024 + ((k0 & 63) >> 3));
                  const uint64_t b_ch = dST + (uint64_t)(stage * (CHUNK >> 4));
#pragma unroll
                  for (int k = 0; k < MMAS_PER_CHUNK; ++k)
                    mma_f16(d, a_ch + (uint64_t)(2 * k), b_ch + (uint64_t)(2 * k), id256,
                            (ch | k) != 0);
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
    const int q = warp & 3, hf = (warp - 2) >> 2;  // lane quadrant, column quarter
    const int r = 32 * q + lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    float cn[2][kCond], x[2][4], xm[2][4], ka[2][4];
    uint32_t dph[2] = {0, 0};
    bool ok = true;
    for (int64_t ip = 0; ip < n_iter && ok; ++ip) {
      const int64_t pr = blockIdx.x + ip * gridDim.x;
      for (int T = 0; T < 2; ++T) {
        const int64_t g = (2 * pr + T) * TM + r;
        const bool valid = g < P.n;
        if (hf == 0) {
#pragma unroll
          for (int k = 0; k < kCond; ++k)
            cn[T][k] = valid ? (P.cond[k * P.n + g] - P.st.cond_mean[k]) * P.st.cond_inv_std[k] : 0.0f;
          if (!valid) {
#pragma unroll
            for (int d = 0; d < 4; ++d) x[T][d] = 0.0f;
          } else if (P.noise) {
#pragma unroll
            for (int d = 0; d < 4; ++d) x[T][d] = P.noise[d * P.n + g];
          } else {
            const float4 z = box_muller4(philox_draw(P.seed, P.id0 + (uint64_t)g, 0u, kTagNoise));
            x[T][0] = z.x;
            x[T][1] = z.y;
            x[T][2] = z.z;
            x[T][3] = z.w;
          }
          write_a1(sbase + (T ? S_A1 : S_A0), r, cn[T], x[T]);
          fence_proxy_async_smem();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.a_ready[T]);
      }
      for (int e = 0; e < P.n_eval && ok; ++e) {
        for (int L = 0; L < 4 && ok; ++L)
          for (int T = 0; T < 2; ++T) {
            if (!mbar_wait(&B.mma_done[T], dph[T] & 1u, abort)) {
              fail(B, P.err, 5);
              ok = false;
              break;
            }
            ++dph[T];
            tc_fence_after();
            const float *bias = L == 0 ? P.bias1 + (size_t)e * 256 : P.bias + L * 256;
            const uint32_t a_base = sbase + (T ? S_A1 : S_A0);
            const uint32_t tcol = tmem + lane_off + (uint32_t)T * 256u + (uint32_t)(hf * EPI_COLS);
            // the load of the next 32 columns is in flight while the current
            // ones are converted and stored
            uint32_t buf[2][32];
            tmem_ld32_raw(tcol, buf[0]);
            tmem_wait_ld_regs(buf[0]);
#pragma unroll
            for (int j = 0; j < EPI_CH; ++j) {
              if (j + 1 < EPI_CH) tmem_ld32_raw(tcol + 32u * (uint32_t)(j + 1), buf[(j + 1) & 1]);
              epi32(buf[j & 1], bias, hf * EPI_COLS + 32 * j, a_base, r);
              if (j + 1 < EPI_CH) tmem_wait_ld_regs(buf[(j + 1) & 1]);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.a_ready[T]);
          }
        if (!ok) break;
        const bool last = e == P.n_eval - 1;
        for (int T = 0; T < 2; ++T) {
          if (!mbar_wait(&B.mma_done[T], dph[T] & 1u, abort)) {
            fail(B, P.err, 6);
            ok = false;
            break;
          }
          ++dph[T];
          tc_fence_after();
          if (hf == 0) {
            float v[4];
            tmem_ld4(tmem + lane_off + (uint32_t)T * 256u, v);
            tmem_wait_ld_regs4(v);
#pragma unroll
            for (int d = 0; d < 4; ++d) v[d] += __ldg(P.bias + 4 * 256 + d);
            float *xin = x[T];
            if (P.integrator == GMC_MIDPOINT && (e & 1) == 0) {
#pragma unroll
              for (int d = 0; d < 4; ++d) xm[T][d] = fmaf(0.5f * h, v[d], x[T][d]);
              xin = xm[T];
            } else if (P.integrator == GMC_RK4) {
              // evaluation e % 4 = i gives k_{i+1}; ka = k1 + 2 k2 + 2 k3 + k4
              const int i = e & 3;
              if (i == 3) {
#pragma unroll
                for (int d = 0; d < 4; ++d) x[T][d] = fmaf(h * (1.0f / 6.0f), ka[T][d] + v[d], x[T][d]);
              } else {
                const float wgt = i == 0 ? 1.0f : 2.0f, hs = i == 2 ? h : 0.5f * h;
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                  ka[T][d] = i == 0 ? v[d] : fmaf(wgt, v[d], ka[T][d]);
                  xm[T][d] = fmaf(hs, v[d], x[T][d]);
                }
                xin = xm[T];
              }
            } else {
#pragma unroll
              for (int d = 0; d < 4; ++d) x[T][d] = fmaf(h, v[d], x[T][d]);
            }
            if (!last) {
              float xi[4] = {xin[0], xin[1], xin[2], xin[3]};
              write_a1(sbase + (T ? S_A1 : S_A0), r, cn[T], xi);
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
                for (int d = 0; d < 4; ++d) P.y_raw[d * P.n + g] = x[T][d];
              }
              if (P.exitp) {
                bool inward;
                const float4 o = decode_exit(x[T][0], x[T][1], x[T][2], x[T][3], P.st, &inward);
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

// element (row, k) of a 64-byte-swizzled K-major block whose rows are 64 B
size_t sw64_off(int row, int k) {
  const int c = k >> 3, e = k & 7;
  return (size_t)((row >> 3) * 512 + (row & 7) * 64 + ((c ^ ((row >> 1) & 3)) << 4) + e * 2);
}

size_t sw32_off(int row, int k) {
  const int c = k >> 3, e = k & 7;
  return (size_t)((row >> 3) * 256 + (row & 7) * 32 + ((c ^ ((row >> 2) & 1)) << 4) + e * 2);
}

}  // namespace

size_t tc_packed_bytes() { return PACKED; }

void tc_pack_host(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                  float *bias_host) {
  unsigned char *P = (unsigned char *)packed_host;
  std::memset(P, 0, PACKED);
  auto put = [&](size_t off, float v) {
    const uint16_t u = bf16_bits(v);
    std::memcpy(P + off, &u, 2);
  };
  // hidden layers W2..W4: chunk ch holds all 256 output rows and K CHUNK_K ch ..
  for (int L = 0; L < 3; ++L)
    for (int ch = 0; ch < CHUNKS; ++ch) {
      const size_t base = OFF_HID + (size_t)(L * CHUNKS + ch) * CHUNK;
      for (int i = 0; i < 256; ++i)
        for (int j = 0; j < CHUNK_K; ++j)
          put(base + (CHUNK_K == 32 ? sw64_off(i, j) : sw128_off(i, j)),
              0.5f * W[L + 1][i * 256 + ch * CHUNK_K + j]);
    }
  // layer 1: [cond (5), x (4) for x_hi, x (4) again for x_lo, 0 0 0]
  for (int nrow = 0; nrow < 256; ++nrow) {
    const float *w = &W[0][nrow * 25];
    for (int k = 0; k < 5; ++k) put(OFF_B1 + sw32_off(nrow, k), 0.5f * w[k]);
    for (int k = 0; k < 4; ++k) {
      put(OFF_B1 + sw32_off(nrow, 5 + k), 0.5f * w[5 + k]);
      put(OFF_B1 + sw32_off(nrow, 9 + k), 0.5f * w[5 + k]);
    }
  }
  // output layer: 16 rows (4 real) x 256 K in four 128-byte-swizzled K-blocks
  for (int d = 0; d < 4; ++d)
    for (int k = 0; k < 256; ++k)
      put(OFF_B5 + (size_t)(k >> 6) * 2048 + sw128_off(d, k & 63), W[4][d * 256 + k]);
  for (int i = 0; i < 5 * 256; ++i) bias_host[i] = 0.0f;
  for (int L = 1; L < 4; ++L)
    for (int c = 0; c < 256; ++c) bias_host[L * 256 + c] = 0.5f * b[L][c];
  for (int d = 0; d < 4; ++d) bias_host[4 * 256 + d] = b[4][d];
}

cudaError_t launch_sampler_tc(cudaStream_t stream, const void *packed, const float *bias,
                              const NetF32 &f32, const NetStats &st, int64_t n, const float *cond,
                              const float *noise, uint64_t seed, uint64_t id0, int steps,
                              int integrator, float *y_raw, float *exit, int *err,
                              float *bias1_scratch) {
  if (n <= 0) return cudaSuccess;
  const int n_eval = integrator == GMC_RK4 ? 4 * steps : (integrator == GMC_MIDPOINT ? 2 * steps : steps);
  layer1_bias_kernel<<<n_eval, kHidden, 0, stream>>>(f32.w1t, f32.b1, steps, integrator, n_eval,
                                                     bias1_scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(sampler_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (n + TM - 1) / TM, npairs = (ntiles + 1) / 2;
  int64_t g = npairs < sms ? npairs : sms;
  g = (g + CLUSTER - 1) / CLUSTER * CLUSTER;
  if (g > sms / CLUSTER * CLUSTER) g = sms / CLUSTER * CLUSTER;
  const int grid = (int)g;
  Params p;
  p.packed = (const unsigned char *)packed;
  p.bias = bias;
  p.bias1 = bias1_scratch;
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
    if (cudaOccupancyMaxActiveClusters(&mc, sampler_tc_kernel, &lc) != cudaSuccess || mc < 1) {
      cudaGetLastError();
      mc = sms / CLUSTER;
    }
    max_clusters = mc;
  }
  const int grid_fit = grid < max_clusters * CLUSTER ? grid : max_clusters * CLUSTER;
  lc.gridDim = dim3((unsigned)grid_fit);
  e = cudaLaunchKernelEx(&lc, sampler_tc_kernel, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace gmc
