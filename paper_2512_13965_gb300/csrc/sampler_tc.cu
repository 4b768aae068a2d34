// BF16 tensor-core flow-ODE sampler (Eq. 8) for sm_103a: tcgen05 MMA with
// FP32 accumulators in tensor memory, the hidden activations kept in tensor
// memory as the next layer's A operand, weights streamed by bulk async copies.
//
// Work unit: a tile of 128 particles. One persistent CTA per SM owns two
// tiles (X, Y) at a time and runs all K steps of both, alternating them: the
// tensor core computes one tile's layer while the epilogue warps turn the
// other tile's previous layer into activations:
//
//   MMA warp:   L(X)   L(Y)   L+1(X)   L+1(Y) ...
//   epilogue:          E(X)   E(Y)     E(X)  ...     (SiLU, BF16)
//
// Tensor memory (512 columns): A_X, A_Y (cols 0-127, 128-255): the 128 x 256
// BF16 operand of each tile (row m in lane m, two K values per column); D
// (256-511): one 128 x 256 FP32 accumulator that the tiles use in turn. The
// epilogue reads the accumulator into registers and releases it at once (the
// other tile's MMAs may start), then writes the activations back to A_T with
// tcgen05.st: no shared-memory traffic for activations. Two accumulators would
// not fit beside the two operands.
//
// Per evaluation of v_theta and tile (M = 128 rows):
//   L1: [x_hi | x_lo | cn | 1 1 0] (K = 16, BF16, shared memory) x B1 -> D
//       (the time-embedding columns of layer 1 are the same for every row,
//        so W1[:, emb] emb(t) + b1 is folded into an FP32 per-evaluation bias)
//   L2..L4: A_T (tensor memory) x W (shared memory, streamed in chunks of
//       all 256 output rows x 128 bytes of K) -> D, N = 256 per MMA
//   L5: A_T x W5 (N = 16, rows 4..15 zero) -> D columns 0..15
// Epilogue: SiLU(z) = h + h tanh(h) with h = z/2 (layers 1-4 are packed with
// weights and biases halved, so the accumulator holds h), in packed BF16x2.
// The biases of layers 2-4 enter the accumulator through one extra K = 16 MMA
// (two constant-1 columns of the layer-1 operand against the bias split into
// BF16 hi + lo); layer 1's bias, which depends on t, is added in the epilogue.
// The ODE state x of tile T stays in FP32 registers of group T's threads.
//
// Roles: warp 0 streams weights, warp 1 owns tensor memory and issues MMAs,
// warps 2..17 are the epilogue: two groups of 8 warps (group g: accumulator
// columns 128 g .. 128 g + 127, and the ODE state of tile g), two threads per
// row and group, each loading its 64 columns at once and converting them in
// 16-column pieces.
// Each CTA streams every weight chunk from L2 into its own stages with a
// plain bulk copy (the whole network is 424 KB, L2-resident); a stage is
// refilled once this CTA's MMAs have released it. CTAs never wait on one
// another.
// Every wait is bounded; a timeout sets *err and the CTA drains and exits.
//
// FP8 variant (template argument FP8): the three 256 x 256 layers (97% of the
// FLOPs) run as kind::f8f6f4 MMAs on E4M3 operands. Each output row c of
// W2..W4 is stored as E4M3 codes of W[c][:] / s_c with s_c = max_k |W[c][k]| / 448
// (per-output-channel scale, FP32); the bias enters the accumulator as b_c / s_c
// through the bias MMA, and the epilogue applies h = acc s_c / 2. Activations entering layers 2-4 are E4M3 with unit
// scale (SiLU outputs are >= -0.279 and far below E4M3's 448), four per
// tensor-memory column. Layer 1 keeps BF16 operands (the ODE state enters
// through them) and layer 4's epilogue writes BF16, so layer 5 (the velocity)
// is the same BF16 MMA as above. A 32 KB weight chunk then holds 128 inputs
// instead of 64; a K step is 32 bytes (8 A columns) in both variants.
//
// Residual-modulated variant (template argument RM, BF16 only): layers 2-4
// are residual blocks a_l = a_{l-1} + SiLU(g z_l). The condition shift M_l c
// of z_l enters through the bias MMA like the bias (the condition columns of
// the layer-1 operand against M_l / 2 in the bias block), so the accumulator
// already holds z_l / 2. The epilogue scales it by the channel modulation
// g = 1 + G_l[0] c_3 + G_l[1] c_4 in packed BF16 (G as BF16 pairs in shared
// memory, the row's standardized ln tau and c in a per-thread shared slot),
// applies the SiLU and adds the block input, which it reads from A_T (the
// MMA that read it has completed) just before overwriting it: the residual
// stream is the BF16 operand itself and costs no tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstring>

#include "decode.cuh"
#include "gmc_internal.cuh"
#include "philox.cuh"
#include "sampler_common.cuh"
#include "tc_ptx.cuh"

namespace gmc {
namespace {

using namespace ptx;
using namespace smp;

constexpr int TM = 128;
constexpr int EPI_WARPS = 16;                 // two groups of 8, one per 128 output columns
constexpr int GROUP_WARPS = EPI_WARPS / 2;    // 2 per TMEM lane quadrant, 64 columns each
constexpr int THREADS = 32 * (2 + EPI_WARPS);
constexpr int NH = 128;                       // output columns of one epilogue group
constexpr int MMAS_PER_CHUNK = 4;             // 32 bytes of K per MMA
#ifndef GMC_TC_STAGES
#define GMC_TC_STAGES 5
#endif
constexpr int NST = GMC_TC_STAGES;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_A = 0;                 // + 128 T: operand of tile T
constexpr uint32_t COL_D = 256;               // the 128 x 256 FP32 accumulator

// shared memory (offsets from a 1024-byte aligned base)
constexpr uint32_t S_A1 = 0;                     // layer-1 operands of tiles X, Y: 2 x 4 KB
constexpr uint32_t S_B1 = 8192;                  // 8 KB
constexpr uint32_t S_B5 = 16384;                 // 8 KB
constexpr uint32_t S_BIAS = 24576;               // 24 KB (BF16 variant)
constexpr uint32_t S_ST = 49152;                 // NST weight stages
constexpr uint32_t S_BAR = S_ST + NST * CHUNK;   // barriers and flags
// residual-modulated network: (ln tau, c) standardized as BF16 pairs (each
// value in both halves), per tile, epilogue thread and row ([T][epilogue
// warp][lane] uint2; each thread reads only what it wrote, so registers are
// spared without a barrier)
constexpr uint32_t S_U = S_BAR + 256;
constexpr uint32_t S_G = S_U + 2 * EPI_WARPS * 32 * 8;  // RM: G as BF16 pairs [3][2][128]
constexpr uint32_t S_TOTAL = S_G + 3 * 2 * 128 * 4;
constexpr uint32_t SMEM_BYTES = S_TOTAL + 1024;  // + alignment slack
// More than half of the SM's shared memory, so no second CTA (which would
// wait for the 512 tensor-memory columns this one holds) shares the SM.
static_assert(SMEM_BYTES > 116 * 1024 && SMEM_BYTES <= 227 * 1024, "shared memory per CTA");

struct Bars {
  uint64_t full[NST];
  uint64_t empty[NST];
  uint64_t res_full;
  uint64_t ar[2][2];    // [T][g]: group g's part of tile T's next operand written
  uint64_t dfull;       // accumulator computed (MMA commit)
  uint64_t dfree;       // accumulator read out (all epilogue warps)
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(Bars) <= 256, "barrier block");

__device__ void fail(Bars &b, int *err, int code) {
  b.abort = 1;
  atomicExch(err, code);
}

// Residual blocks (layers 2-4 of the residual-modulated network, L = 1..3):
// rm_scale turns 32 halved pre-activations h = z / 2 (accumulator columns
// col0 ..) into 16 BF16 pairs of g h = h + h d, d = G[0] c_3 + G[1] c_4, in
// packed BF16 (gs: the layer's G as BF16 pairs, [2][128]; u3p, u4p: the row's
// c_3 and c_4 in both halves). Forming h + h d with one FMA rounds once
// where g = 1 + d followed by g h would round twice. rm_finish reads the
// block input of this thread's 64 columns from a_row (BF16 columns col0 / 2
// ..), adds the SiLU and writes the sum back.
__device__ __forceinline__ void rm_scale(const uint32_t (&v)[32], const uint32_t *gs, uint32_t u3p,
                                         uint32_t u4p, int col0, uint32_t (&hp)[16]) {
  const uint4 *g0 = reinterpret_cast<const uint4 *>(gs + (col0 >> 1));
  const uint4 *g1 = reinterpret_cast<const uint4 *>(gs + 128 + (col0 >> 1));
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 a4 = g0[q], b4 = g1[q];
    const uint32_t ga[4] = {a4.x, a4.y, a4.z, a4.w}, gb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t h, t, d;
      const int k = 4 * q + i;
      asm("cvt.rn.bf16x2.f32 %0, %1, %2;"
          : "=r"(h)
          : "f"(__uint_as_float(v[2 * k + 1])), "f"(__uint_as_float(v[2 * k])));
      asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(t) : "r"(gb[i]), "r"(u4p));
      asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(ga[i]), "r"(u3p), "r"(t));
      asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(hp[k]) : "r"(h), "r"(d));
    }
  }
}

__device__ __forceinline__ void rm_finish(const uint32_t (&h0)[16], const uint32_t (&h1)[16], int col0,
                                          uint32_t a_row) {
#pragma unroll
  for (int pc = 0; pc < 4; ++pc) {
    uint32_t a[8];  // the block input, overwritten by the block output
    const uint32_t col = a_row + (uint32_t)((col0 + 16 * pc) >> 1);
    tmem_ld8_raw(col, a);
    tmem_wait_ld_regs8(a);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      uint32_t t, o;
      const uint32_t h = pc < 2 ? h0[8 * pc + i] : h1[8 * (pc - 2) + i];
      asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
      asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(o) : "r"(h), "r"(t));
      asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(a[i]) : "r"(o), "r"(a[i]));
    }
    tmem_st8(col, a);
  }
}

// One 16-column piece of layer L's epilogue: activations of accumulator
// columns col0.. (of 256) written into this thread's row of A_T. BF16: K =
// col0 at column col0 / 2; E4M3 (FP8 layers 1-3): column col0 / 4.
template <bool FP8>
__device__ __forceinline__ void epi_piece(int L, const uint32_t *v, const float *bias,
                                          const float *scale, int col0, uint32_t a_row) {
  uint32_t w[8];
  if constexpr (FP8) {
    if (L < 3) {
      if (L == 0)
        silu16<kPreBias, true>(v, bias, nullptr, col0, w);
      else
        silu16<kPreScale, true>(v, bias, scale + (L - 1) * 256, col0, w);
      tmem_st4(a_row + (uint32_t)(col0 >> 2), w);
      return;
    }
    silu16<kPreScale, false>(v, bias, scale + 2 * 256, col0, w);
  } else {
    if (L == 0)
      silu16<kPreBias, false>(v, bias, nullptr, col0, w);
    else
      silu16<kPreNone, false>(v, bias, nullptr, col0, w);
  }
  tmem_st8(a_row + (uint32_t)(col0 >> 1), w);
}

// INTEG: the integrator (GMC_EULER, GMC_MIDPOINT, GMC_RK4) as a compile-time
// choice, so an Euler kernel holds no midpoint or RK4 state in registers.
// RM: the residual-modulated network (BF16 only).
template <bool FP8, int INTEG, bool RM = false>
__global__ void __launch_bounds__(THREADS, 1) sampler_tc_kernel(Params P) {
  static_assert(!(FP8 && RM), "the residual-modulated network has no FP8 variant");
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
      mbar_init(&B.empty[s], 1);
    }
    mbar_init(&B.res_full, 1);
    for (int t = 0; t < 2; ++t) {
      mbar_init(&B.ar[t][0], GROUP_WARPS);
      mbar_init(&B.ar[t][1], GROUP_WARPS);
    }
    mbar_init(&B.dfull, 1);
    mbar_init(&B.dfree, EPI_WARPS);
    mbar_init(&B.drain, 1);
    B.abort = 0;
    fence_mbar_init();
  }
  if constexpr (RM) {
    // the channel scales of layers 2-4 as BF16 pairs, read by every epilogue
    uint32_t *gs = reinterpret_cast<uint32_t *>(sm + S_G);
    for (int i = threadIdx.x; i < 3 * 2 * 128; i += THREADS) {
      const float lo = P.rmg[2 * i], hi = P.rmg[2 * i + 1];
      uint32_t w;
      asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
      gs[i] = w;
    }
  }
  if (warp == 1) {
    tmem_alloc(&B.tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B.tmem_base;
  volatile int *abort = &B.abort;

  const int64_t ntiles = (P.n + TM - 1) / TM;
  const int64_t npairs = (ntiles + 1) / 2;
  // tile pairs blockIdx.x, blockIdx.x + gridDim.x, ... (grid <= npairs); the
  // last pair may hold one tile, or rows past n, which are computed on zeros
  // and not stored
  const int64_t n_iter = (npairs - blockIdx.x + gridDim.x - 1) / gridDim.x;
  const float h = 1.0f / (float)P.steps;

  if (warp == 0) {
    // ---------------- weight producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      mbar_arrive_expect_tx(&B.res_full, 16384 + 24576);
      bulk_g2s(sm + S_B1, P.packed + PK::OFF_B1, 8192, &B.res_full);
      bulk_g2s(sm + S_B5, P.packed + PK::OFF_B5, 8192, &B.res_full);
      bulk_g2s(sm + S_BIAS, P.packed + PK::OFF_BIAS, 24576, &B.res_full);
      // the MMA warp's order: per hidden layer and tile, its chunks
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
                  bulk_g2s(sm + S_ST + s * CHUNK, P.packed + PK::OFF_HID + (size_t)(L * NCH + ch) * CHUNK,
                           CHUNK, &B.full[s]);
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
    // The whole warp runs the loop with warp-uniform values, and one elected
    // lane issues each tcgen05 instruction, so descriptors and addresses stay
    // uniform and an MMA issues in a few cycles. Descriptors are built once
    // and advanced by constant offsets (the start-address field counts 16-byte
    // units); a barrier phase that has already completed costs one try_wait.
    {
      // every lane waits (and acquires); the result is made warp-uniform
      auto wwait = [&](uint64_t *bar, uint32_t parity) {
        const bool r = mbar_try_wait(bar, parity) || mbar_wait(bar, parity, abort);
        return __all_sync(0xffffffffu, r);
      };
      bool ok = wwait(&B.res_full, 0);
      if (!ok && lane == 0) fail(B, P.err, 2);
      uint32_t aph[2][2] = {{0, 0}, {0, 0}}, fph = 0;
      uint32_t stage = 0, sph = 0;  // next weight stage and its phase parity
      const uint32_t idn = idesc_bf16_m128(256), id16 = idesc_bf16_m128(16);
      const uint32_t idh = FP8 ? idesc_e4m3_m128(256) : idn;  // hidden layers
      const uint64_t dA1[2] = {smem_desc(sbase + S_A1, 256, kSwizzle32B),
                               smem_desc(sbase + S_A1 + 4096, 256, kSwizzle32B)};
      const uint64_t dB1 = smem_desc(sbase + S_B1, 256, kSwizzle32B);
      const uint64_t dB5 = smem_desc(sbase + S_B5, 1024, kSwizzle128B);
      const uint64_t dBias = smem_desc(sbase + S_BIAS, 256, kSwizzle32B);
      const uint64_t dST = smem_desc(sbase + S_ST, 1024, kSwizzle128B);
      auto wait_ar = [&](int T, int g) {
        if (!wwait(&B.ar[T][g], aph[T][g] & 1u)) {
          if (lane == 0) fail(B, P.err, 3);
          return false;
        }
        ++aph[T][g];
        return true;
      };
      for (int64_t ip = 0; ip < n_iter && ok; ++ip)
        for (int e = 0; e < P.n_eval && ok; ++e)
          for (int L = 0; L < 5 && ok; ++L)
            for (int T = 0; T < 2 && ok; ++T) {
              // layer 1 reads the tile's shared-memory operand, written by the
              // group that owns the tile's ODE state; later layers read A_T,
              // written half by each group
              if (L == 0) ok = wait_ar(T, T);
              else ok = wait_ar(T, 0) && wait_ar(T, 1);
              if (!ok) break;
              if (!wwait(&B.dfree, (fph & 1u) ^ 1u)) {
                if (lane == 0) fail(B, P.err, 7);
                ok = false;
                break;
              }
              ++fph;
              tc_fence_after();
              const uint32_t d = tmem + COL_D;
              const uint32_t a = tmem + COL_A + 128u * (uint32_t)T;
              if (L == 0) {
                mma_f16_w(d, dA1[T], dB1, idn, 0);
              } else if (L < 4) {
                // D = bias first (the two constant-1 columns of the tile's
                // layer-1 operand times the bias block's hi/lo columns; a BF16
                // MMA also in the FP8 variant, whose MMAs then accumulate)
                mma_f16_w(d, dA1[T], dBias + (uint64_t)((L - 1) * 512), idn, 0);
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                  if (!wwait(&B.full[stage], sph)) {
                    if (lane == 0) fail(B, P.err, 4);
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                  // chunk ch = operand bytes 128 ch .. of all 256 output rows;
                  // each MMA takes 32 bytes of K = 8 columns of A_T
                  const uint64_t b_ch = dST + (uint64_t)(stage * (CHUNK >> 4));
#pragma unroll
                  for (int k = 0; k < MMAS_PER_CHUNK; ++k) {
                    const uint32_t a_k = a + (uint32_t)(32 * ch + 8 * k);
                    const uint32_t acc = 1u;
                    if constexpr (FP8)
                      mma_ts_f8_w(d, a_k, b_ch + (uint64_t)(2 * k), idh, acc);
                    else
                      mma_ts_f16_w(d, a_k, b_ch + (uint64_t)(2 * k), idh, acc);
                  }
                  mma_commit_w(&B.empty[stage]);
                  if (++stage == NST) {
                    stage = 0;
                    sph ^= 1u;
                  }
                }
                if (!ok) break;
              } else {
                // velocity: K = 256 BF16 = 16 MMAs of 8 columns; B5 in four
                // 2 KB K-blocks of 128-byte rows
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  mma_ts_f16_w(d, a + (uint32_t)(8 * j), dB5 + (uint64_t)((j >> 2) * 128 + (j & 3) * 2),
                             id16, j != 0);
              }
              mma_commit_w(&B.dfull);
            }
      // all issued MMAs complete before tensor memory is released
      mma_commit_w(&B.drain);
      int never = 0;
      mbar_wait(&B.drain, 0, &never, 1000000000ull);
    }
  } else {
    // ---------------- epilogue ----------------
    // Group g (8 warps) converts accumulator columns 128 g .. 128 g + 127 of
    // every layer of both tiles and owns the ODE state of tile g; within a
    // group, warp w serves TMEM lane quadrant w % 4 (rows 32 q ..) and
    // columns 64 p .. 64 p + 63 of the group's 128.
    const int ew = warp - 2;
    const int g = ew / GROUP_WARPS;
    const int p = (ew >> 2) & 1;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const bool owner = p == 0;  // holds the ODE state of tile g's rows
    float x[4], xm[4], ka[4];
    uint2 *u_slot = reinterpret_cast<uint2 *>(sm + S_U) + ew * 32 + lane;  // RM: + 512 T
    uint32_t dph = 0;
    bool ok = true;
    for (int64_t ip = 0; ip < n_iter && ok; ++ip) {
      const int64_t pr = blockIdx.x + ip * gridDim.x;
      if constexpr (RM) {
#pragma unroll
        for (int T = 0; T < 2; ++T) {
          const int64_t gi = (2 * pr + T) * TM + r;
          const bool valid = gi < P.n;
          const float u3 =
              valid ? (P.cond[3 * P.n + gi] - P.st.cond_mean[3]) * P.st.cond_inv_std[3] : 0.0f;
          const float u4 =
              valid ? (P.cond[4 * P.n + gi] - P.st.cond_mean[4]) * P.st.cond_inv_std[4] : 0.0f;
          uint2 up;
          asm("cvt.rn.bf16x2.f32 %0, %1, %1;" : "=r"(up.x) : "f"(u3));
          asm("cvt.rn.bf16x2.f32 %0, %1, %1;" : "=r"(up.y) : "f"(u4));
          u_slot[512 * T] = up;
        }
      }
      {
        const int T = g;
        const int64_t gi = (2 * pr + T) * TM + r;
        const bool valid = gi < P.n;
        if (owner) {
          float cn[kCondRect];
          load_cond(P.cond, P.st, P.n, gi, valid, cn);
          if (!valid) {
#pragma unroll
            for (int d = 0; d < 4; ++d) x[d] = 0.0f;
          } else if (P.noise) {
#pragma unroll
            for (int d = 0; d < 4; ++d) x[d] = P.noise[d * P.n + gi];
          } else {
            const float4 z = box_muller4(philox_draw(P.seed, P.id0 + (uint64_t)gi, 0u, kTagNoise));
            x[0] = z.x;
            x[1] = z.y;
            x[2] = z.z;
            x[3] = z.w;
          }
          write_a1_cond(sbase + S_A1 + (uint32_t)T * 4096u, r, cn);
          write_a1_x(sbase + S_A1 + (uint32_t)T * 4096u, r, x);
          fence_proxy_async_smem();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.ar[T][g]);
      }
      for (int e = 0; e < P.n_eval && ok; ++e) {
        for (int L = 0; L < 4 && ok; ++L)
#pragma unroll
          for (int T = 0; T < 2; ++T) {
            const float *bias = L == 0 ? P.bias1 + (size_t)e * 256 : P.bias + L * 256;
            const uint32_t a_row = tmem + lane_off + COL_A + 128u * (uint32_t)T;
            const uint32_t d_col = tmem + lane_off + COL_D + (uint32_t)(NH * g + 64 * p);
            const int col0 = NH * g + 64 * p;  // of the layer's 256 outputs
            if (!mbar_wait(&B.dfull, dph & 1u, abort)) {
              fail(B, P.err, 5);
              ok = false;
              break;
            }
            ++dph;
            tc_fence_after();
            if constexpr (RM) {
              if (L > 0) {
                // residual block: the accumulator is read out and released at
                // once, then scaled, and the block output overwrites its input
                const uint2 u = u_slot[512 * T];
                uint32_t va[32], vb[32];
                tmem_ld32_raw(d_col, va);
                tmem_ld32_raw(d_col + 32u, vb);
                tmem_wait_ld_regs(va);
                tmem_wait_ld_regs(vb);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&B.dfree);
                uint32_t h0[16], h1[16];
                const uint32_t *gs = reinterpret_cast<const uint32_t *>(sm + S_G) + (L - 1) * 256;
                rm_scale(va, gs, u.x, u.y, col0, h0);
                rm_scale(vb, gs, u.x, u.y, col0 + 32, h1);
                rm_finish(h0, h1, col0, a_row);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&B.ar[T][g]);
                continue;
              }
            }
            // the whole 64-column slice comes into registers first, so the
            // accumulator is released after one load latency; the MMA that
            // read A_T has completed, so the activations overwrite it at once
            uint32_t va[32], vb[32];
            tmem_ld32_raw(d_col, va);
            tmem_ld32_raw(d_col + 32u, vb);
            tmem_wait_ld_regs(va);
            tmem_wait_ld_regs(vb);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.dfree);  // the MMA may overwrite the accumulator now
            epi_piece<FP8>(L, va, bias, P.scale, col0, a_row);
            epi_piece<FP8>(L, va + 16, bias, P.scale, col0 + 16, a_row);
            epi_piece<FP8>(L, vb, bias, P.scale, col0 + 32, a_row);
            epi_piece<FP8>(L, vb + 16, bias, P.scale, col0 + 48, a_row);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.ar[T][g]);
            if (!ok) break;
          }
        if (!ok) break;
        const bool last = e == P.n_eval - 1;
#pragma unroll
        for (int T = 0; T < 2; ++T) {
          // the velocity of tile T: columns 0-3, read by the group owning T
          if (!mbar_wait(&B.dfull, dph & 1u, abort)) {
            fail(B, P.err, 6);
            ok = false;
            break;
          }
          ++dph;
          tc_fence_after();
          const bool mine = owner && g == T;
          float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          if (mine) {
            tmem_ld4(tmem + lane_off + COL_D, v);
            tmem_wait_ld_regs4(v);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&B.dfree);
          if (g != T) continue;
          if (mine) {
#pragma unroll
            for (int d = 0; d < 4; ++d) v[d] += __ldg(P.bias + 4 * 256 + d);
            float *xin = x;
            if (INTEG == GMC_MIDPOINT && (e & 1) == 0) {
#pragma unroll
              for (int d = 0; d < 4; ++d) xm[d] = fmaf(0.5f * h, v[d], x[d]);
              xin = xm;
            } else if (INTEG == GMC_RK4) {
              // evaluation e % 4 = i gives k_{i+1}; ka = k1 + 2 k2 + 2 k3 + k4
              const int i = e & 3;
              if (i == 3) {
#pragma unroll
                for (int d = 0; d < 4; ++d) x[d] = fmaf(h * (1.0f / 6.0f), ka[d] + v[d], x[d]);
              } else {
                const float wgt = i == 0 ? 1.0f : 2.0f, hs = i == 2 ? h : 0.5f * h;
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                  ka[d] = i == 0 ? v[d] : fmaf(wgt, v[d], ka[d]);
                  xm[d] = fmaf(hs, v[d], x[d]);
                }
                xin = xm;
              }
            } else {
#pragma unroll
              for (int d = 0; d < 4; ++d) x[d] = fmaf(h, v[d], x[d]);
            }
            if (!last) {
              float xi[4] = {xin[0], xin[1], xin[2], xin[3]};
              write_a1_x(sbase + S_A1 + (uint32_t)T * 4096u, r, xi);
              fence_proxy_async_smem();
            }
          }
          __syncwarp();
          if (!last && lane == 0) mbar_arrive(&B.ar[T][g]);
          if (last && owner) {
            const int64_t gi = (2 * pr + T) * TM + r;
            if (gi < P.n) {
              if (P.y_raw) {
#pragma unroll
                for (int d = 0; d < 4; ++d) P.y_raw[d * P.n + gi] = x[d];
              }
              if (P.exitp) {
                bool inward;
                const float4 o = decode_exit(x[0], x[1], x[2], x[3], P.st, &inward);
                P.exitp[gi] = o.x;
                P.exitp[P.n + gi] = o.y;
                P.exitp[2 * P.n + gi] = o.z;
                P.exitp[3 * P.n + gi] = o.w;
              }
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
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

}  // namespace

size_t tc_packed_bytes(bool fp8) { return fp8 ? Packed<true>::BYTES : Packed<false>::BYTES; }

static_assert(pack::kPackCond == kCond && pack::kPackIn == kIn, "packing constants");

void tc_pack_host(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                  float *bias_host, const float (*M)[256 * kCond], int nin) {
  pack::tc_pack_host(W, b, packed_host, bias_host, M, nin);
}

void tc_pack_host_fp8(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                      float *bias_host, float *scale_host, int nin) {
  pack::tc_pack_host_fp8(W, b, packed_host, bias_host, scale_host, nin);
}

namespace {
template <bool FP8, int INTEG, bool RM = false>
cudaError_t launch_tc(cudaStream_t stream, const Params &p, int sms) {
  auto kernel = sampler_tc_kernel<FP8, INTEG, RM>;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  // one persistent CTA per SM (its shared memory and 512 tensor-memory
  // columns keep a second one off the SM), never more CTAs than tile pairs
  const int64_t ntiles = (p.n + TM - 1) / TM, npairs = (ntiles + 1) / 2;
  const int grid = (int)(npairs < sms ? npairs : sms);
  kernel<<<grid, THREADS, SMEM_BYTES, stream>>>(p);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_sampler_tc(cudaStream_t stream, const void *packed, const float *bias,
                              const NetF32 &f32, const NetStats &st, int64_t n, const float *cond,
                              const float *noise, uint64_t seed, uint64_t id0, int steps,
                              int integrator, float *y_raw, float *exit, int *err,
                              float *bias1_scratch, const float *fp8_scale, int kernel,
                              bool bias1_ready) {
  if (n <= 0) return cudaSuccess;
  const int n_eval = integrator == GMC_RK4 ? 4 * steps : (integrator == GMC_MIDPOINT ? 2 * steps : steps);
  if (!bias1_ready) {
    layer1_bias_kernel<<<n_eval, kHidden, 0, stream>>>(f32.w1t, f32.b1, steps, integrator, n_eval,
                                                       bias1_scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
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
  p.rmg = f32.rm ? f32.gg : nullptr;
  if (f32.rm) {
    if (fp8_scale || kernel == GMC_KERNEL_PAIR) return cudaErrorNotSupported;
    if (integrator == GMC_RK4) return launch_tc<false, GMC_RK4, true>(stream, p, sms);
    if (integrator == GMC_MIDPOINT) return launch_tc<false, GMC_MIDPOINT, true>(stream, p, sms);
    return launch_tc<false, GMC_EULER, true>(stream, p, sms);
  }
  if (fp8_scale) {
    if (integrator == GMC_RK4) return launch_tc<true, GMC_RK4>(stream, p, sms);
    if (integrator == GMC_MIDPOINT) return launch_tc<true, GMC_MIDPOINT>(stream, p, sms);
    return launch_tc<true, GMC_EULER>(stream, p, sms);
  }
  if (kernel == GMC_KERNEL_PAIR) return launch_sampler_pair(stream, p, sms);
  if (integrator == GMC_RK4) return launch_tc<false, GMC_RK4>(stream, p, sms);
  if (integrator == GMC_MIDPOINT) return launch_tc<false, GMC_MIDPOINT>(stream, p, sms);
  return launch_tc<false, GMC_EULER>(stream, p, sms);
}

}  // namespace gmc
