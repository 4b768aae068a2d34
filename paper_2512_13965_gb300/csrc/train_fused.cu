// The BF16 training step of the velocity network (Eq. 9: conditional flow
// matching loss, its hand-derived gradient, AdamW) in four tcgen05 kernels per
// step instead of one GEMM launch per layer and direction.
//
// Work unit: a tile of 128 batch rows (rows past the batch are zero and carry
// no gradient). Operands live in global memory as BF16 "images": the exact
// bytes that tcgen05.mma reads from shared memory (K-major, 128-byte swizzle,
// chunks of 64 K values = 128 B per row, 8-row groups 1024 B apart), so a
// kernel moves them with plain bulk copies and never converts on the way in.
//
//   fwd   (one CTA per tile, persistent): X0 -> Z1..Z4 -> v, all five layers
//         with the activations in shared memory; writes per layer the
//         transposed activation image A_l^T (rows = channels, K = batch rows,
//         the weight-gradient operand) and S_l = SiLU'(Z_l) (BF16 pairs);
//         the loss (FP64 atomics per warp) and dV = 2 (v - u) / B as two
//         images (rows = batch, and its transpose).
//   bwd   (one CTA per tile): the input-gradient chain
//         dZ4 = (dV W5) S4, dZ_{l-1} = (dZ_l W_l) S_{l-1}, with dZ_l in shared
//         memory as the next A operand; writes dZ_l^T images.
//   wgrad (jobs x batch slices): dW_l = dZ_l^T A_{l-1} and db_l = dZ_l^T 1
//         (an N = 16 MMA against a constant-ones operand), both contracted
//         over the batch on the tensor core, one FP32 slice per batch range.
//   update (elementwise): the slices summed in a fixed order (deterministic)
//         into the gradient, AdamW, and the BF16 weight images of the next
//         step (forward W_l and the transposed W_l^T of the input gradients).
//
// Every wait is bounded; a timeout sets the context's device error word and
// the CTA drains its MMAs and exits.
#include <cuda_bf16.h>

#include <atomic>
#include <cstring>

#include "decode.cuh"
#include "gmc_internal.cuh"
#include "philox.cuh"
#include "tc_ptx.cuh"
#include "train_fused.h"

namespace gmc {
namespace tf {
namespace {

using namespace ptx;

// ---- image layout -----------------------------------------------------------

// Byte offset of element (row r, K index k) in a K-major 128-byte-swizzled
// chunk of 64 K values (rows of 128 B; 8-row groups of 1024 B).
__host__ __device__ __forceinline__ uint32_t img_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) +
                    (k & 7) * 2);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  uint16_t u;
  memcpy(&u, &h, 2);
  return u;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &v, 4);
  return u;
}

__device__ __forceinline__ float lo_f(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float hi_f(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// SiLU and its derivative from h = z / 2 and one MUFU tanh: with
// sigma(z) = (1 + tanh h) / 2, SiLU(z) = h (1 + tanh h) and
// SiLU'(z) = sigma (1 + h (1 - tanh h)). The approximate tanh (relative error
// near 2^-11) sits below the BF16 rounding that both values receive.
__device__ __forceinline__ void silu_and_grad(float h, float &a, float &s) {
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(h));
  a = fmaf(h, th, h);
  const float sg = fmaf(0.5f, th, 0.5f);
  s = fmaf(sg, fmaf(-h, th, h), sg);
}

// Programmatic dependent launch: the kernels of a step are launched so that
// the next one may start while this one finishes. Work before grid_dep_wait()
// touches nothing the previous kernel writes or reads; grid_dep_launch()
// comes after it, so a dependent's early work never overlaps a kernel older
// than its predecessor.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// A whole batch row in the X0 layout and its target, the same values as
// batch_cols (groups 0-3) and batch_u.
__device__ __forceinline__ void batch_row(const Gen &G, int64_t B, int64_t b, float *__restrict__ x0row,
                                          float *__restrict__ urow) {
  const uint64_t rid = (uint64_t)G.step * (uint64_t)B + (uint64_t)b;
  const uint4 r0 = philox_draw(G.seed, rid, 0u, kTagTrain);
  const int64_t idx = (int64_t)(((uint64_t)r0.x * (uint64_t)G.n) >> 32);
  const float t = u01(r0.y);
  const float4 z = box_muller4(philox_draw(G.seed, rid, 1u, kTagTrain));
  const float x0[4] = {z.x, z.y, z.z, z.w};
  float x[32];
#pragma unroll
  for (int k = 0; k < 5; ++k) x[k] = (__ldg(G.cond + k * G.n + idx) - G.sd.cm[k]) * G.sd.cis[k];
  float u[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const float x1 = (__ldg(G.y + d * G.n + idx) - G.sd.ym[d]) * G.sd.yis[d];
    x[5 + d] = (1.0f - t) * x0[d] + t * x1;
    u[d] = x1 - x0[d];
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) x[9 + j] = time_embedding(j, t);
#pragma unroll
  for (int k = 25; k < 32; ++k) x[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < 32; k += 4)
    *reinterpret_cast<float4 *>(x0row + k) = make_float4(x[k], x[k + 1], x[k + 2], x[k + 3]);
  *reinterpret_cast<float4 *>(urow) = make_float4(u[0], u[1], u[2], u[3]);
}

// ---- the update kernel ------------------------------------------------------

// One block per tile of a weight matrix (rows = outputs), four consecutive
// parameters per thread: the batch slices of the gradient are loaded at once
// and summed in slice order (deterministic), AdamW updates the FP32 master
// weights and moments, and the BF16 images of the next step are written
// coalesced: the forward image (rows = outputs, K = inputs) from each
// thread's 4 inputs, the transposed image (rows = inputs, K = outputs)
// through a transpose in shared memory with 16-byte stores.
//   blocks 0-191:   W2..W4, tiles of 16 outputs x 64 inputs
//   blocks 192-207: W1, tiles of 16 outputs x 32 inputs (forward image only)
//   blocks 208-211: W5, 4 outputs x 64 inputs
//   block 212:      the biases (no images)
// mode bit 0: grad = sum of the slices; bit 1: AdamW; bit 2: the images.
constexpr int kUpdBlocks = 213;
constexpr int kMaxSplits = 16;

struct Upd {
  int mode, S;
  const float *ws;
  float *grad, *p, *m, *v;
  float lr, b1, b2, eps, wd, bc1, bc2;
  uint8_t *img;
};

// Parameters i .. i + 3 (i a multiple of 4): slice sum, AdamW; the updated
// weights in w.
__device__ __forceinline__ void upd4(const Upd &U, int64_t i, float (&w)[4]) {
  float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (U.mode & 1) {
    float4 part[kMaxSplits];
#pragma unroll
    for (int s = 0; s < kMaxSplits; ++s)
      if (s < U.S) part[s] = __ldg(reinterpret_cast<const float4 *>(U.ws + (int64_t)s * P_TOTAL + i));
#pragma unroll
    for (int s = 0; s < kMaxSplits; ++s)
      if (s < U.S) {
        g.x += part[s].x;
        g.y += part[s].y;
        g.z += part[s].z;
        g.w += part[s].w;
      }
    *reinterpret_cast<float4 *>(U.grad + i) = g;
  } else if (U.mode & 2) {
    g = *reinterpret_cast<const float4 *>(U.grad + i);
  }
  const float4 p4 = *reinterpret_cast<const float4 *>(U.p + i);
  w[0] = p4.x; w[1] = p4.y; w[2] = p4.z; w[3] = p4.w;
  if (U.mode & 2) {
    const float4 m4 = *reinterpret_cast<const float4 *>(U.m + i), v4 = *reinterpret_cast<const float4 *>(U.v + i);
    const float gi[4] = {g.x, g.y, g.z, g.w}, mo[4] = {m4.x, m4.y, m4.z, m4.w}, vo[4] = {v4.x, v4.y, v4.z, v4.w};
    float mn[4], vn[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      mn[u] = U.b1 * mo[u] + (1.0f - U.b1) * gi[u];
      vn[u] = U.b2 * vo[u] + (1.0f - U.b2) * gi[u] * gi[u];
      const float mh = mn[u] / U.bc1, vh = vn[u] / U.bc2;
      w[u] = w[u] * (1.0f - U.lr * U.wd) - U.lr * mh / (sqrtf(vh) + U.eps);
    }
    *reinterpret_cast<float4 *>(U.m + i) = make_float4(mn[0], mn[1], mn[2], mn[3]);
    *reinterpret_cast<float4 *>(U.v + i) = make_float4(vn[0], vn[1], vn[2], vn[3]);
    *reinterpret_cast<float4 *>(U.p + i) = make_float4(w[0], w[1], w[2], w[3]);
  }
}

__global__ void __launch_bounds__(256) update_kernel(Upd U) {
  __shared__ __align__(16) uint16_t T[64][24];  // transposed tile [input][output], 48-byte rows
  const int blk = blockIdx.x, tid = threadIdx.x;
  grid_dep_wait();  // the gradient slices
  grid_dep_launch();
  const bool pack = (U.mode & 4) != 0;
  if (blk == kUpdBlocks - 1) {  // biases: b1..b4 (256 each) and b5 (4), 257 groups of 4
    for (int j = tid; j < 257; j += 256) {
      const int l = j >> 6;
      const int64_t i = (l == 0 ? P_B1 : l == 1 ? P_B2 : l == 2 ? P_B3 : l == 3 ? P_B4 : P_B5) + 4 * (j & 63);
      float w[4];
      upd4(U, i, w);
    }
    return;
  }
  int64_t base;
  int R, Cn, stride, o0, i0;
  uint32_t fimg, fchunk, timg;
  if (blk < 192) {
    const int l = blk >> 6, sub = blk & 63;
    base = P_W2 + (int64_t)l * (65536 + 256);
    R = 16; Cn = 64; stride = 256; o0 = (sub >> 2) * 16; i0 = (sub & 3) * 64;
    fimg = l == 0 ? WF2 : l == 1 ? WF3 : WF4;
    timg = l == 0 ? WB2 : l == 1 ? WB3 : WB4;
    fchunk = 32768;
  } else if (blk < 208) {
    base = P_W1;
    R = 16; Cn = 32; stride = 32; o0 = (blk - 192) * 16; i0 = 0;
    fimg = WF1; fchunk = 32768; timg = 0;
  } else {
    base = P_W5;
    R = 4; Cn = 64; stride = 256; o0 = 0; i0 = (blk - 208) * 64;
    fimg = WF5; fchunk = 2048; timg = WB5;
  }
  const int groups = Cn / 4;
  const int row = tid / groups, cg = (tid % groups) * 4;
  if (row < R) {
    const int o = o0 + row, i = i0 + cg;
    float w[4];
    upd4(U, base + (int64_t)o * stride + i, w);
    if (pack) {
      *reinterpret_cast<uint2 *>(U.img + fimg + (uint32_t)(i >> 6) * fchunk + img_off(o, i & 63)) =
          make_uint2(pack2(w[0], w[1]), pack2(w[2], w[3]));
      if (timg) {
#pragma unroll
        for (int u = 0; u < 4; ++u) T[cg + u][row] = bf16_bits(w[u]);
      }
    }
  }
  if (!pack || !timg) return;
  __syncthreads();
  if (R == 16) {  // 64 inputs x 2 groups of 8 outputs
    if (tid < 128) {
      const int ii = tid >> 1, og = (tid & 1) * 8;
      const uint4 q = *reinterpret_cast<const uint4 *>(&T[ii][og]);
      const int o = o0 + og, i = i0 + ii;
      *reinterpret_cast<uint4 *>(U.img + timg + (uint32_t)(o >> 6) * 32768u + img_off(i, o & 63)) = q;
    }
  } else if (tid < 64) {  // W5: input rows, K = the 4 outputs (8 bytes)
    const int i = i0 + tid;
    *reinterpret_cast<uint2 *>(U.img + timg + img_off(i, 0)) = *reinterpret_cast<const uint2 *>(&T[tid][0]);
  }
}

// ---- forward and input-gradient kernels ---------------------------------------

constexpr int TR = 128;              // batch rows per tile
constexpr uint32_t WCH = 32768;      // weight chunk: 256 rows x 128 B
constexpr uint32_t ACH = 16384;      // activation chunk: 128 rows x 128 B
constexpr int NEPI = 16;             // epilogue warps: 4 lane quadrants x 4 column quarters
constexpr int FB_THREADS = 32 * (2 + NEPI);
constexpr int NST = 3;               // weight stages
constexpr int kTileChunks = 13;      // fwd: W1, W2..W4 (4 each); bwd: W5^T, W4^T..W2^T
constexpr uint32_t kID256 = idesc_bf16_m128(256), kID32 = idesc_bf16_m128(32),
                   kID16 = idesc_bf16_m128(16);

struct KP {
  int64_t B, ntiles;
  int gen;       // rows drawn in the forward kernel (Gen) instead of read from X0 / U
  int x0_early;  // X0 / U written before the previous kernel: read before the wait
  int gen_next;  // the weight-gradient kernel draws the next step's rows (gn) into x0n / un
  Gen g, gn;
  float *x0n, *un;
  const float *X0, *U, *params;
  const uint8_t *img;
  uint8_t *xt, *at[4], *dzt[4], *dv, *dvt;
  uint32_t *s[4];
  float *ws;
  double *loss;
  int *err;
};

struct Ctl {
  uint64_t full[NST], empty[NST];
  uint64_t aux_full, aux_empty;  // fwd: the resident W5 image; bwd: the tile's dV image
  uint64_t a_full[4];            // K chunk c of the next A operand written by all epilogue warps
  uint64_t acc_full[2];          // accumulator 0 / 1 complete (one barrier each: the MMA
                                 // may finish the other accumulator before a wait)
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

// shared memory (offsets from a 1024-byte aligned base)
constexpr uint32_t S_A = 0;                       // 4 chunks: the A operand (X0 in chunk 0)
constexpr uint32_t S_ST = 4 * ACH;                // NST weight stages
constexpr uint32_t S_AUX = S_ST + NST * WCH;      // fwd: W5 (8 KB); bwd: dV (16 KB)
constexpr uint32_t S_BIAS = S_AUX + ACH;          // fwd: b1..b4, b5 (FP32)
constexpr uint32_t S_CTL = S_BIAS + 4352;
constexpr uint32_t FB_SMEM = S_CTL + 256 + 1024;  // + alignment slack
static_assert(sizeof(Ctl) <= 256, "control block");
static_assert(FB_SMEM <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) { return smem_desc(addr, 1024, kSwizzle128B); }


__device__ __forceinline__ void fail(Ctl &c, int *err, int code) {
  c.abort = 1;
  atomicExch(err, code);
}

// The weight stream of one CTA (warp 0, lane 0): per tile the 13 chunks
// base + g * WCH, g = 0..12; in the backward kernel also the tile's dV image.
// Waits for every copy it issued before returning.
template <bool BWD>
__device__ void produce(Ctl &C, const KP &P, unsigned char *sm, uint32_t base, volatile int *abort) {
  int issued = 0, it = 0;
  bool ok = true;
  // the backward weight images were written before the previous kernel ran:
  // the first stages fill before the wait
  if (BWD)
    for (; issued < NST; ++issued) {
      mbar_arrive_expect_tx(&C.full[issued], WCH);
      bulk_g2s(sm + S_ST + issued * WCH, P.img + base + (uint32_t)issued * WCH, WCH, &C.full[issued]);
    }
  grid_dep_wait();
  grid_dep_launch();
  for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x, ++it) {
    if (BWD) {
      if (it > 0 && !mbar_wait(&C.aux_empty, (uint32_t)(it - 1) & 1u, abort)) {
        ok = false;
        break;
      }
      mbar_arrive_expect_tx(&C.aux_full, ACH);
      bulk_g2s(sm + S_AUX, P.dv + t * TILE_DV, ACH, &C.aux_full);
    }
    for (int g = (BWD && it == 0) ? NST : 0; g < kTileChunks; ++g, ++issued) {
      const int s = issued % NST;
      if (issued >= NST && !mbar_wait(&C.empty[s], (uint32_t)(issued / NST - 1) & 1u, abort)) {
        ok = false;
        break;
      }
      mbar_arrive_expect_tx(&C.full[s], WCH);
      bulk_g2s(sm + S_ST + s * WCH, P.img + base + (uint32_t)g * WCH, WCH, &C.full[s]);
    }
  }
  if (!ok) fail(C, P.err, 21);
  // copies in flight land before the CTA may exit
  int never = 0;
  for (int k = issued > NST ? issued - NST : 0; k < issued; ++k)
    mbar_wait(&C.full[k % NST], (uint32_t)(k / NST) & 1u, &never, 1000000000ull);
  if (BWD && it > 0) mbar_wait(&C.aux_full, (uint32_t)(it - 1) & 1u, &never, 1000000000ull);
}

// Transposed stores of one warp's 32 rows x 16 columns (col0 .. col0 + 15,
// col0 a multiple of 16) into an image whose rows are the columns and whose
// K index is the row r & 63. Lane pairs (r, r + 1) swap halves so that each
// lane writes one 32-bit word per column pair: the even lane rows r, r + 1 of
// column c, the odd lane those of column c + 1. The swizzled offset of word
// jj is (col0 / 8) * 1024 + (jj / 4) * 1024 + off[jj % 4], off[] fixed per lane.
struct TOff {
  uint32_t off[4];
  uint32_t sel;  // byte selector: (own c lo, partner c lo) or (partner c+1 hi, own c+1 hi)
};

__device__ __forceinline__ TOff t_offsets(int r, int lane) {
  const int odd = lane & 1, r0 = r & ~1, rk = (r0 & 63) >> 3;
  TOff o;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int cc = 2 * j + odd;  // the word's image row within its 8-row group
    o.off[j] = (uint32_t)(cc * 128 + ((rk ^ cc) << 4) + (r0 & 7) * 2);
  }
  o.sel = odd ? 0x3276u : 0x5410u;
  return o;
}

// words[jj] holds this row's columns col0 + 2 jj (low) and + 1 (high).
__device__ __forceinline__ void st_transposed16(uint8_t *img, int col0, const uint32_t (&w)[8], const TOff &o) {
  uint8_t *base = img + (uint32_t)(col0 >> 3) * 1024u;
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const uint32_t partner = __shfl_xor_sync(0xffffffffu, w[jj], 1);
    *reinterpret_cast<uint32_t *>(base + (jj >> 2) * 1024 + o.off[jj & 3]) = __byte_perm(w[jj], partner, o.sel);
  }
}

// Columns 8 gq .. 8 gq + 7 of batch row b (the X0 layout: standardized
// condition, x_t, the 16 time-embedding features, zeros).
__device__ __forceinline__ void batch_cols(const Gen &G, int64_t B, int64_t b, int gq, float (&x)[8]) {
  const uint64_t rid = (uint64_t)G.step * (uint64_t)B + (uint64_t)b;
  const uint4 r0 = philox_draw(G.seed, rid, 0u, kTagTrain);
  const int64_t idx = (int64_t)(((uint64_t)r0.x * (uint64_t)G.n) >> 32);
  const float t = u01(r0.y);
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 0.0f;
  if (gq < 2) {
    const float4 z = box_muller4(philox_draw(G.seed, rid, 1u, kTagTrain));
    const float x0[4] = {z.x, z.y, z.z, z.w};
    if (gq == 0) {
#pragma unroll
      for (int k = 0; k < 5; ++k) x[k] = (__ldg(G.cond + k * G.n + idx) - G.sd.cm[k]) * G.sd.cis[k];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float x1 = (__ldg(G.y + d * G.n + idx) - G.sd.ym[d]) * G.sd.yis[d];
        x[5 + d] = (1.0f - t) * x0[d] + t * x1;
      }
    } else {
      const float x1 = (__ldg(G.y + 3 * G.n + idx) - G.sd.ym[3]) * G.sd.yis[3];
      x[0] = (1.0f - t) * x0[3] + t * x1;
#pragma unroll
      for (int j = 0; j < 7; ++j) x[1 + j] = time_embedding(j, t);
    }
  } else if (gq == 2) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = time_embedding(7 + j, t);
  } else {
    x[0] = time_embedding(15, t);
  }
}

// The regression target u = x1 - x0 of batch row b.
__device__ __forceinline__ void batch_u(const Gen &G, int64_t B, int64_t b, float (&u)[4]) {
  const uint64_t rid = (uint64_t)G.step * (uint64_t)B + (uint64_t)b;
  const uint4 r0 = philox_draw(G.seed, rid, 0u, kTagTrain);
  const int64_t idx = (int64_t)(((uint64_t)r0.x * (uint64_t)G.n) >> 32);
  const float4 z = box_muller4(philox_draw(G.seed, rid, 1u, kTagTrain));
  const float x0[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
  for (int d = 0; d < 4; ++d) u[d] = (__ldg(G.y + d * G.n + idx) - G.sd.ym[d]) * G.sd.yis[d] - x0[d];
}

// Setup shared by the forward and input-gradient kernels: barriers, the
// tensor memory of two accumulators (columns 0-255 and 256-511).
__device__ __forceinline__ uint32_t fb_setup(Ctl &C, int warp) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&C.full[s], 1);
      mbar_init(&C.empty[s], 1);
    }
    mbar_init(&C.aux_full, 1);
    mbar_init(&C.aux_empty, 1);
    for (int c = 0; c < 4; ++c) mbar_init(&C.a_full[c], NEPI);
    mbar_init(&C.acc_full[0], 1);
    mbar_init(&C.acc_full[1], 1);
    mbar_init(&C.drain, 1);
    C.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&C.tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return C.tmem_base;
}

// One warp's 32 rows x 16 columns of an accumulator (columns col0 ..).
__device__ __forceinline__ void acc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  tmem_ld16_raw(taddr, r);
  tmem_wait_ld_regs16(r);
}

// K chunk c of the next A operand is in shared memory: this warp's part.
__device__ __forceinline__ void chunk_written(Ctl &C, int c, int lane) {
  tc_fence_before();
  fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0) mbar_arrive(&C.a_full[c]);
}

// Forward: per tile, layer 1 (K = 32) and layers 2-4 (K = 256) with N = 256,
// layer 5 with N = 16 (4 used). The layers alternate between two
// accumulators, and the A operand has a barrier per 64-channel K chunk: the
// epilogue of layer l converts the accumulator chunk by chunk (16 warps: lane
// quadrant q = warp % 4, 16 columns of every chunk each), and the MMAs of
// layer l + 1 start on chunk c as soon as all warps have written it, while the
// epilogue is still on the later chunks.
__global__ void __launch_bounds__(FB_THREADS, 1) fwd_kernel(KP P) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char *sm = smem_raw + pad;
  const uint32_t sb = raw + pad;
  Ctl &C = *reinterpret_cast<Ctl *>(sm + S_CTL);
  float *bias = reinterpret_cast<float *>(sm + S_BIAS);  // [4][256] halved, then b5[4]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const uint32_t tmem = fb_setup(C, warp);
  volatile int *abort = &C.abort;

  if (warp == 0) {
    if (lane == 0) {
      grid_dep_wait();  // the weight images of this step
      mbar_arrive_expect_tx(&C.aux_full, 8192);
      bulk_g2s(sm + S_AUX, P.img + WF5, 8192, &C.aux_full);
      produce<false>(C, P, sm, WF1, abort);
      int never = 0;
      mbar_wait(&C.aux_full, 0, &never, 1000000000ull);
    }
  } else if (warp == 1) {
    int used = 0, gl = 0;
    uint32_t af[4] = {0u, 0u, 0u, 0u};
    bool ok = mbar_wait(&C.aux_full, 0, abort);
    for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
      for (int L = 0; L < 5 && ok; ++L, ++gl) {
        const uint32_t acc = tmem + (uint32_t)(gl & 1) * 256u;
        const int nch = L == 0 ? 1 : 4;
        for (int c = 0; c < nch && ok; ++c) {
          if (!mbar_wait(&C.a_full[c], af[c] & 1u, abort)) {
            ok = false;
            break;
          }
          ++af[c];
          const uint64_t da = sdesc(sb + S_A + (uint32_t)c * ACH);
          if (L < 4) {
            const int s = used % NST;
            if (!mbar_wait(&C.full[s], (uint32_t)(used / NST) & 1u, abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t db = sdesc(sb + S_ST + (uint32_t)s * WCH);
            const int nk = L == 0 ? 2 : 4;
            for (int k = 0; k < nk; ++k)
              mma_f16_w(acc, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), kID256, (c | k) != 0);
            mma_commit_w(&C.empty[s]);
            ++used;
          } else {
            tc_fence_after();
            const uint64_t db = sdesc(sb + S_AUX + (uint32_t)c * 2048);
            for (int k = 0; k < 4; ++k)
              mma_f16_w(acc, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), kID16, (c | k) != 0);
          }
        }
        if (!ok) break;
        mma_commit_w(&C.acc_full[gl & 1]);
      }
    }
    if (!ok && lane == 0) fail(C, P.err, 22);
    // every MMA issued completes before tensor memory is freed
    mma_commit_w(&C.drain);
    int never = 0;
    mbar_wait(&C.drain, 0, &never, 1000000000ull);
  } else {
    const int e = warp - 2, q = warp & 3, p = e >> 2;
    const int r = 32 * q + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
    const TOff toff = t_offsets(r, lane);
    int gl = 0;  // layers so far: accumulator gl & 1, its (gl >> 1)-th use
    bool ok = true;
    if (!P.gen && !P.x0_early) grid_dep_wait();  // rows given in X0 / U by the previous kernel
    for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
      const int64_t b = t * TR + r;
      const bool valid = b < P.B;  // rows past the batch: finite values, zero dV
      float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // the row's target, loaded ahead of layer 5
      if (p == 0 && valid) {
        if (P.gen) {
          batch_u(P.g, P.B, b, u);
        } else {
#pragma unroll
          for (int o = 0; o < 4; ++o) u[o] = __ldg(P.U + b * 4 + o);
        }
      }
      {  // batch rows -> BF16 A image (chunk 0, K 0..31) and the X0^T image
        const int ei = e * 32 + lane, rr = ei >> 2, gq = ei & 3;
        const int64_t bb = t * TR + rr;
        float x[8];
        if (bb < P.B && P.gen) {
          batch_cols(P.g, P.B, bb, gq, x);
        } else if (bb < P.B) {
          const float4 lo = __ldg(reinterpret_cast<const float4 *>(P.X0 + bb * 32 + 8 * gq));
          const float4 hi = __ldg(reinterpret_cast<const float4 *>(P.X0 + bb * 32 + 8 * gq + 4));
          x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w;
          x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) x[j] = 0.0f;
        }
        sts128(sb + S_A + img_off(rr, 8 * gq), pack2(x[0], x[1]), pack2(x[2], x[3]), pack2(x[4], x[5]),
               pack2(x[6], x[7]));
        if (t == blockIdx.x) {
          // the first tile's rows were drawn before the wait; the biases of
          // this step are the previous kernel's output
          grid_dep_wait();
          grid_dep_launch();
          for (int i = e * 32 + lane; i < 1028; i += 32 * NEPI) {
            const int64_t src = i < 1024 ? (i < 256 ? P_B1 : i < 512 ? P_B2 - 256 : i < 768 ? P_B3 - 512 : P_B4 - 768) + i
                                         : P_B5 + (i - 1024);
            bias[i] = i < 1024 ? 0.5f * P.params[src] : P.params[src];  // layers 1-4 halved (h = z / 2)
          }
          asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");  // the epilogue warps only
        }
        chunk_written(C, 0, lane);
        uint8_t *xt = P.xt + t * TILE_XT + (uint32_t)(rr >> 6) * 4096u;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<uint16_t *>(xt + img_off(8 * gq + j, rr & 63)) = bf16_bits(x[j]);
      }
      for (int L = 0; L < 4; ++L, ++gl) {
        if (!mbar_wait(&C.acc_full[gl & 1], (uint32_t)(gl >> 1) & 1u, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tacc = tl + (uint32_t)(gl & 1) * 256u;
        const float *bl = bias + L * 256;
        uint32_t *sl = P.s[L] + t * (TILE_S / 4) + r;
        uint8_t *at = P.at[L] + t * TILE_AT + (uint32_t)(r >> 6) * 32768u;
        // chunk c + 1's accumulator columns load while chunk c converts
        uint32_t acc[2][16];
        acc_ld16(tacc + (uint32_t)(16 * p), acc[0]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int col0 = 64 * c + 16 * p;
          if (c < 3) tmem_ld16_raw(tacc + (uint32_t)(col0 + 64), acc[(c + 1) & 1]);
          uint32_t pa[8];
          float hb[16];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float4 v4 = *reinterpret_cast<const float4 *>(bl + col0 + 4 * i);
            hb[4 * i] = v4.x; hb[4 * i + 1] = v4.y; hb[4 * i + 2] = v4.z; hb[4 * i + 3] = v4.w;
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            float a2[2], s2[2];
#pragma unroll
            for (int u = 0; u < 2; ++u)
              silu_and_grad(fmaf(__uint_as_float(acc[c & 1][2 * jj + u]), 0.5f, hb[2 * jj + u]), a2[u], s2[u]);
            pa[jj] = pack2(a2[0], a2[1]);
            sl[((col0 >> 1) + jj) * TR] = pack2(s2[0], s2[1]);  // S_l for the backward kernel
          }
          const uint32_t dst = sb + S_A + (uint32_t)c * ACH;
          sts128(dst + img_off(r, 16 * p), pa[0], pa[1], pa[2], pa[3]);
          sts128(dst + img_off(r, 16 * p + 8), pa[4], pa[5], pa[6], pa[7]);
          chunk_written(C, c, lane);
          // A_l^T for the weight gradients, off the MMA's critical path
          st_transposed16(at, col0, pa, toff);
          if (c < 3) tmem_wait_ld_regs16(acc[(c + 1) & 1]);
        }
      }
      if (!ok) break;
      // layer 5: v = A4 W5^T + b5, the loss and dV
      if (!mbar_wait(&C.acc_full[gl & 1], (uint32_t)(gl >> 1) & 1u, abort)) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (p == 0) {
        float v[4];
        tmem_ld4(tl + (uint32_t)(gl & 1) * 256u, v);
        tmem_wait_ld_regs4(v);
        double part = 0.0;
        float dv[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          dv[o] = 0.0f;
          if (valid) {
            const float res = (v[o] + bias[1024 + o]) - u[o];
            part += (double)res * res;
            dv[o] = 2.0f * res / (float)P.B;
          }
        }
        uint8_t *dvi = P.dv + t * TILE_DV;
        *reinterpret_cast<uint4 *>(dvi + img_off(r, 0)) =
            make_uint4(pack2(dv[0], dv[1]), pack2(dv[2], dv[3]), 0u, 0u);
        *reinterpret_cast<uint4 *>(dvi + img_off(r, 8)) = make_uint4(0u, 0u, 0u, 0u);
        uint8_t *dvt = P.dvt + t * TILE_DVT + (uint32_t)(r >> 6) * 2048u;
#pragma unroll
        for (int o = 0; o < 4; ++o)
          *reinterpret_cast<uint16_t *>(dvt + img_off(o, r & 63)) = bf16_bits(dv[o]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0 && part != 0.0) atomicAdd(P.loss, part / (double)P.B);
      }
      ++gl;
      tc_fence_before();
    }
    if (!ok && lane == 0) fail(C, P.err, 23);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// Input gradients: per tile the stages dZ4 = (dV W5) S4 (K = 16, the dV image
// from the forward kernel), then dZ3, dZ2, dZ1 (K = 256 against W_l^T), the
// stages alternating between two accumulators. The epilogue of a stage
// writes dZ chunk by chunk as the next stage's A operand (shared memory;
// the MMAs of the next stage start on each chunk once written) and dZ^T for
// the weight gradients; S_l is loaded before the accumulator is ready.
__global__ void __launch_bounds__(FB_THREADS, 1) bwd_kernel(KP P) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char *sm = smem_raw + pad;
  const uint32_t sb = raw + pad;
  Ctl &C = *reinterpret_cast<Ctl *>(sm + S_CTL);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tmem = fb_setup(C, warp);
  volatile int *abort = &C.abort;

  if (warp == 0) {
    if (lane == 0) produce<true>(C, P, sm, WB5, abort);
  } else if (warp == 1) {
    int used = 0, it = 0, gl = 0;
    uint32_t af[4] = {0u, 0u, 0u, 0u};
    bool ok = true;
    for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x, ++it) {
      for (int R = 0; R < 4 && ok; ++R, ++gl) {
        const uint32_t acc = tmem + (uint32_t)(gl & 1) * 256u;
        if (R == 0) {
          const int s = used % NST;
          if (!mbar_wait(&C.aux_full, (uint32_t)it & 1u, abort) ||
              !mbar_wait(&C.full[s], (uint32_t)(used / NST) & 1u, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          mma_f16_w(acc, sdesc(sb + S_AUX), sdesc(sb + S_ST + (uint32_t)s * WCH), kID256, 0u);
          mma_commit_w(&C.empty[s]);
          mma_commit_w(&C.aux_empty);
          ++used;
        } else {
          for (int c = 0; c < 4 && ok; ++c) {
            const int s = used % NST;
            if (!mbar_wait(&C.a_full[c], af[c] & 1u, abort) ||
                !mbar_wait(&C.full[s], (uint32_t)(used / NST) & 1u, abort)) {
              ok = false;
              break;
            }
            ++af[c];
            tc_fence_after();
            const uint64_t da = sdesc(sb + S_A + (uint32_t)c * ACH), db = sdesc(sb + S_ST + (uint32_t)s * WCH);
            for (int k = 0; k < 4; ++k)
              mma_f16_w(acc, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), kID256, (c | k) != 0);
            mma_commit_w(&C.empty[s]);
            ++used;
          }
          if (!ok) break;
        }
        mma_commit_w(&C.acc_full[gl & 1]);
      }
    }
    if (!ok && lane == 0) fail(C, P.err, 24);
    mma_commit_w(&C.drain);
    int never = 0;
    mbar_wait(&C.drain, 0, &never, 1000000000ull);
  } else {
    const int e = warp - 2, q = warp & 3, p = e >> 2;
    const int r = 32 * q + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
    const TOff toff = t_offsets(r, lane);
    int gl = 0;  // rounds so far: accumulator gl & 1, its (gl >> 1)-th use
    bool ok = true;
    grid_dep_wait();  // S_l and the images of the forward kernel
    for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
      for (int R = 0; R < 4; ++R, ++gl) {
        const int Lo = 3 - R;  // dZ of hidden layer Lo + 1
        // S_l of this thread's 16 columns of chunk c: words 32 c + 8 p .. + 7
        // (one chunk ahead of its use)
        uint32_t sv[8], sn[8];
        const uint32_t *sl = P.s[Lo] + t * (TILE_S / 4) + r + (8 * p) * TR;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) sv[jj] = __ldg(sl + jj * TR);
        if (!mbar_wait(&C.acc_full[gl & 1], (uint32_t)(gl >> 1) & 1u, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tacc = tl + (uint32_t)(gl & 1) * 256u;
        uint8_t *dz = P.dzt[Lo] + t * TILE_AT + (uint32_t)(r >> 6) * 32768u;
        // chunk c + 1's accumulator columns and S words load while chunk c converts
        uint32_t acc[2][16];
        acc_ld16(tacc + (uint32_t)(16 * p), acc[0]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int col0 = 64 * c + 16 * p;
          if (c < 3) {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) sn[jj] = __ldg(sl + (32 * (c + 1) + jj) * TR);
            tmem_ld16_raw(tacc + (uint32_t)(col0 + 64), acc[(c + 1) & 1]);
          }
          uint32_t pd[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            pd[jj] = pack2(__uint_as_float(acc[c & 1][2 * jj]) * lo_f(sv[jj]),
                           __uint_as_float(acc[c & 1][2 * jj + 1]) * hi_f(sv[jj]));
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) sv[jj] = sn[jj];
          if (Lo > 0) {
            const uint32_t dst = sb + S_A + (uint32_t)c * ACH;
            sts128(dst + img_off(r, 16 * p), pd[0], pd[1], pd[2], pd[3]);
            sts128(dst + img_off(r, 16 * p + 8), pd[4], pd[5], pd[6], pd[7]);
            chunk_written(C, c, lane);
          }
          st_transposed16(dz, col0, pd, toff);
          if (c < 3) tmem_wait_ld_regs16(acc[(c + 1) & 1]);
        }
      }
    }
    if (!ok && lane == 0) fail(C, P.err, 25);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// ---- weight gradients -------------------------------------------------------

// Job j of the grid's x dimension, batch slice y:
//   j < 8:  hidden layer l = j / 2, output rows 128 h .. (h = j % 2):
//           D[o][i] = sum_b dZ_l^T[o][b] A_{l-1}^T[i][b] (N = 256; N = 32 for
//           layer 1 against X0^T), and db[o] = sum_b dZ_l^T[o][b] (N = 16
//           against the ones image, accumulator columns 256..271)
//   j = 8, 9: W5 with M = its inputs 128 h ..: D[i][o] = sum_b A4^T[i][b] dV^T[o][b]
//           (N = 16, 4 used); j = 8 also db5 (the ones image as A operand).
// The slice's FP32 result goes to ws[y][...] at the parameter's own offset.
constexpr int WG_THREADS = 192;  // producer, MMA, 4 epilogue warps
constexpr int WNST = 4;
constexpr uint32_t W_A = 16384, W_B = 32768, W_STAGE = W_A + W_B;
constexpr uint32_t W_ONES16 = WNST * W_STAGE, W_ONES128 = W_ONES16 + 2048;
constexpr uint32_t W_CTL = W_ONES128 + 16384;
constexpr uint32_t WG_SMEM = W_CTL + 256 + 1024;
static_assert(WG_SMEM <= 227 * 1024, "shared memory per CTA");

struct WCtl {
  uint64_t full[WNST], empty[WNST];
  uint64_t acc_full, drain;
  uint32_t tmem_base;
  int abort;
};

__global__ void __launch_bounds__(WG_THREADS, 1) wgrad_kernel(KP P) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char *sm = smem_raw + pad;
  const uint32_t sb = raw + pad;
  WCtl &C = *reinterpret_cast<WCtl *>(sm + W_CTL);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int job = blockIdx.x, split = blockIdx.y, S = gridDim.y;
  const int64_t t0 = (int64_t)split * P.ntiles / S, t1 = (int64_t)(split + 1) * P.ntiles / S;
  const int nchunks = (int)(2 * (t1 - t0));
  const bool w5 = job >= 8;
  const int layer = w5 ? 4 : job >> 1, h = w5 ? job - 8 : job & 1;
  const uint32_t b_bytes = w5 ? 2048u : (layer == 0 ? 4096u : 32768u);
  const uint32_t nmain = w5 ? 16u : (layer == 0 ? 32u : 256u);
  const bool bias = job != 9;

  // BF16 ones (0x3F80) for the bias contractions
  uint32_t *ones = reinterpret_cast<uint32_t *>(sm + W_ONES16);
  for (int i = threadIdx.x; i < (2048 + 16384) / 4; i += WG_THREADS) ones[i] = 0x3F803F80u;
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int s = 0; s < WNST; ++s) {
      mbar_init(&C.full[s], 1);
      mbar_init(&C.empty[s], 1);
    }
    mbar_init(&C.acc_full, 1);
    mbar_init(&C.drain, 1);
    C.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&C.tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = C.tmem_base;
  volatile int *abort = &C.abort;

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      int k = 0;
      grid_dep_wait();  // dZ^T of the input-gradient kernel
      grid_dep_launch();
      for (; k < nchunks; ++k) {
        const int s = k % WNST;
        if (k >= WNST && !mbar_wait(&C.empty[s], (uint32_t)(k / WNST - 1) & 1u, abort)) {
          ok = false;
          break;
        }
        const int64_t t = t0 + (k >> 1);
        const uint32_t bc = (uint32_t)(k & 1);
        const uint8_t *src_a = w5 ? P.at[3] + t * TILE_AT + bc * 32768u + (uint32_t)h * 16384u
                                  : P.dzt[layer] + t * TILE_AT + bc * 32768u + (uint32_t)h * 16384u;
        const uint8_t *src_b = w5 ? P.dvt + t * TILE_DVT + bc * 2048u
                                  : (layer == 0 ? P.xt + t * TILE_XT + bc * 4096u
                                                : P.at[layer - 1] + t * TILE_AT + bc * 32768u);
        mbar_arrive_expect_tx(&C.full[s], W_A + b_bytes);
        bulk_g2s(sm + (uint32_t)s * W_STAGE, src_a, W_A, &C.full[s]);
        bulk_g2s(sm + (uint32_t)s * W_STAGE + W_A, src_b, b_bytes, &C.full[s]);
      }
      if (!ok) {
        C.abort = 1;
        atomicExch(P.err, 26);
      }
      int never = 0;
      for (int j = k > WNST ? k - WNST : 0; j < k; ++j)
        mbar_wait(&C.full[j % WNST], (uint32_t)(j / WNST) & 1u, &never, 1000000000ull);
    }
  } else if (warp == 1) {
    bool ok = true;
    const uint32_t idm = nmain == 256 ? kID256 : (nmain == 32 ? kID32 : kID16);
    for (int k = 0; k < nchunks; ++k) {
      const int s = k % WNST;
      if (!mbar_wait(&C.full[s], (uint32_t)(k / WNST) & 1u, abort)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = sb + (uint32_t)s * W_STAGE, sbb = sa + W_A;
      const uint64_t da = sdesc(sa), db = sdesc(sbb);
      // bias: dZ^T against ones (layers), or ones against dV^T (W5)
      const uint64_t xa = w5 ? sdesc(sb + W_ONES128) : da, xb = w5 ? db : sdesc(sb + W_ONES16);
      for (int kk = 0; kk < 4; ++kk) {
        mma_f16_w(tmem, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idm, (k | kk) != 0);
        if (bias)
          mma_f16_w(tmem + 256, xa + (uint64_t)(2 * kk), xb + (uint64_t)(2 * kk), kID16, (k | kk) != 0);
      }
      mma_commit_w(&C.empty[s]);
    }
    if (ok) mma_commit_w(&C.acc_full);
    if (!ok && lane == 0) {
      C.abort = 1;
      atomicExch(P.err, 27);
    }
    mma_commit_w(&C.drain);
    int never = 0;
    mbar_wait(&C.drain, 0, &never, 1000000000ull);
  } else {
    const int q = warp & 3, m = 32 * q + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
    if (P.gen_next) {
      // the next step's batch rows (static data only: before any wait),
      // about one per epilogue thread, drawn while the operands stream in
      const int64_t nthr = (int64_t)gridDim.x * gridDim.y * 128;
      for (int64_t b = ((int64_t)split * gridDim.x + job) * 128 + (warp - 2) * 32 + lane; b < P.B; b += nthr)
        batch_row(P.gn, P.B, b, P.x0n + b * 32, P.un + b * 4);
    }
    if (mbar_wait(&C.acc_full, 0, abort)) {
      tc_fence_after();
      float *ws = P.ws + (int64_t)split * P_TOTAL;
      if (!w5) {
        const int64_t wofs = layer == 0 ? P_W1 : layer == 1 ? P_W2 : layer == 2 ? P_W3 : P_W4;
        const int64_t bofs = layer == 0 ? P_B1 : layer == 1 ? P_B2 : layer == 2 ? P_B3 : P_B4;
        const int o = 128 * h + m;
        float *row = ws + wofs + (int64_t)o * nmain;
        for (uint32_t cb = 0; cb < nmain; cb += 32) {
          uint32_t acc[32];
          tmem_ld32_raw(tl + cb, acc);
          tmem_wait_ld_regs(acc);
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4 *>(row + cb + j) =
                make_float4(__uint_as_float(acc[j]), __uint_as_float(acc[j + 1]),
                            __uint_as_float(acc[j + 2]), __uint_as_float(acc[j + 3]));
        }
        float bv[4];
        tmem_ld4(tl + 256, bv);
        tmem_wait_ld_regs4(bv);
        ws[bofs + o] = bv[0];
      } else {
        float v[4];
        tmem_ld4(tl, v);
        tmem_wait_ld_regs4(v);
#pragma unroll
        for (int o = 0; o < 4; ++o) ws[P_W5 + o * 256 + 128 * h + m] = v[o];
        if (bias) {
          float bv[4];
          tmem_ld4(tl + 256, bv);
          tmem_wait_ld_regs4(bv);
          if (m == 0)
#pragma unroll
            for (int o = 0; o < 4; ++o) ws[P_B5 + o] = bv[o];
        }
      }
    } else if (lane == 0) {
      C.abort = 1;
      atomicExch(P.err, 28);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

template <typename Kernel>
cudaError_t set_smem(Kernel k, size_t bytes, std::atomic<bool> (&done)[kMaxDevices]) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < kMaxDevices && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) done[dev].store(true, std::memory_order_release);
  return e;
}

// A launch that may begin while the previous kernel of the stream finishes
// (the kernel's griddepcontrol.wait orders its dependent work).
template <typename Arg>
cudaError_t launch_dep(void (*k)(Arg), dim3 grid, int threads, size_t smem, cudaStream_t s, const Arg &arg) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, arg);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

cudaError_t alloc(Bufs &b, int64_t batch, cudaStream_t s) {
  const int64_t tiles = (batch + TR - 1) / TR;
  if (b.img && b.tiles >= tiles) return cudaSuccess;
  release(b);
  cudaError_t e = cudaMalloc(&b.img, WIMG_BYTES);
  if (e == cudaSuccess) e = cudaMalloc(&b.act, (size_t)tiles * TILE_BYTES);
  b.max_splits = sm_count() / kJobs;
  if (b.max_splits < 1) b.max_splits = 1;
  if (b.max_splits > kMaxSplits) b.max_splits = kMaxSplits;
  if (e == cudaSuccess) e = cudaMalloc(&b.ws, (size_t)b.max_splits * P_TOTAL * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b.x0n, (size_t)tiles * TR * 36 * sizeof(float));
  if (e == cudaSuccess) b.un = b.x0n + (size_t)tiles * TR * 32;
  // zero padding of the images (K beyond the operand, unused rows) stays zero
  if (e == cudaSuccess) e = cudaMemsetAsync(b.img, 0, WIMG_BYTES, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.act, 0, (size_t)tiles * TILE_BYTES, s);
  if (e != cudaSuccess) {
    release(b);
    return e;
  }
  b.tiles = tiles;
  uint8_t *p = b.act;
  b.xt = p;
  p += tiles * TILE_XT;
  for (int l = 0; l < 4; ++l, p += tiles * TILE_AT) b.at[l] = p;
  for (int l = 0; l < 4; ++l, p += tiles * TILE_AT) b.dzt[l] = p;
  for (int l = 0; l < 4; ++l, p += tiles * TILE_S) b.s[l] = reinterpret_cast<uint32_t *>(p);
  b.dv = p;
  p += tiles * TILE_DV;
  b.dvt = p;
  return cudaSuccess;
}

void release(Bufs &b) {
  if (b.img) cudaFree(b.img);
  if (b.act) cudaFree(b.act);
  if (b.ws) cudaFree(b.ws);
  if (b.x0n) cudaFree(b.x0n);
  b = Bufs{};
}

cudaError_t pack(cudaStream_t s, Bufs &b, float *params) {
  if (!b.img) return cudaErrorInvalidValue;
  Upd U{};
  U.mode = 4;
  U.p = params;
  U.bc1 = U.bc2 = 1.0f;
  U.img = b.img;
  update_kernel<<<kUpdBlocks, 256, 0, s>>>(U);
  return cudaGetLastError();
}

cudaError_t step(cudaStream_t s, Bufs &b, int64_t B, const Gen *gen, const float *X0, const float *U,
                 bool rows_early, float *params, float *grad, float *m, float *v, const Adam *adam,
                 double *loss, int *err, const Gen *next) {
  const int64_t ntiles = (B + TR - 1) / TR;
  if (B < 1 || !b.img || ntiles > b.tiles || (!gen && (!X0 || !U))) return cudaErrorInvalidValue;
  static std::atomic<bool> a_fwd[kMaxDevices], a_bwd[kMaxDevices], a_wg[kMaxDevices];
  cudaError_t e = set_smem(fwd_kernel, FB_SMEM, a_fwd);
  if (e == cudaSuccess) e = set_smem(bwd_kernel, FB_SMEM, a_bwd);
  if (e == cudaSuccess) e = set_smem(wgrad_kernel, WG_SMEM, a_wg);
  if (e != cudaSuccess) return e;
  KP P{};
  P.B = B;
  P.ntiles = ntiles;
  P.gen = gen != nullptr;
  if (gen) P.g = *gen;
  P.x0_early = rows_early && !gen;
  P.gen_next = next != nullptr;
  if (next) P.gn = *next;
  P.x0n = b.x0n;
  P.un = b.un;

  P.X0 = X0;
  P.U = U;
  P.params = params;
  P.img = b.img;
  P.xt = b.xt;
  for (int l = 0; l < 4; ++l) {
    P.at[l] = b.at[l];
    P.dzt[l] = b.dzt[l];
    P.s[l] = b.s[l];
  }
  P.dv = b.dv;
  P.dvt = b.dvt;
  P.ws = b.ws;
  P.loss = loss;
  P.err = err;
  const int sms = sm_count();
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
  const int S = (int)(ntiles < b.max_splits ? ntiles : b.max_splits);
  const Adam a = adam ? *adam : Adam{0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f};
  const Upd upd{adam ? 7 : 1, S, b.ws, grad, params, m, v, a.lr, a.b1, a.b2, a.eps, a.wd, a.bc1, a.bc2, b.img};
  e = launch_dep(fwd_kernel, dim3(grid), FB_THREADS, FB_SMEM, s, P);
  if (e == cudaSuccess) e = launch_dep(bwd_kernel, dim3(grid), FB_THREADS, FB_SMEM, s, P);
  if (e == cudaSuccess) e = launch_dep(wgrad_kernel, dim3(kJobs, (unsigned)S), WG_THREADS, WG_SMEM, s, P);
  if (e == cudaSuccess) e = launch_dep(update_kernel, dim3(kUpdBlocks), 256, 0, s, upd);
  return e;
}

}  // namespace tf
}  // namespace gmc
