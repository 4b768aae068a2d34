// BF16 flow-ODE sampler (Eq. 8) on CTA pairs: tcgen05.mma.cta_group::2 with
// M = 256 tiles, two FP32 accumulators per CTA so the tensor core never waits
// for the epilogue to read one, and the hidden activations in shared memory.
//
// Work unit: a tile of 256 particles computed by a cluster of two CTAs on two
// SMs; CTA r holds rows 128 r .. 128 r + 127 of the tile (tensor-memory lanes
// 0-127 and its A operand) and output rows 128 r .. of every weight matrix
// (the B operand is split along N between the pair). The even CTA issues the
// MMAs for both. A persistent pair owns two tiles (X, Y) at a time and
// alternates them: the tensor core computes a layer of one tile while the
// epilogue warps of both CTAs turn the other tile's previous layer into
// activations:
//
//   MMA (even CTA):  L(X)   L(Y)   L+1(X)   L+1(Y) ...
//   epilogue (both):        E(X)   E(Y)     E(X)  ...   (SiLU, BF16)
//
// Tensor memory of each CTA (512 columns): D_X (0-255) and D_Y (256-511),
// the 128 x 256 FP32 accumulators of its rows of the two tiles. A layer of
// tile T starts as soon as both CTAs have written T's activations: the
// accumulator of T was read before that, and the other tile's accumulator is
// never touched, so no tile waits for the other's epilogue.
//
// Shared memory of each CTA: A_X, A_Y (its 128 rows x 256 BF16 of the
// tile's activations, 4 K-blocks of 128 B rows, 128-byte swizzle, written by
// the epilogue with 16-byte stores), its half of every weight chunk streamed
// in 4 stages (128 output rows x 128 B of K, 16 KB), and resident: the
// layer-1 operands of X and Y, its halves of layer 1, layer 5 and the bias
// blocks of layers 2-4. Per tile-layer and SM the shared memory moves 64 KB
// of A and 64 KB of B to the tensor core, 64 KB of activations in and 64 KB
// of weights in: half the B traffic of a single-CTA M = 128 tile.
//
// Layers and numerics are those of sampler_tc.cu (same packed weights): L1
// [x_hi | x_lo | cn | 1 1 0] (K = 16) x B1 with the per-evaluation FP32 bias
// W1[:, emb] emb(t) + b1 added in the epilogue; L2-L4 with the bias entering
// through one K = 16 MMA against the constant-1 columns; L5 (N = 16) the
// velocity. SiLU(z) = h + h tanh(h), h = z/2, in packed BF16x2.
//
// Roles (576 threads per CTA): warp 0 streams this CTA's weight halves;
// warp 1 issues the MMAs (even CTA) or relays the odd CTA's copy completions
// to the even CTA (odd CTA); warps 2-17 are the epilogue, warp w serving
// tensor-memory lane quadrant w % 4 and accumulator columns 64 p .. 64 p + 63,
// p = (w - 2) / 4; the warps with p = 0 (p = 1) keep the ODE state of tile X
// (Y) in registers.
//
// Synchronization: the MMA completion is committed to the
// even CTA's barriers only, and threads relay it to the odd CTA with remote
// mbarrier arrivals (mapa + mbarrier.arrive.release.cluster); the odd CTA's
// copy completions and activation writes reach the even CTA the same way.
// Every wait is bounded; a timeout sets *err, raises both CTAs' abort flags,
// and the CTAs drain and exit.
#include <cuda_bf16.h>

#include <atomic>
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

using PK = Packed<false>;
constexpr int PM = 128;                      // rows per CTA of an M = 256 tile
constexpr int EPI_WARPS = 16;
constexpr int THREADS = 32 * (2 + EPI_WARPS);
constexpr int NCH = PK::NCH;                 // 4 chunks per hidden layer
constexpr uint32_t HCHUNK = 128u * 128u;     // this CTA's half of a chunk: 16 KB
constexpr int NST = 4;                       // weight stages
constexpr uint32_t TMEM_COLS = 512;

// shared memory (offsets from a 1024-byte aligned base)
constexpr uint32_t KB_BYTES = PM * 128;            // one K-block of A: 128 rows x 128 B
constexpr uint32_t A_BYTES = 4 * KB_BYTES;         // A_T: 64 KB
constexpr uint32_t S_A = 0;                        // A_X, A_Y
constexpr uint32_t S_ST = 2 * A_BYTES;             // NST weight stages
constexpr uint32_t S_A1 = S_ST + NST * HCHUNK;     // layer-1 operands of X, Y: 2 x 4 KB
constexpr uint32_t S_B1 = S_A1 + 8192;             // 128 rows x 32 B
constexpr uint32_t S_B5 = S_B1 + 4096;             // 4 K-blocks x 8 rows x 128 B
constexpr uint32_t S_BIAS = S_B5 + 4096;           // 3 layers x 128 rows x 32 B
constexpr uint32_t S_BAR = S_BIAS + 12288;
constexpr uint32_t SMEM_BYTES = S_BAR + 256 + 1024;  // + alignment slack
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
static_assert(SMEM_BYTES > 116 * 1024, "one CTA per SM");

struct Bars {
  uint64_t full[NST];   // even CTA: its copy (tx) + the odd CTA's relay; odd: its copy
  uint64_t empty[NST];  // even: the MMA commit; odd: relay of it by the even producer
  uint64_t res_full;    // this CTA's resident halves landed
  uint64_t res_peer;    // even CTA: the odd CTA's resident halves landed (relay)
  uint64_t ar[2];       // even CTA: tile T's next operand written by all 32 epilogue warps
  uint64_t dfull[2];    // accumulator T complete: even = commit, odd = relay
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(Bars) <= 256, "barrier block");

// A timeout: this CTA's and the other CTA's abort flags, and the error word.
__device__ void fail(Bars &b, int *err, int code, uint32_t other) {
  b.abort = 1;
  st_cluster_u32(peer_smem(&b.abort, other), 1u);
  atomicExch(err, code);
}

// 16-byte chunk c (0..7) of row r of one K-block of A (128-byte swizzle).
__device__ __forceinline__ uint32_t sw128(uint32_t kb_base, int r, int c) {
  return kb_base + (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// Arrival of one epilogue warp (lane 0) on the even CTA's barrier `bar`.
__device__ __forceinline__ void arrive_even(uint64_t *bar, bool even) {
  if (even) mbar_arrive(bar);
  else mbar_arrive_remote(peer_smem(bar, 0));
}

template <int INTEG>
__global__ void __launch_bounds__(THREADS, 1) sampler_pair_kernel(Params P) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw_addr & 1023u)) & 1023u;
  unsigned char *sm = smem_raw + pad;
  const uint32_t sbase = raw_addr + pad;
  Bars &B = *reinterpret_cast<Bars *>(sm + S_BAR);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank(), other = rank ^ 1u;
  const bool even = rank == 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&B.full[s], even ? 2 : 1);
      mbar_init(&B.empty[s], 1);
    }
    mbar_init(&B.res_full, 1);
    mbar_init(&B.res_peer, 1);
    for (int t = 0; t < 2; ++t) {
      mbar_init(&B.ar[t], 2 * EPI_WARPS);
      mbar_init(&B.dfull[t], 1);
    }
    mbar_init(&B.drain, 1);
    B.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(&B.tmem_base, TMEM_COLS);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_barrier();  // the other CTA's barriers exist before any remote arrival
  tc_fence_after();
  const uint32_t tmem = B.tmem_base;
  volatile int *abort = &B.abort;

  const int64_t ntiles = (P.n + 2 * PM - 1) / (2 * PM);
  const int64_t npairs = (ntiles + 1) / 2;
  const int64_t cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  // tile pairs cl, cl + ncl, ... (ncl <= npairs); both CTAs count alike
  const int64_t n_iter = (npairs - cl + ncl - 1) / ncl;
  const float h = 1.0f / (float)P.steps;

  if (warp == 0) {
    // ---------------- weight producer (this CTA's halves) ----------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      mbar_arrive_expect_tx(&B.res_full, 4096 + 4096 + 12288);
      bulk_g2s(sm + S_B1, P.packed + PK::OFF_B1 + rank * 4096u, 4096, &B.res_full);
      for (int j = 0; j < 4; ++j)
        bulk_g2s(sm + S_B5 + j * 1024, P.packed + PK::OFF_B5 + j * 2048 + rank * 1024u, 1024,
                 &B.res_full);
      for (int L = 0; L < 3; ++L)
        bulk_g2s(sm + S_BIAS + L * 4096, P.packed + PK::OFF_BIAS + L * 8192 + rank * 4096u, 4096,
                 &B.res_full);
      for (int64_t ip = 0; ip < n_iter && ok; ++ip)
        for (int e = 0; e < P.n_eval && ok; ++e)
          for (int L = 0; L < 3 && ok; ++L)
            for (int T = 0; T < 2 && ok; ++T)
              for (int ch = 0; ch < NCH; ++ch) {
                const int s = it % NST;
                const uint32_t round = it / NST;
                if (!mbar_wait_cluster(&B.empty[s], (round & 1u) ^ 1u, abort)) {
                  fail(B, P.err, 11, other);
                  ok = false;
                  break;
                }
                // the odd CTA's half of stage s is free once the MMA that read
                // the even CTA's half has completed: relay it
                if (even && round > 0) mbar_arrive_remote(peer_smem(&B.empty[s], 1));
                mbar_arrive_expect_tx(&B.full[s], HCHUNK);
                bulk_g2s(sm + S_ST + s * HCHUNK,
                         P.packed + PK::OFF_HID + (size_t)(L * NCH + ch) * CHUNK + rank * HCHUNK,
                         HCHUNK, &B.full[s]);
                ++it;
              }
      if (!ok) {
        // every issued copy lands before the CTA exits
        int never = 0;
        for (uint32_t k = (it > NST ? it - NST : 0); k < it; ++k)
          mbar_wait_cluster(&B.full[k % NST], (k / NST) & 1u, &never, 1000000000ull);
        mbar_wait(&B.res_full, 0, &never, 1000000000ull);
      }
    }
  } else if (warp == 1 && !even) {
    // ---------------- relay of the odd CTA's copies ----------------
    if (lane == 0) {
      bool ok = mbar_wait(&B.res_full, 0, abort);
      if (ok) mbar_arrive_remote(peer_smem(&B.res_peer, 0));
      else fail(B, P.err, 12, other);
      uint32_t it = 0;
      for (int64_t ip = 0; ip < n_iter && ok; ++ip)
        for (int e = 0; e < P.n_eval && ok; ++e)
          for (int L = 0; L < 3 && ok; ++L)
            for (int T = 0; T < 2 && ok; ++T)
              for (int ch = 0; ch < NCH; ++ch) {
                const int s = it % NST;
                if (!mbar_wait(&B.full[s], (it / NST) & 1u, abort)) {
                  fail(B, P.err, 13, other);
                  ok = false;
                  break;
                }
                mbar_arrive_remote(peer_smem(&B.full[s], 0));
                ++it;
              }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (even CTA) ----------------
    // warp-uniform loop; one elected lane issues each instruction
    auto wwait = [&](uint64_t *bar, uint32_t parity) {
      const bool r = mbar_try_wait_cluster(bar, parity) || mbar_wait_cluster(bar, parity, abort);
      return __all_sync(0xffffffffu, r);
    };
    bool ok = wwait(&B.res_full, 0) && wwait(&B.res_peer, 0);
    if (!ok && lane == 0) fail(B, P.err, 14, other);
    uint32_t aph[2] = {0, 0};
    uint32_t stage = 0, sph = 0;
    const uint32_t idn = idesc_bf16(256, 256), id16 = idesc_bf16(256, 16);
    const uint64_t dA1[2] = {smem_desc(sbase + S_A1, 256, kSwizzle32B),
                             smem_desc(sbase + S_A1 + 4096, 256, kSwizzle32B)};
    const uint64_t dA[2] = {smem_desc(sbase + S_A, 1024, kSwizzle128B),
                            smem_desc(sbase + S_A + A_BYTES, 1024, kSwizzle128B)};
    const uint64_t dB1 = smem_desc(sbase + S_B1, 256, kSwizzle32B);
    const uint64_t dB5 = smem_desc(sbase + S_B5, 1024, kSwizzle128B);
    const uint64_t dBias = smem_desc(sbase + S_BIAS, 256, kSwizzle32B);
    const uint64_t dST = smem_desc(sbase + S_ST, 1024, kSwizzle128B);
    for (int64_t ip = 0; ip < n_iter && ok; ++ip)
      for (int e = 0; e < P.n_eval && ok; ++e)
        for (int L = 0; L < 5 && ok; ++L)
          for (int T = 0; T < 2 && ok; ++T) {
            // tile T's operand for this layer written by every epilogue warp
            // of both CTAs (which also means its accumulator has been read)
            if (!wwait(&B.ar[T], aph[T] & 1u)) {
              if (lane == 0) fail(B, P.err, 15, other);
              ok = false;
              break;
            }
            ++aph[T];
            tc_fence_after();
            const uint32_t d = tmem + 256u * (uint32_t)T;
            if (L == 0) {
              mma_pair_f16_w(d, dA1[T], dB1, idn, 0);
            } else if (L < 4) {
              mma_pair_f16_w(d, dA1[T], dBias + (uint64_t)((L - 1) * (4096 >> 4)), idn, 0);
#pragma unroll
              for (int ch = 0; ch < NCH; ++ch) {
                if (!wwait(&B.full[stage], sph)) {
                  if (lane == 0) fail(B, P.err, 16, other);
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint64_t b_ch = dST + (uint64_t)(stage * (HCHUNK >> 4));
                const uint64_t a_ch = dA[T] + (uint64_t)(ch * (KB_BYTES >> 4));
#pragma unroll
                for (int k = 0; k < 4; ++k)
                  mma_pair_f16_w(d, a_ch + (uint64_t)(2 * k), b_ch + (uint64_t)(2 * k), idn, 1);
                mma_pair_commit_w(&B.empty[stage]);
                if (++stage == NST) {
                  stage = 0;
                  sph ^= 1u;
                }
              }
              if (!ok) break;
            } else {
              // velocity: K = 256 = 16 MMAs of K = 16; B5 in four 1 KB K-blocks
#pragma unroll
              for (int j = 0; j < 16; ++j)
                mma_pair_f16_w(d, dA[T] + (uint64_t)((j >> 2) * (KB_BYTES >> 4) + (j & 3) * 2),
                               dB5 + (uint64_t)((j >> 2) * (1024 >> 4) + (j & 3) * 2), id16, j != 0);
            }
            mma_pair_commit_w(&B.dfull[T]);
          }
    // all issued MMAs complete before tensor memory is released
    mma_pair_commit_w(&B.drain);
    int never = 0;
    mbar_wait(&B.drain, 0, &never, 1000000000ull);
  } else {
    // ---------------- epilogue (both CTAs) ----------------
    const int ew = warp - 2;
    const int p = ew >> 2;          // accumulator columns 64 p .. 64 p + 63
    const int q = warp & 3;         // tensor-memory lane quadrant
    const int r = 32 * q + lane;    // row of this CTA's half tile
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const int own = p < 2 ? p : -1;  // tile whose ODE state this warp keeps
    float x[4], xm[4], ka[4];
    uint32_t dph[2] = {0, 0};
    bool ok = true;
    auto wait_d = [&](int T) {
      if (!mbar_wait_cluster(&B.dfull[T], dph[T] & 1u, abort)) {
        fail(B, P.err, 17, other);
        return false;
      }
      ++dph[T];
      // the odd CTA learns of the accumulator from the even CTA
      if (even && ew == 0 && lane == 0) mbar_arrive_remote(peer_smem(&B.dfull[T], 1));
      tc_fence_after();
      return true;
    };
    for (int64_t ip = 0; ip < n_iter && ok; ++ip) {
      const int64_t pr = cl + ip * ncl;
#pragma unroll
      for (int T = 0; T < 2; ++T) {
        if (own == T) {
          const int64_t gi = (2 * pr + T) * (2 * PM) + (int64_t)rank * PM + r;
          const bool valid = gi < P.n;
          float cn[kCondRect];
          load_cond(P.cond, P.st, P.n, gi, valid, cn);
          if (!valid) {
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) x[dd] = 0.0f;
          } else if (P.noise) {
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) x[dd] = P.noise[dd * P.n + gi];
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
        if (lane == 0) arrive_even(&B.ar[T], even);
      }
      for (int e = 0; e < P.n_eval && ok; ++e) {
        for (int L = 0; L < 4 && ok; ++L)
#pragma unroll
          for (int T = 0; T < 2; ++T) {
            if (!wait_d(T)) {
              ok = false;
              break;
            }
            // SiLU of the 64 columns -> K-block p of the tile's next operand,
            // in two halves of 32 columns (each: one tensor-memory load, then
            // four 16-byte stores of 8 BF16)
            const uint32_t d_col = tmem + lane_off + 256u * (uint32_t)T + (uint32_t)(64 * p);
            const float *bias = P.bias1 + (size_t)e * 256;
            const uint32_t kb = sbase + S_A + (uint32_t)T * A_BYTES + (uint32_t)p * KB_BYTES;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              uint32_t va[32];
              tmem_ld32_raw(d_col + 32u * (uint32_t)half, va);
              tmem_wait_ld_regs(va);
#pragma unroll
              for (int i = 0; i < 2; ++i) {
                uint32_t w[8];
                const int col0 = 64 * p + 32 * half + 16 * i;
                if (L == 0) silu16<kPreBias, false>(va + 16 * i, bias, nullptr, col0, w);
                else silu16<kPreNone, false>(va + 16 * i, bias, nullptr, col0, w);
                const int c = 4 * half + 2 * i;  // 16-byte chunk of the 128-byte row
                st_shared_v4(sw128(kb, r, c), w[0], w[1], w[2], w[3]);
                st_shared_v4(sw128(kb, r, c + 1), w[4], w[5], w[6], w[7]);
              }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) arrive_even(&B.ar[T], even);
          }
        if (!ok) break;
        const bool last = e == P.n_eval - 1;
#pragma unroll
        for (int T = 0; T < 2; ++T) {
          // the velocity of tile T: columns 0-3, read by the warps keeping T's state
          if (!wait_d(T)) {
            ok = false;
            break;
          }
          const bool mine = own == T;
          float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          if (mine) {
            tmem_ld4(tmem + lane_off + 256u * (uint32_t)T, v);
            tmem_wait_ld_regs4(v);
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) v[dd] += __ldg(P.bias + 4 * 256 + dd);
            float *xin = x;
            if (INTEG == GMC_MIDPOINT && (e & 1) == 0) {
#pragma unroll
              for (int dd = 0; dd < 4; ++dd) xm[dd] = fmaf(0.5f * h, v[dd], x[dd]);
              xin = xm;
            } else if (INTEG == GMC_RK4) {
              // evaluation e % 4 = i gives k_{i+1}; ka = k1 + 2 k2 + 2 k3 + k4
              const int i = e & 3;
              if (i == 3) {
#pragma unroll
                for (int dd = 0; dd < 4; ++dd) x[dd] = fmaf(h * (1.0f / 6.0f), ka[dd] + v[dd], x[dd]);
              } else {
                const float wgt = i == 0 ? 1.0f : 2.0f, hs = i == 2 ? h : 0.5f * h;
#pragma unroll
                for (int dd = 0; dd < 4; ++dd) {
                  ka[dd] = i == 0 ? v[dd] : fmaf(wgt, v[dd], ka[dd]);
                  xm[dd] = fmaf(hs, v[dd], x[dd]);
                }
                xin = xm;
              }
            } else {
#pragma unroll
              for (int dd = 0; dd < 4; ++dd) x[dd] = fmaf(h, v[dd], x[dd]);
            }
            if (!last) {
              float xi[4] = {xin[0], xin[1], xin[2], xin[3]};
              write_a1_x(sbase + S_A1 + (uint32_t)T * 4096u, r, xi);
              fence_proxy_async_smem();
            }
          }
          tc_fence_before();
          __syncwarp();
          if (!last && lane == 0) arrive_even(&B.ar[T], even);
          if (last && mine) {
            const int64_t gi = (2 * pr + T) * (2 * PM) + (int64_t)rank * PM + r;
            if (gi < P.n) {
              if (P.y_raw) {
#pragma unroll
                for (int dd = 0; dd < 4; ++dd) P.y_raw[dd * P.n + gi] = x[dd];
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
  cluster_barrier();  // no MMA, copy or remote arrival touches this CTA after this point
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc_pair(tmem, TMEM_COLS);
  }
}

template <int INTEG>
cudaError_t launch_pair(cudaStream_t stream, const Params &p, int sms) {
  auto kernel = sampler_pair_kernel<INTEG>;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.n + 2 * PM - 1) / (2 * PM), npairs = (ntiles + 1) / 2;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  lc.blockDim = dim3(THREADS);
  lc.dynamicSmemBytes = SMEM_BYTES;
  lc.stream = stream;
  // a persistent grid of clusters that are resident at once (queried once
  // per device), never more clusters than tile pairs
  static std::atomic<int> cached[kMaxDevices];
  int dev = 0;
  cudaGetDevice(&dev);
  int fit = (dev >= 0 && dev < kMaxDevices) ? cached[dev].load(std::memory_order_relaxed) : 0;
  if (fit < 1) {
    lc.gridDim = dim3((unsigned)(sms / 2 * 2));
    int mc = 0;
    if (cudaOccupancyMaxActiveClusters(&mc, kernel, &lc) != cudaSuccess || mc < 1) {
      cudaGetLastError();
      mc = sms / 2;
    }
    fit = mc;
    if (dev >= 0 && dev < kMaxDevices) cached[dev].store(fit, std::memory_order_relaxed);
  }
  const int64_t clusters = npairs < fit ? npairs : fit;
  lc.gridDim = dim3((unsigned)(2 * clusters));
  e = cudaLaunchKernelEx(&lc, kernel, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sampler_pair(cudaStream_t stream, const Params &p, int sms) {
  if (p.integrator == GMC_RK4) return launch_pair<GMC_RK4>(stream, p, sms);
  if (p.integrator == GMC_MIDPOINT) return launch_pair<GMC_MIDPOINT>(stream, p, sms);
  return launch_pair<GMC_EULER>(stream, p, sms);
}

}  // namespace gmc
