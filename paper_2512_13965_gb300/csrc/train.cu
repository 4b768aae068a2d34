// Training of the velocity network by conditional flow matching (Eq. 9) on
// transmissions generated by the GPU random walk.
//
//  gmc_train_data   a11: tau log-uniform, c uniform, xi uniform, sin(theta)
//                   uniform (Philox tag 5, one block per sample), then the
//                   implicit-capture walk (flights at rate c) from the left
//                   face -> targets y = (p, cos theta_out, sin theta_out, ln s).
//  gmc_train_begin  standardization statistics of the data (FP64 sums), FP32
//                   master weights copied from the loaded network, AdamW state.
//  gmc_train_steps  a12 + a13 per step: batch rows drawn with Philox (tag 6):
//                   sample index, t ~ U(0,1], x0 ~ N(0, I); x_t = (1-t) x0 + t x1,
//                   target x1 - x0; forward through the MLP keeping
//                   pre-activations; loss = mean_b ||v - (x1 - x0)||^2;
//                   hand-derived backward; AdamW (decoupled weight decay).
//
// The dense layers run either on tcgen05 tensor cores with BF16 operands
// (train_fused.cu; the default of the command-line trainer) or on a tiled
// FP32 SIMT GEMM with fused epilogues (bias + SiLU forward, SiLU' backward),
// both with FP32 accumulation; master weights and AdamW moments are FP32.
// The residual-modulated network (a loaded network with weight-file flag 1)
// trains on the FP32 path: its blocks' epilogue adds the condition shift,
// applies the channel scale and the residual, and the reverse pass carries
// the block gradient through the residual path (fwd_bwd_rm).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "ckpt.h"
#include "decode.cuh"
#include "gmc_internal.cuh"
#include "host_rules.h"
#include "philox.cuh"
#include "train_fused.h"
#include "walk.cuh"

namespace gmc {

constexpr uint32_t kTagData = 5u, kTagDataInternal = 7u, kTagDataXY = 8u,
                   kTagDataInternalXY = 9u, kTagDataRect = 10u;  // kTagTrain: train_fused.h

struct TrainState {
  int64_t n = 0;
  const float *cond = nullptr, *y = nullptr;
  // standardization: cond mean [ncond], cond sd [ncond], y mean [4], y sd [4]
  float stats[20];
  gmc_train_config cfg{};
  bool rm = false;         // residual-modulated network
  int ncond = 5;           // condition components (6: a network of rectangular cells)
  int64_t np = P_TOTAL;    // parameters (P_TOTAL_RM with rm)
  int64_t step = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  int64_t B = 0;
  float *X0 = nullptr, *U = nullptr, *Z[4] = {}, *A[4] = {}, *V = nullptr, *dZ[2] = {},
        *dV = nullptr;
  double *loss = nullptr;  // [max steps per call]
  int64_t loss_cap = 0;
  double *stat_acc = nullptr;  // sums and sums of squares of the ncond + 4 features
  float *colpart = nullptr;    // partial column sums of the bias gradients (FP32 path)
  float *ws = nullptr;         // K-split partial products of the weight gradients (FP32 path)
  tf::Bufs fb;                 // operand images of the BF16 tensor-core step
  int *err = nullptr;          // device error word of the context
};

namespace {

__global__ void data_kernel(int64_t n, uint64_t seed, float ltau_lo, float ltau_hi, float c_lo,
                            float c_hi, float *__restrict__ cond, float *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox_draw(seed, (uint64_t)i, 0u, kTagData);
  const float ltau = ltau_lo + (ltau_hi - ltau_lo) * u01(r.x);
  const float tau = expf(ltau);
  const float c = c_lo + (c_hi - c_lo) * u01(r.y);
  const float xi = u01(r.z);
  const float sn = fmaf(2.0f, u01(r.w), -1.0f);
  const float cs = sqrtf(fmaxf(1.0f - sn * sn, 0.0f));
  const WalkResult w = walk_cell(tau, c, 1, 0.0f, xi, cs, sn, seed, (uint64_t)i, 1u);
  cond[i] = xi;
  cond[n + i] = cs;
  cond[2 * n + i] = sn;
  cond[3 * n + i] = ltau;
  cond[4 * n + i] = c;
  y[i] = (float)(w.face < 0 ? 0 : w.face) + w.q;
  y[n + i] = w.ux;
  y[2 * n + i] = w.uy;
  y[3 * n + i] = logf(fmaxf(w.s, kSMin));
}

// Training data of the internal (volumetric-source) model: a birth at a
// uniform point (X, Y) of the cell with an isotropic direction, walked with
// implicit capture to its exit. Philox block (i, 0, tag 7): ln tau, c, X, Y;
// (i, 1, tag 7): the direction; the walk draws from event 2 on.
// cond = (X, Y, ln tau, c, min(X, Y, 1 - X, 1 - Y)); y = (p, ux, uy, ln s)
// in the cell's own frame (p counter-clockwise from corner (0, 0)).
__global__ void internal_data_kernel(int64_t n, uint64_t seed, float ltau_lo, float ltau_hi,
                                     float c_lo, float c_hi, float *__restrict__ cond,
                                     float *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox_draw(seed, (uint64_t)i, 0u, kTagDataInternal);
  const float ltau = ltau_lo + (ltau_hi - ltau_lo) * u01(r.x);
  const float tau = expf(ltau);
  const float c = c_lo + (c_hi - c_lo) * u01(r.y);
  const float X = u01(r.z), Y = u01(r.w);
  float ux, uy;
  sincospif(2.0f * u01(philox_draw(seed, (uint64_t)i, 1u, kTagDataInternal).x), &uy, &ux);
  const WalkResult w = walk_cell(tau, c, 1, X, Y, ux, uy, seed, (uint64_t)i, 2u);
  cond[i] = X;
  cond[n + i] = Y;
  cond[2 * n + i] = ltau;
  cond[3 * n + i] = c;
  cond[4 * n + i] = fminf(fminf(X, Y), fminf(1.0f - X, 1.0f - Y));
  y[i] = (float)(w.face < 0 ? 0 : w.face) + w.q;
  y[n + i] = w.ux;
  y[2 * n + i] = w.uy;
  y[3 * n + i] = logf(fmaxf(w.s, kSMin));
}

// Training data of the boundary model for rectangular cells: Philox block
// (i, 0, tag 10) gives ln tau_x uniform in [ln tau_lo, ln tau_hi], c uniform,
// xi uniform and sin theta = 2 u - 1 (the cosine-law entry of the square
// data); (i, 1, tag 10) the aspect, ln(tau_y / tau_x) uniform in
// [ln a_lo, ln a_hi]. The implicit-capture walk in the cell [0, tau_x] x
// [0, tau_y] runs from (0, xi tau_y), flights from event 2 (FP64 positions
// when a side exceeds kTau64). cond = (xi, cos, sin, ln tau_x, c,
// ln(tau_y / tau_x)); y = (p, ux, uy, ln s), q normalized per face.
__global__ void rect_data_kernel(int64_t n, uint64_t seed, float ltau_lo, float ltau_hi,
                                 float la_lo, float la_hi, float c_lo, float c_hi,
                                 float *__restrict__ cond, float *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox_draw(seed, (uint64_t)i, 0u, kTagDataRect);
  const float ltau = ltau_lo + (ltau_hi - ltau_lo) * u01(r.x);
  const float c = c_lo + (c_hi - c_lo) * u01(r.y);
  const float xi = u01(r.z);
  const float sn = 2.0f * u01(r.w) - 1.0f;
  const float cs = sqrtf(fmaxf(1.0f - sn * sn, 0.0f));
  const float la = la_lo + (la_hi - la_lo) * u01(philox_draw(seed, (uint64_t)i, 1u, kTagDataRect).x);
  const float tx = expf(ltau), ty = expf(ltau + la);
  const WalkResult w =
      fmaxf(tx, ty) > kTau64
          ? walk_rect<double>((double)tx, (double)ty, c, 1, 0.0, (double)xi * ty, cs, sn, seed,
                              (uint64_t)i, 2u)
          : walk_rect<float>(tx, ty, c, 1, 0.0f, xi * ty, cs, sn, seed, (uint64_t)i, 2u);
  cond[i] = xi;
  cond[n + i] = cs;
  cond[2 * n + i] = sn;
  cond[3 * n + i] = ltau;
  cond[4 * n + i] = c;
  cond[5 * n + i] = la;
  y[i] = (float)(w.face < 0 ? 0 : w.face) + w.q;
  y[n + i] = w.ux;
  y[2 * n + i] = w.uy;
  y[3 * n + i] = logf(fmaxf(w.s, kSMin));
}

// Training data of the internal model in x-y geometry (a birth inside the
// cross-section of an infinite prism, 3-D isotropic direction): Philox block
// (i, 0, tag 9) gives ln tau, c, X, Y as internal_data_kernel; (i, 1, tag 9)
// the direction, azimuth 2 pi u0 and polar cosine 2 u1 - 1, projected on the
// plane. The implicit-capture walk with scattering on the sphere runs from
// event 2 (FP64 positions in cells thicker than kTau64). cond = (X, Y,
// ln tau, c, min(X, Y, 1 - X, 1 - Y)); y = (p, ux, uy, ln s) in the cell's own
// frame, s the 3-D track length.
__global__ void internal_xy_data_kernel(int64_t n, uint64_t seed, float ltau_lo, float ltau_hi,
                                        float c_lo, float c_hi, float *__restrict__ cond,
                                        float *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox_draw(seed, (uint64_t)i, 0u, kTagDataInternalXY);
  const float ltau = ltau_lo + (ltau_hi - ltau_lo) * u01(r.x);
  const float tau = expf(ltau);
  const float c = c_lo + (c_hi - c_lo) * u01(r.y);
  const float X = u01(r.z), Y = u01(r.w);
  const uint4 r1 = philox_draw(seed, (uint64_t)i, 1u, kTagDataInternalXY);
  float sp, cp;
  sincospif(2.0f * u01(r1.x), &sp, &cp);
  const float mu = 2.0f * u01(r1.y) - 1.0f;
  const float rr = sqrtf(fmaxf(1.0f - mu * mu, 0.0f));
  const float ux = rr * cp, uy = rr * sp;
  const WalkResult w =
      tau > kTau64 ? walk_xy<double>((double)tau, (double)tau, c, 1, (double)X * tau,
                                     (double)Y * tau, ux, uy, seed, (uint64_t)i, 2u)
                   : walk_xy<float>(tau, tau, c, 1, X * tau, Y * tau, ux, uy, seed, (uint64_t)i, 2u);
  cond[i] = X;
  cond[n + i] = Y;
  cond[2 * n + i] = ltau;
  cond[3 * n + i] = c;
  cond[4 * n + i] = fminf(fminf(X, Y), fminf(1.0f - X, 1.0f - Y));
  y[i] = (float)(w.face < 0 ? 0 : w.face) + w.q;
  y[n + i] = w.ux;
  y[2 * n + i] = w.uy;
  y[3 * n + i] = logf(fmaxf(w.s, kSMin));
}

// Training data of the boundary model in x-y geometry (the cell is the
// cross-section of an infinite prism; directions are 3-D and enter the
// network as their projection on the unit disk): Philox block (i, 0, tag 8)
// gives ln tau, c, xi and mu = sqrt(u), the cosine of the entry direction to
// the face normal (the cosine-law inflow of an isotropic flux); (i, 1, tag 8)
// its azimuth 2 pi u about the normal, so the projection is (mu, sqrt(1 -
// mu^2) cos phi). The implicit-capture walk with scattering on the sphere
// runs from event 2 (FP64 positions in cells thicker than kTau64).
// cond = (xi, ux, uy, ln tau, c); y = (p, ux_out, uy_out, ln s), s the 3-D
// track length.
__global__ void xy_data_kernel(int64_t n, uint64_t seed, float ltau_lo, float ltau_hi, float c_lo,
                               float c_hi, float *__restrict__ cond, float *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox_draw(seed, (uint64_t)i, 0u, kTagDataXY);
  const float ltau = ltau_lo + (ltau_hi - ltau_lo) * u01(r.x);
  const float tau = expf(ltau);
  const float c = c_lo + (c_hi - c_lo) * u01(r.y);
  const float xi = u01(r.z);
  const float mu = sqrtf(u01(r.w));
  float sp, cp;
  sincospif(2.0f * u01(philox_draw(seed, (uint64_t)i, 1u, kTagDataXY).x), &sp, &cp);
  const float ux = mu, uy = sqrtf(fmaxf(1.0f - mu * mu, 0.0f)) * cp;
  const WalkResult w =
      tau > kTau64 ? walk_xy<double>((double)tau, (double)tau, c, 1, 0.0, (double)xi * tau, ux, uy,
                                     seed, (uint64_t)i, 2u)
                   : walk_xy<float>(tau, tau, c, 1, 0.0f, xi * tau, ux, uy, seed, (uint64_t)i, 2u);
  cond[i] = xi;
  cond[n + i] = ux;
  cond[2 * n + i] = uy;
  cond[3 * n + i] = ltau;
  cond[4 * n + i] = c;
  y[i] = (float)(w.face < 0 ? 0 : w.face) + w.q;
  y[n + i] = w.ux;
  y[2 * n + i] = w.uy;
  y[3 * n + i] = logf(fmaxf(w.s, kSMin));
}

// sums and sums of squares of the nc + 4 features (FP64): acc[k] and
// acc[nf + k], nf = nc + 4 (nc = 5, or 6 for rectangular cells)
__global__ void stats_kernel(int64_t n, int nc, const float *__restrict__ cond,
                             const float *__restrict__ y, double *acc) {
  constexpr int kMaxF = 10;
  const int nf = nc + 4;
  __shared__ double sh[2 * kMaxF];
  if (threadIdx.x < 2 * kMaxF) sh[threadIdx.x] = 0.0;
  __syncthreads();
  double loc[2 * kMaxF];
  for (int k = 0; k < 2 * kMaxF; ++k) loc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < nf; ++k) {
      const double v = k < nc ? cond[k * n + i] : y[(k - nc) * n + i];
      loc[k] += v;
      loc[nf + k] += v * v;
    }
  }
  for (int k = 0; k < 2 * nf; ++k) {
    double v = loc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sh[k], v);
  }
  __syncthreads();
  if (threadIdx.x < 2 * nf) atomicAdd(&acc[threadIdx.x], sh[threadIdx.x]);
}

// One batch row: sample index, t, x0 -> X0 row [cn, x_t, emb(t), aspect, 0...]
// (the aspect, column 25, for a network of rectangular cells: nc = 6), U row.
__global__ void batch_kernel(int64_t B, int64_t n, int nc, const float *__restrict__ cond,
                             const float *__restrict__ y, Std sd, uint64_t seed, int64_t step,
                             float *__restrict__ X0, float *__restrict__ U) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const uint64_t rid = (uint64_t)step * (uint64_t)B + (uint64_t)b;
  const uint4 r = philox_draw(seed, rid, 0u, kTagTrain);
  const int64_t idx = (int64_t)(((uint64_t)r.x * (uint64_t)n) >> 32);
  const float t = u01(r.y);
  const float4 z = box_muller4(philox_draw(seed, rid, 1u, kTagTrain));
  const float x0[4] = {z.x, z.y, z.z, z.w};
  float *row = X0 + b * 32;
  for (int k = 0; k < 5; ++k) row[k] = (cond[k * n + idx] - sd.cm[k]) * sd.cis[k];
  for (int d = 0; d < 4; ++d) {
    const float x1 = (y[d * n + idx] - sd.ym[d]) * sd.yis[d];
    row[5 + d] = (1.0f - t) * x0[d] + t * x1;
    U[b * 4 + d] = x1 - x0[d];
  }
  for (int j = 0; j < 16; ++j) row[9 + j] = time_embedding(j, t);
  row[25] = nc > 5 ? (cond[5 * n + idx] - sd.cm[5]) * sd.cis[5] : 0.0f;
  for (int k = 26; k < 32; ++k) row[k] = 0.0f;
}

// Batch rows from explicit inputs (gradient check): cn [B][nc], x1, x0 [B][4], t [B].
__global__ void batch_explicit_kernel(int64_t B, int nc, const float *cn, const float *x1,
                                      const float *x0, const float *tt, float *X0, float *U) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float t = tt[b];
  float *row = X0 + b * 32;
  for (int k = 0; k < 5; ++k) row[k] = cn[b * nc + k];
  for (int d = 0; d < 4; ++d) {
    row[5 + d] = (1.0f - t) * x0[b * 4 + d] + t * x1[b * 4 + d];
    U[b * 4 + d] = x1[b * 4 + d] - x0[b * 4 + d];
  }
  for (int j = 0; j < 16; ++j) row[9 + j] = time_embedding(j, t);
  row[25] = nc > 5 ? cn[b * nc + 5] : 0.0f;
  for (int k = 26; k < 32; ++k) row[k] = 0.0f;
}

enum Epi { kEpiStore = 0, kEpiBiasSilu = 1, kEpiBias = 2, kEpiDSilu = 3, kEpiRM = 4, kEpiAdd = 5 };

// Extra operands of a residual-modulated block's forward epilogue: M [256][5],
// G [2][256] and the batch rows X0 (standardized condition in columns 0..4).
struct RMArgs {
  const float *M = nullptr, *G = nullptr, *X0 = nullptr;
};

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

// C[M][N] = sum_k A(m,k) B(k,n), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].
// 64x64 tile, 256 threads, 4x4 outputs per thread, K in slices of 16.
template <int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *__restrict__ A,
                                                   int64_t sam, int64_t sak,
                                                   const float *__restrict__ Bm, int64_t sbk,
                                                   int64_t sbn, float *__restrict__ C,
                                                   const float *__restrict__ bias,
                                                   float *__restrict__ C2,
                                                   const float *__restrict__ Zp, RMArgs rm,
                                                   int kslice) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  // K split over blockIdx.z (kEpiStore only): slice z covers [z kslice,
  // (z + 1) kslice) and writes its partial product to C + z M N
  const int kb = blockIdx.z * kslice;
  const int ke = K < kb + kslice ? K : kb + kslice;
  if (EPI == kEpiStore) C += (int64_t)blockIdx.z * M * N;
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e & 15, mm = e >> 4;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < ke) ? A[gm * sam + gk * sak] : 0.0f;
      const int nn = e & 63, kr = e >> 6;
      const int gn = n0 + nn, gk2 = k0 + kr;
      Bs[kr][nn] = (gn < N && gk2 < ke) ? Bm[gk2 * sbk + gn * sbn] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = n0 + tx + 16 * j;
      if (nn >= N) continue;
      float v = acc[i][j];
      const int64_t o = (int64_t)m * N + nn;
      if (EPI == kEpiBiasSilu) {
        v += bias[nn];
        C[o] = v;                       // pre-activation z (kept for backward)
        C2[o] = v * sigmoidf_(v);       // SiLU(z)
      } else if (EPI == kEpiBias) {
        C[o] = v + bias[nn];
      } else if (EPI == kEpiDSilu) {
        const float z = Zp[o], s = sigmoidf_(z);
        C[o] = v * (s * (1.0f + z * (1.0f - s)));
      } else if (EPI == kEpiRM) {
        // z = acc + b + M c; output a_prev + SiLU(g z), g = 1 + G0 c_3 + G1 c_4
        const float *cn = rm.X0 + (int64_t)m * 32;
        float z = v + bias[nn];
#pragma unroll
        for (int k = 0; k < 5; ++k) z = fmaf(rm.M[nn * 5 + k], cn[k], z);
        const float g = fmaf(rm.G[nn], cn[3], fmaf(rm.G[256 + nn], cn[4], 1.0f));
        const float pz = g * z;
        C[o] = z;
        C2[o] = Zp[o] + pz * sigmoidf_(pz);
      } else if (EPI == kEpiAdd) {
        C[o] += v;
      } else {
        C[o] = v;
      }
    }
  }
}

template <int EPI>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const float *A, int64_t sam, int64_t sak,
                 const float *B, int64_t sbk, int64_t sbn, float *C, const float *bias = nullptr,
                 float *C2 = nullptr, const float *Zp = nullptr, RMArgs rm = RMArgs()) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  gemm_kernel<EPI><<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, bias, C2, Zp, rm, K);
  return cudaGetLastError();
}

// out[i] = sum_z part[z][i], z in order (deterministic)
__global__ void ksum_kernel(int64_t mn, int S, const float *__restrict__ part, float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mn) return;
  float t = 0.0f;
  for (int z = 0; z < S; ++z) t += part[z * mn + i];
  out[i] = t;
}

constexpr int kMaxKSplit = 16;
constexpr int64_t kKSplitWs = (int64_t)kMaxKSplit * 256 * 256;  // workspace floats

// C = A B for a weight gradient (K = the batch): the few output tiles of a
// 256 x 256 product would occupy 16 SMs, so K is split into up to 16 slices
// of at least 1024 rows, each slice's partial product goes to ws, and one
// pass adds the slices in a fixed order.
cudaError_t gemm_wgrad(cudaStream_t s, int M, int N, int K, const float *A, int64_t sam, int64_t sak,
                       const float *B, int64_t sbk, int64_t sbn, float *C, float *ws) {
  int S = K / 1024;
  if (S > kMaxKSplit) S = kMaxKSplit;
  if (S < 2 || (int64_t)S * M * N > kKSplitWs) return gemm<kEpiStore>(s, M, N, K, A, sam, sak, B, sbk, sbn, C);
  const int kslice = ((K + S - 1) / S + 15) / 16 * 16;
  S = (K + kslice - 1) / kslice;
  dim3 grid((N + 63) / 64, (M + 63) / 64, S);
  gemm_kernel<kEpiStore><<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, ws, nullptr, nullptr,
                                              nullptr, RMArgs(), kslice);
  const int64_t mn = (int64_t)M * N;
  ksum_kernel<<<(unsigned)((mn + 255) / 256), 256, 0, s>>>(mn, S, ws, C);
  return cudaGetLastError();
}

// loss and dV = 2 (v - u) / B
__global__ void loss_kernel(int64_t B, const float *__restrict__ V, const float *__restrict__ U,
                            float *__restrict__ dV, double *loss) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double part = 0.0;
  if (b < B) {
    for (int d = 0; d < 4; ++d) {
      const float r = V[b * 4 + d] - U[b * 4 + d];
      part += (double)r * r;
      dV[b * 4 + d] = 2.0f * r / (float)B;
    }
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(loss, part / (double)B);
}

// db[n] = sum_b dZ[b][n] in two passes: blocks of kColRows rows give partial
// sums (grid: column groups of 32 x row blocks), then one thread per column
// adds the partials in block order (a fixed order: deterministic).
constexpr int kColRows = 128;

__global__ void colsum_partial_kernel(int64_t B, int N, const float *__restrict__ dZ,
                                      float *__restrict__ partial) {
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;  // 8 row groups
  const int n = blockIdx.x * 32 + lane;
  const int64_t b0 = (int64_t)blockIdx.y * kColRows;
  const int64_t b1 = b0 + kColRows < B ? b0 + kColRows : B;
  float acc = 0.0f;
  if (n < N)
    for (int64_t b = b0 + rg; b < b1; b += 8) acc += dZ[b * N + n];
  __shared__ float sh[8][33];
  sh[rg][lane] = acc;
  __syncthreads();
  if (rg == 0 && n < N) {
    float t = 0.0f;
    for (int r = 0; r < 8; ++r) t += sh[r][lane];
    partial[(int64_t)blockIdx.y * N + n] = t;
  }
}

// One warp per column: lane l adds partials l, l + 32, ..., then a fixed
// shuffle tree combines the lanes (the same order on every run).
__global__ void colsum_final_kernel(int P, int N, const float *__restrict__ partial,
                                    float *__restrict__ db) {
  const int n = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (n >= N) return;  // whole warps leave together
  float t = 0.0f;
  for (int p = lane; p < P; p += 32) t += partial[(int64_t)p * N + n];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) db[n] = t;
}

cudaError_t colsum(cudaStream_t s, int64_t B, int N, const float *dZ, float *partial, float *db) {
  const int P = (int)((B + kColRows - 1) / kColRows);
  colsum_partial_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)P), 256, 0, s>>>(B, N, dZ, partial);
  colsum_final_kernel<<<(N * 32 + 255) / 256, 256, 0, s>>>(P, N, partial, db);
  return cudaGetLastError();
}

__global__ void adamw_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g,
                             float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                             float b2, float eps, float wd, float bc1, float bc2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / bc1, vh = vi / bc2;
  p[i] = p[i] * (1.0f - lr * wd) - lr * mh / (sqrtf(vh) + eps);
}

inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Reverse pass of a residual-modulated block's scale and SiLU: from dA (the
// gradient reaching the block output) and z, dp = dA silu'(g z), dz = dp g
// (out), and dp z replaces z (the factor of the channel-scale gradients).
__global__ void rm_back_kernel(int64_t n, const float *__restrict__ dA, float *__restrict__ Z,
                               const float *__restrict__ X0, const float *__restrict__ G,
                               float *__restrict__ dz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = i >> 8;
  const int c = (int)(i & 255);
  const float g = fmaf(G[c], X0[b * 32 + 3], fmaf(G[256 + c], X0[b * 32 + 4], 1.0f));
  const float z = Z[i], pz = g * z, s = sigmoidf_(pz);
  const float dp = dA[i] * (s * (1.0f + pz * (1.0f - s)));
  dz[i] = dp * g;
  Z[i] = dp * z;
}

// out = dA silu'(z), elementwise
__global__ void dsilu_kernel(int64_t n, const float *__restrict__ dA, const float *__restrict__ Z,
                             float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float z = Z[i], s = sigmoidf_(z);
  out[i] = dA[i] * (s * (1.0f + z * (1.0f - s)));
}

// forward + loss + backward of the residual-modulated network (the gradient
// of each block as the reverse pass of the oracle states it); grads overwritten
cudaError_t fwd_bwd_rm(cudaStream_t s, TrainState &T, double *loss_slot) {
  const int B = (int)T.B;
  const int64_t nh = (int64_t)B * 256;
  float *P = T.params, *G = T.grads;
  const int64_t wofs[4] = {P_W1, P_W2, P_W3, P_W4}, bofs[4] = {P_B1, P_B2, P_B3, P_B4};
  cudaError_t e = gemm<kEpiBiasSilu>(s, B, 256, 32, T.X0, 32, 1, P + P_W1, 1, 32, T.Z[0], P + P_B1, T.A[0]);
  if (e) return e;
  for (int l = 1; l < 4; ++l) {
    const int j = l - 1;
    RMArgs ra;
    ra.M = P + P_RM_M + j * 1280;
    ra.G = P + P_RM_G + j * 512;
    ra.X0 = T.X0;
    e = gemm<kEpiRM>(s, B, 256, 256, T.A[l - 1], 256, 1, P + wofs[l], 1, 256, T.Z[l], P + bofs[l],
                     T.A[l], T.A[l - 1], ra);
    if (e) return e;
  }
  e = gemm<kEpiBias>(s, B, 4, 256, T.A[3], 256, 1, P + P_W5, 1, 256, T.V, P + P_B5);
  if (e) return e;
  loss_kernel<<<nb(B, 256), 256, 0, s>>>(B, T.V, T.U, T.dV, loss_slot);
  e = gemm_wgrad(s, 4, 256, B, T.dV, 1, 4, T.A[3], 256, 1, G + P_W5, T.ws);
  if (e) return e;
  e = colsum(s, B, 4, T.dV, T.colpart, G + P_B5);
  if (e) return e;
  float *dA = T.dZ[0], *dz = T.dZ[1];
  e = gemm<kEpiStore>(s, B, 256, 4, T.dV, 4, 1, P + P_W5, 256, 1, dA);  // dA = dV W5
  if (e) return e;
  for (int l = 3; l >= 1; --l) {
    const int j = l - 1;
    rm_back_kernel<<<nb(nh, 256), 256, 0, s>>>(nh, dA, T.Z[l], T.X0, P + P_RM_G + j * 512, dz);
    // dW_l = dz^T A_{l-1}, db_l = sum dz, dM_j = dz^T c, dG_j = [c_3 c_4]^T (dp z)
    e = gemm_wgrad(s, 256, 256, B, dz, 1, 256, T.A[l - 1], 256, 1, G + wofs[l], T.ws);
    if (e) return e;
    e = colsum(s, B, 256, dz, T.colpart, G + bofs[l]);
    if (e) return e;
    e = gemm_wgrad(s, 256, 5, B, dz, 1, 256, T.X0, 32, 1, G + P_RM_M + j * 1280, T.ws);
    if (e) return e;
    e = gemm_wgrad(s, 2, 256, B, T.X0 + 3, 1, 32, T.Z[l], 256, 1, G + P_RM_G + j * 512, T.ws);
    if (e) return e;
    // the residual path: dA <- dA + dz W_l
    e = gemm<kEpiAdd>(s, B, 256, 256, dz, 256, 1, P + wofs[l], 256, 1, dA);
    if (e) return e;
  }
  dsilu_kernel<<<nb(nh, 256), 256, 0, s>>>(nh, dA, T.Z[0], dz);
  e = gemm_wgrad(s, 256, 32, B, dz, 1, 256, T.X0, 32, 1, G + P_W1, T.ws);
  if (e) return e;
  e = colsum(s, B, 256, dz, T.colpart, G + P_B1);
  if (e) return e;
  return cudaGetLastError();
}

// forward + loss + backward for the batch already in X0/U; grads overwritten
cudaError_t fwd_bwd(cudaStream_t s, TrainState &T, double *loss_slot) {
  if (T.rm) return fwd_bwd_rm(s, T, loss_slot);
  const int B = (int)T.B;
  float *P = T.params, *G = T.grads;
  const float *W[4] = {P + P_W1, P + P_W2, P + P_W3, P + P_W4};
  const float *bb[4] = {P + P_B1, P + P_B2, P + P_B3, P + P_B4};
  cudaError_t e;
  // forward: Z_l = A_{l-1} W_l^T + b_l, A_l = SiLU(Z_l)
  e = gemm<kEpiBiasSilu>(s, B, 256, 32, T.X0, 32, 1, W[0], 1, 32, T.Z[0], bb[0], T.A[0]);
  if (e) return e;
  for (int l = 1; l < 4; ++l) {
    e = gemm<kEpiBiasSilu>(s, B, 256, 256, T.A[l - 1], 256, 1, W[l], 1, 256, T.Z[l], bb[l], T.A[l]);
    if (e) return e;
  }
  e = gemm<kEpiBias>(s, B, 4, 256, T.A[3], 256, 1, P + P_W5, 1, 256, T.V, P + P_B5);
  if (e) return e;
  loss_kernel<<<nb(B, 256), 256, 0, s>>>(B, T.V, T.U, T.dV, loss_slot);
  // output layer: dW5 = dV^T A4, db5 = sum dV, dZ4 = (dV W5) * SiLU'(Z4)
  e = gemm_wgrad(s, 4, 256, B, T.dV, 1, 4, T.A[3], 256, 1, G + P_W5, T.ws);
  if (e) return e;
  e = colsum(s, B, 4, T.dV, T.colpart, G + P_B5);
  if (e) return e;
  e = gemm<kEpiDSilu>(s, B, 256, 4, T.dV, 4, 1, P + P_W5, 256, 1, T.dZ[0], nullptr, nullptr, T.Z[3]);
  if (e) return e;
  int cur = 0;
  const int64_t wofs[4] = {P_W1, P_W2, P_W3, P_W4}, bofs[4] = {P_B1, P_B2, P_B3, P_B4};
  for (int l = 3; l >= 0; --l) {
    const float *dz = T.dZ[cur];
    const float *ain = l == 0 ? T.X0 : T.A[l - 1];
    const int kin = l == 0 ? 32 : 256;
    // dW_l = dZ_l^T A_{l-1}; db_l = column sums of dZ_l
    e = gemm_wgrad(s, 256, kin, B, dz, 1, 256, ain, kin, 1, G + wofs[l], T.ws);
    if (e) return e;
    e = colsum(s, B, 256, dz, T.colpart, G + bofs[l]);
    if (e) return e;
    if (l > 0) {
      // dZ_{l-1} = (dZ_l W_l) * SiLU'(Z_{l-1})
      e = gemm<kEpiDSilu>(s, B, 256, 256, dz, 256, 1, P + wofs[l], 256, 1, T.dZ[cur ^ 1], nullptr,
                          nullptr, T.Z[l - 1]);
      if (e) return e;
      cur ^= 1;
    }
  }
  return cudaGetLastError();
}

// The gradient of the batch in X0/U into T.grads; on the BF16 path with
// `adam` the same launches also apply AdamW (train_fused.cu).
cudaError_t step_grads(cudaStream_t s, TrainState &T, double *loss_slot, const tf::Adam *adam = nullptr,
                       const tf::Gen *gen = nullptr, const tf::Gen *next = nullptr) {
  if (T.cfg.precision == GMC_BF16) {
    if (!gen)  // rows in X0 / U from the kernel just before
      return tf::step(s, T.fb, T.B, nullptr, T.X0, T.U, false, T.params, T.grads, T.m, T.v, adam,
                      loss_slot, T.err);
    // a training step: its rows were drawn during the previous step when
    // that step knew it (same seed, step and data), else in the forward kernel
    const bool have = T.fb.pregen_step == gen->step;
    const cudaError_t e = tf::step(s, T.fb, T.B, have ? nullptr : gen, T.fb.x0n, T.fb.un, have,
                                   T.params, T.grads, T.m, T.v, adam, loss_slot, T.err, next);
    T.fb.pregen_step = next ? next->step : -1;
    return e;
  }
  return fwd_bwd(s, T, loss_slot);
}

void free_train(TrainState *T) {
  if (!T) return;
  float *bufs[] = {T->params, T->grads, T->m, T->v, T->X0, T->U, T->V, T->dV, T->Z[0], T->Z[1],
                   T->Z[2], T->Z[3], T->A[0], T->A[1], T->A[2], T->A[3], T->dZ[0], T->dZ[1]};
  for (float *b : bufs)
    if (b) cudaFree(b);
  if (T->loss) cudaFree(T->loss);
  if (T->stat_acc) cudaFree(T->stat_acc);
  if (T->colpart) cudaFree(T->colpart);
  if (T->ws) cudaFree(T->ws);
  tf::release(T->fb);
  delete T;
}

// Batch buffers: X0 and U always; the FP32 path's activations, or the
// operand images of the BF16 tensor-core step.
cudaError_t alloc_batch(TrainState &T, int64_t B, cudaStream_t s) {
  if (T.B >= B) return cudaSuccess;
  const bool f32 = T.cfg.precision != GMC_BF16;
  float **bufs[] = {&T.X0, &T.U, &T.V, &T.dV, &T.Z[0], &T.Z[1], &T.Z[2], &T.Z[3],
                    &T.A[0], &T.A[1], &T.A[2], &T.A[3], &T.dZ[0], &T.dZ[1]};
  const int64_t sizes[] = {B * 32, B * 4, B * 4, B * 4, B * 256, B * 256, B * 256, B * 256,
                           B * 256, B * 256, B * 256, B * 256, B * 256, B * 256};
  for (int i = 0; i < 14; ++i) {
    if (*bufs[i]) cudaFree(*bufs[i]);
    *bufs[i] = nullptr;
    if (i >= 2 && !f32) continue;
    cudaError_t e = cudaMalloc(bufs[i], sizes[i] * sizeof(float));
    if (e) return e;
  }
  if (T.colpart) cudaFree(T.colpart);
  T.colpart = nullptr;
  cudaError_t e = f32 ? cudaMalloc(&T.colpart, ((B + kColRows - 1) / kColRows) * 256 * sizeof(float))
                      : tf::alloc(T.fb, B, s);
  if (e) return e;
  if (f32 && !T.ws) {
    e = cudaMalloc(&T.ws, kKSplitWs * sizeof(float));
    if (e) return e;
  }
  T.B = B;
  return cudaSuccess;
}

}  // namespace

void train_state_free(TrainState *T) { free_train(T); }

}  // namespace gmc

using namespace gmc;

extern "C" {

gmc_status gmc_train_data(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo, float tau_hi,
                          float c_lo, float c_hi, float *cond, float *y) {
  if (!ctx) return GMC_EINVAL;
  if (n < 0 || (n > 0 && (!cond || !y))) return set_error(ctx, GMC_EINVAL, "gmc_train_data: bad arguments");
  if (!data_ranges_ok(tau_lo, tau_hi, c_lo, c_hi))
    return set_error(ctx, GMC_EINVAL,
                     "gmc_train_data: need 0 < tau_lo <= tau_hi (finite), 0 <= c_lo <= c_hi <= 1");
  if (n == 0) return GMC_OK;
  if (!is_device_pointer(cond, ctx->device) || !is_device_pointer(y, ctx->device))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data: cond and y must be device memory");
  cudaSetDevice(ctx->device);
  data_kernel<<<nb(n, 128), 128, 0, ctx->stream>>>(n, seed, logf(tau_lo), logf(tau_hi), c_lo, c_hi,
                                                   cond, y);
  GMC_CUDA_TRY(ctx, cudaGetLastError());
  return GMC_OK;
}

gmc_status gmc_train_data_internal(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo,
                                   float tau_hi, float c_lo, float c_hi, float *cond, float *y) {
  if (!ctx) return GMC_EINVAL;
  if (n < 0 || (n > 0 && (!cond || !y)))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data_internal: bad arguments");
  if (!data_ranges_ok(tau_lo, tau_hi, c_lo, c_hi))
    return set_error(ctx, GMC_EINVAL,
                     "gmc_train_data_internal: need 0 < tau_lo <= tau_hi (finite), 0 <= c_lo <= c_hi <= 1");
  if (n == 0) return GMC_OK;
  if (!is_device_pointer(cond, ctx->device) || !is_device_pointer(y, ctx->device))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data_internal: cond and y must be device memory");
  cudaSetDevice(ctx->device);
  internal_data_kernel<<<nb(n, 128), 128, 0, ctx->stream>>>(n, seed, logf(tau_lo), logf(tau_hi), c_lo,
                                                            c_hi, cond, y);
  GMC_CUDA_TRY(ctx, cudaGetLastError());
  return GMC_OK;
}

gmc_status gmc_train_data_xy(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo, float tau_hi,
                             float c_lo, float c_hi, float *cond, float *y) {
  if (!ctx) return GMC_EINVAL;
  if (n < 0 || (n > 0 && (!cond || !y)))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data_xy: bad arguments");
  if (!data_ranges_ok(tau_lo, tau_hi, c_lo, c_hi))
    return set_error(ctx, GMC_EINVAL,
                     "gmc_train_data_xy: need 0 < tau_lo <= tau_hi (finite), 0 <= c_lo <= c_hi <= 1");
  if (n == 0) return GMC_OK;
  if (!is_device_pointer(cond, ctx->device) || !is_device_pointer(y, ctx->device))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data_xy: cond and y must be device memory");
  cudaSetDevice(ctx->device);
  xy_data_kernel<<<nb(n, 128), 128, 0, ctx->stream>>>(n, seed, logf(tau_lo), logf(tau_hi), c_lo, c_hi,
                                                      cond, y);
  GMC_CUDA_TRY(ctx, cudaGetLastError());
  return GMC_OK;
}

gmc_status gmc_train_data_rect(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo, float tau_hi,
                               float aspect_lo, float aspect_hi, float c_lo, float c_hi, float *cond,
                               float *y) {
  if (!ctx) return GMC_EINVAL;
  if (n < 0 || (n > 0 && (!cond || !y)))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data_rect: bad arguments");
  if (!data_ranges_ok(tau_lo, tau_hi, c_lo, c_hi, aspect_lo, aspect_hi))
    return set_error(ctx, GMC_EINVAL,
                     "gmc_train_data_rect: need 0 < tau_lo <= tau_hi, 0 < aspect_lo <= aspect_hi "
                     "(finite), 0 <= c_lo <= c_hi <= 1");
  if (n == 0) return GMC_OK;
  if (!is_device_pointer(cond, ctx->device) || !is_device_pointer(y, ctx->device))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data_rect: cond and y must be device memory");
  cudaSetDevice(ctx->device);
  rect_data_kernel<<<nb(n, 128), 128, 0, ctx->stream>>>(n, seed, logf(tau_lo), logf(tau_hi),
                                                        logf(aspect_lo), logf(aspect_hi), c_lo, c_hi,
                                                        cond, y);
  GMC_CUDA_TRY(ctx, cudaGetLastError());
  return GMC_OK;
}

gmc_status gmc_train_data_internal_xy(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo,
                                      float tau_hi, float c_lo, float c_hi, float *cond, float *y) {
  if (!ctx) return GMC_EINVAL;
  if (n < 0 || (n > 0 && (!cond || !y)))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data_internal_xy: bad arguments");
  if (!data_ranges_ok(tau_lo, tau_hi, c_lo, c_hi))
    return set_error(ctx, GMC_EINVAL,
                     "gmc_train_data_internal_xy: need 0 < tau_lo <= tau_hi (finite), 0 <= c_lo <= c_hi <= 1");
  if (n == 0) return GMC_OK;
  if (!is_device_pointer(cond, ctx->device) || !is_device_pointer(y, ctx->device))
    return set_error(ctx, GMC_EINVAL, "gmc_train_data_internal_xy: cond and y must be device memory");
  cudaSetDevice(ctx->device);
  internal_xy_data_kernel<<<nb(n, 128), 128, 0, ctx->stream>>>(n, seed, logf(tau_lo), logf(tau_hi),
                                                               c_lo, c_hi, cond, y);
  GMC_CUDA_TRY(ctx, cudaGetLastError());
  return GMC_OK;
}

gmc_status gmc_train_begin(gmc_ctx *ctx, int64_t n, const float *cond, const float *y,
                           const gmc_train_config *cfg) {
  if (!ctx || !cfg) return GMC_EINVAL;
  if (n < 2 || !cond || !y) return set_error(ctx, GMC_EINVAL, "gmc_train_begin: need n >= 2 samples");
  switch (train_config_check(*cfg)) {
    case 0: break;
    case 1:
    case 2: return set_error(ctx, GMC_EINVAL, "gmc_train_begin: batch in [1, 2^20], lr > 0 (finite)");
    case 3:
      return set_error(ctx, GMC_EINVAL, "gmc_train_begin: precision must be GMC_FP32 or GMC_BF16");
    default:
      return set_error(ctx, GMC_EINVAL,
                       "gmc_train_begin: need betas in [0, 1), eps > 0, weight decay >= 0 (finite)");
  }
  if (!ctx->net.loaded) return set_error(ctx, GMC_ENOWEIGHTS, "gmc_train_begin: load initial weights first");
  if (ctx->net.rm && cfg->precision != GMC_FP32)
    return set_error(ctx, GMC_EINVAL, "gmc_train_begin: the residual-modulated network trains at GMC_FP32");
  if (ctx->net.stats.ncond != kCond && cfg->precision != GMC_FP32)
    return set_error(ctx, GMC_EINVAL, "gmc_train_begin: the rectangular-cell network trains at GMC_FP32");
  if (!is_device_pointer(cond, ctx->device) || !is_device_pointer(y, ctx->device))
    return set_error(ctx, GMC_EINVAL, "gmc_train_begin: data must be device memory");
  cudaSetDevice(ctx->device);
  if (ctx->train) free_train(ctx->train);
  TrainState *T = new TrainState();
  ctx->train = T;
  T->n = n;
  T->cond = cond;
  T->y = y;
  T->cfg = *cfg;
  T->rm = ctx->net.rm;
  T->ncond = ctx->net.stats.ncond;
  T->np = T->rm ? P_TOTAL_RM : P_TOTAL;
  T->step = 0;
  cudaStream_t s = ctx->stream;
  const int nc = T->ncond, nf = nc + 4;
  GMC_CUDA_TRY(ctx, cudaMalloc(&T->stat_acc, 20 * sizeof(double)));
  GMC_CUDA_TRY(ctx, cudaMemsetAsync(T->stat_acc, 0, 20 * sizeof(double), s));
  stats_kernel<<<1024, 256, 0, s>>>(n, nc, cond, y, T->stat_acc);
  GMC_CUDA_TRY(ctx, cudaGetLastError());
  double acc[20];
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(acc, T->stat_acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  for (int k = 0; k < nf; ++k) {
    const double mean = acc[k] / n;
    double var = acc[nf + k] / n - mean * mean;
    const double sd = var > 1e-12 ? std::sqrt(var) : 1.0;
    if (k < nc) {
      T->stats[k] = (float)mean;
      T->stats[nc + k] = (float)sd;
    } else {
      T->stats[2 * nc + (k - nc)] = (float)mean;
      T->stats[2 * nc + 4 + (k - nc)] = (float)sd;
    }
  }
  // master weights from the loaded network
  const int64_t np = T->np;
  std::vector<float> h(np, 0.0f);
  for (int c = 0; c < 256; ++c)
    for (int k = 0; k < ctx->net.nin; ++k) h[P_W1 + c * 32 + k] = ctx->net.host_w[0][c * ctx->net.nin + k];
  std::memcpy(&h[P_B1], ctx->net.host_b[0], 256 * 4);
  const int64_t wo[3] = {P_W2, P_W3, P_W4}, bo[3] = {P_B2, P_B3, P_B4};
  for (int l = 0; l < 3; ++l) {
    std::memcpy(&h[wo[l]], ctx->net.host_w[l + 1], 65536 * 4);
    std::memcpy(&h[bo[l]], ctx->net.host_b[l + 1], 256 * 4);
  }
  std::memcpy(&h[P_W5], ctx->net.host_w[4], 1024 * 4);
  std::memcpy(&h[P_B5], ctx->net.host_b[4], 4 * 4);
  if (T->rm) {
    std::memcpy(&h[P_RM_M], ctx->net.host_m, 3 * 256 * 5 * 4);
    std::memcpy(&h[P_RM_G], ctx->net.host_g, 3 * 512 * 4);
  }
  GMC_CUDA_TRY(ctx, cudaMalloc(&T->params, np * 4));
  GMC_CUDA_TRY(ctx, cudaMalloc(&T->grads, np * 4));
  GMC_CUDA_TRY(ctx, cudaMalloc(&T->m, np * 4));
  GMC_CUDA_TRY(ctx, cudaMalloc(&T->v, np * 4));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(T->params, h.data(), np * 4, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemsetAsync(T->grads, 0, np * 4, s));
  GMC_CUDA_TRY(ctx, cudaMemsetAsync(T->m, 0, np * 4, s));
  GMC_CUDA_TRY(ctx, cudaMemsetAsync(T->v, 0, np * 4, s));
  GMC_CUDA_TRY(ctx, alloc_batch(*T, cfg->batch, s));
  T->err = ctx->d_err;
  if (cfg->precision == GMC_BF16) GMC_CUDA_TRY(ctx, tf::pack(s, T->fb, T->params));
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return GMC_OK;
}

gmc_status gmc_train_steps(gmc_ctx *ctx, int64_t n_steps, float *losses) {
  if (!ctx) return GMC_EINVAL;
  TrainState *T = ctx->train;
  if (!T) return set_error(ctx, GMC_EINVAL, "gmc_train_steps: call gmc_train_begin first");
  if (n_steps < 0) return set_error(ctx, GMC_EINVAL, "gmc_train_steps: n_steps < 0");
  if (n_steps == 0) return GMC_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  if (T->loss_cap < n_steps) {
    if (T->loss) cudaFree(T->loss);
    T->loss = nullptr;
    GMC_CUDA_TRY(ctx, cudaMalloc(&T->loss, n_steps * sizeof(double)));
    T->loss_cap = n_steps;
  }
  GMC_CUDA_TRY(ctx, cudaMemsetAsync(T->loss, 0, n_steps * sizeof(double), s));
  Std sd;
  const int nc = T->ncond;
  for (int k = 0; k < 6; ++k) {
    sd.cm[k] = k < nc ? T->stats[k] : 0.0f;
    sd.cis[k] = k < nc ? 1.0f / T->stats[nc + k] : 1.0f;
  }
  for (int k = 0; k < 4; ++k) {
    sd.ym[k] = T->stats[2 * nc + k];
    sd.yis[k] = 1.0f / T->stats[2 * nc + 4 + k];
  }
  const gmc_train_config &c = T->cfg;
  for (int64_t i = 0; i < n_steps; ++i) {
    if (c.precision != GMC_BF16)
      batch_kernel<<<nb(T->B, 256), 256, 0, s>>>(T->B, T->n, T->ncond, T->cond, T->y, sd, c.seed,
                                                 T->step, T->X0, T->U);
    const float bc1 = 1.0f - (float)std::pow(c.beta1, (double)(T->step + 1));
    const float bc2 = 1.0f - (float)std::pow(c.beta2, (double)(T->step + 1));
    if (c.precision == GMC_BF16) {
      const tf::Adam adam{(float)c.lr, (float)c.beta1, (float)c.beta2, (float)c.eps,
                          (float)c.weight_decay, bc1, bc2};
      const tf::Gen gen{T->cond, T->y, T->n, sd, c.seed, T->step};
      const tf::Gen next{T->cond, T->y, T->n, sd, c.seed, T->step + 1};
      GMC_CUDA_TRY(ctx, step_grads(s, *T, T->loss + i, &adam, &gen, &next));
    } else {
      GMC_CUDA_TRY(ctx, step_grads(s, *T, T->loss + i));
      adamw_kernel<<<nb(T->np, 256), 256, 0, s>>>(T->np, T->params, T->grads, T->m, T->v,
                                                    (float)c.lr, (float)c.beta1, (float)c.beta2,
                                                    (float)c.eps, (float)c.weight_decay, bc1, bc2);
    }
    ++T->step;
    GMC_CUDA_TRY(ctx, cudaGetLastError());
  }
  if (losses) {
    std::vector<double> hl(n_steps);
    GMC_CUDA_TRY(ctx, cudaMemcpyAsync(hl.data(), T->loss, n_steps * sizeof(double), cudaMemcpyDeviceToHost, s));
    GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    for (int64_t i = 0; i < n_steps; ++i) losses[i] = (float)hl[i];
    return check_device_error(ctx);
  }
  return GMC_OK;
}

gmc_status gmc_train_grad(gmc_ctx *ctx, int64_t B, const float *cn, const float *x1,
                          const float *x0, const float *t, double *loss, float *grad) {
  if (!ctx) return GMC_EINVAL;
  TrainState *T = ctx->train;
  if (!T) return set_error(ctx, GMC_EINVAL, "gmc_train_grad: call gmc_train_begin first");
  if (B < 1 || B > T->B || !cn || !x1 || !x0 || !t || !loss || !grad)
    return set_error(ctx, GMC_EINVAL, "gmc_train_grad: 1 <= B <= batch and non-null arrays");
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  float *d;
  const int nc = T->ncond;
  const size_t nbytes = (size_t)B * (nc + 4 + 4 + 1) * 4;
  GMC_CUDA_TRY(ctx, ensure(ctx->stage[0], nbytes));
  d = (float *)ctx->stage[0].ptr;
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(d, cn, B * nc * 4, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(d + B * nc, x1, B * 16, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(d + B * (nc + 4), x0, B * 16, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(d + B * (nc + 8), t, B * 4, cudaMemcpyHostToDevice, s));
  batch_explicit_kernel<<<nb(B, 256), 256, 0, s>>>(B, nc, d, d + B * nc, d + B * (nc + 4),
                                                   d + B * (nc + 8), T->X0, T->U);
  const int64_t saveB = T->B;
  T->B = B;
  double *ls;
  GMC_CUDA_TRY(ctx, ensure(ctx->stage[1], sizeof(double)));
  ls = (double *)ctx->stage[1].ptr;
  GMC_CUDA_TRY(ctx, cudaMemsetAsync(ls, 0, sizeof(double), s));
  cudaError_t e = step_grads(s, *T, ls);
  T->B = saveB;
  GMC_CUDA_TRY(ctx, e);
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(loss, ls, sizeof(double), cudaMemcpyDeviceToHost, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(grad, T->grads, T->np * 4, cudaMemcpyDeviceToHost, s));
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return check_device_error(ctx);
}

int64_t gmc_train_param_count(void) { return P_TOTAL; }

gmc_status gmc_train_param_count_ctx(const gmc_ctx *ctx, int64_t *count) {
  if (!ctx || !count) return GMC_EINVAL;
  if (!ctx->train) return GMC_EINVAL;
  *count = ctx->train->np;
  return GMC_OK;
}

gmc_status gmc_train_set_lr(gmc_ctx *ctx, double lr) {
  if (!ctx) return GMC_EINVAL;
  if (!ctx->train) return set_error(ctx, GMC_EINVAL, "gmc_train_set_lr: call gmc_train_begin first");
  if (!(lr > 0.0) || !std::isfinite(lr))
    return set_error(ctx, GMC_EINVAL, "gmc_train_set_lr: lr must be > 0 and finite");
  ctx->train->cfg.lr = lr;
  return GMC_OK;
}

gmc_status gmc_train_params(gmc_ctx *ctx, float *out) {
  if (!ctx || !out) return GMC_EINVAL;
  if (!ctx->train) return set_error(ctx, GMC_EINVAL, "gmc_train_params: call gmc_train_begin first");
  cudaSetDevice(ctx->device);
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->train->params, ctx->train->np * 4, cudaMemcpyDeviceToHost,
                                    ctx->stream));
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return GMC_OK;
}

int32_t ckpt_arch(const TrainState &T) { return ckpt_arch_bits(T.rm, T.ncond); }

gmc_status gmc_train_state_size(const gmc_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return GMC_EINVAL;
  const int64_t np = ctx->train ? ctx->train->np : P_TOTAL;
  *bytes = sizeof(TrainCkpt) + 3 * (size_t)np * sizeof(float);
  return GMC_OK;
}

gmc_status gmc_train_save_state(gmc_ctx *ctx, void *blob, size_t nbytes) {
  if (!ctx) return GMC_EINVAL;
  TrainState *T = ctx->train;
  if (!T) return set_error(ctx, GMC_EINVAL, "gmc_train_save_state: call gmc_train_begin first");
  size_t need = 0;
  gmc_train_state_size(ctx, &need);
  if (!blob || nbytes != need)
    return set_error(ctx, GMC_EINVAL, "gmc_train_save_state: need a host buffer of %zu bytes", need);
  TrainCkpt h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "GMCT", 4);
  h.version = kCkptVersion;
  h.params = T->np;
  h.arch = ckpt_arch(*T);
  h.step = T->step;
  h.batch = T->cfg.batch;
  h.n = T->n;
  h.precision = T->cfg.precision;
  h.lr = T->cfg.lr;
  h.beta1 = T->cfg.beta1;
  h.beta2 = T->cfg.beta2;
  h.eps = T->cfg.eps;
  h.weight_decay = T->cfg.weight_decay;
  h.seed = T->cfg.seed;
  std::memcpy(h.stats, T->stats, sizeof(h.stats));
  unsigned char *out = (unsigned char *)blob;
  std::memcpy(out, &h, sizeof(h));
  float *body = (float *)(out + sizeof(h));
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  const int64_t np = T->np;
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(body, T->params, np * 4, cudaMemcpyDeviceToHost, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(body + np, T->m, np * 4, cudaMemcpyDeviceToHost, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(body + 2 * np, T->v, np * 4, cudaMemcpyDeviceToHost, s));
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return check_device_error(ctx);
}

gmc_status gmc_train_load_state(gmc_ctx *ctx, const void *blob, size_t nbytes) {
  if (!ctx) return GMC_EINVAL;
  TrainState *T = ctx->train;
  if (!T) return set_error(ctx, GMC_EINVAL, "gmc_train_load_state: call gmc_train_begin first");
  size_t need = 0;
  gmc_train_state_size(ctx, &need);
  if (!blob || nbytes != need)
    return set_error(ctx, GMC_EFORMAT, "gmc_train_load_state: a checkpoint is %zu bytes", need);
  TrainCkpt h;
  std::memcpy(&h, blob, sizeof(h));
  static_assert(sizeof(T->stats) == sizeof(h.stats), "checkpoint statistics");
  const CkptTarget tgt{T->np, T->cfg.batch, T->n, T->cfg.precision, ckpt_arch(*T), T->ncond, T->stats};
  switch (ckpt_check(h, tgt)) {
    case kCkptOk: break;
    case kCkptNotThisNetwork:
      return set_error(ctx, GMC_EFORMAT,
                       "gmc_train_load_state: not a version-3 training checkpoint of this network");
    case kCkptBadStats:
      return set_error(ctx, GMC_EFORMAT, "gmc_train_load_state: bad standardization statistics");
    case kCkptBadHyper:
      return set_error(ctx, GMC_EFORMAT,
                       "gmc_train_load_state: bad hyperparameters (lr > 0, betas in [0, 1), "
                       "eps > 0, weight decay >= 0, all finite)");
    case kCkptOtherRun:
      return set_error(ctx, GMC_EINVAL,
                       "gmc_train_load_state: begin training with the checkpoint's batch and precision");
    default:
      return set_error(ctx, GMC_EINVAL,
                       "gmc_train_load_state: the checkpoint was saved on other data (size %lld, "
                       "or different statistics) than this training state's (size %lld)",
                       (long long)h.n, (long long)T->n);
  }
  const float *body = (const float *)((const unsigned char *)blob + sizeof(h));
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  const int64_t np = T->np;
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(T->params, body, np * 4, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(T->m, body + np, np * 4, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(T->v, body + 2 * np, np * 4, cudaMemcpyHostToDevice, s));
  if (T->cfg.precision == GMC_BF16) {
    GMC_CUDA_TRY(ctx, tf::pack(s, T->fb, T->params));
    T->fb.pregen_step = -1;  // rows drawn for another step or seed
  }
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  T->step = h.step;
  T->cfg.lr = h.lr;
  T->cfg.beta1 = h.beta1;
  T->cfg.beta2 = h.beta2;
  T->cfg.eps = h.eps;
  T->cfg.weight_decay = h.weight_decay;
  T->cfg.seed = h.seed;
  return GMC_OK;
}

gmc_status gmc_train_commit(gmc_ctx *ctx, const char *path) {
  if (!ctx) return GMC_EINVAL;
  TrainState *T = ctx->train;
  if (!T) return set_error(ctx, GMC_EINVAL, "gmc_train_commit: call gmc_train_begin first");
  if (ctx->server) return set_error(ctx, GMC_EBUSY, "gmc_train_commit: the server is running");
  cudaSetDevice(ctx->device);
  std::vector<float> h(T->np);
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), T->params, T->np * 4, cudaMemcpyDeviceToHost, ctx->stream));
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  // GMCW version 1 blob
  std::vector<unsigned char> blob;
  auto u32 = [&](uint32_t v) { const unsigned char *p = (const unsigned char *)&v; blob.insert(blob.end(), p, p + 4); };
  auto f32 = [&](const float *v, size_t n) { const unsigned char *p = (const unsigned char *)v; blob.insert(blob.end(), p, p + 4 * n); };
  blob.insert(blob.end(), {'G', 'M', 'C', 'W'});
  u32(1); u32(5);
  const int nc = T->ncond, nin = nc + kState + kEmb;
  const uint32_t dims[6] = {(uint32_t)nin, 256, 256, 256, 256, 4};
  for (uint32_t dd : dims) u32(dd);
  u32((uint32_t)nc); u32(4); u32(16); u32(T->rm ? kFlagRM : 0u);
  f32(T->stats, 2 * nc + 8);
  std::vector<float> w1(256 * nin);
  for (int c = 0; c < 256; ++c)
    for (int k = 0; k < nin; ++k) w1[c * nin + k] = h[P_W1 + c * 32 + k];
  f32(w1.data(), w1.size());
  f32(&h[P_B1], 256);
  f32(&h[P_W2], 65536); f32(&h[P_B2], 256);
  f32(&h[P_W3], 65536); f32(&h[P_B3], 256);
  f32(&h[P_W4], 65536); f32(&h[P_B4], 256);
  f32(&h[P_W5], 1024); f32(&h[P_B5], 4);
  if (T->rm) {
    f32(&h[P_RM_M], 3 * 256 * 5);
    f32(&h[P_RM_G], 3 * 512);
  }
  if (path) {
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(ctx, GMC_EIO, "cannot write '%s'", path);
    const size_t wrote = std::fwrite(blob.data(), 1, blob.size(), f);
    const bool bad = std::fclose(f) != 0 || wrote != blob.size();
    if (bad) return set_error(ctx, GMC_EIO, "short write to '%s'", path);
  }
  TrainState *keep = ctx->train;
  ctx->train = nullptr;  // loading weights must not drop the training state
  gmc_status st = gmc_load_weights_buffer(ctx, blob.data(), blob.size());
  ctx->train = keep;
  return st;
}

}  // extern "C"
