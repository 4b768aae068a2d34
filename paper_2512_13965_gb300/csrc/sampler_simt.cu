// FP32 SIMT flow-ODE sampler (Eq. 8): the parity path of gmc_transmit.
//
// One CTA owns 64 particles for all K steps. Their activations live in
// shared memory (one 64 x 256 buffer, overwritten in place layer by layer
// because every thread keeps its outputs in registers until all reads of the
// layer are done); weights stream through a 32 x 256 shared tile. Each of the
// 256 threads computes a 4-row x 16-column register tile, columns
// {4 cg + 64 q + e} so that a warp's float4 reads of a weight row are
// contiguous. Accurate expf keeps SiLU within FP32 rounding.
// Residual-modulated network (net.rm): hidden layers 2-4 add the condition
// shift M_j c to the pre-activation, scale it by g = 1 + G_j[0] c_3 +
// G_j[1] c_4 and add SiLU(g z) to the layer's input (the residual), each
// thread reading the old activations of exactly the cells it overwrites.
#include "decode.cuh"
#include "gmc_internal.cuh"
#include "philox.cuh"

namespace gmc {
namespace {

constexpr int R = 64;       // particles per CTA
constexpr int KC = 32;      // K rows per weight tile
constexpr int LDA = 260;    // padded activation row (floats)
constexpr int THREADS = 256;

struct Smem {
  float act[R][LDA];
  float wc[KC][kHidden];
  float x[R][4];
  float xm[R][4];
  float ka[R][4];
  float v[R][4];
  float cn[R][kCondRect];  // [5]: the aspect of a rectangular cell (0 otherwise)
  float emb[kEmb];
};

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

// act[:, 0:K] (K = 32 or 256) times wt [K][256] (+ b) -> SiLU -> act[:, 0:256];
// with mt non-null (a residual-modulated block, K = 256): act += SiLU(g z),
// z = acc + b + mt^T cn, g = 1 + gg[0] cn_3 + gg[1] cn_4
__device__ void dense_silu(Smem &s, const float *__restrict__ wt, const float *__restrict__ b,
                           int K, const float *__restrict__ mt = nullptr,
                           const float *__restrict__ gg = nullptr) {
  const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
  float acc[4][16];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += KC) {
    __syncthreads();
    const float4 *src = reinterpret_cast<const float4 *>(wt + (size_t)k0 * kHidden);
    float4 *dst = reinterpret_cast<float4 *>(&s.wc[0][0]);
#pragma unroll
    for (int i = 0; i < KC * kHidden / 4 / THREADS; ++i) dst[t + i * THREADS] = __ldg(src + t + i * THREADS);
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < KC; kk += 4) {
      float4 a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4 *>(&s.act[rg * 4 + i][k0 + kk]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float4 w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = *reinterpret_cast<const float4 *>(&s.wc[kk + u][cg * 4 + 64 * q]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float av = u == 0 ? a[i].x : (u == 1 ? a[i].y : (u == 2 ? a[i].z : a[i].w));
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc[i][q * 4 + 0] = fmaf(av, w[q].x, acc[i][q * 4 + 0]);
            acc[i][q * 4 + 1] = fmaf(av, w[q].y, acc[i][q * 4 + 1]);
            acc[i][q * 4 + 2] = fmaf(av, w[q].z, acc[i][q * 4 + 2]);
            acc[i][q * 4 + 3] = fmaf(av, w[q].w, acc[i][q * 4 + 3]);
          }
        }
      }
    }
  }
  __syncthreads();  // every read of act is done: overwrite in place
  if (mt) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = cg * 4 + 64 * q + e;
        const float bc = __ldg(b + c), g0 = __ldg(gg + c), g1 = __ldg(gg + kHidden + c);
        float m[kCond];
#pragma unroll
        for (int k = 0; k < kCond; ++k) m[k] = __ldg(mt + k * kHidden + c);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = rg * 4 + i;
          float z = acc[i][q * 4 + e] + bc;
#pragma unroll
          for (int k = 0; k < kCond; ++k) z = fmaf(m[k], s.cn[r][k], z);
          const float g = fmaf(g0, s.cn[r][3], fmaf(g1, s.cn[r][4], 1.0f));
          s.act[r][c] += silu(g * z);
        }
      }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 bb = __ldg(reinterpret_cast<const float4 *>(b + cg * 4 + 64 * q));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4 o;
      o.x = silu(acc[i][q * 4 + 0] + bb.x);
      o.y = silu(acc[i][q * 4 + 1] + bb.y);
      o.z = silu(acc[i][q * 4 + 2] + bb.z);
      o.w = silu(acc[i][q * 4 + 3] + bb.w);
      *reinterpret_cast<float4 *>(&s.act[rg * 4 + i][cg * 4 + 64 * q]) = o;
    }
  }
  __syncthreads();
}

// v = W5 act + b5 for the CTA's rows, evaluated at state xs and time t.
__device__ void velocity(Smem &s, const NetF32 &net, const float (*xs)[4], float t) {
  const int tid = threadIdx.x;
  if (tid < kEmb) s.emb[tid] = time_embedding(tid, t);
  __syncthreads();
  // layer-1 input [cn(5), x(4), emb(16), aspect, 0 x 6] (the aspect is 0 for
  // a square-cell network, whose w1t row 25 is zero)
  for (int e = tid; e < R * kIn1Pad; e += THREADS) {
    const int r = e / kIn1Pad, k = e % kIn1Pad;
    float v = 0.0f;
    if (k < kCond) v = s.cn[r][k];
    else if (k < kCond + kState) v = xs[r][k - kCond];
    else if (k < kIn) v = s.emb[k - kCond - kState];
    else if (k == kIn) v = s.cn[r][kCond];
    s.act[r][k] = v;
  }
  dense_silu(s, net.w1t, net.b1, kIn1Pad);
  if (net.rm) {
    dense_silu(s, net.w2t, net.b2, kHidden, net.mt, net.gg);
    dense_silu(s, net.w3t, net.b3, kHidden, net.mt + kCond * kHidden, net.gg + 2 * kHidden);
    dense_silu(s, net.w4t, net.b4, kHidden, net.mt + 2 * kCond * kHidden, net.gg + 4 * kHidden);
  } else {
    dense_silu(s, net.w2t, net.b2, kHidden);
    dense_silu(s, net.w3t, net.b3, kHidden);
    dense_silu(s, net.w4t, net.b4, kHidden);
  }
  {
    const int r = tid >> 2, d = tid & 3;
    const float4 *w = reinterpret_cast<const float4 *>(net.w5 + d * kHidden);
    const float4 *a = reinterpret_cast<const float4 *>(&s.act[r][0]);
    float acc = 0.0f;
#pragma unroll 8
    for (int k = 0; k < kHidden / 4; ++k) {
      const float4 wv = __ldg(w + k), av = a[k];
      acc = fmaf(av.x, wv.x, acc);
      acc = fmaf(av.y, wv.y, acc);
      acc = fmaf(av.z, wv.z, acc);
      acc = fmaf(av.w, wv.w, acc);
    }
    s.v[r][d] = acc + __ldg(net.b5 + d);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(THREADS) sampler_f32_kernel(
    NetF32 net, NetStats st, int64_t n, const float *__restrict__ cond,
    const float *__restrict__ noise, uint64_t seed, uint64_t id0, int steps, int integrator,
    float *__restrict__ y_raw, float *__restrict__ exitp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &s = *reinterpret_cast<Smem *>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * R;
  // condition (standardized) and x(0)
  if (tid < R) {
    const int64_t g = row0 + tid;
    if (g < n) {
#pragma unroll
      for (int k = 0; k < kCondRect; ++k)
        s.cn[tid][k] = k < st.ncond ? (cond[k * n + g] - st.cond_mean[k]) * st.cond_inv_std[k] : 0.0f;
      if (noise) {
#pragma unroll
        for (int d = 0; d < 4; ++d) s.x[tid][d] = noise[d * n + g];
      } else {
        const float4 z = box_muller4(philox_draw(seed, id0 + (uint64_t)g, 0u, kTagNoise));
        s.x[tid][0] = z.x;
        s.x[tid][1] = z.y;
        s.x[tid][2] = z.z;
        s.x[tid][3] = z.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kCondRect; ++k) s.cn[tid][k] = 0.0f;
#pragma unroll
      for (int d = 0; d < 4; ++d) s.x[tid][d] = 0.0f;
    }
  }
  __syncthreads();
  const float h = 1.0f / (float)steps;
  const int rr = tid >> 2, dd = tid & 3;
  for (int k = 0; k < steps; ++k) {
    const float t = (float)k * h;
    velocity(s, net, s.x, t);
    if (integrator == GMC_MIDPOINT) {
      s.xm[rr][dd] = fmaf(0.5f * h, s.v[rr][dd], s.x[rr][dd]);
      __syncthreads();
      velocity(s, net, s.xm, t + 0.5f * h);
    } else if (integrator == GMC_RK4) {
      // k1 .. k4 accumulate into ka = k1 + 2 k2 + 2 k3 + k4
      s.ka[rr][dd] = s.v[rr][dd];
      s.xm[rr][dd] = fmaf(0.5f * h, s.v[rr][dd], s.x[rr][dd]);
      __syncthreads();
      velocity(s, net, s.xm, t + 0.5f * h);
      s.ka[rr][dd] = fmaf(2.0f, s.v[rr][dd], s.ka[rr][dd]);
      s.xm[rr][dd] = fmaf(0.5f * h, s.v[rr][dd], s.x[rr][dd]);
      __syncthreads();
      velocity(s, net, s.xm, t + 0.5f * h);
      s.ka[rr][dd] = fmaf(2.0f, s.v[rr][dd], s.ka[rr][dd]);
      s.xm[rr][dd] = fmaf(h, s.v[rr][dd], s.x[rr][dd]);
      __syncthreads();
      velocity(s, net, s.xm, t + h);
      s.v[rr][dd] = (s.ka[rr][dd] + s.v[rr][dd]) * (1.0f / 6.0f);
    }
    s.x[rr][dd] = fmaf(h, s.v[rr][dd], s.x[rr][dd]);
    __syncthreads();
  }
  if (tid < R) {
    const int64_t g = row0 + tid;
    if (g < n) {
      if (y_raw) {
#pragma unroll
        for (int d = 0; d < 4; ++d) y_raw[d * n + g] = s.x[tid][d];
      }
      if (exitp) {
        bool inward;
        const float4 e = decode_exit(s.x[tid][0], s.x[tid][1], s.x[tid][2], s.x[tid][3], st, &inward);
        exitp[0 * n + g] = e.x;
        exitp[1 * n + g] = e.y;
        exitp[2 * n + g] = e.z;
        exitp[3 * n + g] = e.w;
      }
    }
  }
}

}  // namespace

cudaError_t launch_sampler_f32(cudaStream_t stream, const NetF32 &net, const NetStats &st,
                               int64_t n, const float *cond, const float *noise, uint64_t seed,
                               uint64_t id0, int steps, int integrator, float *y_raw,
                               float *exit) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = sizeof(Smem);
  cudaError_t e = cudaFuncSetAttribute(sampler_f32_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (n + R - 1) / R;
  sampler_f32_kernel<<<(unsigned)blocks, THREADS, smem, stream>>>(net, st, n, cond, noise, seed,
                                                                   id0, steps, integrator, y_raw,
                                                                   exit);
  return cudaGetLastError();
}

}  // namespace gmc
