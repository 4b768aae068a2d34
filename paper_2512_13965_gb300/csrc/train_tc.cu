// BF16 tensor-core GEMMs of the training step (Eq. 9 forward and backward):
//
//   C[m][n] = epilogue( sum_k A(m,k) B(n,k) ),
//   A(m,k) = A[m sam + k sak],  B(n,k) = B[n sbn + k sbk]   (FP32 in global memory)
//
// One CTA computes a 128 x BN tile over a K range. Each K chunk of 64 is read
// from global memory (float4 when the K index is contiguous, else lanes over
// rows so that every load instruction is coalesced), rounded to BF16 and
// stored into shared memory in the 128-byte-swizzled K-major layout that
// tcgen05.mma reads; two stages let the loads of chunk i+1 overlap the MMAs of
// chunk i. Accumulation is FP32 in tensor memory; the epilogue reads it back
// with tcgen05.ld and applies bias + SiLU (keeping the pre-activation),
// bias, SiLU' (backward), or a plain store into a split-K slice that a
// second kernel sums in a fixed order. The master weights and every stored
// activation and gradient stay FP32: only the MMA operands are BF16.
//
// Every wait is bounded; a timeout sets the context's device error word.
#include <cuda_bf16.h>

#include <atomic>
#include <cstring>

#include "gmc_internal.cuh"
#include "tc_ptx.cuh"

namespace gmc {
namespace {

using namespace ptx;

constexpr int TG_THREADS = 256;
constexpr int KC = 64;                 // K per staged chunk (128 bytes of BF16)
constexpr uint32_t A_BYTES = 128u * 128u;  // 128 rows x 128 B

struct TgParams {
  int M, N, K;
  const float *A;
  int64_t sam, sak;
  const float *B;
  int64_t sbn, sbk;
  float *C;          // [M][N] (+ split slice offset)
  const float *bias;  // [N]
  float *C2;         // [M][N] SiLU output (kTgBiasSilu)
  const float *Zp;   // [M][N] pre-activation (kTgDSilu)
  int kps;           // K per split slice (multiple of KC)
  int64_t cstride;   // C offset between split slices
  int *err;
};

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &v, 4);
  return u;
}

__device__ __forceinline__ uint32_t sw128_addr(uint32_t base, int r, int c) {
  return base + (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// The chunk when rows are contiguous and K is strided (s_row == 1, s_k a
// multiple of 4: the backward GEMMs' transposed operands). Work item = (group
// of 4 rows, 8-column group c): 8 float4 loads, one per K index, each
// covering the 4 rows (lanes take consecutive row groups, so a warp's load is
// 512 contiguous bytes), transposed in registers into 4 rows of 8 BF16.
// Row groups that cross nrows, or loads off 16-byte alignment, take scalar
// loads; out-of-range entries are zero.
template <int ROWS>
__device__ __forceinline__ void stage_rows(uint32_t sbase, const float *__restrict__ P, int64_t s_k,
                                           int row0, int nrows, int k0, int kend) {
  constexpr int RG = ROWS / 4;
  constexpr int ITEMS = RG * 8;
  constexpr int PER = (ITEMS + TG_THREADS - 1) / TG_THREADS;
  float v[PER][8][4];
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int i = threadIdx.x + it * TG_THREADS;
    const int rg = i % RG, c = i / RG;
    const int gr = row0 + 4 * rg, gk = k0 + 8 * c;
    const bool whole = i < ITEMS && gr + 4 <= nrows;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float *src = P + (int64_t)gr + (int64_t)(gk + j) * s_k;
      if (whole && gk + j < kend && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(src));
        v[it][j][0] = a.x; v[it][j][1] = a.y; v[it][j][2] = a.z; v[it][j][3] = a.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          v[it][j][u] = (i < ITEMS && gr + u < nrows && gk + j < kend)
                            ? __ldg(P + (int64_t)(gr + u) + (int64_t)(gk + j) * s_k)
                            : 0.0f;
      }
    }
  }
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int i = threadIdx.x + it * TG_THREADS;
    if (i >= ITEMS) break;
    const int rg = i % RG, c = i / RG;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      sts128(sw128_addr(sbase, 4 * rg + u, c), bf16x2(v[it][0][u], v[it][1][u]),
             bf16x2(v[it][2][u], v[it][3][u]), bf16x2(v[it][4][u], v[it][5][u]),
             bf16x2(v[it][6][u], v[it][7][u]));
  }
}

// ROWS x 64 operand chunk (rows row0.., K k0..) into shared memory as BF16.
// Work item = (row r, 8-column group c); out-of-range entries are zero. Each
// thread first issues the loads of all its items, then converts and stores
// them, so a chunk costs about one memory latency, not one per item.
template <int ROWS>
__device__ __forceinline__ void stage(uint32_t sbase, const float *__restrict__ P, int64_t s_row,
                                      int64_t s_k, int row0, int nrows, int k0, int kend) {
  if (s_row == 1 && s_k != 1 && (s_k & 3) == 0 && ROWS % 4 == 0) {
    stage_rows<ROWS>(sbase, P, s_k, row0, nrows, k0, kend);
    return;
  }
  constexpr int ITEMS = ROWS * 8;
  constexpr int PER = (ITEMS + TG_THREADS - 1) / TG_THREADS;
  const bool kcontig = s_k == 1;
  float v[PER][8];
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int i = threadIdx.x + it * TG_THREADS;
    const int r = kcontig ? (i >> 3) : (i % ROWS);
    const int c = kcontig ? (i & 7) : (i / ROWS);
    const int gr = row0 + r, gk = k0 + 8 * c;
    const float *src = P + (int64_t)gr * s_row + (int64_t)gk * s_k;
    if (i < ITEMS && gr < nrows && kcontig && gk + 8 <= kend &&
        ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
      const float4 a = __ldg(reinterpret_cast<const float4 *>(src));
      const float4 b = __ldg(reinterpret_cast<const float4 *>(src) + 1);
      v[it][0] = a.x; v[it][1] = a.y; v[it][2] = a.z; v[it][3] = a.w;
      v[it][4] = b.x; v[it][5] = b.y; v[it][6] = b.z; v[it][7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[it][j] = (i < ITEMS && gr < nrows && gk + j < kend)
                       ? __ldg(P + (int64_t)gr * s_row + (int64_t)(gk + j) * s_k)
                       : 0.0f;
    }
  }
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int i = threadIdx.x + it * TG_THREADS;
    if (i >= ITEMS) break;
    const int r = kcontig ? (i >> 3) : (i % ROWS);
    const int c = kcontig ? (i & 7) : (i / ROWS);
    sts128(sw128_addr(sbase, r, c), bf16x2(v[it][0], v[it][1]), bf16x2(v[it][2], v[it][3]),
           bf16x2(v[it][4], v[it][5]), bf16x2(v[it][6], v[it][7]));
  }
}

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

template <int EPI>
__device__ __forceinline__ void epi_store(const TgParams &P, float *C, int m, int n0c, const float *v,
                                          int cnt) {
  // cnt consecutive columns n0c .. of row m (cnt a multiple of 4, n0c of 4)
  const int64_t row = (int64_t)m * P.N;
  for (int j = 0; j < cnt; j += 4) {
    const int n = n0c + j;
    if (n >= P.N) break;
    float o[4], o2[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int nn = n + u;
      float x = v[j + u];
      if (nn < P.N) {
        if (EPI == kTgBiasSilu) {
          x += __ldg(P.bias + nn);
          o2[u] = x * sigm(x);
        } else if (EPI == kTgBias) {
          x += __ldg(P.bias + nn);
        } else if (EPI == kTgDSilu) {
          const float z = __ldg(P.Zp + row + nn), s = sigm(z);
          x *= s * (1.0f + z * (1.0f - s));
        }
      }
      o[u] = x;
    }
    if (n + 4 <= P.N && (P.N & 3) == 0) {
      *reinterpret_cast<float4 *>(C + row + n) = make_float4(o[0], o[1], o[2], o[3]);
      if (EPI == kTgBiasSilu)
        *reinterpret_cast<float4 *>(P.C2 + row + n) = make_float4(o2[0], o2[1], o2[2], o2[3]);
    } else {
      for (int u = 0; u < 4 && n + u < P.N; ++u) {
        C[row + n + u] = o[u];
        if (EPI == kTgBiasSilu) P.C2[row + n + u] = o2[u];
      }
    }
  }
}

template <int BN, int EPI>
__global__ void __launch_bounds__(TG_THREADS) tgemm_kernel(TgParams P) {
  constexpr uint32_t B_BYTES = (uint32_t)BN * 128u;
  constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = BN < 32 ? 32u : (uint32_t)BN;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char *sm = smem_raw + pad;
  const uint32_t sbase = raw + pad;
  uint64_t *done = reinterpret_cast<uint64_t *>(sm + 2 * STAGE);
  uint32_t *tbase = reinterpret_cast<uint32_t *>(sm + 2 * STAGE + 16);
  int *abort_flag = reinterpret_cast<int *>(sm + 2 * STAGE + 20);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tbase, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;
  volatile int *abort = abort_flag;

  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * P.kps;
  const int kend = min(P.K, kbeg + P.kps);
  const int nch = kend > kbeg ? (kend - kbeg + KC - 1) / KC : 0;
  const uint32_t idesc = idesc_bf16_m128((uint32_t)BN);
  bool ok = true;
  for (int kc = 0; kc < nch; ++kc) {
    const int s = kc & 1;
    if (kc >= 2) {
      const bool w = mbar_wait(&done[s], (uint32_t)((kc - 2) >> 1) & 1u, abort);
      if (!__syncthreads_and(w)) {
        ok = false;
        break;
      }
    }
    const uint32_t a_s = sbase + (uint32_t)s * STAGE, b_s = a_s + A_BYTES;
    const int k0 = kbeg + kc * KC;
    stage<128>(a_s, P.A, P.sam, P.sak, m0, P.M, k0, kend);
    stage<BN>(b_s, P.B, P.sbn, P.sbk, n0, P.N, k0, kend);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint64_t da = smem_desc(a_s, 1024, kSwizzle128B), db = smem_desc(b_s, 1024, kSwizzle128B);
#pragma unroll
      for (int k = 0; k < KC / 16; ++k)
        mma_f16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (kc | k) != 0);
      mma_commit(&done[s]);
    }
  }
  if (ok && nch > 0) {
    const int last = nch - 1;
    ok = __syncthreads_and(mbar_wait(&done[last & 1], (uint32_t)(last >> 1) & 1u, abort));
  }
  tc_fence_after();
  if (ok) {
    float *C = P.C + (int64_t)blockIdx.z * P.cstride;
    const int q = warp & 3, half = warp >> 2;
    const int m = m0 + 32 * q + lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    constexpr int COLS = BN / 2;  // per thread
    if constexpr (COLS >= 32) {
#pragma unroll 1
      for (int j = 0; j < COLS; j += 32) {
        uint32_t r[32];
        tmem_ld32_raw(tmem + lane_off + (uint32_t)(half * COLS + j), r);
        tmem_wait_ld_regs(r);
        if (m < P.M) {
          float v[32];
#pragma unroll
          for (int u = 0; u < 32; ++u) v[u] = nch > 0 ? __uint_as_float(r[u]) : 0.0f;
          epi_store<EPI>(P, C, m, n0 + half * COLS + j, v, 32);
        }
      }
    } else {
      float v[COLS];
#pragma unroll
      for (int j = 0; j < COLS; j += 4) {
        float t[4];
        tmem_ld4(tmem + lane_off + (uint32_t)(half * COLS + j), t);
        tmem_wait_ld_regs4(t);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[j + u] = nch > 0 ? t[u] : 0.0f;
      }
      if (m < P.M) epi_store<EPI>(P, C, m, n0 + half * COLS, v, COLS);
    }
  } else if (threadIdx.x == 0) {
    atomicExch(P.err, 7);
    // drain: the MMAs issued so far complete before tensor memory is freed
    int never = 0;
    if (nch > 0) mbar_wait(&done[(nch - 1) & 1], (uint32_t)((nch - 1) >> 1) & 1u, &never, 1000000000ull);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

// out[i] = sum over s of ws[s * n + i], in slice order
__global__ void splitk_reduce_kernel(int64_t n, int S, const float *__restrict__ ws,
                                     float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.0f;
  for (int s = 0; s < S; ++s) acc += ws[(int64_t)s * n + i];
  out[i] = acc;
}

template <int BN, int EPI>
cudaError_t launch_bn(cudaStream_t st, const TgParams &p, int splits) {
  constexpr size_t smem = 2 * ((size_t)A_BYTES + (size_t)BN * 128) + 64 + 1024;
  // the attribute is per device: set it once on each device this process uses
  static std::atomic<bool> attr[kMaxDevices];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDevices || !attr[dev].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(tgemm_kernel<BN, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) attr[dev].store(true, std::memory_order_release);
  }
  dim3 grid((unsigned)((p.M + 127) / 128), (unsigned)((p.N + BN - 1) / BN), (unsigned)splits);
  tgemm_kernel<BN, EPI><<<grid, TG_THREADS, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tgemm(cudaStream_t st, int epi, int M, int N, int K, const float *A, int64_t sam,
                  int64_t sak, const float *B, int64_t sbn, int64_t sbk, float *C,
                  const float *bias, float *C2, const float *Zp, int splits, float *ws,
                  size_t ws_floats, int *err) {
  if (M <= 0 || N <= 0 || N > 256) return cudaErrorInvalidValue;
  TgParams p{};
  p.M = M;
  p.N = N;
  p.K = K;
  p.A = A;
  p.sam = sam;
  p.sak = sak;
  p.B = B;
  p.sbn = sbn;
  p.sbk = sbk;
  p.bias = bias;
  p.C2 = C2;
  p.Zp = Zp;
  p.err = err;
  int S = splits < 1 ? 1 : splits;
  int kps = (K + S - 1) / S;
  kps = (kps + KC - 1) / KC * KC;
  if (kps < KC) kps = KC;
  S = (K + kps - 1) / kps;
  if (S < 1) S = 1;
  const bool split = S > 1;
  if (split && (epi != kTgStore || !ws || (size_t)S * M * N > ws_floats)) return cudaErrorInvalidValue;
  p.kps = kps;
  p.C = split ? ws : C;
  p.cstride = (int64_t)M * N;
  cudaError_t e;
  if (N <= 16) {
    switch (epi) {
      case kTgStore: e = launch_bn<16, kTgStore>(st, p, S); break;
      case kTgBias: e = launch_bn<16, kTgBias>(st, p, S); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (epi) {
      case kTgStore: e = launch_bn<256, kTgStore>(st, p, S); break;
      case kTgBiasSilu: e = launch_bn<256, kTgBiasSilu>(st, p, S); break;
      case kTgDSilu: e = launch_bn<256, kTgDSilu>(st, p, S); break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess || !split) return e;
  const int64_t n = (int64_t)M * N;
  splitk_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, S, ws, C);
  return cudaGetLastError();
}

}  // namespace gmc
