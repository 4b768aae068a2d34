// transport_solve: the four-stage GMC transport algorithm (and the standard
// MC walk it replaces) as an event loop over waves of in-flight particles.
//
// Particle bank (structure of arrays, double-buffered, capacity C):
//   hist u64 (history id = Philox id), cell i32, face i32 (global face the
//   particle entered through), xi f32 (canonical entry position), gx, gy f32
//   (global direction), w f32 (weight), ev u32 (next Philox event).
// One wave:
//   births   new histories fill free slots: birth point and direction from
//            Philox (id, 0, tag 4), walked to the first face crossing of the
//            birth cell with implicit capture (the paper's separate
//            internal-source network is not built);
//   GMC      prep: rotate into the canonical left-entry frame (stage 1),
//            build the condition and draw z ~ N(0, I) at (id, ev, tag 2);
//            sampler: the fused flow-ODE kernel (stage 2);
//            post: attenuate and tally (stage 3, Eq. 5-7), rotate back,
//            roulette, cross into the neighbour, compact survivors (stage 4);
//   ANALOG   one kernel walks each particle through its cell (Eq. 4) and
//            does stages 3-4 the same way.
// Tally: FP64 atomics into flux[ny*nx]; Delta w / (V sigma_a) with V = 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "decode.cuh"
#include "gmc_internal.cuh"
#include "philox.cuh"
#include "walk.cuh"

namespace gmc {
namespace {

struct Bank {
  uint64_t *hist;
  int32_t *cell, *face;
  float *xi, *gx, *gy, *w;
  uint32_t *ev;
};

struct DevStats {
  double leaked, absorbed, roulette_net;
  unsigned long long transmissions, collisions, kills, inward;
};

struct Grid {
  int nx, ny;
  const float *tau, *c;
};

struct Rules {
  uint64_t seed;
  float w_cut, p_survive;
};

// rotate (ux, uy) by k quarter turns counter-clockwise
__device__ __forceinline__ void rot(float &ux, float &uy, int k) {
  const float a = ux, b = uy;
  switch (k & 3) {
    case 0: ux = a; uy = b; break;
    case 1: ux = -b; uy = a; break;
    case 2: ux = -a; uy = -b; break;
    default: ux = b; uy = -a; break;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Stage 3 and 4 for one finished cell transmission: deposit, attenuate,
// roulette, cross. Appends the survivor to `out` (warp-aggregated). Every
// lane of the warp must call this (inactive lanes with active = false).
struct Exit {
  bool active;
  uint64_t hist;
  int cell, gface;   // cell crossed, global exit face
  float q;           // counter-clockwise position on that face
  float gx, gy;      // global direction
  float w, s;        // weight on entry, track length (optical)
  uint32_t ev;       // next Philox event
  uint32_t ncoll;
  bool inward;
};

__device__ void finish_transmission(const Exit &x, const Grid &G, const Rules &R, double *flux,
                                    Bank out, int *out_count, DevStats *st) {
  double dabs = 0.0, dleak = 0.0, droul = 0.0;
  unsigned long long kills = 0;
  bool keep = false;
  int ncell = 0, nface = 0;
  float w = 0.0f;
  if (x.active) {
    const float tau = G.tau[x.cell], cc = G.c[x.cell];
    const float a = 1.0f - cc;
    float dw;
    double score;
    if (a > 0.0f) {
      dw = x.w * (-expm1f(-a * x.s));                       // Eq. 6
      score = (double)dw / ((double)a * (double)tau);       // Eq. 7
    } else {
      dw = 0.0f;
      score = (double)x.w * (double)x.s / (double)tau;
    }
    atomicAdd(&flux[x.cell], score);
    dabs = dw;
    w = x.w - dw;                                           // Eq. 5
    bool alive = true;
    if (w < R.w_cut) {
      const float u = u01(philox_draw(R.seed, x.hist, x.ev, kTagRoulette).x);
      if (u <= R.p_survive) {
        droul = (double)(w / R.p_survive) - (double)w;
        w = w / R.p_survive;
      } else {
        droul = -(double)w;
        kills = 1;
        alive = false;
      }
    }
    if (alive) {
      const int i = x.cell % G.nx, j = x.cell / G.nx;
      const int ni = i + (x.gface == 1) - (x.gface == 3);
      const int nj = j + (x.gface == 2) - (x.gface == 0);
      if (ni < 0 || ni >= G.nx || nj < 0 || nj >= G.ny) {
        dleak = w;
      } else {
        keep = true;
        ncell = nj * G.nx + ni;
        nface = (x.gface + 2) & 3;
      }
    }
  }
  // warp-aggregated append of survivors
  const unsigned mask = __ballot_sync(0xffffffffu, keep);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && mask) base = atomicAdd(out_count, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (keep) {
    const int k = base + __popc(mask & ((1u << lane) - 1u));
    out.hist[k] = x.hist;
    out.cell[k] = ncell;
    out.face[k] = nface;
    out.xi[k] = x.q;
    out.gx[k] = x.gx;
    out.gy[k] = x.gy;
    out.w[k] = w;
    out.ev[k] = x.ev;
  }
  // warp-reduced statistics
  dabs = warp_sum(dabs);
  dleak = warp_sum(dleak);
  droul = warp_sum(droul);
  const unsigned long long nt = warp_sum_u(x.active ? 1ull : 0ull);
  const unsigned long long nc = warp_sum_u(x.active ? (unsigned long long)x.ncoll : 0ull);
  const unsigned long long nk = warp_sum_u(kills);
  const unsigned long long ni = warp_sum_u(x.active && x.inward ? 1ull : 0ull);
  if (lane == 0 && nt) {
    atomicAdd(&st->absorbed, dabs);
    atomicAdd(&st->leaked, dleak);
    atomicAdd(&st->roulette_net, droul);
    atomicAdd(&st->transmissions, nt);
    atomicAdd(&st->collisions, nc);
    atomicAdd(&st->kills, nk);
    atomicAdd(&st->inward, ni);
  }
}

__device__ __forceinline__ int64_t cdf_search(const double *cdf, int64_t n, double target) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (cdf[mid] >= target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Births of histories first .. first+count-1.
__global__ void birth_kernel(int64_t first, int64_t count, const double *__restrict__ cdf,
                             double total, Grid G, Rules R, double *flux, Bank out,
                             int *out_count, DevStats *st) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Exit x;
  x.active = k < count;
  x.inward = false;
  if (x.active) {
    const uint64_t h = (uint64_t)(first + k);
    const uint4 r = philox_draw(R.seed, h, 0u, kTagBirth);
    const double u0 = ((double)r.x + 1.0) * (1.0 / 4294967296.0);
    const int64_t cell = cdf_search(cdf, (int64_t)G.nx * G.ny, u0 * total);
    float ux, uy;
    sincospif(2.0f * u01(r.w), &uy, &ux);
    const float tau = G.tau[cell], cc = G.c[cell];
    const WalkResult wr = walk_cell(tau, cc, 1, u01(r.y), u01(r.z), ux, uy, R.seed, h, 0u);
    x.hist = h;
    x.cell = (int)cell;
    x.gface = wr.face < 0 ? 0 : wr.face;
    x.q = wr.q;
    x.gx = wr.ux;
    x.gy = wr.uy;
    x.w = 1.0f;
    x.s = wr.s;
    x.ev = wr.event;
    x.ncoll = wr.ncoll;
  }
  finish_transmission(x, G, R, flux, out, out_count, st);
}

// ANALOG: walk each bank particle through its cell in the cell's own
// (global-oriented) frame, entering at the point its entry face and xi give.
__global__ void analog_wave_kernel(int64_t live, Bank in, Grid G, Rules R, double *flux, Bank out,
                                   int *out_count, DevStats *st) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Exit x;
  x.active = k < live;
  x.inward = false;
  if (x.active) {
    const int cell = in.cell[k], F = in.face[k];
    const float xi = in.xi[k];
    // point on face F with counter-clockwise parameter 1 - xi
    float X, Y;
    switch (F) {
      case 0: X = 1.0f - xi; Y = 0.0f; break;
      case 1: X = 1.0f; Y = 1.0f - xi; break;
      case 2: X = xi; Y = 1.0f; break;
      default: X = 0.0f; Y = xi; break;
    }
    const uint64_t h = in.hist[k];
    const WalkResult wr = walk_cell(G.tau[cell], G.c[cell], 1, X, Y, in.gx[k], in.gy[k], R.seed, h,
                                    in.ev[k]);
    x.hist = h;
    x.cell = cell;
    x.gface = wr.face < 0 ? 0 : wr.face;
    x.q = wr.q;
    x.gx = wr.ux;
    x.gy = wr.uy;
    x.w = in.w[k];
    x.s = wr.s;
    x.ev = wr.event;
    x.ncoll = wr.ncoll;
  }
  finish_transmission(x, G, R, flux, out, out_count, st);
}

// GMC stage 1 and the noise of stage 2.
__global__ void gmc_prep_kernel(int64_t live, Bank in, Grid G, uint64_t seed, float *cond,
                                float *noise) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= live) return;
  const int cell = in.cell[k], F = in.face[k];
  float ux = in.gx[k], uy = in.gy[k];
  rot(ux, uy, -((F + 1) & 3));
  cond[k] = in.xi[k];
  cond[live + k] = ux;
  cond[2 * live + k] = uy;
  cond[3 * live + k] = logf(G.tau[cell]);
  cond[4 * live + k] = G.c[cell];
  const float4 z = box_muller4(philox_draw(seed, in.hist[k], in.ev[k], kTagNoise));
  noise[k] = z.x;
  noise[live + k] = z.y;
  noise[2 * live + k] = z.z;
  noise[3 * live + k] = z.w;
}

// GMC stages 3 and 4 from the sampler's decoded exits (p, ux, uy, s).
__global__ void gmc_post_kernel(int64_t live, Bank in, const float *__restrict__ ex, Grid G,
                                Rules R, double *flux, Bank out, int *out_count, DevStats *st) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Exit x;
  x.active = k < live;
  x.inward = false;
  if (x.active) {
    const int F = in.face[k], r = (F + 1) & 3;
    const float p = ex[k];
    float ux = ex[live + k], uy = ex[2 * live + k];
    const int fc = min((int)p, 3);
    x.hist = in.hist[k];
    x.cell = in.cell[k];
    x.gface = (fc + r) & 3;
    x.q = fminf(fmaxf(p - (float)fc, 0.0f), 1.0f);
    // the sampler reflected inward directions; count them for the statistics
    rot(ux, uy, r);
    x.gx = ux;
    x.gy = uy;
    x.w = in.w[k];
    x.s = ex[3 * live + k];
    x.ev = in.ev[k] + 1u;
    x.ncoll = 0;
  }
  finish_transmission(x, G, R, flux, out, out_count, st);
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

Bank carve(void *base, int64_t C) {
  Bank b;
  char *p = (char *)base;
  b.hist = (uint64_t *)p; p += 8 * C;
  b.cell = (int32_t *)p; p += 4 * C;
  b.face = (int32_t *)p; p += 4 * C;
  b.xi = (float *)p; p += 4 * C;
  b.gx = (float *)p; p += 4 * C;
  b.gy = (float *)p; p += 4 * C;
  b.w = (float *)p; p += 4 * C;
  b.ev = (uint32_t *)p;
  return b;
}

constexpr size_t kBankBytesPerParticle = 36;

}  // namespace
}  // namespace gmc

using namespace gmc;

extern "C" gmc_status transport_solve(gmc_ctx *ctx, int nx, int ny, const float *tau,
                                      const float *c, const float *source, int64_t n_histories,
                                      int method, uint64_t seed, double *flux,
                                      gmc_solve_stats *stats) {
  if (!ctx) return GMC_EINVAL;
  if (nx < 1 || ny < 1 || (int64_t)nx * ny > (1 << 26))
    return set_error(ctx, GMC_EINVAL, "transport_solve: grid must be 1..2^26 cells");
  if (!tau || !c || !source || !flux) return set_error(ctx, GMC_EINVAL, "transport_solve: null array");
  if (n_histories < 0) return set_error(ctx, GMC_EINVAL, "transport_solve: n_histories < 0");
  if (method != GMC_METHOD_ANALOG && method != GMC_METHOD_GMC)
    return set_error(ctx, GMC_EINVAL, "transport_solve: unknown method");
  const int64_t ncell = (int64_t)nx * ny;
  std::vector<double> cdf(ncell);
  double acc = 0.0;
  for (int64_t k = 0; k < ncell; ++k) {
    if (!(tau[k] > 0.0f) || !std::isfinite(tau[k]) || !(c[k] >= 0.0f && c[k] <= 1.0f))
      return set_error(ctx, GMC_EINVAL, "transport_solve: cell %lld needs tau > 0, c in [0,1]",
                       (long long)k);
    if (method == GMC_METHOD_GMC && (tau[k] < 0.05f || tau[k] > 2000.0f || c[k] < 0.4f))
      return set_error(ctx, GMC_EINVAL,
                       "transport_solve: cell %lld outside the sampler's range (tau in [0.05, 2000], c >= 0.4)",
                       (long long)k);
    if (!(source[k] >= 0.0f) || !std::isfinite(source[k]))
      return set_error(ctx, GMC_EINVAL, "transport_solve: source must be finite and >= 0");
    acc += source[k] > 0.0f ? (double)source[k] : 0.0;
    cdf[k] = acc;
  }
  if (n_histories > 0 && !(acc > 0.0)) return set_error(ctx, GMC_EINVAL, "transport_solve: zero source");
  if (method == GMC_METHOD_GMC && !ctx->has_weights)
    return set_error(ctx, GMC_ENOWEIGHTS, "transport_solve: GMC needs gmc_load_weights");
  const gmc_config cfg = ctx->cfg;
  if (method == GMC_METHOD_GMC && cfg.precision == GMC_FP8)
    return set_error(ctx, GMC_ENOTIMPL, "transport_solve: FP8 sampler not built");
  const int64_t C = cfg.bank_capacity;

  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  // scratch: grid (tau, c), cdf, flux, stats+counters, two banks, cond, noise, exits
  GMC_CUDA_TRY(ctx, ensure(ctx->solve[0], (size_t)ncell * 8));
  GMC_CUDA_TRY(ctx, ensure(ctx->solve[1], (size_t)ncell * 8));
  GMC_CUDA_TRY(ctx, ensure(ctx->solve[2], (size_t)ncell * 8));
  GMC_CUDA_TRY(ctx, ensure(ctx->solve[3], sizeof(DevStats) + 64));
  GMC_CUDA_TRY(ctx, ensure(ctx->solve[4], (size_t)C * kBankBytesPerParticle));
  GMC_CUDA_TRY(ctx, ensure(ctx->solve[5], (size_t)C * kBankBytesPerParticle));
  if (method == GMC_METHOD_GMC) {
    GMC_CUDA_TRY(ctx, ensure(ctx->solve[6], (size_t)C * 5 * 4));
    GMC_CUDA_TRY(ctx, ensure(ctx->solve[7], (size_t)C * 4 * 4));
    GMC_CUDA_TRY(ctx, ensure(ctx->solve[8], (size_t)C * 4 * 4));
    GMC_CUDA_TRY(ctx, ensure(ctx->bias1, (size_t)2 * cfg.steps * 256 * sizeof(float)));
  }
  float *d_tau = (float *)ctx->solve[0].ptr;
  float *d_c = d_tau + ncell;
  double *d_cdf = (double *)ctx->solve[1].ptr;
  double *d_flux = (double *)ctx->solve[2].ptr;
  DevStats *d_st = (DevStats *)ctx->solve[3].ptr;
  int *d_count = (int *)((char *)ctx->solve[3].ptr + sizeof(DevStats) + 16);
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(d_tau, tau, ncell * 4, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(d_c, c, ncell * 4, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(d_cdf, cdf.data(), ncell * 8, cudaMemcpyHostToDevice, s));
  GMC_CUDA_TRY(ctx, cudaMemsetAsync(d_flux, 0, ncell * 8, s));
  GMC_CUDA_TRY(ctx, cudaMemsetAsync(d_st, 0, sizeof(DevStats) + 64, s));

  Grid G{nx, ny, d_tau, d_c};
  Rules R{seed, (float)cfg.w_cut, (float)cfg.p_survive};
  Bank bank[2] = {carve(ctx->solve[4].ptr, C), carve(ctx->solve[5].ptr, C)};
  int cur = 0;
  int64_t live = 0, next_hist = 0, waves = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  int h_count = 0;
  for (;;) {
    // births into the free slots of the current bank
    const int64_t room = C - live;
    const int64_t m = std::min(room, n_histories - next_hist);
    if (m > 0) {
      GMC_CUDA_TRY(ctx, cudaMemcpyAsync(d_count, &live, 4, cudaMemcpyHostToDevice, s));
      birth_kernel<<<nblocks(m, 256), 256, 0, s>>>(next_hist, m, d_cdf, acc, G, R, d_flux,
                                                   bank[cur], d_count, d_st);
      GMC_CUDA_TRY(ctx, cudaGetLastError());
      GMC_CUDA_TRY(ctx, cudaMemcpyAsync(&h_count, d_count, 4, cudaMemcpyDeviceToHost, s));
      GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
      next_hist += m;
      live = h_count;
    }
    if (live == 0) {
      if (next_hist >= n_histories) break;
      continue;
    }
    ++waves;
    GMC_CUDA_TRY(ctx, cudaMemsetAsync(d_count, 0, 4, s));
    const int nxt = cur ^ 1;
    if (method == GMC_METHOD_ANALOG) {
      analog_wave_kernel<<<nblocks(live, 128), 128, 0, s>>>(live, bank[cur], G, R, d_flux, bank[nxt],
                                                           d_count, d_st);
      GMC_CUDA_TRY(ctx, cudaGetLastError());
    } else {
      float *d_cond = (float *)ctx->solve[6].ptr;
      float *d_noise = (float *)ctx->solve[7].ptr;
      float *d_exit = (float *)ctx->solve[8].ptr;
      gmc_prep_kernel<<<nblocks(live, 256), 256, 0, s>>>(live, bank[cur], G, seed, d_cond, d_noise);
      GMC_CUDA_TRY(ctx, cudaGetLastError());
      cudaError_t e;
      if (cfg.precision == GMC_FP32)
        e = launch_sampler_f32(s, ctx->f32, ctx->stats, live, d_cond, d_noise, seed, 0, cfg.steps,
                               cfg.integrator, nullptr, d_exit);
      else
        e = launch_sampler_tc(s, ctx->d_tc, ctx->d_tc_bias, ctx->f32, ctx->stats, live, d_cond,
                              d_noise, seed, 0, cfg.steps, cfg.integrator, nullptr, d_exit,
                              ctx->d_err, (float *)ctx->bias1.ptr);
      if (e != cudaSuccess) return cuda_error(ctx, e, "transport_solve sampler");
      gmc_post_kernel<<<nblocks(live, 256), 256, 0, s>>>(live, bank[cur], d_exit, G, R, d_flux,
                                                         bank[nxt], d_count, d_st);
      GMC_CUDA_TRY(ctx, cudaGetLastError());
    }
    GMC_CUDA_TRY(ctx, cudaMemcpyAsync(&h_count, d_count, 4, cudaMemcpyDeviceToHost, s));
    GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    live = h_count;
    cur = nxt;
    if (method == GMC_METHOD_GMC) {
      gmc_status es = check_device_error(ctx);
      if (es != GMC_OK) return es;
    }
  }
  cudaEventRecord(e1, s);
  std::vector<double> hf(ncell);
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(hf.data(), d_flux, ncell * 8, cudaMemcpyDeviceToHost, s));
  DevStats hs;
  GMC_CUDA_TRY(ctx, cudaMemcpyAsync(&hs, d_st, sizeof(hs), cudaMemcpyDeviceToHost, s));
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double inv = n_histories > 0 ? 1.0 / (double)n_histories : 0.0;
  for (int64_t k = 0; k < ncell; ++k) flux[k] = hf[k] * inv;
  if (stats) {
    stats->leaked = hs.leaked;
    stats->absorbed = hs.absorbed;
    stats->roulette_net = hs.roulette_net;
    stats->transmissions = (int64_t)hs.transmissions;
    stats->collisions = (int64_t)hs.collisions;
    stats->roulette_kills = (int64_t)hs.kills;
    stats->waves = waves;
    stats->inward_fixes = (int64_t)hs.inward;
    stats->seconds = ms * 1e-3;
  }
  return check_device_error(ctx);
}
