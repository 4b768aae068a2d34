// Batched kernels: raw Philox blocks, Box-Muller normals, and the analog
// random-walk cell transmission (one thread per particle).
#include "gmc_internal.cuh"
#include "philox.cuh"
#include "walk.cuh"

namespace gmc {
namespace {

__global__ void philox_kernel(int64_t n, uint64_t seed, uint64_t id0, uint32_t event, uint32_t tag,
                              uint4 *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox_draw(seed, id0 + (uint64_t)i, event, tag);
}

__global__ void normals_kernel(int64_t n, uint64_t seed, uint64_t id0, uint32_t event,
                               uint32_t tag, float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 z = box_muller4(philox_draw(seed, id0 + (uint64_t)i, event, tag));
  out[i] = z.x;
  out[n + i] = z.y;
  out[2 * n + i] = z.z;
  out[3 * n + i] = z.w;
}

// One walk per particle, entering the left face at y = xi tau; persistent,
// with lane refill (walk.cuh): lanes claim particles from *next.
constexpr int kAnalogThreads = 256;

__global__ void __launch_bounds__(kAnalogThreads) analog_kernel(
    int64_t n, const float *__restrict__ xi, const float *__restrict__ cos_in,
    const float *__restrict__ sin_in, const float *__restrict__ tau, const float *__restrict__ c,
    int mode, uint64_t seed, uint64_t id0, uint32_t event0, int32_t *__restrict__ status,
    float *__restrict__ exitp, uint32_t *__restrict__ ncoll, unsigned long long *next) {
  const int implicit = mode == GMC_ABSORB_IMPLICIT;
  int64_t i = n;  // this lane's particle (n: none)
  bool drained = false;
  WalkState ws{};
  float t = 0.0f, cc = 0.0f;
  for (;;) {
    const bool need = i == n && !drained;
    if (__any_sync(0xffffffffu, need)) {
      const int64_t k = warp_claim(need, next, n);
      if (need) {
        if (k < n) {
          i = k;
          t = tau[i];
          cc = c[i];
          ws = walk_start(t, 0.0f, xi[i], cos_in[i], sin_in[i], event0);
        } else {
          drained = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, i < n)) break;
    if (i < n) {
      const WalkResult w = walk_cell_resume(t, cc, implicit, ws, kWalkRound, seed, id0 + (uint64_t)i);
      if (w.status != kTruncated || ws.ncoll >= kMaxFlights) {
        status[i] = w.status;
        exitp[i] = w.status == kExited ? (float)w.face + w.q : -1.0f;
        exitp[n + i] = w.ux;
        exitp[2 * n + i] = w.uy;
        exitp[3 * n + i] = w.s;
        if (ncoll) ncoll[i] = w.ncoll;
        i = n;
      }
    }
  }
}

// Rectangular cells: entry on the left face at y = xi * ty.
__global__ void analog_rect_kernel(int64_t n, const float *__restrict__ xi,
                                   const float *__restrict__ cos_in,
                                   const float *__restrict__ sin_in, const float *__restrict__ tx,
                                   const float *__restrict__ ty, const float *__restrict__ c,
                                   int mode, uint64_t seed, uint64_t id0, uint32_t event0,
                                   int32_t *__restrict__ status, float *__restrict__ exitp,
                                   uint32_t *__restrict__ ncoll) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int implicit = mode == GMC_ABSORB_IMPLICIT;
  const float a = tx[i], b = ty[i];
  const WalkResult w =
      fmaxf(a, b) > kTau64
          ? walk_rect<double>((double)a, (double)b, c[i], implicit, 0.0, (double)xi[i] * b,
                              cos_in[i], sin_in[i], seed, id0 + (uint64_t)i, event0)
          : walk_rect<float>(a, b, c[i], implicit, 0.0f, xi[i] * b, cos_in[i], sin_in[i], seed,
                             id0 + (uint64_t)i, event0);
  status[i] = w.status;
  exitp[i] = w.status == kExited ? (float)w.face + w.q : -1.0f;
  exitp[n + i] = w.ux;
  exitp[2 * n + i] = w.uy;
  exitp[3 * n + i] = w.s;
  if (ncoll) ncoll[i] = w.ncoll;
}

// x-y geometry: entry on the left face at y = xi * ty with the projected
// direction (ux_in, uy_in); exits report the projected direction.
__global__ void analog_xy_kernel(int64_t n, const float *__restrict__ xi,
                                 const float *__restrict__ ux_in, const float *__restrict__ uy_in,
                                 const float *__restrict__ tx, const float *__restrict__ ty,
                                 const float *__restrict__ c, int mode, uint64_t seed,
                                 uint64_t id0, uint32_t event0, int32_t *__restrict__ status,
                                 float *__restrict__ exitp, uint32_t *__restrict__ ncoll) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int implicit = mode == GMC_ABSORB_IMPLICIT;
  const float a = tx[i], b = ty[i];
  const WalkResult w =
      fmaxf(a, b) > kTau64
          ? walk_xy<double>((double)a, (double)b, c[i], implicit, 0.0, (double)xi[i] * b,
                            ux_in[i], uy_in[i], seed, id0 + (uint64_t)i, event0)
          : walk_xy<float>(a, b, c[i], implicit, 0.0f, xi[i] * b, ux_in[i], uy_in[i], seed,
                           id0 + (uint64_t)i, event0);
  status[i] = w.status;
  exitp[i] = w.status == kExited ? (float)w.face + w.q : -1.0f;
  exitp[n + i] = w.ux;
  exitp[2 * n + i] = w.uy;
  exitp[3 * n + i] = w.s;
  if (ncoll) ncoll[i] = w.ncoll;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_philox(cudaStream_t stream, int64_t n, uint64_t seed, uint64_t id0,
                          uint32_t event, uint32_t tag, uint32_t *out) {
  if (n <= 0) return cudaSuccess;
  philox_kernel<<<blocks_for(n, 256), 256, 0, stream>>>(n, seed, id0, event, tag,
                                                         reinterpret_cast<uint4 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_normals(cudaStream_t stream, int64_t n, uint64_t seed, uint64_t id0,
                           uint32_t event, uint32_t tag, float *out) {
  if (n <= 0) return cudaSuccess;
  normals_kernel<<<blocks_for(n, 256), 256, 0, stream>>>(n, seed, id0, event, tag, out);
  return cudaGetLastError();
}

cudaError_t launch_analog(cudaStream_t stream, int64_t n, const float *xi, const float *cos_in,
                          const float *sin_in, const float *tau, const float *c, int mode,
                          uint64_t seed, uint64_t id0, uint32_t event0, int32_t *status,
                          float *exit, uint32_t *ncoll, unsigned long long *next) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const unsigned grid = persistent_blocks(analog_kernel, kAnalogThreads, n);
  analog_kernel<<<grid, kAnalogThreads, 0, stream>>>(n, xi, cos_in, sin_in, tau, c, mode, seed,
                                                      id0, event0, status, exit, ncoll, next);
  return cudaGetLastError();
}

cudaError_t launch_analog_rect(cudaStream_t stream, int64_t n, const float *xi, const float *cos_in,
                               const float *sin_in, const float *tx, const float *ty,
                               const float *c, int mode, uint64_t seed, uint64_t id0,
                               uint32_t event0, int32_t *status, float *exit, uint32_t *ncoll) {
  if (n <= 0) return cudaSuccess;
  analog_rect_kernel<<<blocks_for(n, 128), 128, 0, stream>>>(n, xi, cos_in, sin_in, tx, ty, c, mode,
                                                              seed, id0, event0, status, exit,
                                                              ncoll);
  return cudaGetLastError();
}

cudaError_t launch_analog_xy(cudaStream_t stream, int64_t n, const float *xi, const float *ux_in,
                             const float *uy_in, const float *tx, const float *ty, const float *c,
                             int mode, uint64_t seed, uint64_t id0, uint32_t event0,
                             int32_t *status, float *exit, uint32_t *ncoll) {
  if (n <= 0) return cudaSuccess;
  analog_xy_kernel<<<blocks_for(n, 128), 128, 0, stream>>>(n, xi, ux_in, uy_in, tx, ty, c, mode,
                                                            seed, id0, event0, status, exit,
                                                            ncoll);
  return cudaGetLastError();
}

}  // namespace gmc
