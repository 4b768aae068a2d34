// gmc_transmit_noalloc: the BF16 tensor-core sampler for callers that must
// not allocate device memory during the call.
//
// Who needs it: code that runs under a framework owning the device allocator
// (a caching or pooled allocator that must see every allocation), code that
// records work into CUDA graphs or runs in a latency-critical loop where a
// cudaMalloc would synchronize the device or fail under memory pressure, and
// embedded or real-time hosts that only allow allocation at start-up. Such
// callers create the context and load weights once at start-up; after that,
// this entry point touches only memory that already exists.
//
// The only scratch the sampler needs beyond its inputs and outputs is the
// per-evaluation layer-1 bias table (W1[:, emb] emb(t_e) + b1, FP32,
// 256 floats per network evaluation). Here it lives in a file-scope device
// array sized for 512 evaluations (256 Euler or midpoint steps, 128 RK4
// steps), 512 KiB, which every GPU that loads the library holds until the process
// exits. All calls on a device share that one array: two calls whose
// kernels overlap on the GPU (different streams, or different host threads)
// race on it and must be serialized by the caller. Each call rewrites every
// row it reads, so nothing has to be cleared between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "gmc_internal.cuh"

namespace gmc {
namespace {

constexpr int kNoallocMaxEvals = 512;
constexpr int kNoallocMaxSteps = 256;
constexpr int kMaxDevices = 64;

// Device scratch. In host code `g_noalloc_bias1` names a host-side shadow
// symbol, not a device address: a kernel handed it directly would fault or
// silently use the wrong memory, so host code passes the address that
// cudaGetSymbolAddress returns for the current device instead.
__device__ __align__(256) float g_noalloc_bias1[kNoallocMaxEvals * kHidden];

std::mutex g_mu;
float *g_addr[kMaxDevices] = {};

// Once per device, with that device current: resolve the array's device
// address. The first call on a device does this (it may also load the
// library's device code), so make that first call before any stream capture.
gmc_status scratch_address(gmc_ctx *ctx, float **out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return set_error(ctx, GMC_EINVAL, "gmc_transmit_noalloc: device index %d not supported", ctx->device);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[ctx->device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_bias1);
    if (e != cudaSuccess) return cuda_error(ctx, e, "cudaGetSymbolAddress(g_noalloc_bias1)");
    g_addr[ctx->device] = (float *)p;
  }
  *out = g_addr[ctx->device];
  return GMC_OK;
}

}  // namespace
}  // namespace gmc

using namespace gmc;

extern "C" gmc_status gmc_transmit_noalloc(gmc_ctx *ctx, int64_t n, const float *cond,
                                           const float *noise, uint64_t seed, uint64_t id0,
                                           int steps, int integrator, float *y_raw, float *exit) {
  if (!ctx) return GMC_EINVAL;
  if (n < 0) return set_error(ctx, GMC_EINVAL, "gmc_transmit_noalloc: n < 0");
  if (integrator != GMC_EULER && integrator != GMC_MIDPOINT && integrator != GMC_RK4)
    return set_error(ctx, GMC_EINVAL, "gmc_transmit_noalloc: unknown integrator");
  const int evals_per_step = integrator == GMC_RK4 ? 4 : (integrator == GMC_MIDPOINT ? 2 : 1);
  const int max_steps = integrator == GMC_RK4 ? kNoallocMaxEvals / 4 : kNoallocMaxSteps;
  if (steps < 1 || steps > max_steps)
    return set_error(ctx, GMC_EINVAL,
                     "gmc_transmit_noalloc: steps must be in [1, %d] for this integrator (the "
                     "static scratch holds %d layer-1 bias rows, %d per step), got %d",
                     max_steps, kNoallocMaxEvals, evals_per_step, steps);
  if (!ctx->net.loaded || !ctx->net.d_tc)
    return set_error(ctx, GMC_ENOWEIGHTS, "gmc_transmit_noalloc: no weights loaded");
  if (check_net_path(ctx, ctx->net, GMC_BF16, ctx->cfg.sampler_kernel, "gmc_transmit_noalloc") != GMC_OK)
    return GMC_EINVAL;
  if (ctx->net.stats.ncond != kCond)
    return set_error(ctx, GMC_EINVAL, "gmc_transmit_noalloc: takes [5][n] conditions (not a "
                                      "rectangular-cell network)");
  if (n == 0) return GMC_OK;
  if (!cond || (!y_raw && !exit)) return set_error(ctx, GMC_EINVAL, "gmc_transmit_noalloc: null array");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(ctx, e, "cudaSetDevice");
  // host pointers would need staging buffers: only device memory of the
  // context's GPU (or managed memory) is accepted
  if (!is_device_pointer(cond, ctx->device) || (noise && !is_device_pointer(noise, ctx->device)) ||
      (y_raw && !is_device_pointer(y_raw, ctx->device)) || (exit && !is_device_pointer(exit, ctx->device)))
    return set_error(ctx, GMC_EINVAL, "gmc_transmit_noalloc: every array must be device memory of the context's GPU");
  float *scratch = nullptr;
  gmc_status st = scratch_address(ctx, &scratch);
  if (st != GMC_OK) return st;
  e = launch_sampler_tc(ctx->stream, ctx->net.d_tc, ctx->net.d_tc_bias, ctx->net.f32, ctx->net.stats, n, cond,
                        noise, seed, id0, steps, integrator, y_raw, exit, ctx->d_err, scratch,
                        nullptr, ctx->cfg.sampler_kernel);
  if (e != cudaSuccess) return cuda_error(ctx, e, "gmc_transmit_noalloc launch");
  return GMC_OK;
}
