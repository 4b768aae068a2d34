// gmc_selftest_wait: exercises the failure path of the bounded device waits
// without faulting anything. One thread initializes an mbarrier that nothing
// ever arrives at and waits on it with the same bounded wait the tensor-core
// kernels use; the wait gives up after the given time, sets the context's
// device error word and the kernel returns. The host then reads the word as
// every blocking call does (GMC_ETIMEOUT) and the context stays usable.
#include <cuda_runtime.h>

#include "gmc_internal.cuh"
#include "tc_ptx.cuh"

namespace gmc {
namespace {

__global__ void wait_never_kernel(int *err, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  ptx::mbar_init(&bar, 1);
  ptx::fence_mbar_init();
  int no_abort = 0;
  if (!ptx::mbar_wait(&bar, 0u, &no_abort, limit_ns)) atomicExch(err, 9);
}

}  // namespace
}  // namespace gmc

using namespace gmc;

extern "C" gmc_status gmc_selftest_wait(gmc_ctx *ctx, double limit_ms) {
  if (!ctx) return GMC_EINVAL;
  if (!(limit_ms > 0.0) || limit_ms > 2000.0)
    return set_error(ctx, GMC_EINVAL, "gmc_selftest_wait: limit_ms in (0, 2000]");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(ctx, e, "cudaSetDevice");
  wait_never_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_err, (uint64_t)(limit_ms * 1e6));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(ctx, e, "gmc_selftest_wait launch");
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_error(ctx, e, "gmc_selftest_wait");
  return check_device_error(ctx);
}
