// Tensor-core flow-ODE sampler (placeholder until the tcgen05 kernel lands).
#include "gmc_internal.cuh"

namespace gmc {
size_t tc_packed_bytes() { return 0; }
void tc_pack_host(const float (*)[256 * 256], const float (*)[256], void *, float *) {}
cudaError_t launch_sampler_tc(cudaStream_t, const void *, const float *, const NetStats &, int64_t,
                              const float *, const float *, uint64_t, uint64_t, int, int, float *,
                              float *, int *) {
  return cudaErrorNotSupported;
}
}  // namespace gmc
