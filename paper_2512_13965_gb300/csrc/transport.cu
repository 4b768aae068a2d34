// Transport solve (placeholder until the event loop lands).
#include "gmc_internal.cuh"

extern "C" gmc_status transport_solve(gmc_ctx *ctx, int, int, const float *, const float *,
                                      const float *, int64_t, int, uint64_t, double *,
                                      gmc_solve_stats *) {
  return gmc::set_error(ctx, GMC_ENOTIMPL, "transport_solve: not built");
}
