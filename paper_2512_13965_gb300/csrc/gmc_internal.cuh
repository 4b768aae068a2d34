// Internal declarations shared by the translation units of libgmc.so.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/gmc.h"
#include "ptr_kind.h"

namespace gmc {

constexpr int kCond = 5, kState = 4, kEmb = 16, kIn = kCond + kState + kEmb, kHidden = 256;
// a network for rectangular cells has a sixth condition component, the
// aspect ln(tau_y / tau_x), as input column kIn (after the time embedding)
constexpr int kCondRect = kCond + 1;
constexpr int kIn1Pad = 32;  // layer-1 input padded to 32 columns
constexpr int kMaxDevices = 64;  // per-device launch caches (attributes, occupancy)
constexpr float kSMin = 1e-7f;

// FP32 network, transposed for the SIMT path: w1t [32][256] (rows 25..31
// zero), w2t..w4t [256][256] with wt[k][c] = W[c][k]; w5 [4][256] as in the
// file; biases as in the file. The residual-modulated network (rm = 1) also
// has mt [3][5][256] (mt[j][k][c] = M_j[c][k], the condition shift of hidden
// layer j + 2) and gg [3][2][256] (its channel scales G_j).
struct NetF32 {
  const float *w1t, *b1, *w2t, *b2, *w3t, *b3, *w4t, *b4, *w5, *b5;
  const float *mt, *gg;
  int rm;
};
constexpr uint32_t kFlagRM = 1u;  // weight-file flag of the residual-modulated network

// Standardization of the file: cond_mean[ncond], cond_std[ncond], y_mean[4],
// y_std[4]; ncond = 5, or 6 for a network of rectangular cells (entries past
// ncond are 0 and 1).
struct NetStats {
  float cond_mean[kCondRect], cond_inv_std[kCondRect], y_mean[kState], y_std[kState];
  int ncond;
  int disk;  // exits decoded for x-y geometry (direction projected on the unit disk)
};

// Packed operands of the tensor-core path (built by sampler_tc.cu).
struct NetTC;
// Training state (train.cu).
struct TrainState;
void train_state_free(TrainState *t);
// Wave engine of transport_solve and the serving thread (transport.cu).
class Engine;
struct Server;
void engine_free(Engine *e);
void server_free(Server *s);

struct Buffer {
  void *ptr = nullptr;
  size_t bytes = 0;
};

// One loaded velocity network: host copy of the file's layers, the FP32
// transposed block of the SIMT path, and the packed BF16 and FP8 operands of
// the tensor-core path.
struct NetDev {
  bool loaded = false;
  bool rm = false;  // residual-modulated network (weight-file flag 1)
  int nin = kIn;    // layer-1 inputs: 25, or 26 for rectangular cells
  uint64_t generation = 0;  // counts loads: cached per-network data keys on it
  float host_w[5][256 * 256];  // W_l[out][in] as in the file (unused tail for small layers)
  float host_b[5][256];
  float host_m[3][256 * kCond];  // M_j[c][k] (rm only)
  float host_g[3][2 * 256];      // G_j[0..1][c] (rm only)
  NetStats stats{};
  float *d_f32 = nullptr;  // FP32 transposed block
  NetF32 f32{};
  void *d_tc = nullptr;  // packed BF16 operands
  size_t tc_bytes = 0;
  float *d_tc_bias = nullptr;    // per-layer biases for the tensor-core path
  void *d_tc8 = nullptr;         // packed operands of the FP8 variant (E4M3 W2..W4)
  float *d_tc8_scale = nullptr;  // [3][256] per-output-channel scales of W2..W4, halved
};

}  // namespace gmc

struct gmc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  std::string last_error;
  mutable std::mutex err_mu;  // last_error is also written by the serving thread
  gmc_config cfg{};

  // networks: the boundary model (cell transmissions, gmc_load_weights) and
  // the internal model (births inside a source cell, gmc_load_internal_weights)
  gmc::NetDev net;
  gmc::NetDev internal;
  // the boundary model of x-y geometry (gmc_load_xy_weights, gmc_transmit_xy)
  gmc::NetDev xy;
  // the internal model of x-y geometry (gmc_load_internal_xy_weights): births
  // of x-y GMC solves
  gmc::NetDev internal_xy;
  int *d_err = nullptr;  // device error word (bounded waits)

  // training state (gmc_train_begin .. gmc_destroy)
  gmc::TrainState *train = nullptr;

  // staging buffers for host-pointer calls
  gmc::Buffer stage[9];
  // per-evaluation layer-1 bias of the tensor-core sampler
  gmc::Buffer bias1;
  // work counter of the persistent random-walk kernel (8 bytes)
  gmc::Buffer walk_next;
  // transport_solve engine (kept between calls) and the serving thread
  gmc::Engine *solver = nullptr;
  gmc::Server *server = nullptr;
};

namespace gmc {

gmc_status set_error(gmc_ctx *ctx, gmc_status s, const char *fmt, ...);
// GMC_EINVAL (context error naming `who`) when network N cannot run on the
// sampler path of `precision` and `kernel`: the residual-modulated network has
// the FP32 and the BF16 one-CTA-per-SM tensor-core path only.
gmc_status check_net_path(gmc_ctx *ctx, const NetDev &N, int precision, int kernel, const char *who);
gmc_status cuda_error(gmc_ctx *ctx, cudaError_t e, const char *what);
// Device memory of GPU ctx_device, or managed memory (not another GPU's memory).
bool is_device_pointer(const void *p, int ctx_device);
PtrKind pointer_kind(const void *p, int ctx_device);
// Reads and clears the device error word (set by bounded waits that gave up).
gmc_status check_device_error(gmc_ctx *ctx);
// Grows buffer `b` to at least `bytes` (never shrinks).
cudaError_t ensure(Buffer &b, size_t bytes);

#define GMC_CUDA_TRY(ctx, expr)                                   \
  do {                                                            \
    cudaError_t e__ = (expr);                                     \
    if (e__ != cudaSuccess) return ::gmc::cuda_error(ctx, e__, #expr); \
  } while (0)

// Blocks of a persistent launch of `kernel` with `threads` threads per block
// and no dynamic shared memory: as many as are resident on the current device
// at once (occupancy queried once per device and kernel), at most
// ceil(items / threads).
template <typename Kernel>
unsigned persistent_blocks(Kernel kernel, int threads, int64_t items) {
  static std::atomic<int> cached[kMaxDevices];
  int dev = 0;
  cudaGetDevice(&dev);
  int fit = (dev >= 0 && dev < kMaxDevices) ? cached[dev].load(std::memory_order_relaxed) : 0;
  if (fit < 1) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    fit = per_sm * (sms > 0 ? sms : 1);
    if (dev >= 0 && dev < kMaxDevices) cached[dev].store(fit, std::memory_order_relaxed);
  }
  const int64_t need = (items + threads - 1) / threads;
  return (unsigned)(need < fit ? (need > 0 ? need : 1) : fit);
}

// Launchers implemented in the kernel translation units. All are
// asynchronous on `stream` and take device pointers only.
cudaError_t launch_philox(cudaStream_t stream, int64_t n, uint64_t seed, uint64_t id0,
                          uint32_t event, uint32_t tag, uint32_t *out);
cudaError_t launch_normals(cudaStream_t stream, int64_t n, uint64_t seed, uint64_t id0,
                           uint32_t event, uint32_t tag, float *out);
cudaError_t launch_sampler_f32(cudaStream_t stream, const NetF32 &net, const NetStats &st,
                               int64_t n, const float *cond, const float *noise, uint64_t seed,
                               uint64_t id0, int steps, int integrator, float *y_raw, float *exit);
// next: 8 bytes of device scratch (the persistent kernel's work counter),
// cleared by the launcher.
cudaError_t launch_analog(cudaStream_t stream, int64_t n, const float *xi, const float *cos_in,
                          const float *sin_in, const float *tau, const float *c, int mode,
                          uint64_t seed, uint64_t id0, uint32_t event0, int32_t *status,
                          float *exit, uint32_t *ncoll, unsigned long long *next);
cudaError_t launch_analog_rect(cudaStream_t stream, int64_t n, const float *xi, const float *cos_in,
                               const float *sin_in, const float *tx, const float *ty,
                               const float *c, int mode, uint64_t seed, uint64_t id0,
                               uint32_t event0, int32_t *status, float *exit, uint32_t *ncoll);
cudaError_t launch_analog_xy(cudaStream_t stream, int64_t n, const float *xi, const float *ux_in,
                             const float *uy_in, const float *tx, const float *ty, const float *c,
                             int mode, uint64_t seed, uint64_t id0, uint32_t event0,
                             int32_t *status, float *exit, uint32_t *ncoll);

// Tensor-core sampler (sampler_tc.cu). The BF16 and FP8 variants share the
// bias vector ([5][256]); the FP8 one also takes per-channel weight scales.
size_t tc_packed_bytes(bool fp8);
// M: the condition shifts of the residual-modulated network (null for the
// MLP), packed into the bias blocks of layers 2-4.
// nin: layer-1 inputs (25, or 26 with the aspect of rectangular cells);
// W[0] holds W1 as [256][nin].
void tc_pack_host(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                  float *bias_host, const float (*M)[256 * kCond] = nullptr, int nin = kIn);
void tc_pack_host_fp8(const float (*W)[256 * 256], const float (*b)[256], void *packed_host,
                      float *bias_host, float *scale_host, int nin = kIn);
// packed: from tc_pack_host (fp8_scale null) or tc_pack_host_fp8 (fp8_scale =
// its [3][256] scales on the device). kernel: gmc_sampler_kernel of the BF16
// path (GMC_KERNEL_PAIR: sampler_pair.cu). bias1_ready: bias1_scratch already
// holds this network's per-evaluation layer-1 bias for these steps and
// integrator, so its kernel is skipped. A residual-modulated network (f32.rm)
// runs on the BF16 tile kernel only (cudaErrorNotSupported otherwise).
cudaError_t launch_sampler_tc(cudaStream_t stream, const void *packed, const float *bias,
                              const NetF32 &f32, const NetStats &st, int64_t n, const float *cond,
                              const float *noise, uint64_t seed, uint64_t id0, int steps,
                              int integrator, float *y_raw, float *exit, int *err,
                              float *bias1_scratch, const float *fp8_scale,
                              int kernel = GMC_KERNEL_TILE, bool bias1_ready = false);

}  // namespace gmc
