// C ABI: contexts, errors, configuration, weight loading, and the batched
// entry points gmc_philox, gmc_normals, gmc_transmit and analog_transmit.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gmc_internal.cuh"
#include "gmcw.h"
#include "host_rules.h"

namespace gmc {

gmc_status set_error(gmc_ctx *ctx, gmc_status s, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    ctx->last_error = buf;
  }
  return s;
}

gmc_status cuda_error(gmc_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation)
    return set_error(ctx, GMC_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorInvalidDevicePointer)  // stage_in / stage_out_prepare: another GPU's memory
    return set_error(ctx, GMC_EINVAL, "%s: an array is device memory of another GPU than the "
                     "context's", what);
  return set_error(ctx, GMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

PtrKind pointer_kind(const void *p, int ctx_device) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kPtrHost;
  }
  return classify_pointer((int)a.type, a.device, ctx_device, a.devicePointer != nullptr);
}

bool is_device_pointer(const void *p, int ctx_device) {
  return p && pointer_kind(p, ctx_device) == kPtrDevice;
}

gmc_status check_device_error(gmc_ctx *ctx) {
  int h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpy(h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(ctx, e, "reading the device error word");
  if (h[0] != 0) {
    cudaMemset(ctx->d_err, 0, sizeof(h));
    return set_error(ctx, GMC_ETIMEOUT, "a bounded device wait gave up (code %d)", h[0]);
  }
  return GMC_OK;
}

cudaError_t ensure(Buffer &b, size_t bytes) {
  if (b.bytes >= bytes && b.ptr) return cudaSuccess;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
  size_t want = bytes < 256 ? 256 : bytes;
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e == cudaSuccess) b.bytes = want;
  return e;
}

namespace {

// One array argument of a batched call: device pointers pass through;
// page-locked host memory (cudaHostAlloc / cudaHostRegister) is read and
// written in place by the kernels over the CPU-GPU link (mapped); other host
// memory is staged through a context buffer (host).
struct Arg {
  const void *user = nullptr;
  void *dev = nullptr;
  size_t bytes = 0;
  bool host = false;
  bool mapped = false;
};

// Device address of page-locked host memory, or null for anything else.
void *mapped_host_pointer(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Device memory of the context's GPU and managed memory pass through,
// page-locked host memory is used in place; another GPU's memory is refused
// with cudaErrorInvalidDevicePointer (cuda_error turns it into GMC_EINVAL).
cudaError_t stage_direct(gmc_ctx *ctx, Arg &a, bool *done) {
  *done = true;
  switch (pointer_kind(a.user, ctx->device)) {
    case kPtrDevice: a.dev = const_cast<void *>(a.user); return cudaSuccess;
    case kPtrOtherDevice: return cudaErrorInvalidDevicePointer;
    case kPtrMappedHost:
      if (void *m = mapped_host_pointer(a.user)) {
        a.dev = m;
        a.mapped = true;
        return cudaSuccess;
      }
      break;
    case kPtrHost: break;
  }
  *done = false;
  return cudaSuccess;
}

cudaError_t stage_in(gmc_ctx *ctx, int slot, Arg &a) {
  if (!a.user) return cudaSuccess;
  bool done = false;
  cudaError_t d = stage_direct(ctx, a, &done);
  if (done) return d;
  a.host = true;
  cudaError_t e = ensure(ctx->stage[slot], a.bytes);
  if (e != cudaSuccess) return e;
  a.dev = ctx->stage[slot].ptr;
  return cudaMemcpyAsync(a.dev, a.user, a.bytes, cudaMemcpyHostToDevice, ctx->stream);
}

cudaError_t stage_out_prepare(gmc_ctx *ctx, int slot, Arg &a) {
  if (!a.user) return cudaSuccess;
  bool done = false;
  cudaError_t d = stage_direct(ctx, a, &done);
  if (done) return d;
  a.host = true;
  cudaError_t e = ensure(ctx->stage[slot], a.bytes);
  if (e != cudaSuccess) return e;
  a.dev = ctx->stage[slot].ptr;
  return cudaSuccess;
}

cudaError_t stage_out_finish(gmc_ctx *ctx, Arg &a) {
  if (!a.user || !a.host) return cudaSuccess;
  return cudaMemcpyAsync(const_cast<void *>(a.user), a.dev, a.bytes, cudaMemcpyDeviceToHost,
                         ctx->stream);
}

gmc_config default_config() {
  gmc_config c;
  c.steps = 16;
  c.integrator = GMC_EULER;
  c.precision = GMC_BF16;
  c.w_cut = 1e-4;
  c.p_survive = 0.1;
  c.bank_capacity = (int64_t)1 << 21;
  c.flights_per_wave = 512;
  c.gmc_min_tau = 0.0;
  c.net_tau_lo = 0.1;
  c.net_tau_hi = 1000.0;
  c.net_c_lo = 0.5;
  c.net_c_hi = 0.999;
  c.sampler_kernel = GMC_KERNEL_TILE;
  return c;
}

}  // namespace
}  // namespace gmc

using namespace gmc;

extern "C" {

const char *gmc_status_str(gmc_status s) {
  switch (s) {
    case GMC_OK: return "GMC_OK";
    case GMC_EINVAL: return "GMC_EINVAL";
    case GMC_ENOMEM: return "GMC_ENOMEM";
    case GMC_ECUDA: return "GMC_ECUDA";
    case GMC_ETIMEOUT: return "GMC_ETIMEOUT";
    case GMC_EFORMAT: return "GMC_EFORMAT";
    case GMC_ENOTIMPL: return "GMC_ENOTIMPL";
    case GMC_EBUSY: return "GMC_EBUSY";
    case GMC_ENOWEIGHTS: return "GMC_ENOWEIGHTS";
    case GMC_EIO: return "GMC_EIO";
  }
  return "GMC_UNKNOWN";
}

const char *gmc_last_error(const gmc_ctx *ctx) {
  if (!ctx) return "null context";
  // a copy per calling thread: the serving thread may replace the message
  thread_local std::string copy;
  std::lock_guard<std::mutex> lk(ctx->err_mu);
  copy = ctx->last_error;
  return copy.c_str();
}

gmc_status gmc_create(gmc_ctx **out, int device) {
  if (!out) return GMC_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return GMC_EINVAL;
  }
  gmc_ctx *ctx = new (std::nothrow) gmc_ctx();
  if (!ctx) return GMC_ENOMEM;
  ctx->device = device;
  ctx->cfg = default_config();
  cudaError_t e = cudaSetDevice(device);
  // a blocking stream: ordered with work on the legacy default stream, so
  // buffers a caller fills there are ready before the library reads them
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamDefault);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int) * 4);
  if (e != cudaSuccess) {
    gmc_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? GMC_ENOMEM : GMC_ECUDA;
  }
  ctx->stream = ctx->own_stream;
  *out = ctx;
  return GMC_OK;
}

gmc_status gmc_destroy(gmc_ctx *ctx) {
  if (!ctx) return GMC_OK;
  cudaSetDevice(ctx->device);
  if (ctx->server) server_free(ctx->server);
  if (ctx->solver) engine_free(ctx->solver);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto &b : ctx->stage)
    if (b.ptr) cudaFree(b.ptr);
  if (ctx->bias1.ptr) cudaFree(ctx->bias1.ptr);
  if (ctx->walk_next.ptr) cudaFree(ctx->walk_next.ptr);
  if (ctx->train) train_state_free(ctx->train);
  if (ctx->net.d_f32) cudaFree(ctx->net.d_f32);
  if (ctx->net.d_tc) cudaFree(ctx->net.d_tc);
  if (ctx->net.d_tc_bias) cudaFree(ctx->net.d_tc_bias);
  if (ctx->net.d_tc8) cudaFree(ctx->net.d_tc8);
  if (ctx->net.d_tc8_scale) cudaFree(ctx->net.d_tc8_scale);
  if (ctx->internal.d_f32) cudaFree(ctx->internal.d_f32);
  if (ctx->internal.d_tc) cudaFree(ctx->internal.d_tc);
  if (ctx->internal.d_tc_bias) cudaFree(ctx->internal.d_tc_bias);
  if (ctx->internal.d_tc8) cudaFree(ctx->internal.d_tc8);
  if (ctx->internal.d_tc8_scale) cudaFree(ctx->internal.d_tc8_scale);
  if (ctx->xy.d_f32) cudaFree(ctx->xy.d_f32);
  if (ctx->xy.d_tc) cudaFree(ctx->xy.d_tc);
  if (ctx->xy.d_tc_bias) cudaFree(ctx->xy.d_tc_bias);
  if (ctx->xy.d_tc8) cudaFree(ctx->xy.d_tc8);
  if (ctx->xy.d_tc8_scale) cudaFree(ctx->xy.d_tc8_scale);
  if (ctx->internal_xy.d_f32) cudaFree(ctx->internal_xy.d_f32);
  if (ctx->internal_xy.d_tc) cudaFree(ctx->internal_xy.d_tc);
  if (ctx->internal_xy.d_tc_bias) cudaFree(ctx->internal_xy.d_tc_bias);
  if (ctx->internal_xy.d_tc8) cudaFree(ctx->internal_xy.d_tc8);
  if (ctx->internal_xy.d_tc8_scale) cudaFree(ctx->internal_xy.d_tc8_scale);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
  return GMC_OK;
}

gmc_status gmc_set_stream(gmc_ctx *ctx, void *cuda_stream) {
  if (!ctx) return GMC_EINVAL;
  ctx->stream = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own_stream;
  return GMC_OK;
}

gmc_status gmc_synchronize(gmc_ctx *ctx) {
  if (!ctx) return GMC_EINVAL;
  cudaSetDevice(ctx->device);
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return check_device_error(ctx);
}

gmc_status gmc_get_config(const gmc_ctx *ctx, gmc_config *out) {
  if (!ctx || !out) return GMC_EINVAL;
  *out = ctx->cfg;
  return GMC_OK;
}

gmc_status gmc_set_config(gmc_ctx *ctx, const gmc_config *cfg) {
  if (!ctx || !cfg) return GMC_EINVAL;
  if (ctx->server) return set_error(ctx, GMC_EBUSY, "gmc_set_config: the server is running");
  switch (config_check(*cfg)) {
    case 0: break;
    case 1: return set_error(ctx, GMC_EINVAL, "steps must be in [1, 256], got %d", cfg->steps);
    case 2: return set_error(ctx, GMC_EINVAL, "unknown integrator %d", cfg->integrator);
    case 3: return set_error(ctx, GMC_EINVAL, "unknown precision %d", cfg->precision);
    case 4: return set_error(ctx, GMC_EINVAL, "need w_cut >= 0 and p_survive in (0, 1]");
    case 5: return set_error(ctx, GMC_EINVAL, "bank_capacity must be in [1024, 2^28]");
    case 6: return set_error(ctx, GMC_EINVAL, "flights_per_wave must be >= 1");
    case 7: return set_error(ctx, GMC_EINVAL, "gmc_min_tau must be >= 0");
    case 8:
      return set_error(ctx, GMC_EINVAL,
                       "need 0 < net_tau_lo <= net_tau_hi (finite), 0 < net_c_lo <= net_c_hi <= 1");
    default: return set_error(ctx, GMC_EINVAL, "unknown sampler_kernel %d", cfg->sampler_kernel);
  }
  ctx->cfg = *cfg;
  return GMC_OK;
}

gmc_status gmc_philox(gmc_ctx *ctx, int64_t n, uint64_t seed, uint64_t id0, uint32_t event,
                      uint32_t tag, uint32_t *out) {
  if (!ctx || n < 0 || (n > 0 && !out)) return set_error(ctx, GMC_EINVAL, "gmc_philox: bad arguments");
  if (n == 0) return GMC_OK;
  cudaSetDevice(ctx->device);
  Arg o;
  o.user = out;
  o.bytes = (size_t)n * 16;
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 0, o));
  GMC_CUDA_TRY(ctx, launch_philox(ctx->stream, n, seed, id0, event, tag, (uint32_t *)o.dev));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, o));
  if (o.host || o.mapped) GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return GMC_OK;
}

gmc_status gmc_normals(gmc_ctx *ctx, int64_t n, uint64_t seed, uint64_t id0, uint32_t event,
                       uint32_t tag, float *out) {
  if (!ctx || n < 0 || (n > 0 && !out)) return set_error(ctx, GMC_EINVAL, "gmc_normals: bad arguments");
  if (n == 0) return GMC_OK;
  cudaSetDevice(ctx->device);
  Arg o;
  o.user = out;
  o.bytes = (size_t)n * 16;
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 0, o));
  GMC_CUDA_TRY(ctx, launch_normals(ctx->stream, n, seed, id0, event, tag, (float *)o.dev));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, o));
  if (o.host || o.mapped) GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return GMC_OK;
}

}  // extern "C"

namespace gmc {
gmc_status check_net_path(gmc_ctx *ctx, const NetDev &N, int precision, int kernel, const char *who) {
  const bool special = N.rm || N.stats.ncond != kCond;
  if (!special || precision == GMC_FP32 || (precision == GMC_BF16 && kernel == GMC_KERNEL_TILE))
    return GMC_OK;
  return set_error(ctx, GMC_EINVAL,
                   "%s: the %s network runs at GMC_FP32, or GMC_BF16 with GMC_KERNEL_TILE", who,
                   N.rm ? "residual-modulated" : "rectangular-cell");
}

// Parses a GMCW version 1 blob into N and uploads its FP32, BF16 and FP8 copies.
// Flag 1 (the residual-modulated network) adds M[3][256][5] and G[3][2][256]
// after the layers. n_cond = 6 with 26 inputs is a network for rectangular
// cells (the aspect as input column 25; not with flag 1).
// Nothing of N changes unless the blob parses; N stays marked unloaded from
// the first change until every device copy is in place.
gmc_status load_net(gmc_ctx *ctx, NetDev &N, const void *blob, size_t nbytes) {
  static_assert(kGmcwCond == kCond && kGmcwCondRect == kCondRect && kGmcwState == kState &&
                    kGmcwEmb == kEmb && kGmcwHidden == kHidden && kGmcwFlagRM == kFlagRM,
                "weight-file constants");
  if (ctx->server) return set_error(ctx, GMC_EBUSY, "loading weights: the server is running");
  GmcwNet P;
  int bad_layer = -1;
  const int ps = gmcw_parse(blob, nbytes, &P, &bad_layer);
  if (ps == kGmcwTruncatedLayer)
    return set_error(ctx, GMC_EFORMAT, "weight file: truncated layer %d", bad_layer);
  if (ps != kGmcwOk) return set_error(ctx, GMC_EFORMAT, "weight file: %s", gmcw_status_text(ps));
  const bool rm = P.rm;
  const int nc = P.ncond, nin = P.nin;
  const float *st = P.stats.data();

  N.loaded = false;
  for (int l = 0; l < 5; ++l) {
    std::memset(N.host_w[l], 0, sizeof(N.host_w[l]));
    std::memset(N.host_b[l], 0, sizeof(N.host_b[l]));
    std::memcpy(N.host_w[l], P.w[l].data(), P.w[l].size() * sizeof(float));
    std::memcpy(N.host_b[l], P.b[l].data(), P.b[l].size() * sizeof(float));
  }
  N.rm = rm;
  N.nin = nin;
  std::memset(N.host_m, 0, sizeof(N.host_m));
  std::memset(N.host_g, 0, sizeof(N.host_g));
  if (rm) {
    std::memcpy(N.host_m, P.m.data(), P.m.size() * sizeof(float));
    std::memcpy(N.host_g, P.g.data(), P.g.size() * sizeof(float));
  }
  NetStats ns;
  for (int k = 0; k < kCondRect; ++k) {
    ns.cond_mean[k] = k < nc ? st[k] : 0.0f;
    ns.cond_inv_std[k] = k < nc ? 1.0f / st[nc + k] : 1.0f;
  }
  for (int k = 0; k < 4; ++k) {
    ns.y_mean[k] = st[2 * nc + k];
    ns.y_std[k] = st[2 * nc + 4 + k];
  }
  ns.ncond = nc;
  // the x-y geometry slots decode into the unit disk
  ns.disk = (&N == &ctx->xy || &N == &ctx->internal_xy) ? 1 : 0;

  // FP32 transposed block (room for the modulation arrays in every load, so
  // a later load of either network reuses it)
  const size_t n1 = 32 * 256, nh = 256 * 256;
  const size_t nm = 3 * kCond * 256, ng = 3 * 2 * 256;
  const size_t total = n1 + 256 + 3 * (nh + 256) + 4 * 256 + 4 + nm + ng;
  std::vector<float> h(total, 0.0f);
  float *p = h.data();
  float *w1t = p; p += n1;
  float *b1 = p; p += 256;
  float *wt[3], *bt[3];
  for (int l = 0; l < 3; ++l) { wt[l] = p; p += nh; bt[l] = p; p += 256; }
  float *w5 = p; p += 4 * 256;
  float *b5 = p; p += 4;
  float *mt = p; p += nm;
  float *gg = p; p += ng;
  for (int c = 0; c < 256; ++c)
    for (int k = 0; k < nin; ++k) w1t[k * 256 + c] = N.host_w[0][c * nin + k];
  std::memcpy(b1, N.host_b[0], 256 * 4);
  for (int l = 0; l < 3; ++l) {
    for (int c = 0; c < 256; ++c)
      for (int k = 0; k < 256; ++k) wt[l][k * 256 + c] = N.host_w[l + 1][c * 256 + k];
    std::memcpy(bt[l], N.host_b[l + 1], 256 * 4);
  }
  std::memcpy(w5, N.host_w[4], 4 * 256 * 4);
  std::memcpy(b5, N.host_b[4], 4 * 4);
  for (int j = 0; j < 3; ++j)
    for (int c = 0; c < 256; ++c)
      for (int k = 0; k < kCond; ++k) mt[(j * kCond + k) * 256 + c] = N.host_m[j][c * kCond + k];
  std::memcpy(gg, N.host_g, ng * sizeof(float));

  cudaSetDevice(ctx->device);
  GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (!N.d_f32) GMC_CUDA_TRY(ctx, cudaMalloc(&N.d_f32, total * sizeof(float)));
  GMC_CUDA_TRY(ctx, cudaMemcpy(N.d_f32, h.data(), total * sizeof(float), cudaMemcpyHostToDevice));
  float *d = N.d_f32;
  N.f32.w1t = d; d += n1;
  N.f32.b1 = d; d += 256;
  N.f32.w2t = d; d += nh;
  N.f32.b2 = d; d += 256;
  N.f32.w3t = d; d += nh;
  N.f32.b3 = d; d += 256;
  N.f32.w4t = d; d += nh;
  N.f32.b4 = d; d += 256;
  N.f32.w5 = d; d += 4 * 256;
  N.f32.b5 = d; d += 4;
  N.f32.mt = d; d += nm;
  N.f32.gg = d;
  N.f32.rm = rm ? 1 : 0;

  // packed operands of the tensor-core path (BF16 and FP8 variants)
  {
    const size_t tcb = tc_packed_bytes(false), tcb8 = tc_packed_bytes(true);
    std::vector<unsigned char> packed(tcb), packed8(tcb8);
    std::vector<float> bias(5 * 256, 0.0f), scale(3 * 256, 0.0f);
    tc_pack_host(N.host_w, N.host_b, packed.data(), bias.data(), rm ? N.host_m : nullptr, nin);
    tc_pack_host_fp8(N.host_w, N.host_b, packed8.data(), bias.data(), scale.data(), nin);
    if (!N.d_tc) GMC_CUDA_TRY(ctx, cudaMalloc(&N.d_tc, tcb));
    if (!N.d_tc8) GMC_CUDA_TRY(ctx, cudaMalloc(&N.d_tc8, tcb8));
    if (!N.d_tc_bias) GMC_CUDA_TRY(ctx, cudaMalloc(&N.d_tc_bias, 5 * 256 * sizeof(float)));
    if (!N.d_tc8_scale) GMC_CUDA_TRY(ctx, cudaMalloc(&N.d_tc8_scale, 3 * 256 * sizeof(float)));
    GMC_CUDA_TRY(ctx, cudaMemcpy(N.d_tc, packed.data(), tcb, cudaMemcpyHostToDevice));
    GMC_CUDA_TRY(ctx, cudaMemcpy(N.d_tc8, packed8.data(), tcb8, cudaMemcpyHostToDevice));
    GMC_CUDA_TRY(ctx, cudaMemcpy(N.d_tc_bias, bias.data(), 5 * 256 * sizeof(float),
                                 cudaMemcpyHostToDevice));
    GMC_CUDA_TRY(ctx, cudaMemcpy(N.d_tc8_scale, scale.data(), 3 * 256 * sizeof(float),
                                 cudaMemcpyHostToDevice));
    N.tc_bytes = tcb;
  }
  N.stats = ns;
  N.loaded = true;
  ++N.generation;
  return GMC_OK;
}


// Reads a whole file; false (with the context error set) on failure.
bool read_file(gmc_ctx *ctx, const char *path, std::vector<unsigned char> &blob, gmc_status *st) {
  FILE *f = std::fopen(path, "rb");
  if (!f) {
    *st = set_error(ctx, GMC_EIO, "cannot open weight file '%s'", path);
    return false;
  }
  unsigned char buf[1 << 16];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) blob.insert(blob.end(), buf, buf + got);
  const bool err = std::ferror(f) != 0;
  std::fclose(f);
  if (err) {
    *st = set_error(ctx, GMC_EIO, "read error on '%s'", path);
    return false;
  }
  return true;
}

}  // namespace gmc

extern "C" {

gmc_status gmc_load_weights(gmc_ctx *ctx, const char *path) {
  if (!ctx || !path) return set_error(ctx, GMC_EINVAL, "gmc_load_weights: null argument");
  std::vector<unsigned char> blob;
  gmc_status st;
  if (!read_file(ctx, path, blob, &st)) return st;
  return load_net(ctx, ctx->net, blob.data(), blob.size());
}

gmc_status gmc_load_internal_weights(gmc_ctx *ctx, const char *path) {
  if (!ctx || !path) return set_error(ctx, GMC_EINVAL, "gmc_load_internal_weights: null argument");
  std::vector<unsigned char> blob;
  gmc_status st;
  if (!read_file(ctx, path, blob, &st)) return st;
  return load_net(ctx, ctx->internal, blob.data(), blob.size());
}

gmc_status gmc_load_xy_weights(gmc_ctx *ctx, const char *path) {
  if (!ctx || !path) return set_error(ctx, GMC_EINVAL, "gmc_load_xy_weights: null argument");
  std::vector<unsigned char> blob;
  gmc_status st;
  if (!read_file(ctx, path, blob, &st)) return st;
  return load_net(ctx, ctx->xy, blob.data(), blob.size());
}

gmc_status gmc_load_internal_xy_weights(gmc_ctx *ctx, const char *path) {
  if (!ctx || !path) return set_error(ctx, GMC_EINVAL, "gmc_load_internal_xy_weights: null argument");
  std::vector<unsigned char> blob;
  gmc_status st;
  if (!read_file(ctx, path, blob, &st)) return st;
  return load_net(ctx, ctx->internal_xy, blob.data(), blob.size());
}

gmc_status gmc_load_internal_xy_weights_buffer(gmc_ctx *ctx, const void *blob, size_t nbytes) {
  if (!ctx || !blob)
    return set_error(ctx, GMC_EINVAL, "gmc_load_internal_xy_weights_buffer: null argument");
  return load_net(ctx, ctx->internal_xy, blob, nbytes);
}

gmc_status gmc_load_weights_buffer(gmc_ctx *ctx, const void *blob, size_t nbytes) {
  if (!ctx || !blob) return set_error(ctx, GMC_EINVAL, "gmc_load_weights_buffer: null argument");
  return load_net(ctx, ctx->net, blob, nbytes);
}

gmc_status gmc_load_internal_weights_buffer(gmc_ctx *ctx, const void *blob, size_t nbytes) {
  if (!ctx || !blob) return set_error(ctx, GMC_EINVAL, "gmc_load_internal_weights_buffer: null argument");
  return load_net(ctx, ctx->internal, blob, nbytes);
}

gmc_status gmc_load_xy_weights_buffer(gmc_ctx *ctx, const void *blob, size_t nbytes) {
  if (!ctx || !blob) return set_error(ctx, GMC_EINVAL, "gmc_load_xy_weights_buffer: null argument");
  return load_net(ctx, ctx->xy, blob, nbytes);
}

}  // extern "C"

namespace gmc {
// gmc_transmit with network N (the boundary or the internal model).
gmc_status transmit_net(gmc_ctx *ctx, const NetDev &N, int64_t n, const float *cond,
                        const float *noise, uint64_t seed, uint64_t id0, int steps, int integrator,
                        int precision, float *y_raw, float *exit) {
  if (n < 0) return set_error(ctx, GMC_EINVAL, "gmc_transmit: n < 0");
  if (n == 0) return GMC_OK;
  if (!cond || (!y_raw && !exit)) return set_error(ctx, GMC_EINVAL, "gmc_transmit: null array");
  if (steps < 1 || steps > 256) return set_error(ctx, GMC_EINVAL, "gmc_transmit: steps in [1,256]");
  if (integrator != GMC_EULER && integrator != GMC_MIDPOINT && integrator != GMC_RK4)
    return set_error(ctx, GMC_EINVAL, "gmc_transmit: unknown integrator");
  if (!N.loaded) return set_error(ctx, GMC_ENOWEIGHTS, "gmc_transmit: no weights loaded for this model");
  if (precision != GMC_FP32 && precision != GMC_BF16 && precision != GMC_FP8)
    return set_error(ctx, GMC_EINVAL, "gmc_transmit: unknown precision");
  if (check_net_path(ctx, N, precision, ctx->cfg.sampler_kernel, "gmc_transmit") != GMC_OK)
    return GMC_EINVAL;
  cudaSetDevice(ctx->device);
  Arg a_cond, a_noise, a_y, a_exit;
  a_cond.user = cond; a_cond.bytes = (size_t)n * N.stats.ncond * 4;
  a_noise.user = noise; a_noise.bytes = (size_t)n * 4 * 4;
  a_y.user = y_raw; a_y.bytes = (size_t)n * 4 * 4;
  a_exit.user = exit; a_exit.bytes = (size_t)n * 4 * 4;
  GMC_CUDA_TRY(ctx, stage_in(ctx, 0, a_cond));
  GMC_CUDA_TRY(ctx, stage_in(ctx, 1, a_noise));
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 2, a_y));
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 3, a_exit));
  if (precision == GMC_FP32) {
    GMC_CUDA_TRY(ctx, launch_sampler_f32(ctx->stream, N.f32, N.stats, n, (const float *)a_cond.dev,
                                         (const float *)a_noise.dev, seed, id0, steps, integrator,
                                         (float *)a_y.dev, (float *)a_exit.dev));
  } else {
    const bool fp8 = precision == GMC_FP8;
    GMC_CUDA_TRY(ctx, ensure(ctx->bias1, (size_t)4 * steps * 256 * sizeof(float)));
    cudaError_t e = launch_sampler_tc(ctx->stream, fp8 ? N.d_tc8 : N.d_tc, N.d_tc_bias,
                                      N.f32, N.stats, n, (const float *)a_cond.dev,
                                      (const float *)a_noise.dev, seed, id0, steps, integrator,
                                      (float *)a_y.dev, (float *)a_exit.dev, ctx->d_err,
                                      (float *)ctx->bias1.ptr, fp8 ? N.d_tc8_scale : nullptr,
                                      ctx->cfg.sampler_kernel);
    if (e != cudaSuccess) return cuda_error(ctx, e, "launch_sampler_tc");
  }
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, a_y));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, a_exit));
  if (a_cond.host || a_noise.host || a_y.host || a_exit.host || a_cond.mapped || a_noise.mapped ||
      a_y.mapped || a_exit.mapped) {
    GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
  }
  return GMC_OK;
}

}  // namespace gmc

namespace gmc {
using Walk6Launch = cudaError_t (*)(cudaStream_t, int64_t, const float *, const float *,
                                    const float *, const float *, const float *, const float *,
                                    int, uint64_t, uint64_t, uint32_t, int32_t *, float *,
                                    uint32_t *);

// Marshalling of the batched walks with six per-particle inputs (rectangular
// cells, x-y geometry): staging, launch, copies back.
static gmc_status walk6(gmc_ctx *ctx, const char *name, Walk6Launch launch, int64_t n,
                        const float *const ins[6], int mode, uint64_t seed, uint64_t id0,
                        uint32_t event0, int32_t *status, float *exit, uint32_t *ncoll) {
  if (!ctx) return GMC_EINVAL;
  if (n < 0) return set_error(ctx, GMC_EINVAL, "%s: n < 0", name);
  if (n == 0) return GMC_OK;
  for (int k = 0; k < 6; ++k)
    if (!ins[k]) return set_error(ctx, GMC_EINVAL, "%s: null array", name);
  if (!status || !exit) return set_error(ctx, GMC_EINVAL, "%s: null array", name);
  if (mode != GMC_ABSORB_ANALOG && mode != GMC_ABSORB_IMPLICIT)
    return set_error(ctx, GMC_EINVAL, "%s: unknown mode", name);
  cudaSetDevice(ctx->device);
  Arg in[6], o_status, o_exit, o_ncoll;
  for (int k = 0; k < 6; ++k) {
    in[k].user = ins[k];
    in[k].bytes = (size_t)n * 4;
    GMC_CUDA_TRY(ctx, stage_in(ctx, k, in[k]));
  }
  o_status.user = status; o_status.bytes = (size_t)n * 4;
  o_exit.user = exit; o_exit.bytes = (size_t)n * 16;
  o_ncoll.user = ncoll; o_ncoll.bytes = (size_t)n * 4;
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 6, o_status));
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 7, o_exit));
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 8, o_ncoll));
  GMC_CUDA_TRY(ctx, launch(ctx->stream, n, (const float *)in[0].dev, (const float *)in[1].dev,
                           (const float *)in[2].dev, (const float *)in[3].dev,
                           (const float *)in[4].dev, (const float *)in[5].dev, mode, seed, id0,
                           event0, (int32_t *)o_status.dev, (float *)o_exit.dev,
                           (uint32_t *)o_ncoll.dev));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, o_status));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, o_exit));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, o_ncoll));
  bool host = o_status.host || o_exit.host || o_ncoll.host || o_status.mapped || o_exit.mapped ||
              o_ncoll.mapped;
  for (auto &a : in) host = host || a.host || a.mapped;
  if (host) GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return GMC_OK;
}
}  // namespace gmc

extern "C" {

gmc_status gmc_transmit(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                        uint64_t seed, uint64_t id0, int steps, int integrator, int precision,
                        float *y_raw, float *exit) {
  if (!ctx) return GMC_EINVAL;
  return transmit_net(ctx, ctx->net, n, cond, noise, seed, id0, steps, integrator, precision,
                      y_raw, exit);
}

gmc_status gmc_sample_internal(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                               uint64_t seed, uint64_t id0, int steps, int integrator,
                               int precision, float *y_raw, float *exit) {
  if (!ctx) return GMC_EINVAL;
  return transmit_net(ctx, ctx->internal, n, cond, noise, seed, id0, steps, integrator, precision,
                      y_raw, exit);
}

gmc_status gmc_sample_internal_xy(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                                  uint64_t seed, uint64_t id0, int steps, int integrator,
                                  int precision, float *y_raw, float *exit) {
  if (!ctx) return GMC_EINVAL;
  return transmit_net(ctx, ctx->internal_xy, n, cond, noise, seed, id0, steps, integrator,
                      precision, y_raw, exit);
}

gmc_status gmc_transmit_xy(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                           uint64_t seed, uint64_t id0, int steps, int integrator, int precision,
                           float *y_raw, float *exit) {
  if (!ctx) return GMC_EINVAL;
  return transmit_net(ctx, ctx->xy, n, cond, noise, seed, id0, steps, integrator, precision,
                      y_raw, exit);
}

gmc_status analog_transmit(gmc_ctx *ctx, int64_t n, const float *xi, const float *cos_in,
                           const float *sin_in, const float *tau, const float *c, int mode,
                           uint64_t seed, uint64_t id0, uint32_t event0, int32_t *status,
                           float *exit, uint32_t *ncoll) {
  if (!ctx) return GMC_EINVAL;
  if (n < 0) return set_error(ctx, GMC_EINVAL, "analog_transmit: n < 0");
  if (n == 0) return GMC_OK;
  if (!xi || !cos_in || !sin_in || !tau || !c || !status || !exit)
    return set_error(ctx, GMC_EINVAL, "analog_transmit: null array");
  if (mode != GMC_ABSORB_ANALOG && mode != GMC_ABSORB_IMPLICIT)
    return set_error(ctx, GMC_EINVAL, "analog_transmit: unknown mode");
  cudaSetDevice(ctx->device);
  Arg in[5], o_status, o_exit, o_ncoll;
  const float *ins[5] = {xi, cos_in, sin_in, tau, c};
  for (int k = 0; k < 5; ++k) {
    in[k].user = ins[k];
    in[k].bytes = (size_t)n * 4;
    GMC_CUDA_TRY(ctx, stage_in(ctx, k, in[k]));
  }
  o_status.user = status; o_status.bytes = (size_t)n * 4;
  o_exit.user = exit; o_exit.bytes = (size_t)n * 16;
  o_ncoll.user = ncoll; o_ncoll.bytes = (size_t)n * 4;
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 5, o_status));
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 6, o_exit));
  GMC_CUDA_TRY(ctx, stage_out_prepare(ctx, 7, o_ncoll));
  GMC_CUDA_TRY(ctx, ensure(ctx->walk_next, sizeof(unsigned long long)));
  GMC_CUDA_TRY(ctx, launch_analog(ctx->stream, n, (const float *)in[0].dev, (const float *)in[1].dev,
                                  (const float *)in[2].dev, (const float *)in[3].dev,
                                  (const float *)in[4].dev, mode, seed, id0, event0,
                                  (int32_t *)o_status.dev, (float *)o_exit.dev,
                                  (uint32_t *)o_ncoll.dev,
                                  (unsigned long long *)ctx->walk_next.ptr));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, o_status));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, o_exit));
  GMC_CUDA_TRY(ctx, stage_out_finish(ctx, o_ncoll));
  bool host = o_status.host || o_exit.host || o_ncoll.host || o_status.mapped || o_exit.mapped ||
              o_ncoll.mapped;
  for (auto &a : in) host = host || a.host || a.mapped;
  if (host) GMC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return GMC_OK;
}

gmc_status analog_transmit_rect(gmc_ctx *ctx, int64_t n, const float *xi, const float *cos_in,
                                const float *sin_in, const float *tau_x, const float *tau_y,
                                const float *c, int mode, uint64_t seed, uint64_t id0,
                                uint32_t event0, int32_t *status, float *exit, uint32_t *ncoll) {
  const float *in[6] = {xi, cos_in, sin_in, tau_x, tau_y, c};
  return walk6(ctx, "analog_transmit_rect", launch_analog_rect, n, in, mode, seed, id0, event0,
               status, exit, ncoll);
}

gmc_status analog_transmit_xy(gmc_ctx *ctx, int64_t n, const float *xi, const float *ux_in,
                              const float *uy_in, const float *tau_x, const float *tau_y,
                              const float *c, int mode, uint64_t seed, uint64_t id0,
                              uint32_t event0, int32_t *status, float *exit, uint32_t *ncoll) {
  const float *in[6] = {xi, ux_in, uy_in, tau_x, tau_y, c};
  return walk6(ctx, "analog_transmit_xy", launch_analog_xy, n, in, mode, seed, id0, event0,
               status, exit, ncoll);
}

}  // extern "C"
