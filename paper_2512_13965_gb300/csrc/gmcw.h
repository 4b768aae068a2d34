// Parsing of "GMCW" version-1 weight files into host arrays. Plain C++ with
// no CUDA headers, so a host-only unit test checks it against the oracle's
// reader without a GPU.
//
// Layout (little-endian): magic "GMCW", u32 version = 1, u32 n_layers = 5,
// u32 dims[6] = {n_in, 256, 256, 256, 256, 4}, u32 n_cond (5, or 6 for
// rectangular cells), u32 n_state = 4, u32 n_emb = 16, u32 flags (bit 0: the
// residual-modulated network, not with n_cond 6); f32 cond_mean[n_cond],
// cond_std[n_cond], y_mean[4], y_std[4]; per layer l = 0..4 f32
// W_l[dims[l+1]][dims[l]] then b_l[dims[l+1]]; with flag 1, f32
// M_j[256][5] for j = 0..2, then G_j[2][256] for j = 0..2. n_in =
// n_cond + 4 + 16.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

namespace gmc {

constexpr uint32_t kGmcwFlagRM = 1u;
constexpr int kGmcwCond = 5, kGmcwCondRect = 6, kGmcwState = 4, kGmcwEmb = 16, kGmcwHidden = 256;

struct GmcwNet {
  int ncond = 0;  // 5, or 6 for rectangular cells
  int nin = 0;    // layer-1 inputs: ncond + 4 + 16
  bool rm = false;
  std::vector<float> stats;       // cond_mean[ncond], cond_std[ncond], y_mean[4], y_std[4]
  std::vector<float> w[5], b[5];  // W_l [out][in] and b_l [out] as stored
  std::vector<float> m, g;        // M_j [3][256][5] and G_j [3][2][256]; empty unless rm
};

enum GmcwStatus {
  kGmcwOk = 0,
  kGmcwBadMagic,
  kGmcwTruncatedHeader,
  kGmcwUnsupported,
  kGmcwBadDims,
  kGmcwTruncatedStats,
  kGmcwTruncatedLayer,
  kGmcwTruncatedModulation,
  kGmcwTrailing,
  kGmcwBadStd,
  kGmcwNonFinite,
};

inline const char *gmcw_status_text(int s) {
  switch (s) {
    case kGmcwOk: return "ok";
    case kGmcwBadMagic: return "bad magic";
    case kGmcwTruncatedHeader: return "truncated header";
    case kGmcwUnsupported: return "unsupported version, layout or flags";
    case kGmcwBadDims: return "layer dims must be 25-256-256-256-256-4 (26-... with n_cond 6)";
    case kGmcwTruncatedStats: return "truncated statistics";
    case kGmcwTruncatedLayer: return "truncated layer";
    case kGmcwTruncatedModulation: return "truncated modulation arrays";
    case kGmcwTrailing: return "trailing bytes";
    case kGmcwBadStd: return "cond_std must be > 0";
    case kGmcwNonFinite: return "non-finite statistics";
    default: return "unknown";
  }
}

namespace gmcw_detail {
struct Reader {
  const unsigned char *p;
  size_t n, off;
  bool u32(uint32_t *v) {
    if (n - off < 4) return false;
    std::memcpy(v, p + off, 4);
    off += 4;
    return true;
  }
  bool f32(std::vector<float> &v, size_t count) {
    if ((n - off) / 4 < count) return false;
    v.resize(count);
    std::memcpy(v.data(), p + off, 4 * count);
    off += 4 * count;
    return true;
  }
};
}  // namespace gmcw_detail

// Parses `nbytes` bytes at `blob` into *out (left unchanged on failure).
// Returns a GmcwStatus; for kGmcwTruncatedLayer, *layer is the layer index.
// The weights themselves are taken as stored; the statistics must be finite
// with every cond_std > 0.
inline int gmcw_parse(const void *blob, size_t nbytes, GmcwNet *out, int *layer) {
  if (!blob || nbytes < 4 || std::memcmp(blob, "GMCW", 4) != 0) return kGmcwBadMagic;
  gmcw_detail::Reader rd{(const unsigned char *)blob, nbytes, 4};
  uint32_t version, nl, dims[6], ncond, nstate, nemb, flags;
  bool ok = rd.u32(&version) && rd.u32(&nl);
  for (int i = 0; i < 6 && ok; ++i) ok = rd.u32(&dims[i]);
  ok = ok && rd.u32(&ncond) && rd.u32(&nstate) && rd.u32(&nemb) && rd.u32(&flags);
  if (!ok) return kGmcwTruncatedHeader;
  if (version != 1 || nl != 5 || (ncond != (uint32_t)kGmcwCond && ncond != (uint32_t)kGmcwCondRect) ||
      nstate != (uint32_t)kGmcwState || nemb != (uint32_t)kGmcwEmb || (flags & ~kGmcwFlagRM) ||
      (ncond != (uint32_t)kGmcwCond && (flags & kGmcwFlagRM)))
    return kGmcwUnsupported;
  GmcwNet P;
  P.ncond = (int)ncond;
  P.nin = P.ncond + kGmcwState + kGmcwEmb;
  P.rm = (flags & kGmcwFlagRM) != 0;
  const uint32_t want[6] = {(uint32_t)P.nin, kGmcwHidden, kGmcwHidden, kGmcwHidden, kGmcwHidden,
                            (uint32_t)kGmcwState};
  for (int i = 0; i < 6; ++i)
    if (dims[i] != want[i]) return kGmcwBadDims;
  const int nst = 2 * P.ncond + 2 * kGmcwState;
  if (!rd.f32(P.stats, nst)) return kGmcwTruncatedStats;
  for (int l = 0; l < 5; ++l) {
    if (!rd.f32(P.w[l], (size_t)dims[l + 1] * dims[l]) || !rd.f32(P.b[l], dims[l + 1])) {
      if (layer) *layer = l;
      return kGmcwTruncatedLayer;
    }
  }
  if (P.rm && (!rd.f32(P.m, 3 * kGmcwHidden * kGmcwCond) || !rd.f32(P.g, 3 * 2 * kGmcwHidden)))
    return kGmcwTruncatedModulation;
  if (rd.off != nbytes) return kGmcwTrailing;
  for (int k = 0; k < P.ncond; ++k)
    if (!(P.stats[P.ncond + k] > 0.0f)) return kGmcwBadStd;
  for (int k = 0; k < nst; ++k)
    if (!std::isfinite(P.stats[k])) return kGmcwNonFinite;
  *out = std::move(P);
  return kGmcwOk;
}

}  // namespace gmc
