// Header of a training checkpoint and the checks a restore applies to it
// before anything of the training state changes. Plain C++ with no CUDA
// headers, so a host-only unit test checks every refusal without a GPU.
//
// A checkpoint is this header, then the FP32 master weights and Adam's first
// and second moments (params floats each). The batch of step k draws its
// rows from Philox at (seed, k), so restoring these and the step count
// resumes the run exactly where it stopped. The dataset is identified by its
// size n and its FP64-accumulated standardization statistics (stored as
// FP32), which gmc_train_begin recomputes from the data: a checkpoint
// restores only into a training state begun on data with the same n and
// bit-identical statistics.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

namespace gmc {

struct TrainCkpt {
  char magic[4];
  uint32_t version;
  int64_t params, step, batch, n;
  int32_t precision, arch;  // arch bit 0: residual-modulated; bit 1: rectangular cells
  double lr, beta1, beta2, eps, weight_decay;
  uint64_t seed;
  float stats[20];  // cond_mean, cond_std [n_cond each], y_mean, y_std [4 each]; 2 n_cond + 8 used
};
constexpr uint32_t kCkptVersion = 3;

// arch bits of a network: residual-modulated, and rectangular cells (a
// condition of more than the square cell's five components)
inline int32_t ckpt_arch_bits(bool rm, int ncond) { return (rm ? 1 : 0) | (ncond != 5 ? 2 : 0); }

// The training state a checkpoint is restored into (from gmc_train_begin).
struct CkptTarget {
  int64_t params, batch, n;
  int32_t precision, arch;
  int ncond;
  const float *stats;  // [20], as the header stores them
};

enum CkptCheck {
  kCkptOk = 0,
  kCkptNotThisNetwork,  // magic, version, parameter count or network form
  kCkptBadStats,        // a non-finite statistic or a standard deviation <= 0
  kCkptBadHyper,        // lr, betas, eps or weight decay outside their ranges
  kCkptOtherRun,        // another batch size or precision, or a negative step
  kCkptOtherData,       // another dataset size or statistics
};

inline int ckpt_check(const TrainCkpt &h, const CkptTarget &t) {
  if (std::memcmp(h.magic, "GMCT", 4) != 0 || h.version != kCkptVersion || h.params != t.params ||
      h.arch != t.arch)
    return kCkptNotThisNetwork;
  const int nc = t.ncond;
  for (int k = 0; k < 2 * nc + 8; ++k)
    if (!std::isfinite(h.stats[k]) ||
        (((k >= nc && k < 2 * nc) || k >= 2 * nc + 4) && !(h.stats[k] > 0.0f)))
      return kCkptBadStats;
  if (!(h.lr > 0.0) || !std::isfinite(h.lr) || !(h.beta1 >= 0.0 && h.beta1 < 1.0) ||
      !(h.beta2 >= 0.0 && h.beta2 < 1.0) || !(h.eps > 0.0) || !std::isfinite(h.eps) ||
      !(h.weight_decay >= 0.0) || !std::isfinite(h.weight_decay))
    return kCkptBadHyper;
  if (h.batch != t.batch || h.precision != t.precision || h.step < 0) return kCkptOtherRun;
  if (h.n != t.n || std::memcmp(h.stats, t.stats, sizeof(h.stats)) != 0) return kCkptOtherData;
  return kCkptOk;
}

}  // namespace gmc
