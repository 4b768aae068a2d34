// Host-side rules that decide what the kernels are given: each cell's
// network condition and routing, the checks of a solve's grid and source and
// the source CDF births search, the sizes a solve on rectangular cells
// accepts, the ranges of the configuration, of the training data and of the
// training configuration the C ABI accepts, and the bookkeeping of the
// serving engine's device-memory pool. Plain C++ with no CUDA headers (the C
// ABI's gmc.h only), so a host-only unit test checks them (against the
// oracle where it has a counterpart) without a GPU.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

#include "gmc.h"

namespace gmc {

// The scattering-equivalent condition of a cell (tau, c) in the training box
// [t_lo, t_hi] x [c_lo, c_hi] of the networks. The networks learn the
// implicit-capture walk (flights at rate c, absorption applied afterwards as
// exp(-(1 - c) s), Eq. 4-5), which in a cell of side tau is the walk at rate
// 1 in a cell of side c tau with every length divided by c: a cell (tau', c')
// with c' tau' = c tau has the same exits, and s = s' c' / c. Inside the box
// (tau', c') = (tau, c); outside, c' is the value of [max(c_lo, c tau / t_hi),
// min(c_hi, c tau / t_lo)] nearest c and tau' = c tau / c' (clamped into the
// box against rounding). Returns false where that interval is empty or
// c tau = 0: no equivalent.
inline bool equivalent_condition(double tau, double c, double t_lo, double t_hi, double c_lo,
                                 double c_hi, double *tau_n, double *c_n) {
  *tau_n = tau;
  *c_n = c;
  if (tau >= t_lo && tau <= t_hi && c >= c_lo && c <= c_hi) return true;
  const double w = c * tau;
  const double lo = std::max(c_lo, w / t_hi), hi = std::min(c_hi, w / t_lo);
  if (!(w > 0.0) || !(lo <= hi)) return false;
  *c_n = std::min(std::max(c, lo), std::max(lo, hi));
  *tau_n = std::min(std::max(w / *c_n, t_lo), t_hi);
  return true;
}

// equivalent_condition for a rectangular cell with optical sides tx, ty: the
// implicit-capture walk in the rectangle depends on (c tx, c ty) only, and
// the network sees either side as the depth behind the entry face, so both
// must lie in [t_lo, t_hi]: c' is c moved into [c_lo, c_hi] and
// [c max(tx, ty) / t_hi, c min(tx, ty) / t_lo], tx' = c tx / c' (clamped into
// the box against rounding), ty' = tx' ty / tx. Cells inside the box keep
// (tx, c). Returns false where that interval is empty or c = 0. With
// tx = ty this is equivalent_condition.
inline bool equivalent_condition_rect(double tx, double ty, double c, double t_lo, double t_hi,
                                      double c_lo, double c_hi, double *tx_n, double *c_n) {
  *tx_n = tx;
  *c_n = c;
  if (tx >= t_lo && tx <= t_hi && ty >= t_lo && ty <= t_hi && c >= c_lo && c <= c_hi) return true;
  const double big = std::max(tx, ty), small = std::min(tx, ty);
  const double lo = std::max(c_lo, c * big / t_hi), hi = std::min(c_hi, c * small / t_lo);
  if (!(c * small > 0.0) || !(lo <= hi)) return false;
  *c_n = std::min(std::max(c, lo), std::max(lo, hi));
  *tx_n = std::min(std::max(c * tx / *c_n, t_lo), t_hi);
  return true;
}

// What stage 1 and stage 3 of a GMC solve read per cell: the network's
// condition (ln tau', c'), the track-length factor c' / c, and whether the
// random walk crosses the cell instead (no equivalent condition, or thinner
// than min_tau when min_tau > 0). FP64 arithmetic, stored as the kernels
// read it.
struct CellCondition {
  float ltau_n;
  float c_n;
  float s_scale;
  uint8_t walk;
};

// ty > 0: a rectangular cell of optical sides tau (along x) and ty, whose
// condition holds ln tx' (the kernels add ln(ty / tau) for entries through
// the bottom or top face); ty <= 0: a square cell of side tau.
inline CellCondition cell_condition(double tau, double c, double t_lo, double t_hi, double c_lo,
                                    double c_hi, double min_tau, double ty = 0.0) {
  double tn, cn;
  const bool ok = ty > 0.0 ? equivalent_condition_rect(tau, ty, c, t_lo, t_hi, c_lo, c_hi, &tn, &cn)
                           : equivalent_condition(tau, c, t_lo, t_hi, c_lo, c_hi, &tn, &cn);
  CellCondition r;
  r.ltau_n = (float)std::log(tn);
  r.c_n = (float)cn;
  r.s_scale = ok ? (float)(cn / c) : 1.0f;
  r.walk = (!ok || (min_tau > 0.0 && tau < min_tau)) ? 1 : 0;
  return r;
}

// Checks a solve's cells and source and accumulates the source CDF that
// births search (FP64, in cell order): every cell needs tau > 0 (finite) and
// c in [0, 1]; a volumetric source (wall false) has ncell strengths, a
// surface source on the left boundary (wall true) ny, each finite and >= 0.
// cdf[k] is the sum of the first k + 1 strengths (ncell entries, or ny), and
// *total the sum of all. Returns 0, or for the first defect in cell order
// (a cell's tau and c before its source strength) 1 (tau or c of cell
// *bad), 2 (the volumetric strength of cell *bad) or 3 (the wall strength
// of row *bad).
inline int grid_source_check(int64_t ncell, int ny, const float *tau, const float *c,
                             const float *source, bool wall, double *cdf, double *total,
                             int64_t *bad) {
  double acc = 0.0;
  for (int64_t k = 0; k < ncell; ++k) {
    if (!(tau[k] > 0.0f) || !std::isfinite(tau[k]) || !(c[k] >= 0.0f && c[k] <= 1.0f)) {
      *bad = k;
      return 1;
    }
    if (wall) continue;
    if (!(source[k] >= 0.0f) || !std::isfinite(source[k])) {
      *bad = k;
      return 2;
    }
    acc += source[k] > 0.0f ? (double)source[k] : 0.0;
    cdf[k] = acc;
  }
  for (int j = 0; wall && j < ny; ++j) {
    if (!(source[j] >= 0.0f) || !std::isfinite(source[j])) {
      *bad = j;
      return 3;
    }
    acc += source[j] > 0.0f ? (double)source[j] : 0.0;
    cdf[j] = acc;
  }
  *total = acc;
  return 0;
}

// Sizes of a solve on rectangular cells dx x dy with cross sections sigma[n]:
// the kernels form a cell's height as its optical width sigma dx times
// dy / dx in FP32, so dx and dy must be finite and > 0, dy / dx within
// [1e-37, 1e37], and every sigma dy within (0, 1e38] (room for the rounding
// of the product). Returns 0 when the sizes are accepted; 1 for dx or dy,
// 2 for the aspect, 3 for a cell, whose index goes to *bad_cell.
inline int rect_sizes_check(const float *sigma, size_t n, float dx, float dy, size_t *bad_cell) {
  if (!(dx > 0.0f) || !(dy > 0.0f) || !std::isfinite(dx) || !std::isfinite(dy)) return 1;
  const double ry = (double)dy / (double)dx;
  if (!(ry >= 1e-37 && ry <= 1e37)) return 2;
  for (size_t k = 0; k < n; ++k) {
    const double h = (double)sigma[k] * dy;
    if (!(h > 0.0 && h <= 1e38)) {
      *bad_cell = k;
      return 3;
    }
  }
  return 0;
}

// The ranges gmc_set_config accepts. Returns 0, or the first field out of
// range: 1 steps (1..256), 2 integrator, 3 precision, 4 w_cut (>= 0) or
// p_survive ((0, 1]), 5 bank_capacity (1024..2^28), 6 flights_per_wave
// (>= 1), 7 gmc_min_tau (>= 0), 8 the networks' box (0 < tau_lo <= tau_hi
// finite, 0 < c_lo <= c_hi <= 1), 9 sampler_kernel.
inline int config_check(const gmc_config &c) {
  if (c.steps < 1 || c.steps > 256) return 1;
  if (c.integrator != GMC_EULER && c.integrator != GMC_MIDPOINT && c.integrator != GMC_RK4) return 2;
  if (c.precision < GMC_FP32 || c.precision > GMC_FP8) return 3;
  if (!(c.w_cut >= 0.0) || !(c.p_survive > 0.0 && c.p_survive <= 1.0)) return 4;
  if (c.bank_capacity < 1024 || c.bank_capacity > ((int64_t)1 << 28)) return 5;
  if (c.flights_per_wave < 1) return 6;
  if (!(c.gmc_min_tau >= 0.0)) return 7;
  if (!(c.net_tau_lo > 0.0 && c.net_tau_hi >= c.net_tau_lo && std::isfinite(c.net_tau_hi)) ||
      !(c.net_c_lo > 0.0 && c.net_c_hi >= c.net_c_lo && c.net_c_hi <= 1.0))
    return 8;
  if (c.sampler_kernel != GMC_KERNEL_TILE && c.sampler_kernel != GMC_KERNEL_PAIR) return 9;
  return 0;
}

// The ranges a training-data generator draws from: tau log-uniform in
// [tau_lo, tau_hi] with 0 < tau_lo <= tau_hi finite, c uniform in
// [c_lo, c_hi] within [0, 1], and for rectangular cells the aspect
// tau_y / tau_x log-uniform in [aspect_lo, aspect_hi] with
// 0 < aspect_lo <= aspect_hi finite (1, 1 for square cells).
inline bool data_ranges_ok(float tau_lo, float tau_hi, float c_lo, float c_hi,
                           float aspect_lo = 1.0f, float aspect_hi = 1.0f) {
  return tau_lo > 0.0f && tau_hi >= tau_lo && std::isfinite(tau_hi) && c_lo >= 0.0f &&
         c_hi >= c_lo && c_hi <= 1.0f && aspect_lo > 0.0f && aspect_hi >= aspect_lo &&
         std::isfinite(aspect_hi);
}

// The training configuration gmc_train_begin accepts. Returns 0, or 1 batch
// (1..2^20), 2 lr (> 0, finite), 3 precision (GMC_FP32 or GMC_BF16), 4 the
// optimizer's constants (betas in [0, 1), eps > 0, weight decay >= 0, all
// finite): the ranges a checkpoint's hyperparameters are held to as well.
inline int train_config_check(const gmc_train_config &c) {
  if (c.batch < 1 || c.batch > (1 << 20)) return 1;
  if (!(c.lr > 0.0) || !std::isfinite(c.lr)) return 2;
  if (c.precision != GMC_FP32 && c.precision != GMC_BF16) return 3;
  if (!(c.beta1 >= 0.0 && c.beta1 < 1.0) || !(c.beta2 >= 0.0 && c.beta2 < 1.0) ||
      !(c.eps > 0.0) || !std::isfinite(c.eps) || !(c.weight_decay >= 0.0) ||
      !std::isfinite(c.weight_decay))
    return 4;
  return 0;
}

// Free regions of the serving engine's device-memory pool: first fit by
// offset (a request takes the lowest-addressed free region that holds its
// footprint, from that region's start), and a released region merges with
// free neighbours, so releasing everything leaves one region again.
class FreeList {
 public:
  void reset(size_t bytes) {
    free_.clear();
    if (bytes) free_[0] = bytes;
  }
  bool alloc(size_t bytes, size_t *off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  // offset -> length of every free region, in address order
  const std::map<size_t, size_t> &regions() const { return free_; }

 private:
  std::map<size_t, size_t> free_;
};

}  // namespace gmc
