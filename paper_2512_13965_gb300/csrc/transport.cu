// Transport solves: the four-stage GMC transport algorithm (and the standard
// MC walk it replaces) as an event loop over waves of in-flight particles,
// with several solves ("requests") sharing one particle bank.
//
// Particle banks (structure of arrays, double-buffered, capacity C each):
//   face bank: particles entering a cell through a face -- hist u64 (history
//     id = Philox id), slot i32 (request), cell i32, face i32 (global face the
//     particle entered through), xi f32 (canonical entry position), gx, gy f32
//     (global direction), w f32 (weight), ev u32 (next Philox event): 40 B;
//   inside bank: random walks in progress inside a cell -- position and track
//     length (f64, in the precision the cell walks in), direction, weight,
//     next Philox event, collisions so far: 64 B.
// One wave:
//   births   new histories of every admitted request fill free room of the
//            banks (fair share), birth cell and point from Philox (id, 0,
//            tag 4). GMC with an internal (volumetric-source) network loaded:
//            one batch of the internal model samples every birth's exit from
//            its cell (condition X, Y, ln tau, c and the distance to the
//            nearest face; noise at (id, 0, tag 2)), then stages 3-4 as below.
//            Otherwise (and for ANALOG) the birth direction from the same draw
//            starts a random walk in the inside bank;
//   inside   every walk in progress takes up to flights_per_wave more
//            flights of the implicit-capture walk (Eq. 4); a walk that leaves
//            its cell does stages 3-4 below, the others stay in the bank, so
//            no wave waits for the longest walk;
//   GMC      face particles -- prep: rotate into the canonical left-entry
//            frame (stage 1), build the condition and draw z ~ N(0, I) at
//            (id, ev, tag 2); sampler: the fused flow-ODE kernel (stage 2);
//            post: attenuate and tally (stage 3, Eq. 5-7), rotate back,
//            roulette, cross into the neighbour, compact survivors (stage 4);
//   ANALOG   face particles start their walk through the cell (Eq. 4), up
//            to flights_per_wave flights, then as for the inside bank.
// A resumed walk draws the same random numbers as an uninterrupted one, so
// the cap changes no result.
// Tallies: per request, FP64 atomics into flux[ny*nx]; Delta w / (V sigma_a)
// with V = 1. Per-history random numbers depend only on (request seed,
// history id, event), and sampler rows are independent, so a request's
// result does not depend on which other requests share its waves (up to the
// order of FP64 additions).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "decode.cuh"
#include "gmc_internal.cuh"
#include "host_rules.h"
#include "philox.cuh"
#include "walk.cuh"

namespace gmc {

constexpr int kMaxSlots = 64;

namespace {

struct Bank {
  uint64_t *hist;
  int32_t *slot, *cell, *face;
  float *xi, *gx, *gy, *w;
  uint32_t *ev;
};
constexpr size_t kBankBytesPerParticle = 40;

// Walks in progress inside a cell.
struct IBank {
  uint64_t *hist;
  double *x, *y, *s;
  int32_t *slot, *cell;
  float *ux, *uy, *w;
  uint32_t *ev, *ncoll;
};
constexpr size_t kIBankBytesPerParticle = 64;

struct DevStats {
  double leaked, absorbed, roulette_net;
  unsigned long long transmissions, collisions, kills, inward;
};

// one admitted request, as the kernels see it
struct Slot {
  int nx, ny;
  const float *tau, *c;
  double *flux;
  uint64_t seed;
  // GMC solves, per cell: the networks' condition (ln tau', c'), the factor
  // c'/c of a sampled track length (scattering-equivalent condition, 1 inside
  // the training box), and whether the random walk crosses the cell instead
  // (no equivalent condition, or thinner than gmc_min_tau)
  const float *ltau_n, *c_n, *s_scale;
  const uint8_t *walk;
  // x-y geometry: every cell the cross-section of an infinite prism,
  // directions 3-D (carried as their projection on the plane)
  int xy;
  // rectangular cells (transport_solve_rect): tau holds the optical width
  // tx = sigma dx, the height is tx ry (ry = dy / dx, lry = ln ry), and a
  // flux score is divided by dy as well (Delta w / (sigma_a dx dy))
  int rect;
  float ry, lry, dy;
};

struct Rules {
  float w_cut, p_survive;
};

// Where stage 4 appends the survivors: the face bank, or, in a GMC solve
// (gmc set) for a destination cell the random walk crosses (Slot::walk), the
// bank of face particles the random walk transmits.
struct Route {
  Bank out;
  int *count;
  Bank thin;
  int *thin_count;
  bool gmc;
};

// rotate (ux, uy) by k quarter turns counter-clockwise
__device__ __forceinline__ void rot(float &ux, float &uy, int k) {
  const float a = ux, b = uy;
  switch (k & 3) {
    case 0: ux = a; uy = b; break;
    case 1: ux = -b; uy = a; break;
    case 2: ux = -a; uy = -b; break;
    default: ux = b; uy = -a; break;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// A finished cell transmission of one lane.
struct Exit {
  bool active;
  int slot;
  uint64_t hist;
  int cell, gface;   // cell crossed, global exit face
  float q;           // counter-clockwise position on that face
  float gx, gy;      // global direction
  float w, s;        // weight on entry, track length (optical)
  uint32_t ev;       // next Philox event
  uint32_t ncoll;
};

// Stages 3 and 4: deposit, attenuate, roulette, cross; appends survivors to
// `out` (warp-aggregated) and counts them per request. Every lane of the
// warp calls this (inactive lanes with active = false).
__device__ __forceinline__ void put_face(Bank out, int k, const Exit &x, int ncell, int nface,
                                         float w) {
  out.hist[k] = x.hist;
  out.slot[k] = x.slot;
  out.cell[k] = ncell;
  out.face[k] = nface;
  out.xi[k] = x.q;
  out.gx[k] = x.gx;
  out.gy[k] = x.gy;
  out.w[k] = w;
  out.ev[k] = x.ev;
}

// BLOCK: every thread of the block calls this exactly once (grid kernels);
// the per-request statistics are then combined over the block before the
// atomics, one set per block when all its warps serve one request.
template <bool BLOCK = false>
__device__ void finish_transmission(const Exit &x, const Slot *__restrict__ slots, Rules R,
                                    const Route &rt, DevStats *st, int *slot_live) {
  double dabs = 0.0, dleak = 0.0, droul = 0.0;
  unsigned long long kills = 0;
  bool keep = false, thin = false;
  int ncell = 0, nface = 0;
  float w = 0.0f;
  if (x.active) {
    const Slot S = slots[x.slot];
    const float tau = S.tau[x.cell], cc = S.c[x.cell];
    const float a = 1.0f - cc;
    float dw;
    double score;
    if (a > 0.0f) {
      dw = x.w * (-expm1f(-a * x.s));                       // Eq. 6
      score = (double)dw / ((double)a * (double)tau);       // Eq. 7
    } else {
      dw = 0.0f;
      score = (double)x.w * (double)x.s / (double)tau;
    }
    if (S.rect) score /= (double)S.dy;                      // per unit area dx dy
    atomicAdd(&S.flux[x.cell], score);
    dabs = dw;
    w = x.w - dw;                                           // Eq. 5
    bool alive = true;
    if (w < R.w_cut) {
      const float u = u01(philox_draw(S.seed, x.hist, x.ev, kTagRoulette).x);
      if (u <= R.p_survive) {
        droul = (double)(w / R.p_survive) - (double)w;
        w = w / R.p_survive;
      } else {
        droul = -(double)w;
        kills = 1;
        alive = false;
      }
    }
    if (alive) {
      const int i = x.cell % S.nx, j = x.cell / S.nx;
      const int ni = i + (x.gface == 1) - (x.gface == 3);
      const int nj = j + (x.gface == 2) - (x.gface == 0);
      if (ni < 0 || ni >= S.nx || nj < 0 || nj >= S.ny) {
        dleak = w;
      } else {
        keep = true;
        ncell = nj * S.nx + ni;
        nface = (x.gface + 2) & 3;
        thin = rt.gmc && S.walk[ncell] != 0;
      }
    }
  }
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const unsigned mask_f = __ballot_sync(0xffffffffu, keep && !thin);
  const unsigned mask_t = __ballot_sync(0xffffffffu, keep && thin);
  const unsigned mask = mask_f | mask_t;
  int base_f = 0, base_t = 0;
  if (lane == 0 && mask_f) base_f = atomicAdd(rt.count, __popc(mask_f));
  if (lane == 0 && mask_t) base_t = atomicAdd(rt.thin_count, __popc(mask_t));
  base_f = __shfl_sync(0xffffffffu, base_f, 0);
  base_t = __shfl_sync(0xffffffffu, base_t, 0);
  if (keep && !thin) put_face(rt.out, base_f + __popc(mask_f & below), x, ncell, nface, w);
  if (keep && thin) put_face(rt.thin, base_t + __popc(mask_t & below), x, ncell, nface, w);
  // statistics and survivor counts per request: warp-reduced when every
  // active lane belongs to the same request (the common case: births of a
  // request are contiguous and compaction keeps warp order), per lane otherwise
  const unsigned act = __ballot_sync(0xffffffffu, x.active);
  if (!BLOCK && !act) return;
  const int lead = act ? __ffs(act) - 1 : 0;
  const int slot0 = __shfl_sync(0xffffffffu, x.slot, lead);
  const bool uniform = __all_sync(0xffffffffu, !x.active || x.slot == slot0);
  if constexpr (BLOCK) {
    __shared__ double s_d[32][3];              // absorbed, leaked, roulette per warp
    __shared__ unsigned long long s_u[32][4];  // transmissions, collisions, kills, survivors
    __shared__ int s_slot[32];                 // the warp's request; -1 none, -2 mixed
    const int wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    double ab = 0.0, lk = 0.0, ro = 0.0;
    unsigned long long nc = 0, nk = 0;
    if (uniform) {
      ab = warp_sum(dabs);
      lk = warp_sum(dleak);
      ro = warp_sum(droul);
      nc = warp_sum((unsigned long long)(x.active ? x.ncoll : 0u));
      nk = warp_sum(kills);
    }
    if (lane == 0) {
      s_slot[wid] = !act ? -1 : (uniform ? slot0 : -2);
      s_d[wid][0] = ab;
      s_d[wid][1] = lk;
      s_d[wid][2] = ro;
      s_u[wid][0] = (unsigned long long)__popc(act);
      s_u[wid][1] = nc;
      s_u[wid][2] = nk;
      s_u[wid][3] = (unsigned long long)__popc(mask);
    }
    __syncthreads();
    int bslot = -1;
    bool same = true;
    for (int i = 0; i < nw; ++i) {
      const int si = s_slot[i];
      if (si == -2 || (si >= 0 && bslot >= 0 && si != bslot)) same = false;
      if (si >= 0 && bslot < 0) bslot = si;
    }
    if (same) {
      if (threadIdx.x == 0 && bslot >= 0) {
        double t[3] = {0.0, 0.0, 0.0};
        unsigned long long u[4] = {0, 0, 0, 0};
        for (int i = 0; i < nw; ++i) {  // warp order: a fixed summation order
          for (int j = 0; j < 3; ++j) t[j] += s_d[i][j];
          for (int j = 0; j < 4; ++j) u[j] += s_u[i][j];
        }
        DevStats *sp = st + bslot;
        atomicAdd(&sp->absorbed, t[0]);
        atomicAdd(&sp->leaked, t[1]);
        atomicAdd(&sp->roulette_net, t[2]);
        atomicAdd(&sp->transmissions, u[0]);
        atomicAdd(&sp->collisions, u[1]);
        atomicAdd(&sp->kills, u[2]);
        if (u[3]) atomicAdd(&slot_live[bslot], (int)u[3]);
      }
      return;
    }
    if (!act) return;
    if (uniform) {
      if (lane == 0) {
        DevStats *sp = st + slot0;
        atomicAdd(&sp->absorbed, ab);
        atomicAdd(&sp->leaked, lk);
        atomicAdd(&sp->roulette_net, ro);
        atomicAdd(&sp->transmissions, (unsigned long long)__popc(act));
        atomicAdd(&sp->collisions, nc);
        atomicAdd(&sp->kills, nk);
        if (mask) atomicAdd(&slot_live[slot0], __popc(mask));
      }
      return;
    }
  }
  if (uniform) {
    dabs = warp_sum(dabs);
    dleak = warp_sum(dleak);
    droul = warp_sum(droul);
    const unsigned long long nc = warp_sum((unsigned long long)(x.active ? x.ncoll : 0u));
    const unsigned long long nk = warp_sum(kills);
    if (lane == 0) {
      DevStats *s = st + slot0;
      atomicAdd(&s->absorbed, dabs);
      atomicAdd(&s->leaked, dleak);
      atomicAdd(&s->roulette_net, droul);
      atomicAdd(&s->transmissions, (unsigned long long)__popc(act));
      atomicAdd(&s->collisions, nc);
      atomicAdd(&s->kills, nk);
      if (mask) atomicAdd(&slot_live[slot0], __popc(mask));
    }
  } else if (x.active) {
    DevStats *s = st + x.slot;
    atomicAdd(&s->absorbed, dabs);
    atomicAdd(&s->leaked, dleak);
    atomicAdd(&s->roulette_net, droul);
    atomicAdd(&s->transmissions, 1ull);
    atomicAdd(&s->collisions, (unsigned long long)x.ncoll);
    atomicAdd(&s->kills, kills);
    if (keep) atomicAdd(&slot_live[x.slot], 1);
  }
}

// Appends the lanes with `keep` set to the inside bank (warp-aggregated) and
// counts them per request. Every lane of the warp must call it.
__device__ void append_inside(bool keep, int slot, uint64_t hist, int cell, const WalkState &ws,
                              float w, IBank out, int *count, int *slot_live) {
  const int lane = threadIdx.x & 31;
  const unsigned mask = __ballot_sync(0xffffffffu, keep);
  if (!mask) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(count, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (keep) {
    const int k = base + __popc(mask & ((1u << lane) - 1u));
    out.hist[k] = hist;
    out.x[k] = ws.x;
    out.y[k] = ws.y;
    out.s[k] = ws.s;
    out.slot[k] = slot;
    out.cell[k] = cell;
    out.ux[k] = ws.ux;
    out.uy[k] = ws.uy;
    out.w[k] = w;
    out.ev[k] = ws.event;
    out.ncoll[k] = ws.ncoll;
  }
  const int lead = __ffs(mask) - 1;
  const int slot0 = __shfl_sync(0xffffffffu, slot, lead);
  const bool uniform = __all_sync(0xffffffffu, !keep || slot == slot0);
  if (uniform) {
    if (lane == 0) atomicAdd(&slot_live[slot0], __popc(mask));
  } else if (keep) {
    atomicAdd(&slot_live[slot], 1);
  }
}

// Direction of a volumetric birth: isotropic on the circle (angle 2 pi u3 of
// the birth draw) or, in x-y geometry, on the sphere with that azimuth and
// polar cosine 2 u - 1, u the first uniform of the draw (h, 1, tag 4),
// projected on the plane.
__device__ __forceinline__ void birth_direction(const Slot &S, uint64_t h, const uint4 &r,
                                                float &ux, float &uy) {
  if (S.xy) {
    float sp, cp;
    sincospif(2.0f * u01(r.w), &sp, &cp);
    const float mu = 2.0f * u01(philox_draw(S.seed, h, 1u, kTagBirth).x) - 1.0f;
    const float rr = sqrtf(fmaxf(1.0f - mu * mu, 0.0f));
    ux = rr * cp;
    uy = rr * sp;
  } else {
    sincospif(2.0f * u01(r.w), &uy, &ux);
  }
}

__device__ __forceinline__ int64_t cdf_search(const double *cdf, int64_t n, double target) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (cdf[mid] >= target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Births of histories first .. first+count-1 of the request in `slot`: a
// walk starting at the birth point (walked by the next wave).
__global__ void birth_kernel(int slot, int64_t first, int64_t count, const double *__restrict__ cdf,
                             double total, const Slot *__restrict__ slots, IBank out, int *in_count,
                             int *slot_live) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool keep = k < count;
  WalkState ws{};
  int cell = 0;
  uint64_t h = 0;
  if (keep) {
    const Slot S = slots[slot];
    h = (uint64_t)(first + k);
    const uint4 r = philox_draw(S.seed, h, 0u, kTagBirth);
    const double u0 = ((double)r.x + 1.0) * (1.0 / 4294967296.0);
    cell = (int)cdf_search(cdf, (int64_t)S.nx * S.ny, u0 * total);
    float ux, uy;
    birth_direction(S, h, r, ux, uy);
    ws = S.rect ? walk_start_rect(S.tau[cell], S.tau[cell] * S.ry, u01(r.y), u01(r.z), ux, uy, 0u)
                : walk_start(S.tau[cell], u01(r.y), u01(r.z), ux, uy, 0u);
  }
  append_inside(keep, slot, h, cell, ws, 1.0f, out, in_count, slot_live);
}

// Births of a surface source on the left boundary (x = 0): history h of the
// request in `slot` draws (u0, u1, u2, -) at (h, 0, tag 4), enters boundary
// row j (the first whose cumulative wall strength reaches u0 total) through
// the west face of cell (0, j) at canonical position xi = u1, with the cosine
// law for its direction, sin theta = 2 u2 - 1 (an isotropic radiance seen
// through the boundary), and joins the face bank at base + k with weight 1.
// In x-y geometry the cosine law is the 3-D one: cosine to the inward normal
// mu = sqrt(u2), azimuth about it 2 pi u3, projection (mu, sqrt(1 - mu^2)
// cos(2 pi u3)).
__global__ void birth_wall_kernel(int slot, int64_t first, int64_t count,
                                  const double *__restrict__ cdf, double total,
                                  const Slot *__restrict__ slots, Route rt, int *slot_live) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = k < count;
  const Slot S = slots[slot];
  uint64_t h = 0;
  int cell = 0;
  float xi = 0.0f, gx = 0.0f, gy = 0.0f;
  bool thin = false;
  if (valid) {
    h = (uint64_t)(first + k);
    const uint4 r = philox_draw(S.seed, h, 0u, kTagBirth);
    const double u0 = ((double)r.x + 1.0) * (1.0 / 4294967296.0);
    const int j = (int)cdf_search(cdf, (int64_t)S.ny, u0 * total);
    cell = j * S.nx;
    xi = u01(r.y);
    if (S.xy) {
      gx = sqrtf(u01(r.z));
      gy = sqrtf(fmaxf(1.0f - gx * gx, 0.0f)) * cospif(2.0f * u01(r.w));
    } else {
      const float sn = 2.0f * u01(r.z) - 1.0f;
      gx = sqrtf(fmaxf(1.0f - sn * sn, 0.0f));
      gy = sn;
    }
    thin = rt.gmc && S.walk[cell] != 0;  // a cell the random walk crosses
  }
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const unsigned mask_f = __ballot_sync(0xffffffffu, valid && !thin);
  const unsigned mask_t = __ballot_sync(0xffffffffu, valid && thin);
  int base_f = 0, base_t = 0;
  if (lane == 0 && mask_f) base_f = atomicAdd(rt.count, __popc(mask_f));
  if (lane == 0 && mask_t) base_t = atomicAdd(rt.thin_count, __popc(mask_t));
  if (lane == 0 && (mask_f | mask_t)) atomicAdd(&slot_live[slot], __popc(mask_f | mask_t));
  base_f = __shfl_sync(0xffffffffu, base_f, 0);
  base_t = __shfl_sync(0xffffffffu, base_t, 0);
  if (!valid) return;
  const Bank out = thin ? rt.thin : rt.out;
  const int64_t o = thin ? base_t + __popc(mask_t & below) : base_f + __popc(mask_f & below);
  out.hist[o] = h;
  out.slot[o] = slot;
  out.cell[o] = cell;
  out.face[o] = 3;
  out.xi[o] = xi;
  out.gx[o] = gx;
  out.gy[o] = gy;
  out.w[o] = 1.0f;
  out.ev[o] = 0u;
}

// Ends or parks one lane's walk: an exit (or absorption) becomes the Exit of
// stages 3-4, a walk cut by the flight cap goes back to the inside bank.
__device__ __forceinline__ void settle(const WalkResult &wr, const WalkState &ws, int slot,
                                       uint64_t h, int cell, float w, Exit &x, bool &park) {
  park = wr.status == kTruncated && ws.ncoll < kMaxFlights;
  x.active = !park;
  x.slot = slot;
  x.hist = h;
  x.cell = cell;
  x.gface = wr.face < 0 ? 0 : wr.face;
  x.q = wr.q;
  x.gx = wr.ux;
  x.gy = wr.uy;
  x.w = w;
  x.s = wr.s;
  x.ev = wr.event;
  x.ncoll = wr.ncoll;
}

// Up to `cap` more flights of every walk in progress (FROM_FACE false: the
// inside bank `iin`), or the start of the walk of every face particle
// through its cell (FROM_FACE true: the face bank `fin`; the ANALOG method
// and the thin cells of a hybrid GMC solve) in the cell's own
// (global-oriented) frame, entering at the point its entry face and xi give.
// A walk that leaves its cell does stages 3-4; one cut by the cap is parked
// in `iout` for the next wave. Persistent, with lane refill (walk.cuh): the
// lanes claim particles from *next in rounds of kWalkRound flights, and the
// warp-collective stage 3-4 and parking run only in rounds where a lane's
// walk ended.
constexpr int kWalkThreads = 256;

template <bool FROM_FACE>
__global__ void __launch_bounds__(kWalkThreads) walk_wave_kernel(
    int64_t live, Bank fin, IBank iin, const Slot *__restrict__ slots, Rules R, uint32_t cap,
    Route rt, IBank iout, int *in_count, DevStats *st, int *slot_live, unsigned long long *next) {
  int64_t k = live;  // this lane's particle (live: none)
  bool drained = false;
  WalkState ws{};
  int slot = 0, cell = 0;
  uint64_t h = 0, seed = 0;
  float w = 0.0f, tau = 0.0f, cc = 0.0f;
  uint32_t budget = 0;
  bool sph = false, rect = false;
  float ty = 0.0f;
  for (;;) {
    const bool need = k == live && !drained;
    if (__any_sync(0xffffffffu, need)) {
      const int64_t kk = warp_claim(need, next, live);
      if (need) {
        if (kk < live) {
          k = kk;
          if constexpr (FROM_FACE) {
            slot = fin.slot[k];
            cell = fin.cell[k];
            h = fin.hist[k];
            w = fin.w[k];
          } else {
            slot = iin.slot[k];
            cell = iin.cell[k];
            h = iin.hist[k];
            w = iin.w[k];
          }
          const Slot S = slots[slot];
          tau = S.tau[cell];
          cc = S.c[cell];
          seed = S.seed;
          sph = S.xy != 0;
          rect = S.rect != 0;
          ty = tau * S.ry;
          budget = cap;
          if constexpr (FROM_FACE) {
            // point on face F with counter-clockwise parameter 1 - xi
            const float xi = fin.xi[k];
            float X, Y;
            switch (fin.face[k]) {
              case 0: X = 1.0f - xi; Y = 0.0f; break;
              case 1: X = 1.0f; Y = 1.0f - xi; break;
              case 2: X = xi; Y = 1.0f; break;
              default: X = 0.0f; Y = xi; break;
            }
            ws = rect ? walk_start_rect(tau, ty, X, Y, fin.gx[k], fin.gy[k], fin.ev[k])
                      : walk_start(tau, X, Y, fin.gx[k], fin.gy[k], fin.ev[k]);
          } else {
            ws.x = iin.x[k];
            ws.y = iin.y[k];
            ws.s = iin.s[k];
            ws.ux = iin.ux[k];
            ws.uy = iin.uy[k];
            ws.event = iin.ev[k];
            ws.ncoll = iin.ncoll[k];
          }
        } else {
          drained = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, k < live)) break;
    bool ended = false;
    WalkResult wr;
    if (k < live) {
      const uint32_t r = budget < kWalkRound ? budget : kWalkRound;
      wr = rect ? walk_cell_resume_rect(tau, ty, cc, 1, ws, r, seed, h)
                : walk_cell_resume(tau, cc, 1, ws, r, seed, h, sph);
      budget -= r;
      ended = wr.status != kTruncated || budget == 0 || ws.ncoll >= kMaxFlights;
    }
    if (__any_sync(0xffffffffu, ended)) {
      Exit x;
      x.active = false;
      x.slot = 0;
      bool park = false;
      if (ended) settle(wr, ws, slot, h, cell, w, x, park);
      finish_transmission(x, slots, R, rt, st, slot_live);
      append_inside(ended && park, slot, h, cell, ws, w, iout, in_count, slot_live);
      if (ended) k = live;
    }
  }
}

// GMC births with the internal model, stage 1: rows base .. base+count-1 of
// the birth batch (row stride M): history, request and cell, the internal
// condition (X, Y, ln tau, c, min(X, Y, 1 - X, 1 - Y)) and z ~ N(0, I) at
// (id, 0, tag 2). Birth point and cell are those of birth_kernel; the
// condition takes the cell's network condition (ln tau', c'). A birth in a
// cell the random walk crosses (Slot::walk) starts a random walk in the
// inside bank instead (direction from the same draw) and its batch row is
// marked unused.
__global__ void birth_gmc_kernel(int slot, int64_t first, int64_t count, int64_t base, int64_t M,
                                 const double *__restrict__ cdf, double total,
                                 const Slot *__restrict__ slots, uint64_t *bhist, int32_t *bslot,
                                 int32_t *bcell, float *cond, float *noise,
                                 IBank iout, int *in_count, int *slot_live) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool walk = false;
  WalkState ws{};
  int cell = 0;
  uint64_t h = 0;
  if (k < count) {
    const Slot S = slots[slot];
    h = (uint64_t)(first + k);
    const uint4 r = philox_draw(S.seed, h, 0u, kTagBirth);
    const double u0 = ((double)r.x + 1.0) * (1.0 / 4294967296.0);
    cell = (int)cdf_search(cdf, (int64_t)S.nx * S.ny, u0 * total);
    const float X = u01(r.y), Y = u01(r.z);
    const float tau = S.tau[cell];
    const int64_t row = base + k;
    bhist[row] = h;
    bcell[row] = cell;
    walk = S.walk[cell] != 0;
    bslot[row] = walk ? -1 : slot;
    cond[row] = X;
    cond[M + row] = Y;
    cond[2 * M + row] = S.ltau_n[cell];
    cond[3 * M + row] = S.c_n[cell];
    cond[4 * M + row] = fminf(fminf(X, Y), fminf(1.0f - X, 1.0f - Y));
    const float4 z = box_muller4(philox_draw(S.seed, h, 0u, kTagNoise));
    noise[row] = z.x;
    noise[M + row] = z.y;
    noise[2 * M + row] = z.z;
    noise[3 * M + row] = z.w;
    if (walk) {
      float ux, uy;
      birth_direction(S, h, r, ux, uy);
      ws = walk_start(tau, X, Y, ux, uy, 0u);
    }
  }
  append_inside(walk, slot, h, cell, ws, 1.0f, iout, in_count, slot_live);
}

// GMC births, stages 3-4 from the internal model's decoded exits (p, ux, uy,
// s), which are already in the cell's own (global-oriented) frame.
__global__ void birth_gmc_post_kernel(int64_t M, const uint64_t *__restrict__ bhist,
                                      const int32_t *__restrict__ bslot,
                                      const int32_t *__restrict__ bcell, const float *__restrict__ ex,
                                      const Slot *__restrict__ slots, Rules R, Route rt,
                                      DevStats *st, int *slot_live) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Exit x;
  x.active = k < M && bslot[k] >= 0;  // rows of walked births are unused
  x.slot = 0;
  if (x.active) {
    const float p = ex[k];
    const int fc = min((int)p, 3);
    x.slot = bslot[k];
    x.hist = bhist[k];
    x.cell = bcell[k];
    x.gface = fc;
    x.q = fminf(fmaxf(p - (float)fc, 0.0f), 1.0f);
    x.gx = ex[M + k];
    x.gy = ex[2 * M + k];
    x.w = 1.0f;
    x.s = ex[3 * M + k] * slots[x.slot].s_scale[x.cell];
    x.ev = 1u;  // event 0 held the birth draw and the noise
    x.ncoll = 0;
  }
  finish_transmission<true>(x, slots, R, rt, st, slot_live);
}

// GMC stage 1 and the noise of stage 2.
__global__ void gmc_prep_kernel(int64_t live, Bank in, const Slot *__restrict__ slots, float *cond,
                                float *noise) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= live) return;
  const Slot S = slots[in.slot[k]];
  const int cell = in.cell[k], F = in.face[k];
  float ux = in.gx[k], uy = in.gy[k];
  rot(ux, uy, -((F + 1) & 3));
  cond[k] = in.xi[k];
  cond[live + k] = ux;
  cond[2 * live + k] = uy;
  cond[3 * live + k] = S.ltau_n[cell];
  cond[4 * live + k] = S.c_n[cell];
  if (S.rect) {
    // canonical sides: a quarter turn exchanges width and height
    const bool odd = ((F + 1) & 1) != 0;
    cond[3 * live + k] = S.ltau_n[cell] + (odd ? S.lry : 0.0f);
    cond[5 * live + k] = odd ? -S.lry : S.lry;
  }
  const float4 z = box_muller4(philox_draw(S.seed, in.hist[k], in.ev[k], kTagNoise));
  noise[k] = z.x;
  noise[live + k] = z.y;
  noise[2 * live + k] = z.z;
  noise[3 * live + k] = z.w;
}

// GMC stages 3 and 4 from the sampler's decoded exits (p, ux, uy, s).
__global__ void gmc_post_kernel(int64_t live, Bank in, const float *__restrict__ ex,
                                const Slot *__restrict__ slots, Rules R, Route rt, DevStats *st,
                                int *slot_live) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Exit x;
  x.active = k < live;
  x.slot = 0;
  if (x.active) {
    const int F = in.face[k], r = (F + 1) & 3;
    const float p = ex[k];
    float ux = ex[live + k], uy = ex[2 * live + k];
    const int fc = min((int)p, 3);
    x.slot = in.slot[k];
    x.hist = in.hist[k];
    x.cell = in.cell[k];
    x.gface = (fc + r) & 3;
    x.q = fminf(fmaxf(p - (float)fc, 0.0f), 1.0f);
    rot(ux, uy, r);
    x.gx = ux;
    x.gy = uy;
    x.w = in.w[k];
    x.s = ex[3 * live + k] * slots[x.slot].s_scale[x.cell];
    x.ev = in.ev[k] + 1u;
    x.ncoll = 0;
  }
  finish_transmission<true>(x, slots, R, rt, st, slot_live);
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

Bank carve(void *base, int64_t C) {
  Bank b;
  char *p = (char *)base;
  b.hist = (uint64_t *)p; p += 8 * C;
  b.slot = (int32_t *)p; p += 4 * C;
  b.cell = (int32_t *)p; p += 4 * C;
  b.face = (int32_t *)p; p += 4 * C;
  b.xi = (float *)p; p += 4 * C;
  b.gx = (float *)p; p += 4 * C;
  b.gy = (float *)p; p += 4 * C;
  b.w = (float *)p; p += 4 * C;
  b.ev = (uint32_t *)p;
  return b;
}

IBank carve_inside(void *base, int64_t C) {
  IBank b;
  char *p = (char *)base;
  b.hist = (uint64_t *)p; p += 8 * C;
  b.x = (double *)p; p += 8 * C;
  b.y = (double *)p; p += 8 * C;
  b.s = (double *)p; p += 8 * C;
  b.slot = (int32_t *)p; p += 4 * C;
  b.cell = (int32_t *)p; p += 4 * C;
  b.ux = (float *)p; p += 4 * C;
  b.uy = (float *)p; p += 4 * C;
  b.w = (float *)p; p += 4 * C;
  b.ev = (uint32_t *)p; p += 4 * C;
  b.ncoll = (uint32_t *)p;
  return b;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// ----------------------------------------------------------------------------
// Host side: requests, a device-memory pool, the wave engine, the server.

struct Request {
  uint64_t ticket = 0;
  int nx = 0, ny = 0;
  int64_t ncell = 0;
  std::vector<float> tau, c;
  std::vector<float> ltau_n, c_n, s_scale;  // network condition and track-length factor
  std::vector<uint8_t> walk;                // cells the random walk crosses (GMC)
  std::vector<double> cdf;
  double total = 0.0;
  int64_t n_hist = 0;
  uint64_t seed = 0;
  int method = GMC_METHOD_ANALOG;
  bool wall = false;  // source on the left boundary (cdf over the ny rows)
  bool xy = false;    // x-y geometry (transport_solve_xy, transport_solve_wall_xy)
  bool rect = false;  // rectangular cells dx x dy (transport_solve_rect); tau holds sigma dx
  float dx = 1.0f, dy = 1.0f;
  // engine state
  int slot = -1;
  int64_t next_hist = 0;
  int live = 0;
  int64_t wave0 = 0;  // engine wave count at admission
  size_t pool_off = 0, footprint = 0;
  double *d_cdf = nullptr, *d_flux = nullptr;
  float *d_tau = nullptr, *d_c = nullptr;
  float *d_ltau_n = nullptr, *d_c_n = nullptr, *d_s_scale = nullptr;
  uint8_t *d_walk = nullptr;
  // result
  std::vector<double> flux;
  gmc_solve_stats st{};
  gmc_status status = GMC_OK;
  bool done = false;
  double t_submit = 0.0, t_done = 0.0;
  cudaEvent_t ev0 = nullptr;
};

// Device bytes of one request: tau, c, ln tau', c', c'/c (float), walk flags
// (byte), source CDF and FP64 tally.
size_t request_footprint(int64_t ncell) {
  return 5 * align256(ncell * 4) + align256(ncell) + 2 * align256(ncell * 8);
}

// Validates a solve description and copies it into a Request.
// wall: `source` holds ny strengths of a surface source on the left boundary
// instead of ny*nx volumetric strengths.
gmc_status make_request(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                        const float *source, int64_t n_histories, int method, uint64_t seed,
                        Request &R, bool wall = false, bool xy = false, bool rect = false,
                        double aspect = 1.0) {
  if (nx < 1 || ny < 1 || (int64_t)nx * ny > (1 << 26))
    return set_error(ctx, GMC_EINVAL, "solve: grid must be 1..2^26 cells");
  if (!tau || !c || !source) return set_error(ctx, GMC_EINVAL, "solve: null array");
  if (n_histories < 0) return set_error(ctx, GMC_EINVAL, "solve: n_histories < 0");
  if (method != GMC_METHOD_ANALOG && method != GMC_METHOD_GMC)
    return set_error(ctx, GMC_EINVAL, "solve: unknown method");
  const int64_t ncell = (int64_t)nx * ny;
  R.nx = nx;
  R.ny = ny;
  R.ncell = ncell;
  R.tau.assign(tau, tau + ncell);
  R.c.assign(c, c + ncell);
  R.cdf.resize(ncell);
  double acc = 0.0;
  int64_t bad = 0;
  switch (grid_source_check(ncell, ny, tau, c, source, wall, R.cdf.data(), &acc, &bad)) {
    case 0: break;
    case 1:
      return set_error(ctx, GMC_EINVAL, "solve: cell %lld needs tau > 0, c in [0,1]", (long long)bad);
    case 2: return set_error(ctx, GMC_EINVAL, "solve: source must be finite and >= 0");
    default: return set_error(ctx, GMC_EINVAL, "solve: wall source must be finite and >= 0");
  }
  // the networks' condition per cell (GMC): the scattering-equivalent one,
  // or the random walk where there is none or the cell is thinner than
  // gmc_min_tau; FP64 on the host
  const gmc_config &cf = ctx->cfg;
  R.ltau_n.resize(ncell);
  R.c_n.resize(ncell);
  R.s_scale.resize(ncell);
  R.walk.assign(ncell, 0);
  for (int64_t k = 0; k < ncell; ++k) {
    // rectangular cells: tau holds the optical width, the height is tau dy/dx
    const CellCondition cc =
        cell_condition((double)tau[k], (double)c[k], cf.net_tau_lo, cf.net_tau_hi, cf.net_c_lo,
                       cf.net_c_hi, cf.gmc_min_tau, rect ? (double)tau[k] * aspect : 0.0);
    R.ltau_n[k] = cc.ltau_n;
    R.c_n[k] = cc.c_n;
    R.s_scale[k] = cc.s_scale;
    R.walk[k] = cc.walk;
  }
  R.wall = wall;
  R.xy = xy;
  R.rect = rect;
  if (rect && method == GMC_METHOD_GMC) {
    // rectangular cells: the boundary network must take the aspect (six
    // condition rows); births are walked
    if (!ctx->net.loaded || ctx->net.stats.ncond != kCondRect)
      return set_error(ctx, GMC_EINVAL,
                       "rectangular-cell solve: GMC needs a network of rectangular cells");
    if (check_net_path(ctx, ctx->net, ctx->cfg.precision, ctx->cfg.sampler_kernel,
                       "rectangular-cell solve") != GMC_OK)
      return GMC_EINVAL;
  }
  // the square solves' cells: a network of rectangular cells (six
  // condition rows) has no place in them
  if (method == GMC_METHOD_GMC && !rect) {
    const NetDev *nets[4] = {&ctx->net, &ctx->internal, &ctx->xy, &ctx->internal_xy};
    for (const NetDev *N : nets)
      if (N->loaded && N->stats.ncond != kCond &&
          (xy ? (N == &ctx->xy || N == &ctx->internal_xy) : (N == &ctx->net || N == &ctx->internal)))
        return set_error(ctx, GMC_EINVAL, "solve: a rectangular-cell network cannot sample square cells");
  }
  if (n_histories > 0 && !(acc > 0.0)) return set_error(ctx, GMC_EINVAL, "solve: zero source");
  if (xy && method == GMC_METHOD_GMC) {
    // the x-y boundary network; births by the x-y internal model when loaded,
    // walked otherwise
    if (!ctx->xy.loaded)
      return set_error(ctx, GMC_ENOWEIGHTS, "x-y solve: GMC needs gmc_load_xy_weights");
    if (check_net_path(ctx, ctx->xy, ctx->cfg.precision, ctx->cfg.sampler_kernel, "x-y solve") != GMC_OK ||
        (ctx->internal_xy.loaded && check_net_path(ctx, ctx->internal_xy, ctx->cfg.precision,
                                                   ctx->cfg.sampler_kernel, "x-y solve") != GMC_OK))
      return GMC_EINVAL;
  } else if (method == GMC_METHOD_GMC && !ctx->net.loaded) {
    return set_error(ctx, GMC_ENOWEIGHTS, "solve: GMC needs gmc_load_weights");
  }
  if (method == GMC_METHOD_GMC && !xy && !rect) {
    const gmc_config &cf = ctx->cfg;
    if (check_net_path(ctx, ctx->net, cf.precision, cf.sampler_kernel, "solve") != GMC_OK ||
        (ctx->internal.loaded &&
         check_net_path(ctx, ctx->internal, cf.precision, cf.sampler_kernel, "solve") != GMC_OK))
      return GMC_EINVAL;
  }
  R.total = acc;
  R.n_hist = n_histories;
  R.method = method;
  R.seed = seed;
  R.footprint = request_footprint(ncell);
  return GMC_OK;
}

// First-fit sub-allocator over one device buffer (admission by memory).
class Pool {
 public:
  cudaError_t init(size_t bytes) {
    bytes_ = align256(bytes);
    cudaError_t e = cudaMalloc(&base_, bytes_);
    if (e == cudaSuccess) list_.reset(bytes_);
    return e;
  }
  ~Pool() {
    if (base_) cudaFree(base_);
  }
  size_t capacity() const { return bytes_; }
  bool alloc(size_t bytes, size_t *off) { return list_.alloc(bytes, off); }
  void release(size_t off, size_t bytes) { list_.release(off, bytes); }
  char *base() const { return (char *)base_; }

 private:
  void *base_ = nullptr;
  size_t bytes_ = 0;
  FreeList list_;
};

// The wave engine: every admitted request owns a slot, a pool region (grid,
// CDF, tally) and its share of the particle bank.
class Engine {
 public:
  Engine(gmc_ctx *ctx, int method, int64_t capacity, size_t pool_bytes, cudaStream_t stream)
      : ctx_(ctx), method_(method), C_(capacity), pool_bytes_(pool_bytes), s_(stream) {}

  ~Engine() {
    cudaStreamSynchronize(s_);
    void *bufs[] = {bank_mem_[0], bank_mem_[1], ibank_mem_[0], ibank_mem_[1], tbank_mem_[0],
                    tbank_mem_[1], d_cond_, d_noise_, d_exit_, d_slots_, d_stats_, d_counts_,
                    d_bias1_, d_bmeta_, d_next_};
    for (void *b : bufs)
      if (b) cudaFree(b);
    if (h_counts_) cudaFreeHost(h_counts_);
  }

  gmc_status init() {
    GMC_CUDA_TRY(ctx_, pool_.init(pool_bytes_));
    GMC_CUDA_TRY(ctx_, cudaMalloc(&bank_mem_[0], C_ * kBankBytesPerParticle));
    GMC_CUDA_TRY(ctx_, cudaMalloc(&bank_mem_[1], C_ * kBankBytesPerParticle));
    GMC_CUDA_TRY(ctx_, cudaMalloc(&ibank_mem_[0], C_ * kIBankBytesPerParticle));
    GMC_CUDA_TRY(ctx_, cudaMalloc(&ibank_mem_[1], C_ * kIBankBytesPerParticle));
    if (method_ == GMC_METHOD_GMC) {
      GMC_CUDA_TRY(ctx_, cudaMalloc(&d_cond_, C_ * 6 * sizeof(float)));  // 6 rows: rectangular cells
      GMC_CUDA_TRY(ctx_, cudaMalloc(&d_noise_, C_ * 4 * sizeof(float)));
      GMC_CUDA_TRY(ctx_, cudaMalloc(&d_exit_, C_ * 4 * sizeof(float)));
      GMC_CUDA_TRY(ctx_, cudaMalloc(&d_bias1_, 2 * kBias1Floats * sizeof(float)));
      GMC_CUDA_TRY(ctx_, cudaMalloc(&d_bmeta_, C_ * 16));  // birth batch: hist, slot, cell
      GMC_CUDA_TRY(ctx_, cudaMalloc(&tbank_mem_[0], C_ * kBankBytesPerParticle));
      GMC_CUDA_TRY(ctx_, cudaMalloc(&tbank_mem_[1], C_ * kBankBytesPerParticle));
    }
    GMC_CUDA_TRY(ctx_, cudaMalloc(&d_slots_, kMaxSlots * sizeof(Slot)));
    GMC_CUDA_TRY(ctx_, cudaMalloc(&d_stats_, kMaxSlots * sizeof(DevStats)));
    GMC_CUDA_TRY(ctx_, cudaMalloc(&d_counts_, kCounts * sizeof(int)));
    GMC_CUDA_TRY(ctx_, cudaMalloc(&d_next_, 3 * sizeof(unsigned long long)));
    GMC_CUDA_TRY(ctx_, cudaMallocHost(&h_counts_, kCounts * sizeof(int)));
    bank_[0] = carve(bank_mem_[0], C_);
    bank_[1] = carve(bank_mem_[1], C_);
    ibank_[0] = carve_inside(ibank_mem_[0], C_);
    ibank_[1] = carve_inside(ibank_mem_[1], C_);
    // the thin-cell face banks exist for GMC solves only; ANALOG routes nothing there
    tbank_[0] = carve(tbank_mem_[0] ? tbank_mem_[0] : bank_mem_[0], C_);
    tbank_[1] = carve(tbank_mem_[1] ? tbank_mem_[1] : bank_mem_[1], C_);
    for (auto &r : reqs_) r = nullptr;
    return GMC_OK;
  }

  int method() const { return method_; }
  cudaStream_t stream() const { return s_; }
  int64_t capacity() const { return C_; }
  size_t pool_capacity() const { return pool_.capacity(); }
  bool idle() const { return active_ == 0; }
  int active() const { return active_; }

  // Admits R if a slot and its pool footprint are free; false otherwise.
  // The requests in the engine at one time share a geometry (their face
  // particles go through one network).
  bool try_admit(Request *R, gmc_status *err) {
    *err = GMC_OK;
    if (active_ >= kMaxSlots) return false;
    if (active_ > 0 && (R->xy != xy_ || R->rect != rect_)) return false;
    size_t off;
    if (!pool_.alloc(R->footprint, &off)) return false;
    int slot = -1;
    for (int k = 0; k < kMaxSlots; ++k)
      if (!reqs_[k]) {
        slot = k;
        break;
      }
    char *p = pool_.base() + off;
    const int64_t n = R->ncell;
    R->pool_off = off;
    const size_t a4 = align256(n * 4), a8 = align256(n * 8);
    R->d_tau = (float *)p;
    R->d_c = (float *)(p + a4);
    R->d_ltau_n = (float *)(p + 2 * a4);
    R->d_c_n = (float *)(p + 3 * a4);
    R->d_s_scale = (float *)(p + 4 * a4);
    R->d_cdf = (double *)(p + 5 * a4);
    R->d_flux = (double *)(p + 5 * a4 + a8);
    R->d_walk = (uint8_t *)(p + 5 * a4 + 2 * a8);
    Slot S{R->nx, R->ny, R->d_tau, R->d_c, R->d_flux, R->seed,
           R->d_ltau_n, R->d_c_n, R->d_s_scale, R->d_walk, R->xy ? 1 : 0,
           R->rect ? 1 : 0, R->dy / R->dx, std::log(R->dy / R->dx), R->dy};
    cudaError_t e = cudaMemcpyAsync(R->d_tau, R->tau.data(), n * 4, cudaMemcpyHostToDevice, s_);
    if (!e) e = cudaMemcpyAsync(R->d_c, R->c.data(), n * 4, cudaMemcpyHostToDevice, s_);
    if (!e) e = cudaMemcpyAsync(R->d_ltau_n, R->ltau_n.data(), n * 4, cudaMemcpyHostToDevice, s_);
    if (!e) e = cudaMemcpyAsync(R->d_c_n, R->c_n.data(), n * 4, cudaMemcpyHostToDevice, s_);
    if (!e) e = cudaMemcpyAsync(R->d_s_scale, R->s_scale.data(), n * 4, cudaMemcpyHostToDevice, s_);
    if (!e) e = cudaMemcpyAsync(R->d_walk, R->walk.data(), n, cudaMemcpyHostToDevice, s_);
    if (!e) e = cudaMemcpyAsync(R->d_cdf, R->cdf.data(), n * 8, cudaMemcpyHostToDevice, s_);
    if (!e) e = cudaMemsetAsync(R->d_flux, 0, n * 8, s_);
    if (!e) e = cudaMemcpyAsync(d_slots_ + slot, &S, sizeof(Slot), cudaMemcpyHostToDevice, s_);
    if (!e) e = cudaMemsetAsync(d_stats_ + slot, 0, sizeof(DevStats), s_);
    if (!e) e = cudaStreamSynchronize(s_);  // host vectors and S are read by the copies
    if (e) {
      pool_.release(off, R->footprint);
      *err = cuda_error(ctx_, e, "admitting a solve");
      return false;
    }
    if (!R->ev0) cudaEventCreate(&R->ev0);
    cudaEventRecord(R->ev0, s_);
    R->slot = slot;
    R->next_hist = 0;
    R->live = 0;
    R->wave0 = waves_;
    reqs_[slot] = R;
    ++active_;
    xy_ = R->xy;
    rect_ = R->rect;
    return true;
  }

  // One wave: births for every request with histories left, one step of
  // every particle in the banks (a transmission of each face particle, up to
  // flights_per_wave flights of each walk in progress), completion of
  // finished requests.
  gmc_status step(std::vector<Request *> &completed) {
    const Rules rules{(float)ctx_->cfg.w_cut, (float)ctx_->cfg.p_survive};
    const uint32_t cap = (uint32_t)ctx_->cfg.flights_per_wave;
    const bool gmc = method_ == GMC_METHOD_GMC;
    int *d_face = d_counts_, *d_in = d_counts_ + 1, *d_thin = d_counts_ + 2,
        *d_slot_live = d_counts_ + 3;
    // births: fair share of the free room among requests with histories left
    int pending = 0, pending_wall = 0;
    for (auto *R : reqs_)
      if (R && R->next_hist < R->n_hist) ++(R->wall ? pending_wall : pending);
    int64_t room = C_ - live_ - live_in_ - live_thin_;
    if (pending_wall > 0 && room > 0) {
      // surface-source births enter the current face banks directly (the
      // random walk's bank for cells it crosses in a GMC solve)
      GMC_CUDA_TRY(ctx_, set_counts());
      const Route wroute{bank_[cur_], d_face, tbank_[ctn_], d_thin, gmc};
      int left = pending + pending_wall;
      for (auto *R : reqs_) {
        if (!R || !R->wall || R->next_hist >= R->n_hist) continue;
        const int64_t m = std::min<int64_t>(room / left, R->n_hist - R->next_hist);
        --left;
        if (m <= 0) continue;
        birth_wall_kernel<<<nblocks(m, 256), 256, 0, s_>>>(R->slot, R->next_hist, m, R->d_cdf,
                                                            R->total, d_slots_, wroute, d_slot_live);
        GMC_CUDA_TRY(ctx_, cudaGetLastError());
        R->next_hist += m;
        room -= m;
      }
      GMC_CUDA_TRY(ctx_, read_counts());
      live_ = h_counts_[0];
      live_thin_ = h_counts_[2];
      for (auto *R : reqs_)
        if (R) R->live += h_counts_[3 + R->slot];
    }
    const NetDev &inet = xy_ ? ctx_->internal_xy : ctx_->internal;
    if (pending > 0 && room > 0 && method_ == GMC_METHOD_GMC && inet.loaded && !rect_) {
      const gmc_status sb = births_internal(pending, room, rules);
      if (sb != GMC_OK) return sb;
    } else if (pending > 0 && room > 0) {
      GMC_CUDA_TRY(ctx_, set_counts());
      int left = pending;
      for (auto *R : reqs_) {
        if (!R || R->wall || R->next_hist >= R->n_hist) continue;
        const int64_t share = room / left;
        const int64_t m = std::min<int64_t>(share, R->n_hist - R->next_hist);
        --left;
        if (m <= 0) continue;
        room -= m;
        birth_kernel<<<nblocks(m, 256), 256, 0, s_>>>(R->slot, R->next_hist, m, R->d_cdf, R->total,
                                                       d_slots_, ibank_[cin_], d_in, d_slot_live);
        GMC_CUDA_TRY(ctx_, cudaGetLastError());
        R->next_hist += m;
      }
      GMC_CUDA_TRY(ctx_, read_counts());
      live_in_ = h_counts_[1];
      for (auto *R : reqs_)
        if (R) R->live += h_counts_[3 + R->slot];
    }
    if (live_ + live_in_ + live_thin_ > 0) {
      ++waves_;
      const int nxt = cur_ ^ 1, nin = cin_ ^ 1, ntn = ctn_ ^ 1;
      const Route route{bank_[nxt], d_face, tbank_[ntn], d_thin, gmc};
      GMC_CUDA_TRY(ctx_, cudaMemsetAsync(d_counts_, 0, kCounts * sizeof(int), s_));
      GMC_CUDA_TRY(ctx_, cudaMemsetAsync(d_next_, 0, 3 * sizeof(unsigned long long), s_));
      if (live_in_ > 0) {
        walk_wave_kernel<false>
            <<<persistent_blocks(walk_wave_kernel<false>, kWalkThreads, live_in_), kWalkThreads, 0,
               s_>>>(live_in_, bank_[cur_], ibank_[cin_], d_slots_, rules, cap, route, ibank_[nin],
                     d_in, d_stats_, d_slot_live, d_next_);
        GMC_CUDA_TRY(ctx_, cudaGetLastError());
      }
      if (live_thin_ > 0) {  // face particles of thin cells in a GMC solve: random walk
        walk_wave_kernel<true>
            <<<persistent_blocks(walk_wave_kernel<true>, kWalkThreads, live_thin_), kWalkThreads,
               0, s_>>>(live_thin_, tbank_[ctn_], ibank_[cin_], d_slots_, rules, cap, route,
                        ibank_[nin], d_in, d_stats_, d_slot_live, d_next_ + 1);
        GMC_CUDA_TRY(ctx_, cudaGetLastError());
      }
      if (live_ > 0 && method_ == GMC_METHOD_ANALOG) {
        walk_wave_kernel<true>
            <<<persistent_blocks(walk_wave_kernel<true>, kWalkThreads, live_), kWalkThreads, 0,
               s_>>>(live_, bank_[cur_], ibank_[cin_], d_slots_, rules, cap, route, ibank_[nin],
                     d_in, d_stats_, d_slot_live, d_next_ + 2);
        GMC_CUDA_TRY(ctx_, cudaGetLastError());
      } else if (live_ > 0) {
        gmc_prep_kernel<<<nblocks(live_, 256), 256, 0, s_>>>(live_, bank_[cur_], d_slots_, d_cond_,
                                                             d_noise_);
        GMC_CUDA_TRY(ctx_, cudaGetLastError());
        gmc_status es = sample(xy_ ? ctx_->xy : ctx_->net, live_);
        if (es != GMC_OK) return es;
        gmc_post_kernel<<<nblocks(live_, 256), 256, 0, s_>>>(live_, bank_[cur_], d_exit_, d_slots_,
                                                             rules, route, d_stats_, d_slot_live);
        GMC_CUDA_TRY(ctx_, cudaGetLastError());
      }
      GMC_CUDA_TRY(ctx_, read_counts());
      live_ = h_counts_[0];
      live_in_ = h_counts_[1];
      live_thin_ = h_counts_[2];
      for (auto *R : reqs_)
        if (R) R->live = h_counts_[3 + R->slot];
      cur_ = nxt;
      cin_ = nin;
      ctn_ = ntn;
      if (method_ == GMC_METHOD_GMC) {
        gmc_status es = check_device_error(ctx_);
        if (es != GMC_OK) return es;
      }
    }
    // completions
    for (int k = 0; k < kMaxSlots; ++k) {
      Request *R = reqs_[k];
      if (!R || R->next_hist < R->n_hist || R->live > 0) continue;
      GMC_CUDA_TRY(ctx_, finish(R));
      completed.push_back(R);
      reqs_[k] = nullptr;
      --active_;
    }
    return GMC_OK;
  }

 private:
  // Stage 2 on `rows` rows of d_cond_ / d_noise_ into d_exit_ with network N.
  gmc_status sample(const NetDev &N, int64_t rows) {
    const gmc_config &cfg = ctx_->cfg;
    cudaError_t e;
    if (cfg.precision == GMC_FP32)
      e = launch_sampler_f32(s_, N.f32, N.stats, rows, d_cond_, d_noise_, 0, 0, cfg.steps,
                             cfg.integrator, nullptr, d_exit_);
    else {
      const bool fp8 = cfg.precision == GMC_FP8;
      // the per-evaluation layer-1 bias depends on the network, the steps and
      // the integrator only: computed once per (network load, setting)
      const int nk = (&N == &ctx_->internal || &N == &ctx_->internal_xy) ? 1 : 0;
      Bias1Key &key = bias1_key_[nk];
      const bool ready = key.net == &N && key.generation == N.generation && key.steps == cfg.steps &&
                         key.integrator == cfg.integrator;
      e = launch_sampler_tc(s_, fp8 ? N.d_tc8 : N.d_tc, N.d_tc_bias, N.f32, N.stats, rows, d_cond_,
                            d_noise_, 0, 0, cfg.steps, cfg.integrator, nullptr, d_exit_,
                            ctx_->d_err, d_bias1_ + nk * kBias1Floats, fp8 ? N.d_tc8_scale : nullptr,
                            cfg.sampler_kernel, ready);
      if (e == cudaSuccess && rows > 0) key = Bias1Key{&N, N.generation, cfg.steps, cfg.integrator};
    }
    if (e != cudaSuccess) return cuda_error(ctx_, e, "solve: sampler");
    return GMC_OK;
  }

  // Births of this wave through the internal model: every request's share of
  // the free room is sampled in one batch, tallied in its birth cell and
  // appended to the face banks, so it crosses its first face in this wave;
  // births in cells the random walk crosses start random walks instead.
  gmc_status births_internal(int pending, int64_t room, const Rules &rules) {
    std::vector<std::pair<Request *, int64_t>> plan;
    int64_t M = 0;
    int left = pending;
    for (auto *R : reqs_) {
      if (!R || R->wall || R->next_hist >= R->n_hist) continue;
      const int64_t share = room / left;
      const int64_t m = std::min<int64_t>(share, R->n_hist - R->next_hist);
      --left;
      if (m <= 0) continue;
      room -= m;
      plan.emplace_back(R, m);
      M += m;
    }
    if (M == 0) return GMC_OK;
    uint64_t *bhist = (uint64_t *)d_bmeta_;
    int32_t *bslot = (int32_t *)((char *)d_bmeta_ + 8 * C_);
    int32_t *bcell = (int32_t *)((char *)d_bmeta_ + 12 * C_);
    int *d_face = d_counts_, *d_in = d_counts_ + 1, *d_thin = d_counts_ + 2,
        *d_slot_live = d_counts_ + 3;
    GMC_CUDA_TRY(ctx_, set_counts());
    int64_t base = 0;
    for (auto &pm : plan) {
      Request *R = pm.first;
      const int64_t m = pm.second;
      birth_gmc_kernel<<<nblocks(m, 256), 256, 0, s_>>>(R->slot, R->next_hist, m, base, M, R->d_cdf,
                                                         R->total, d_slots_, bhist, bslot, bcell,
                                                         d_cond_, d_noise_, ibank_[cin_],
                                                         d_in, d_slot_live);
      GMC_CUDA_TRY(ctx_, cudaGetLastError());
      R->next_hist += m;
      base += m;
    }
    gmc_status st = sample(xy_ ? ctx_->internal_xy : ctx_->internal, M);
    if (st != GMC_OK) return st;
    const Route route{bank_[cur_], d_face, tbank_[ctn_], d_thin, true};
    birth_gmc_post_kernel<<<nblocks(M, 256), 256, 0, s_>>>(M, bhist, bslot, bcell, d_exit_, d_slots_,
                                                           rules, route, d_stats_, d_slot_live);
    GMC_CUDA_TRY(ctx_, cudaGetLastError());
    GMC_CUDA_TRY(ctx_, read_counts());
    live_ = h_counts_[0];
    live_in_ = h_counts_[1];
    live_thin_ = h_counts_[2];
    for (auto *R : reqs_)
      if (R) R->live += h_counts_[3 + R->slot];
    return check_device_error(ctx_);
  }

  // Bank counters <- current live counts, survivor counts per slot <- 0 (for
  // births appending to the current banks).
  cudaError_t set_counts() {
    init_[0] = (int)live_;
    init_[1] = (int)live_in_;
    init_[2] = (int)live_thin_;
    cudaError_t e = cudaMemcpyAsync(d_counts_, init_, 3 * sizeof(int), cudaMemcpyHostToDevice, s_);
    if (e) return e;
    return cudaMemsetAsync(d_counts_ + 3, 0, kMaxSlots * sizeof(int), s_);
  }

  cudaError_t read_counts() {
    cudaError_t e = cudaMemcpyAsync(h_counts_, d_counts_, kCounts * sizeof(int),
                                    cudaMemcpyDeviceToHost, s_);
    if (e) return e;
    return cudaStreamSynchronize(s_);
  }

  cudaError_t finish(Request *R) {
    R->flux.resize(R->ncell);
    DevStats hs;
    cudaError_t e = cudaMemcpyAsync(R->flux.data(), R->d_flux, R->ncell * 8, cudaMemcpyDeviceToHost, s_);
    if (!e) e = cudaMemcpyAsync(&hs, d_stats_ + R->slot, sizeof(hs), cudaMemcpyDeviceToHost, s_);
    cudaEvent_t e1;
    cudaEventCreate(&e1);
    cudaEventRecord(e1, s_);
    if (!e) e = cudaStreamSynchronize(s_);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, R->ev0, e1);
    cudaEventDestroy(e1);
    cudaEventDestroy(R->ev0);
    R->ev0 = nullptr;
    pool_.release(R->pool_off, R->footprint);
    if (e) return e;
    const double inv = R->n_hist > 0 ? 1.0 / (double)R->n_hist : 0.0;
    for (auto &f : R->flux) f *= inv;
    R->st.leaked = hs.leaked;
    R->st.absorbed = hs.absorbed;
    R->st.roulette_net = hs.roulette_net;
    R->st.transmissions = (int64_t)hs.transmissions;
    R->st.collisions = (int64_t)hs.collisions;
    R->st.roulette_kills = (int64_t)hs.kills;
    R->st.waves = waves_ - R->wave0;
    R->st.inward_fixes = (int64_t)hs.inward;
    R->st.seconds = ms * 1e-3;
    R->t_done = now_s();
    R->st.latency = R->t_done - R->t_submit;
    R->done = true;
    return cudaSuccess;
  }

  gmc_ctx *ctx_;
  int method_;
  int64_t C_;
  size_t pool_bytes_;
  cudaStream_t s_;
  Pool pool_;
  // counters: [0] face bank, [1] inside bank, [2] thin-cell face bank,
  // [3 ..] live particles per slot
  static constexpr int kCounts = kMaxSlots + 3;
  void *bank_mem_[2] = {nullptr, nullptr}, *ibank_mem_[2] = {nullptr, nullptr},
       *tbank_mem_[2] = {nullptr, nullptr};
  Bank bank_[2], tbank_[2];
  IBank ibank_[2];
  int cur_ = 0, cin_ = 0, ctn_ = 0;
  int64_t live_ = 0, live_in_ = 0, live_thin_ = 0;
  int init_[3] = {0, 0, 0};  // host source of the counters copied before births
  int64_t waves_ = 0;
  float *d_cond_ = nullptr, *d_noise_ = nullptr, *d_exit_ = nullptr, *d_bias1_ = nullptr;
  // layer-1 bias of the boundary (0) and internal (1) networks: n_eval x 256
  // floats each, n_eval <= 4 x 256 steps; valid for the key it was computed with
  static constexpr size_t kBias1Floats = 4 * 256 * 256;
  struct Bias1Key {
    const NetDev *net = nullptr;
    uint64_t generation = 0;
    int steps = -1, integrator = -1;
  };
  Bias1Key bias1_key_[2];
  void *d_bmeta_ = nullptr;
  Slot *d_slots_ = nullptr;
  DevStats *d_stats_ = nullptr;
  int *d_counts_ = nullptr;
  unsigned long long *d_next_ = nullptr;  // work counters of the persistent walk kernels
  int *h_counts_ = nullptr;
  Request *reqs_[kMaxSlots];
  int active_ = 0;
  bool xy_ = false;    // geometry of the admitted requests
  bool rect_ = false;
};

// The server: a worker thread running the engine over admitted requests.
struct Server {
  gmc_ctx *ctx = nullptr;
  std::unique_ptr<Engine> engine;
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  gmc_status fatal = GMC_OK;
  int method = 0;

  void run() {
    cudaSetDevice(ctx->device);
    std::vector<Request *> done;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        if (!stop && engine->idle() && queue.empty())
          cv_work.wait_for(lk, std::chrono::milliseconds(50));
        if (stop) break;
        while (!queue.empty()) {
          gmc_status err;
          if (!engine->try_admit(queue.front(), &err)) {
            if (err != GMC_OK) {
              queue.front()->status = err;
              queue.front()->done = true;
              queue.pop_front();
              cv_done.notify_all();
              continue;
            }
            break;  // first-come first-served: wait until memory frees up
          }
          queue.pop_front();
        }
      }
      if (engine->idle()) continue;
      done.clear();
      const gmc_status st = engine->step(done);
      std::lock_guard<std::mutex> lk(mu);
      if (st != GMC_OK) {
        fatal = st;
        stop = true;
        cv_done.notify_all();
        break;
      }
      if (!done.empty()) cv_done.notify_all();
    }
  }
};

void server_free(Server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  S->engine.reset();
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

void engine_free(Engine *E) { delete E; }

}  // namespace gmc

using namespace gmc;

extern "C" {

namespace {
gmc_status solve_one(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                     const float *source, int64_t n_histories, int method, uint64_t seed,
                     double *flux, gmc_solve_stats *stats, bool wall, bool xy = false,
                     bool rect = false, float dx = 1.0f, float dy = 1.0f) {
  if (!ctx) return GMC_EINVAL;
  if (!flux) return set_error(ctx, GMC_EINVAL, "transport_solve: null flux");
  Request R;
  gmc_status st = make_request(ctx, nx, ny, tau, c, source, n_histories, method, seed, R, wall, xy,
                               rect, (double)dy / (double)dx);
  if (st != GMC_OK) return st;
  R.dx = dx;
  R.dy = dy;
  cudaSetDevice(ctx->device);
  const int64_t C = ctx->cfg.bank_capacity;
  Engine *E = ctx->solver;
  if (!E || E->method() != method || E->capacity() != C || E->pool_capacity() < R.footprint ||
      E->stream() != ctx->stream) {
    if (E) engine_free(E);
    ctx->solver = nullptr;
    E = new Engine(ctx, method, C, std::max<size_t>(R.footprint, (size_t)1 << 20), ctx->stream);
    st = E->init();
    if (st != GMC_OK) {
      engine_free(E);
      return st;
    }
    ctx->solver = E;
  }
  R.t_submit = now_s();
  gmc_status err;
  if (!E->try_admit(&R, &err)) return err != GMC_OK ? err : set_error(ctx, GMC_ENOMEM, "transport_solve: cannot admit");
  std::vector<Request *> done;
  while (!R.done) {
    st = E->step(done);
    if (st != GMC_OK) {
      engine_free(E);
      ctx->solver = nullptr;
      return st;
    }
  }
  std::memcpy(flux, R.flux.data(), R.ncell * sizeof(double));
  if (stats) *stats = R.st;
  return check_device_error(ctx);
}
}  // namespace

gmc_status transport_solve(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                           const float *source, int64_t n_histories, int method, uint64_t seed,
                           double *flux, gmc_solve_stats *stats) {
  return solve_one(ctx, nx, ny, tau, c, source, n_histories, method, seed, flux, stats, false);
}

gmc_status transport_solve_wall(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                                const float *wall, int64_t n_histories, int method, uint64_t seed,
                                double *flux, gmc_solve_stats *stats) {
  return solve_one(ctx, nx, ny, tau, c, wall, n_histories, method, seed, flux, stats, true);
}

gmc_status transport_solve_rect(gmc_ctx *ctx, int nx, int ny, const float *sigma, const float *c,
                                const float *source, float dx, float dy, int64_t n_histories,
                                int method, uint64_t seed, double *flux, gmc_solve_stats *stats) {
  if (!ctx) return GMC_EINVAL;
  if (nx < 1 || ny < 1 || (int64_t)nx * ny > (1 << 26) || !sigma)
    return set_error(ctx, GMC_EINVAL, "transport_solve_rect: grid must be 1..2^26 cells");
  size_t bad = 0;
  switch (rect_sizes_check(sigma, (size_t)nx * ny, dx, dy, &bad)) {
    case 0: break;
    case 1: return set_error(ctx, GMC_EINVAL, "transport_solve_rect: need finite dx, dy > 0");
    case 2:
      return set_error(ctx, GMC_EINVAL, "transport_solve_rect: dy / dx must lie in [1e-37, 1e37]");
    default:
      return set_error(ctx, GMC_EINVAL, "transport_solve_rect: cell %zu needs 0 < sigma dy <= 1e38",
                       bad);
  }
  // the cells' optical widths sigma dx (the heights follow as sigma dy)
  std::vector<float> tx((size_t)nx * ny);
  for (size_t k = 0; k < tx.size(); ++k) tx[k] = sigma[k] * dx;
  return solve_one(ctx, nx, ny, tx.data(), c, source, n_histories, method, seed, flux, stats, false,
                   false, true, dx, dy);
}

gmc_status transport_solve_xy(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                              const float *source, int64_t n_histories, int method, uint64_t seed,
                              double *flux, gmc_solve_stats *stats) {
  return solve_one(ctx, nx, ny, tau, c, source, n_histories, method, seed, flux, stats, false, true);
}

gmc_status transport_solve_wall_xy(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                                   const float *wall, int64_t n_histories, int method,
                                   uint64_t seed, double *flux, gmc_solve_stats *stats) {
  return solve_one(ctx, nx, ny, tau, c, wall, n_histories, method, seed, flux, stats, true, true);
}

gmc_status gmc_serve_start(gmc_ctx *ctx, const gmc_serve_config *cfg) {
  if (!ctx || !cfg) return GMC_EINVAL;
  if (ctx->server) return set_error(ctx, GMC_EBUSY, "gmc_serve_start: already serving");
  if (cfg->method != GMC_METHOD_ANALOG && cfg->method != GMC_METHOD_GMC)
    return set_error(ctx, GMC_EINVAL, "gmc_serve_start: unknown method");
  if (cfg->memory_budget < ((size_t)1 << 20))
    return set_error(ctx, GMC_EINVAL, "gmc_serve_start: memory_budget must be >= 1 MiB");
  if (cfg->method == GMC_METHOD_GMC && !ctx->net.loaded)
    return set_error(ctx, GMC_ENOWEIGHTS, "gmc_serve_start: GMC needs gmc_load_weights");
  if (cfg->method == GMC_METHOD_GMC &&
      (check_net_path(ctx, ctx->net, ctx->cfg.precision, ctx->cfg.sampler_kernel, "gmc_serve_start") != GMC_OK ||
       (ctx->internal.loaded && check_net_path(ctx, ctx->internal, ctx->cfg.precision,
                                               ctx->cfg.sampler_kernel, "gmc_serve_start") != GMC_OK)))
    return GMC_EINVAL;
  cudaSetDevice(ctx->device);
  Server *S = new Server();
  S->ctx = ctx;
  S->method = cfg->method;
  cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e) {
    delete S;
    return cuda_error(ctx, e, "gmc_serve_start: stream");
  }
  S->engine.reset(new Engine(ctx, cfg->method, ctx->cfg.bank_capacity, cfg->memory_budget, S->stream));
  gmc_status st = S->engine->init();
  if (st != GMC_OK) {
    server_free(S);
    return st;
  }
  S->worker = std::thread([S] { S->run(); });
  ctx->server = S;
  return GMC_OK;
}

gmc_status gmc_submit(gmc_ctx *ctx, const gmc_solve_req *req, uint64_t *ticket) {
  if (!ctx || !req || !ticket) return GMC_EINVAL;
  Server *S = ctx->server;
  if (!S) return set_error(ctx, GMC_EINVAL, "gmc_submit: call gmc_serve_start first");
  std::unique_ptr<Request> R(new Request());
  gmc_status st = make_request(ctx, req->nx, req->ny, req->tau, req->c, req->source,
                               req->n_histories, S->method, req->seed, *R);
  if (st != GMC_OK) return st;
  if (R->footprint > S->engine->pool_capacity())
    return set_error(ctx, GMC_ENOMEM, "gmc_submit: grid needs %zu bytes, budget is %zu",
                     R->footprint, S->engine->pool_capacity());
  R->t_submit = now_s();
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return S->fatal != GMC_OK ? S->fatal : set_error(ctx, GMC_EINVAL, "gmc_submit: server stopped");
  R->ticket = S->next_ticket++;
  *ticket = R->ticket;
  S->queue.push_back(R.get());
  S->all[R->ticket] = std::move(R);
  S->cv_work.notify_one();
  return GMC_OK;
}

static gmc_status take_result(gmc_ctx *ctx, Server *S, std::map<uint64_t, std::unique_ptr<Request>>::iterator it,
                              double *flux, gmc_solve_stats *stats) {
  Request *R = it->second.get();
  gmc_status st = R->status;
  if (st == GMC_OK) {
    if (flux) std::memcpy(flux, R->flux.data(), R->ncell * sizeof(double));
    if (stats) *stats = R->st;
  } else {
    set_error(ctx, st, "request %llu failed", (unsigned long long)R->ticket);
  }
  S->all.erase(it);
  return st;
}

gmc_status gmc_poll(gmc_ctx *ctx, uint64_t ticket, double *flux, gmc_solve_stats *stats) {
  if (!ctx) return GMC_EINVAL;
  Server *S = ctx->server;
  if (!S) return set_error(ctx, GMC_EINVAL, "gmc_poll: not serving");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return set_error(ctx, GMC_EINVAL, "gmc_poll: unknown ticket %llu", (unsigned long long)ticket);
  if (!it->second->done) return S->fatal != GMC_OK ? S->fatal : GMC_EBUSY;
  return take_result(ctx, S, it, flux, stats);
}

gmc_status gmc_wait(gmc_ctx *ctx, uint64_t ticket, double timeout_s, double *flux,
                    gmc_solve_stats *stats) {
  if (!ctx) return GMC_EINVAL;
  Server *S = ctx->server;
  if (!S) return set_error(ctx, GMC_EINVAL, "gmc_wait: not serving");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return set_error(ctx, GMC_EINVAL, "gmc_wait: unknown ticket %llu", (unsigned long long)ticket);
  Request *R = it->second.get();
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (!R->done && S->fatal == GMC_OK) {
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !R->done)
      return set_error(ctx, GMC_ETIMEOUT, "gmc_wait: request %llu not done", (unsigned long long)ticket);
  }
  if (!R->done) return S->fatal;
  return take_result(ctx, S, it, flux, stats);
}

gmc_status gmc_serve_stop(gmc_ctx *ctx) {
  if (!ctx) return GMC_EINVAL;
  Server *S = ctx->server;
  if (!S) return GMC_OK;
  const gmc_status fatal = S->fatal;
  server_free(S);
  ctx->server = nullptr;
  return fatal;
}

}  // extern "C"
