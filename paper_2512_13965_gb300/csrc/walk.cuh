// Random-walk transport through one square cell (section "Monte Carlo
// Method", Eq. 4): free flights d = -ln(u)/sigma with u in (0,1], step
// min(d_b, d), isotropic scattering; analog mode kills at a collision with
// probability 1 - c, implicit-capture mode samples flights with sigma = c and
// never kills. Used by analog_transmit, by the births of transport_solve and
// by its analog method.
//
// Position arithmetic runs in T (float, or double in optically thick cells);
// the variates (log, sincos) are drawn in float. In double cells the exit
// decision of a flight is the FP64 one, reached cheaply: the wall distances
// are first taken in FP32 from the FP64 gaps (flight_exits), and only a
// flight whose length, or whose two wall distances, lie within the FP32
// rounding bound of each other is decided by the FP64 divisions; an exiting
// flight's distance is always the FP64 quotient. Histories are therefore the
// same as with FP64 distances throughout.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "philox.cuh"

namespace gmc {

constexpr uint32_t kMaxFlights = 1u << 28;  // bound on one walk (never reached in practice)
constexpr float kTau64 = 64.0f;             // cells thicker than this walk in FP64

enum : int { kExited = 0, kAbsorbed = 1, kTruncated = 2 };

// Relative margin of the FP32 screen: an FP32 wall distance (the FP64 gap
// rounded to FP32, then divided in FP32) is within 2 roundings (1.2e-7) of
// the FP64 one; decisions closer than this margin are taken in FP64.
constexpr float kScreen = 5e-7f;

// Distance along the direction (ux, uy) from (x, y) to the wall it points at
// in [0, wx] x [0, wy], one axis: +inf when the component is zero.
template <typename T>
__device__ __forceinline__ T wall_distance(T w, T p, float u) {
  if (u > 0.0f) return (w - p) / (T)u;
  if (u < 0.0f) return -p / (T)u;
  return (T)INFINITY;
}

// Whether a flight of length d (a float value) from (x, y) with direction
// (ux, uy) reaches a wall of the box [0, wx] x [0, wy] first (d >= distance,
// ties exit), which wall (xface: a wall x = const; a corner picks x), and, if
// so, the distance db >= 0 in T. Equal to the plain T computation.
template <typename T>
__device__ __forceinline__ bool flight_exits(T wx, T wy, T x, T y, float ux, float uy, float d,
                                             bool &xface, T &db) {
  if constexpr (sizeof(T) == sizeof(double)) {
    bool sure = true;
    float fx = INFINITY, fy = INFINITY;
    if (ux != 0.0f) {
      const float g = (float)(ux > 0.0f ? wx - x : -x);
      sure = sure && fabsf(g) >= 1e-30f;
      fx = g / ux;
    }
    if (uy != 0.0f) {
      const float g = (float)(uy > 0.0f ? wy - y : -y);
      sure = sure && fabsf(g) >= 1e-30f;
      fy = g / uy;
    }
    const float lo = fminf(fx, fy), hi = fmaxf(fx, fy);
    sure = sure && lo > 1e-20f && lo < 1e30f &&
           (hi == INFINITY || lo <= hi * (1.0f - kScreen)) &&
           (d >= lo * (1.0f + kScreen) || d < lo * (1.0f - kScreen));
    if (sure) {
      xface = fx <= fy;
      if (d < lo) return false;
      db = xface ? wall_distance(wx, x, ux) : wall_distance(wy, y, uy);
      if (db < (T)0) db = (T)0;
      return true;
    }
  }
  const T dbx = wall_distance(wx, x, ux), dby = wall_distance(wy, y, uy);
  xface = dbx <= dby;
  db = xface ? dbx : dby;
  if (db < (T)0) db = (T)0;
  return (T)d >= db;
}

struct WalkResult {
  int status;       // kExited / kAbsorbed / kTruncated
  int face;         // exit face 0..3 (cell frame), -1 otherwise
  float q;          // counter-clockwise position on the exit face
  float ux, uy;     // final direction
  float s;          // track length, optical units
  uint32_t ncoll;   // collisions
  uint32_t event;   // next unused Philox event
};

// Up to max_flights flights of a walk in progress: position (x, y), track
// length s, direction, next Philox event and collision count are read and
// updated in place. Status kExited / kAbsorbed ends the walk; kTruncated means
// max_flights were taken and the walk resumes from the updated state, drawing
// exactly the random numbers an uninterrupted walk would. sphere: x-y
// geometry (the cell is the cross-section of an infinite prism): (ux, uy) is
// the projection of a 3-D direction, a flight of 3-D length d moves the
// position by d (ux, uy), and a scattering draws the direction on the sphere
// (azimuth 2 pi u2 as on the circle, polar cosine 2 u3 - 1), as walk_xy.
template <typename T>
__device__ __forceinline__ WalkResult walk_box_from(T tau, float c, int implicit, T &x, T &y, T &s,
                                                    float &ux, float &uy, uint32_t &event,
                                                    uint32_t &ncoll, uint32_t max_flights,
                                                    uint64_t seed, uint64_t id,
                                                    bool sphere = false) {
  const float rate = implicit ? c : 1.0f;
  WalkResult w;
  w.status = kTruncated;
  w.face = -1;
  w.q = 0.0f;
  for (uint32_t it = 0; it < max_flights; ++it) {
    const uint4 r = philox_draw(seed, id, event, kTagWalk);
    ++event;
    const float df = rate > 0.0f ? -logf(u01(r.x)) / rate : INFINITY;
    const T d = (T)df;
    bool xface;
    T db;
    if (flight_exits(tau, tau, x, y, ux, uy, df, xface, db)) {
      s += db;
      int face;
      T along;
      if (xface) {
        face = ux > 0.0f ? 1 : 3;
        along = y + db * (T)uy;
      } else {
        face = uy > 0.0f ? 2 : 0;
        along = x + db * (T)ux;
      }
      // counter-clockwise position: bottom x, right y, top tau - x, left tau - y
      T qn = (face == 0 || face == 1) ? along / tau : (tau - along) / tau;
      float q = (float)qn;
      q = fminf(fmaxf(q, 0.0f), 1.0f);
      w.status = kExited;
      w.face = face;
      w.q = q;
      break;
    }
    s += d;
    x += d * (T)ux;
    y += d * (T)uy;
    ++ncoll;
    if (!implicit && u01(r.y) > c) {
      w.status = kAbsorbed;
      break;
    }
    if (sphere) {
      float sp, cp;
      sincospif(2.0f * u01(r.z), &sp, &cp);
      const float mu = 2.0f * u01(r.w) - 1.0f;
      const float rr = sqrtf(fmaxf(1.0f - mu * mu, 0.0f));
      ux = rr * cp;
      uy = rr * sp;
    } else {
      sincospif(2.0f * u01(r.z), &uy, &ux);
    }
  }
  w.ux = ux;
  w.uy = uy;
  w.s = (float)s;
  w.ncoll = ncoll;
  w.event = event;
  return w;
}

template <typename T>
__device__ __forceinline__ WalkResult walk_box(T tau, float c, int implicit, T x, T y, float ux,
                                               float uy, uint64_t seed, uint64_t id,
                                               uint32_t event) {
  T s = 0;
  uint32_t ncoll = 0;
  return walk_box_from(tau, c, implicit, x, y, s, ux, uy, event, ncoll, kMaxFlights, seed, id);
}

// Persistent walk kernels refill their lanes: every lane walks one particle
// at a time, kWalkRound flights per round, and a lane whose walk has ended
// claims the next unprocessed particle. A warp then never idles while its
// longest walk finishes, and the grid no longer waits for its slowest block.
constexpr uint32_t kWalkRound = 8;

// Claims the next particle index for every lane of the warp with `need` set,
// with one atomic per warp on the counter *next; returns n once the n items
// are exhausted (and for lanes without `need`). Every lane must call it.
__device__ __forceinline__ int64_t warp_claim(bool need, unsigned long long *next, int64_t n) {
  const unsigned m = __ballot_sync(0xffffffffu, need);
  if (!m) return n;
  const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == lead) base = atomicAdd(next, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, lead);
  if (!need || base >= (unsigned long long)n) return n;
  const unsigned long long k = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
  return k < (unsigned long long)n ? (int64_t)k : n;
}

// A walk in progress inside a cell, in optical units. Positions and track
// length hold values of the precision the cell walks in (float below
// kTau64, double above), so a resumed walk continues bit for bit.
struct WalkState {
  double x, y, s;
  float ux, uy;
  uint32_t event, ncoll;
};

// Start of a walk at the point (X, Y) in normalized cell coordinates.
__device__ __forceinline__ WalkState walk_start(float tau, float X, float Y, float ux, float uy,
                                                uint32_t event) {
  WalkState st;
  if (tau > kTau64) {
    st.x = (double)X * (double)tau;
    st.y = (double)Y * (double)tau;
  } else {
    st.x = (double)(X * tau);
    st.y = (double)(Y * tau);
  }
  st.s = 0.0;
  st.ux = ux;
  st.uy = uy;
  st.event = event;
  st.ncoll = 0;
  return st;
}

// Up to max_flights more flights of the walk in `st` (updated in place); a
// walk whose total collisions reach kMaxFlights ends as kTruncated with
// face -1 regardless of max_flights. sphere: x-y geometry (walk_box_from).
__device__ __forceinline__ WalkResult walk_cell_resume(float tau, float c, int implicit,
                                                       WalkState &st, uint32_t max_flights,
                                                       uint64_t seed, uint64_t id,
                                                       bool sphere = false) {
  const uint32_t left = st.ncoll < kMaxFlights ? kMaxFlights - st.ncoll : 0u;
  const uint32_t cap = max_flights < left ? max_flights : left;
  WalkResult w;
  if (tau > kTau64) {
    double x = st.x, y = st.y, s = st.s;
    w = walk_box_from<double>((double)tau, c, implicit, x, y, s, st.ux, st.uy, st.event, st.ncoll,
                              cap, seed, id, sphere);
    st.x = x;
    st.y = y;
    st.s = s;
  } else {
    float x = (float)st.x, y = (float)st.y, s = (float)st.s;
    w = walk_box_from<float>(tau, c, implicit, x, y, s, st.ux, st.uy, st.event, st.ncoll, cap, seed,
                             id, sphere);
    st.x = x;
    st.y = y;
    st.s = s;
  }
  return w;
}

// The walk in a rectangular cell of optical width tx and height ty (the
// geometry variant with unequal sides), from (x, y) to its end; q is
// normalized along the exit face, as for the square, which tx = ty gives.
template <typename T>
__device__ __forceinline__ WalkResult walk_rect(T tx, T ty, float c, int implicit, T x, T y,
                                                float ux, float uy, uint64_t seed, uint64_t id,
                                                uint32_t event) {
  const float rate = implicit ? c : 1.0f;
  T s = 0;
  uint32_t ncoll = 0;
  WalkResult w;
  w.status = kTruncated;
  w.face = -1;
  w.q = 0.0f;
  for (uint32_t it = 0; it < kMaxFlights; ++it) {
    const uint4 r = philox_draw(seed, id, event, kTagWalk);
    ++event;
    const float df = rate > 0.0f ? -logf(u01(r.x)) / rate : INFINITY;
    const T d = (T)df;
    bool xface;
    T db;
    if (flight_exits(tx, ty, x, y, ux, uy, df, xface, db)) {
      s += db;
      int face;
      T qn;
      if (xface) {
        face = ux > 0.0f ? 1 : 3;
        const T along = y + db * (T)uy;
        qn = face == 1 ? along / ty : (ty - along) / ty;
      } else {
        face = uy > 0.0f ? 2 : 0;
        const T along = x + db * (T)ux;
        qn = face == 0 ? along / tx : (tx - along) / tx;
      }
      w.status = kExited;
      w.face = face;
      w.q = fminf(fmaxf((float)qn, 0.0f), 1.0f);
      break;
    }
    s += d;
    x += d * (T)ux;
    y += d * (T)uy;
    ++ncoll;
    if (!implicit && u01(r.y) > c) {
      w.status = kAbsorbed;
      break;
    }
    sincospif(2.0f * u01(r.z), &uy, &ux);
  }
  w.ux = ux;
  w.uy = uy;
  w.s = (float)s;
  w.ncoll = ncoll;
  w.event = event;
  return w;
}

// The walk in x-y geometry (the geometry variant in which the cell is the
// cross-section of an infinite prism and directions are 3-D): (ux, uy) is
// the direction's projection on the plane (a point of the unit disk), a
// flight of 3-D length d moves the position by d (ux, uy), s is the 3-D
// track length, and a scattering draws the direction isotropically on the
// sphere, polar cosine 2 u3 - 1 from the flight's fourth uniform and
// azimuth 2 pi u2. Faces and q as walk_rect.
template <typename T>
__device__ __forceinline__ WalkResult walk_xy(T tx, T ty, float c, int implicit, T x, T y,
                                              float ux, float uy, uint64_t seed, uint64_t id,
                                              uint32_t event) {
  const float rate = implicit ? c : 1.0f;
  T s = 0;
  uint32_t ncoll = 0;
  WalkResult w;
  w.status = kTruncated;
  w.face = -1;
  w.q = 0.0f;
  for (uint32_t it = 0; it < kMaxFlights; ++it) {
    const uint4 r = philox_draw(seed, id, event, kTagWalk);
    ++event;
    const float df = rate > 0.0f ? -logf(u01(r.x)) / rate : INFINITY;
    const T d = (T)df;
    bool xface;
    T db;
    if (flight_exits(tx, ty, x, y, ux, uy, df, xface, db)) {
      s += db;
      int face;
      T qn;
      if (xface) {
        face = ux > 0.0f ? 1 : 3;
        const T along = y + db * (T)uy;
        qn = face == 1 ? along / ty : (ty - along) / ty;
      } else {
        face = uy > 0.0f ? 2 : 0;
        const T along = x + db * (T)ux;
        qn = face == 0 ? along / tx : (tx - along) / tx;
      }
      w.status = kExited;
      w.face = face;
      w.q = fminf(fmaxf((float)qn, 0.0f), 1.0f);
      break;
    }
    s += d;
    x += d * (T)ux;
    y += d * (T)uy;
    ++ncoll;
    if (!implicit && u01(r.y) > c) {
      w.status = kAbsorbed;
      break;
    }
    float sp, cp;
    sincospif(2.0f * u01(r.z), &sp, &cp);
    const float mu = 2.0f * u01(r.w) - 1.0f;
    const float rr = sqrtf(fmaxf(1.0f - mu * mu, 0.0f));
    ux = rr * cp;
    uy = rr * sp;
  }
  w.ux = ux;
  w.uy = uy;
  w.s = (float)s;
  w.ncoll = ncoll;
  w.event = event;
  return w;
}

// walk_box_from in a rectangle [0, tx] x [0, ty] (rectangular cells in the
// solve): the same flights, draws and exit rule, q normalized per face as
// walk_rect. A separate function, so the square cells' walk is unchanged.
template <typename T>
__device__ __forceinline__ WalkResult walk_rect_from(T tx, T ty, float c, int implicit, T &x, T &y,
                                                     T &s, float &ux, float &uy, uint32_t &event,
                                                     uint32_t &ncoll, uint32_t max_flights,
                                                     uint64_t seed, uint64_t id) {
  const float rate = implicit ? c : 1.0f;
  WalkResult w;
  w.status = kTruncated;
  w.face = -1;
  w.q = 0.0f;
  for (uint32_t it = 0; it < max_flights; ++it) {
    const uint4 r = philox_draw(seed, id, event, kTagWalk);
    ++event;
    const float df = rate > 0.0f ? -logf(u01(r.x)) / rate : INFINITY;
    const T d = (T)df;
    bool xface;
    T db;
    if (flight_exits(tx, ty, x, y, ux, uy, df, xface, db)) {
      s += db;
      int face;
      T qn;
      if (xface) {
        face = ux > 0.0f ? 1 : 3;
        const T along = y + db * (T)uy;
        qn = face == 1 ? along / ty : (ty - along) / ty;
      } else {
        face = uy > 0.0f ? 2 : 0;
        const T along = x + db * (T)ux;
        qn = face == 0 ? along / tx : (tx - along) / tx;
      }
      w.status = kExited;
      w.face = face;
      w.q = fminf(fmaxf((float)qn, 0.0f), 1.0f);
      break;
    }
    s += d;
    x += d * (T)ux;
    y += d * (T)uy;
    ++ncoll;
    if (!implicit && u01(r.y) > c) {
      w.status = kAbsorbed;
      break;
    }
    sincospif(2.0f * u01(r.z), &uy, &ux);
  }
  w.ux = ux;
  w.uy = uy;
  w.s = (float)s;
  w.ncoll = ncoll;
  w.event = event;
  return w;
}

// A walk in a rectangle [0, tx] x [0, ty] started at (X, Y) in normalized
// cell coordinates (positions in FP64 when a side exceeds kTau64, as the
// square cell's walk_start), and its resumption (walk_cell_resume).
__device__ __forceinline__ WalkState walk_start_rect(float tx, float ty, float X, float Y, float ux,
                                                     float uy, uint32_t event) {
  WalkState st;
  if (fmaxf(tx, ty) > kTau64) {
    st.x = (double)X * (double)tx;
    st.y = (double)Y * (double)ty;
  } else {
    st.x = (double)(X * tx);
    st.y = (double)(Y * ty);
  }
  st.s = 0.0;
  st.ux = ux;
  st.uy = uy;
  st.event = event;
  st.ncoll = 0;
  return st;
}

__device__ __forceinline__ WalkResult walk_cell_resume_rect(float tx, float ty, float c, int implicit,
                                                            WalkState &st, uint32_t max_flights,
                                                            uint64_t seed, uint64_t id) {
  const uint32_t left = st.ncoll < kMaxFlights ? kMaxFlights - st.ncoll : 0u;
  const uint32_t cap = max_flights < left ? max_flights : left;
  WalkResult w;
  if (fmaxf(tx, ty) > kTau64) {
    double x = st.x, y = st.y, s = st.s;
    w = walk_rect_from<double>((double)tx, (double)ty, c, implicit, x, y, s, st.ux, st.uy, st.event,
                               st.ncoll, cap, seed, id);
    st.x = x;
    st.y = y;
    st.s = s;
  } else {
    float x = (float)st.x, y = (float)st.y, s = (float)st.s;
    w = walk_rect_from<float>(tx, ty, c, implicit, x, y, s, st.ux, st.uy, st.event, st.ncoll, cap,
                              seed, id);
    st.x = x;
    st.y = y;
    st.s = s;
  }
  return w;
}

// Walk from a point given in normalized cell coordinates (X, Y in [0,1]),
// picking the position precision from the cell's optical size.
__device__ __forceinline__ WalkResult walk_cell(float tau, float c, int implicit, float X, float Y,
                                                float ux, float uy, uint64_t seed, uint64_t id,
                                                uint32_t event) {
  if (tau > kTau64)
    return walk_box<double>((double)tau, c, implicit, (double)X * tau, (double)Y * tau, ux, uy,
                            seed, id, event);
  return walk_box<float>(tau, c, implicit, X * tau, Y * tau, ux, uy, seed, id, event);
}

}  // namespace gmc
