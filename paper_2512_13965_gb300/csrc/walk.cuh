// Random-walk transport through one square cell (section "Monte Carlo
// Method", Eq. 4): free flights d = -ln(u)/sigma with u in (0,1], step
// min(d_b, d), isotropic scattering; analog mode kills at a collision with
// probability 1 - c, implicit-capture mode samples flights with sigma = c and
// never kills. Used by analog_transmit, by the births of transport_solve and
// by its analog method.
//
// Position arithmetic runs in T (float, or double in optically thick cells);
// the variates (log, sincos) are drawn in float.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "philox.cuh"

namespace gmc {

constexpr uint32_t kMaxFlights = 1u << 28;  // bound on one walk (never reached in practice)
constexpr float kTau64 = 64.0f;             // cells thicker than this walk in FP64

enum : int { kExited = 0, kAbsorbed = 1, kTruncated = 2 };

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
// exactly the random numbers an uninterrupted walk would.
template <typename T>
__device__ __forceinline__ WalkResult walk_box_from(T tau, float c, int implicit, T &x, T &y, T &s,
                                                    float &ux, float &uy, uint32_t &event,
                                                    uint32_t &ncoll, uint32_t max_flights,
                                                    uint64_t seed, uint64_t id) {
  const float rate = implicit ? c : 1.0f;
  const T inf = (T)INFINITY;
  WalkResult w;
  w.status = kTruncated;
  w.face = -1;
  w.q = 0.0f;
  for (uint32_t it = 0; it < max_flights; ++it) {
    const uint4 r = philox_draw(seed, id, event, kTagWalk);
    ++event;
    const T d = rate > 0.0f ? (T)(-logf(u01(r.x)) / rate) : inf;
    T dbx = inf, dby = inf;
    if (ux > 0.0f) dbx = (tau - x) / (T)ux;
    else if (ux < 0.0f) dbx = -x / (T)ux;
    if (uy > 0.0f) dby = (tau - y) / (T)uy;
    else if (uy < 0.0f) dby = -y / (T)uy;
    const bool xface = dbx <= dby;
    T db = xface ? dbx : dby;
    if (db < (T)0) db = (T)0;
    if (d >= db) {
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
    sincospif(2.0f * u01(r.z), &uy, &ux);
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
// face -1 regardless of max_flights.
__device__ __forceinline__ WalkResult walk_cell_resume(float tau, float c, int implicit,
                                                       WalkState &st, uint32_t max_flights,
                                                       uint64_t seed, uint64_t id) {
  const uint32_t left = st.ncoll < kMaxFlights ? kMaxFlights - st.ncoll : 0u;
  const uint32_t cap = max_flights < left ? max_flights : left;
  WalkResult w;
  if (tau > kTau64) {
    double x = st.x, y = st.y, s = st.s;
    w = walk_box_from<double>((double)tau, c, implicit, x, y, s, st.ux, st.uy, st.event, st.ncoll,
                              cap, seed, id);
    st.x = x;
    st.y = y;
    st.s = s;
  } else {
    float x = (float)st.x, y = (float)st.y, s = (float)st.s;
    w = walk_box_from<float>(tau, c, implicit, x, y, s, st.ux, st.uy, st.event, st.ncoll, cap, seed,
                             id);
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
  const T inf = (T)INFINITY;
  T s = 0;
  uint32_t ncoll = 0;
  WalkResult w;
  w.status = kTruncated;
  w.face = -1;
  w.q = 0.0f;
  for (uint32_t it = 0; it < kMaxFlights; ++it) {
    const uint4 r = philox_draw(seed, id, event, kTagWalk);
    ++event;
    const T d = rate > 0.0f ? (T)(-logf(u01(r.x)) / rate) : inf;
    T dbx = inf, dby = inf;
    if (ux > 0.0f) dbx = (tx - x) / (T)ux;
    else if (ux < 0.0f) dbx = -x / (T)ux;
    if (uy > 0.0f) dby = (ty - y) / (T)uy;
    else if (uy < 0.0f) dby = -y / (T)uy;
    const bool xface = dbx <= dby;
    T db = xface ? dbx : dby;
    if (db < (T)0) db = (T)0;
    if (d >= db) {
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
  const T inf = (T)INFINITY;
  T s = 0;
  uint32_t ncoll = 0;
  WalkResult w;
  w.status = kTruncated;
  w.face = -1;
  w.q = 0.0f;
  for (uint32_t it = 0; it < kMaxFlights; ++it) {
    const uint4 r = philox_draw(seed, id, event, kTagWalk);
    ++event;
    const T d = rate > 0.0f ? (T)(-logf(u01(r.x)) / rate) : inf;
    T dbx = inf, dby = inf;
    if (ux > 0.0f) dbx = (tx - x) / (T)ux;
    else if (ux < 0.0f) dbx = -x / (T)ux;
    if (uy > 0.0f) dby = (ty - y) / (T)uy;
    else if (uy < 0.0f) dby = -y / (T)uy;
    const bool xface = dbx <= dby;
    T db = xface ? dbx : dby;
    if (db < (T)0) db = (T)0;
    if (d >= db) {
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
