// Exit-state decoding (stage 4 of the transport algorithm, Eq. 11): the
// standardized ODE output x(1) = (p, cos theta, sin theta, ln s) is mapped
// back to physical units, p is wrapped onto the perimeter [0,4), the
// direction is renormalized and made to point out of the exit face, and the
// path length is s = max(exp(ln s), 1e-7).
#pragma once
#include "gmc_internal.cuh"

namespace gmc {

// Returns (p, ux, uy, s); *inward is set when the sampled direction pointed
// into the cell and was reflected about the face. With st.disk (x-y
// geometry, Eq. 11 with the direction encoded by its projection on the unit
// disk) the projection is kept, scaled back onto the unit circle only when it
// lies outside the disk, and a projection with no outward component left
// (parallel to the face, or zero) becomes the outward normal.
__device__ __forceinline__ float4 decode_exit(float y0, float y1, float y2, float y3,
                                              const NetStats &st, bool *inward) {
  float p = fmaf(y0, st.y_std[0], st.y_mean[0]);
  float ux = fmaf(y1, st.y_std[1], st.y_mean[1]);
  float uy = fmaf(y2, st.y_std[2], st.y_mean[2]);
  const float ls = fmaf(y3, st.y_std[3], st.y_mean[3]);
  p = p - 4.0f * floorf(p * 0.25f);
  if (!(p < 4.0f)) p = 0.0f;  // rounding of tiny negatives, and NaN
  if (p < 0.0f) p = 0.0f;
  const int face = min((int)p, 3);
  // outward normal of the face: 0 (0,-1), 1 (1,0), 2 (0,1), 3 (-1,0)
  const float nx = face == 1 ? 1.0f : (face == 3 ? -1.0f : 0.0f);
  const float ny = face == 2 ? 1.0f : (face == 0 ? -1.0f : 0.0f);
  const float nrm = sqrtf(ux * ux + uy * uy);
  if (st.disk) {
    if (nrm > 1.0f) {
      ux /= nrm;
      uy /= nrm;
    }
  } else if (nrm > 0.0f) {
    ux /= nrm;
    uy /= nrm;
  } else {
    ux = nx;
    uy = ny;
  }
  const float dot = ux * nx + uy * ny;
  *inward = dot < 0.0f;
  if (dot < 0.0f) {
    ux -= 2.0f * dot * nx;
    uy -= 2.0f * dot * ny;
  } else if (st.disk && dot == 0.0f) {
    ux = nx;
    uy = ny;
  }
  const float s = fmaxf(expf(ls), kSMin);
  return make_float4(p, ux, uy, s);
}

// emb(t) component j: sin(2^j pi t) for j < 8, cos(2^(j-8) pi t) otherwise.
__device__ __forceinline__ float time_embedding(int j, float t) {
  const float a = ldexpf(t, j & 7);
  return j < 8 ? sinpif(a) : cospif(a);
}

}  // namespace gmc
