// Device Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the variates
// the method draws from it: uniforms on (0,1] for free flights (Eq. 4) and
// Box-Muller normals for the flow-ODE seed x(0) ~ N(0, I) (Eq. 8).
//
// Counter (id_lo, id_hi, event, tag), key (seed_lo, seed_hi).
#pragma once
#include <cstdint>

namespace gmc {

enum : uint32_t { kTagWalk = 1u, kTagNoise = 2u, kTagRoulette = 3u, kTagBirth = 4u };

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(m0, c.x), hi1 = __umulhi(m1, c.z);
#else
    const uint32_t hi0 = (uint32_t)(((uint64_t)m0 * c.x) >> 32);
    const uint32_t hi1 = (uint32_t)(((uint64_t)m1 * c.z) >> 32);
#endif
    const uint32_t lo0 = m0 * c.x, lo1 = m1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__host__ __device__ __forceinline__ uint4 philox_draw(uint64_t seed, uint64_t id, uint32_t event,
                                                      uint32_t tag) {
  return philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), event, tag),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// (x + 1) 2^-32 rounded to float: never 0, at most 1.
__device__ __forceinline__ float u01(uint32_t x) {
  return fmaf((float)x, 2.3283064365386963e-10f, 2.3283064365386963e-10f);
}

__device__ __forceinline__ float4 box_muller4(uint4 r) {
  const float u0 = u01(r.x), u1 = u01(r.y), u2 = u01(r.z), u3 = u01(r.w);
  const float a = sqrtf(-2.0f * logf(u0)), b = sqrtf(-2.0f * logf(u2));
  float s1, c1, s3, c3;
  sincospif(2.0f * u1, &s1, &c1);
  sincospif(2.0f * u3, &s3, &c3);
  return make_float4(a * c1, a * s1, b * c3, b * s3);
}

}  // namespace gmc
