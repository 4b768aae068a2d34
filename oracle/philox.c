/*
 * Oracle: Philox4x32-10 counter-based generator (test infrastructure only).
 *
 * Written from the published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter
 * and a 2x32-bit key, ten rounds of two 32x32->64 multiplications, with the
 * key bumped by the Weyl constants between rounds.
 *
 * The paper draws every free-flight length from a uniform variate on (0,1]
 * (Eq. 4) and every Gaussian seed of the flow ODE from N(0, I) (Eq. 8).
 * Uniforms here are u = (x + 1) * 2^-32, which lies in (0, 1] as Eq. 4 asks.
 * Normals are Box-Muller pairs computed in double precision.
 *
 * Counter convention shared (by specification, not by code) with the CUDA
 * path: ctr = (id_lo, id_hi, event, tag), key = (seed_lo, seed_hi).
 */
#include <stdint.h>
#include <math.h>
#include "oracle.h"

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_draw(uint64_t seed, uint64_t id, uint32_t event, uint32_t tag, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), event, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

double orc_u01(uint32_t x)
{
    /* (x + 1) / 2^32, exactly representable in double: in (0, 1]. */
    return ((double)x + 1.0) * (1.0 / 4294967296.0);
}

void orc_uniform4(uint64_t seed, uint64_t id, uint32_t event, uint32_t tag, double u[4])
{
    uint32_t r[4];
    orc_philox_draw(seed, id, event, tag, r);
    for (int i = 0; i < 4; ++i) u[i] = orc_u01(r[i]);
}

void orc_normal4(uint64_t seed, uint64_t id, uint32_t event, uint32_t tag, double z[4])
{
    double u[4];
    orc_uniform4(seed, id, event, tag, u);
    /* Box-Muller: (u0,u1) -> z0,z1 and (u2,u3) -> z2,z3. */
    const double two_pi = 6.283185307179586476925286766559;
    double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    z[0] = r0 * cos(two_pi * u[1]);
    z[1] = r0 * sin(two_pi * u[1]);
    z[2] = r1 * cos(two_pi * u[3]);
    z[3] = r1 * sin(two_pi * u[3]);
}

/* Batched entry points for the Python harness. */
void orc_philox_batch(uint64_t seed, int64_t n, uint64_t id0, uint32_t event, uint32_t tag, uint32_t *out /* [n][4] */)
{
    for (int64_t i = 0; i < n; ++i)
        orc_philox_draw(seed, id0 + (uint64_t)i, event, tag, out + 4 * i);
}

void orc_normal_batch(uint64_t seed, int64_t n, uint64_t id0, uint32_t event, uint32_t tag, double *out /* [4][n] */)
{
    for (int64_t i = 0; i < n; ++i) {
        double z[4];
        orc_normal4(seed, id0 + (uint64_t)i, event, tag, z);
        for (int k = 0; k < 4; ++k) out[k * n + i] = z[k];
    }
}

/* Per-particle counters: ids[i], events[i] at one tag. */
void orc_normal_ids(uint64_t seed, int64_t n, const uint64_t *ids, const uint32_t *events, uint32_t tag,
                    double *out /* [4][n] */)
{
    for (int64_t i = 0; i < n; ++i) {
        double z[4];
        orc_normal4(seed, ids[i], events[i], tag, z);
        for (int k = 0; k < 4; ++k) out[k * n + i] = z[k];
    }
}

void orc_uniform_ids(uint64_t seed, int64_t n, const uint64_t *ids, const uint32_t *events, uint32_t tag,
                     double *out /* [4][n] */)
{
    for (int64_t i = 0; i < n; ++i) {
        double u[4];
        orc_uniform4(seed, ids[i], events[i], tag, u);
        for (int k = 0; k < 4; ++k) out[k * n + i] = u[k];
    }
}
