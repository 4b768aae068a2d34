/*
 * Oracle declarations (test infrastructure only: only tests, the smoke check
 * and the CPU-baseline leg of the benchmark may call into oracle/).
 *
 * Conventions (stated by specification; the CUDA path implements them in
 * code of its own):
 *  - A cell is the square [0,tau]^2 in optical coordinates (sigma_t = 1,
 *    lengths in total mean free paths). Directions lie on the unit circle,
 *    except in the x-y geometry walk, whose directions are 3-D unit vectors.
 *  - Faces are numbered counter-clockwise from the corner (0,0):
 *    0 = bottom (y=0), 1 = right (x=tau), 2 = top (y=tau), 3 = left (x=0).
 *    A point on face f has a counter-clockwise parameter q in [0,1]:
 *    bottom x=q*tau, right y=q*tau, top x=(1-q)*tau, left y=(1-q)*tau.
 *    The unwrapped perimeter coordinate of Eq. 11 is p = f + q in [0,4).
 *  - Philox tags: walk flights 1, flow-ODE noise 2, roulette 3, births 4.
 */
#ifndef GMC_ORACLE_H
#define GMC_ORACLE_H
#include <stdint.h>

#define ORC_TAG_WALK 1u
#define ORC_TAG_NOISE 2u
#define ORC_TAG_ROULETTE 3u
#define ORC_TAG_BIRTH 4u

#define ORC_MODE_ANALOG 0
#define ORC_MODE_IMPLICIT 1

#define ORC_EXITED 0
#define ORC_ABSORBED 1

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox_draw(uint64_t seed, uint64_t id, uint32_t event, uint32_t tag, uint32_t out[4]);
double orc_u01(uint32_t x);
void orc_uniform4(uint64_t seed, uint64_t id, uint32_t event, uint32_t tag, double u[4]);
void orc_normal4(uint64_t seed, uint64_t id, uint32_t event, uint32_t tag, double z[4]);

typedef struct {
    int status;        /* ORC_EXITED or ORC_ABSORBED */
    int face;          /* exit face (valid when EXITED) */
    double q;          /* counter-clockwise parameter on the exit face */
    double x, y;       /* final point (exit point or absorption site), optical units */
    double ux, uy;     /* final direction */
    double s;          /* total track length inside the cell, optical units */
    int64_t ncoll;     /* number of collisions (scatterings, plus the absorbing one) */
    uint32_t event;    /* next unused Philox event counter */
} orc_walk_result;

void orc_walk_box(double tau, double c, int mode, double x, double y, double ux, double uy,
                  uint64_t seed, uint64_t id, uint32_t event0, orc_walk_result *res);
void orc_walk_rect(double tx, double ty, double c, int mode, double x, double y, double ux,
                   double uy, uint64_t seed, uint64_t id, uint32_t event0, orc_walk_result *res);
void orc_walk_xy(double tx, double ty, double c, int mode, int sphere, double x, double y,
                 double ux, double uy, double uz, uint64_t seed, uint64_t id, uint32_t event0,
                 orc_walk_result *res, double *uz_out);
void orc_walk_one_rect(double tx, double ty, double c, int mode, double x, double y, double ux,
                       double uy, uint64_t seed, uint64_t id, uint32_t event0, int32_t *status,
                       int32_t *face, double *out, int64_t *ncoll, uint32_t *event);
void orc_walk_one_xy(double tau, double c, int mode, double x, double y, double ux, double uy,
                     uint64_t seed, uint64_t id, uint32_t event0, int32_t *status, int32_t *face,
                     double *out, int64_t *ncoll, uint32_t *event);

#endif
