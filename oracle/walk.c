/*
 * Oracle: random-walk cell transmission in FP64 (test infrastructure only).
 *
 * Follows the Monte Carlo method section of the paper: a particle streams
 * along its direction until it either scatters or reaches the cell boundary;
 * the free-flight length is d_s = -ln(xi)/sigma (Eq. 4) with xi in (0,1], the
 * step is min(d_b, d_s), a scattering draws a new direction from the
 * (isotropic) kernel, and the track length in the cell accumulates to
 * Delta s_tot (Eq. 5-7).
 *
 * Two absorption modes:
 *  - IMPLICIT (implicit capture, as the paper uses): flights are sampled with
 *    the scattering cross section, sigma = c in optical units; the particle is
 *    never killed, its weight is attenuated afterwards by exp(-(1-c) s) (Eq. 5).
 *  - ANALOG (discrete absorption, the plain method GMC replaces): flights are
 *    sampled with sigma_t = 1; at each collision the particle survives with
 *    probability c, otherwise it is absorbed there.
 *
 * Random numbers: one Philox draw (4 uniforms) per flight, at counter
 * (id, event, TAG_WALK): u0 -> flight length, u1 -> survival test (analog
 * mode: survive iff u1 <= c), u2 -> new direction angle 2*pi*u2.
 */
#include <math.h>
#include <stdint.h>
#include "oracle.h"

static const double ORC_TWO_PI = 6.283185307179586476925286766559;

static void exit_point(double tau, int face, double x, double y, orc_walk_result *res)
{
    double q;
    switch (face) {
    case 0: q = x / tau; y = 0.0; break;
    case 1: q = y / tau; x = tau; break;
    case 2: q = (tau - x) / tau; y = tau; break;
    default: q = (tau - y) / tau; x = 0.0; break;
    }
    if (q < 0.0) q = 0.0;
    if (q > 1.0) q = 1.0;
    res->face = face;
    res->q = q;
    res->x = x;
    res->y = y;
}

void orc_walk_box(double tau, double c, int mode, double x, double y, double ux, double uy,
                  uint64_t seed, uint64_t id, uint32_t event0, orc_walk_result *res)
{
    const double rate = (mode == ORC_MODE_IMPLICIT) ? c : 1.0;
    uint32_t event = event0;
    double s = 0.0;
    int64_t ncoll = 0;
    for (;;) {
        double u[4];
        orc_uniform4(seed, id, event, ORC_TAG_WALK, u);
        ++event;
        double d = (rate > 0.0) ? -log(u[0]) / rate : INFINITY;
        double dbx = INFINITY, dby = INFINITY;
        if (ux > 0.0) dbx = (tau - x) / ux;
        else if (ux < 0.0) dbx = -x / ux;
        if (uy > 0.0) dby = (tau - y) / uy;
        else if (uy < 0.0) dby = -y / uy;
        double db = dbx <= dby ? dbx : dby;
        if (d >= db) {
            /* streams to the boundary: the x-face wins exact corner ties */
            s += db;
            double xe = x + db * ux, ye = y + db * uy;
            int face = (dbx <= dby) ? (ux > 0.0 ? 1 : 3) : (uy > 0.0 ? 2 : 0);
            exit_point(tau, face, xe, ye, res);
            res->status = ORC_EXITED;
            res->ux = ux;
            res->uy = uy;
            break;
        }
        s += d;
        x += d * ux;
        y += d * uy;
        ++ncoll;
        if (mode == ORC_MODE_ANALOG && u[1] > c) {
            res->status = ORC_ABSORBED;
            res->face = -1;
            res->q = 0.0;
            res->x = x;
            res->y = y;
            res->ux = ux;
            res->uy = uy;
            break;
        }
        double phi = ORC_TWO_PI * u[2];
        ux = cos(phi);
        uy = sin(phi);
    }
    res->s = s;
    res->ncoll = ncoll;
    res->event = event;
}

/*
 * Batched canonical-frame transmission: particle i enters the left face at
 * y = xi[i]*tau[i] with direction (cos_in[i], sin_in[i]); Philox id = id0+i,
 * first event ctr0. Outputs are arrays of length n.
 */
void orc_transmit_batch(int64_t n, const double *xi, const double *cos_in, const double *sin_in,
                        const double *tau, const double *c, int mode, uint64_t seed, uint64_t id0,
                        uint32_t ctr0, int32_t *status, int32_t *face, double *q, double *ux,
                        double *uy, double *s, int64_t *ncoll)
{
    for (int64_t i = 0; i < n; ++i) {
        orc_walk_result r;
        orc_walk_box(tau[i], c[i], mode, 0.0, xi[i] * tau[i], cos_in[i], sin_in[i], seed,
                     id0 + (uint64_t)i, ctr0, &r);
        status[i] = r.status;
        face[i] = r.face;
        q[i] = r.q;
        ux[i] = r.ux;
        uy[i] = r.uy;
        s[i] = r.s;
        ncoll[i] = r.ncoll;
    }
}

/* Single general walk, exposed for the Python event-loop oracle. */
void orc_walk_one(double tau, double c, int mode, double x, double y, double ux, double uy,
                  uint64_t seed, uint64_t id, uint32_t event0, int32_t *status, int32_t *face,
                  double *out /* q, x, y, ux, uy, s */, int64_t *ncoll, uint32_t *event)
{
    orc_walk_result r;
    orc_walk_box(tau, c, mode, x, y, ux, uy, seed, id, event0, &r);
    *status = r.status;
    *face = r.face;
    out[0] = r.q;
    out[1] = r.x;
    out[2] = r.y;
    out[3] = r.ux;
    out[4] = r.uy;
    out[5] = r.s;
    *ncoll = r.ncoll;
    *event = r.event;
}

/* Single walk in a rectangular cell [0, tx] x [0, ty] from an arbitrary
   point, for the Python event-loop oracle. Outputs as orc_walk_one (q
   normalized per face). */
void orc_walk_one_rect(double tx, double ty, double c, int mode, double x, double y, double ux,
                       double uy, uint64_t seed, uint64_t id, uint32_t event0, int32_t *status,
                       int32_t *face, double *out /* q, x, y, ux, uy, s */, int64_t *ncoll,
                       uint32_t *event)
{
    orc_walk_result r;
    orc_walk_rect(tx, ty, c, mode, x, y, ux, uy, seed, id, event0, &r);
    *status = r.status;
    *face = r.face;
    out[0] = r.q;
    out[1] = r.x;
    out[2] = r.y;
    out[3] = r.ux;
    out[4] = r.uy;
    out[5] = r.s;
    *ncoll = r.ncoll;
    *event = r.event;
}

/* Single walk in x-y geometry (a square cell of side tau, directions on the
   sphere) from an arbitrary point, for the Python event-loop oracle: (ux, uy)
   is the direction's projection on the plane and |uz| = sqrt(1 - ux^2 - uy^2)
   (the sign of uz does not enter a walk in the plane). Outputs as
   orc_walk_one. */
void orc_walk_one_xy(double tau, double c, int mode, double x, double y, double ux, double uy,
                     uint64_t seed, uint64_t id, uint32_t event0, int32_t *status, int32_t *face,
                     double *out /* q, x, y, ux, uy, s */, int64_t *ncoll, uint32_t *event)
{
    orc_walk_result r;
    double uz_out;
    const double r2 = ux * ux + uy * uy;
    const double uz = r2 < 1.0 ? sqrt(1.0 - r2) : 0.0;
    orc_walk_xy(tau, tau, c, mode, 1, x, y, ux, uy, uz, seed, id, event0, &r, &uz_out);
    *status = r.status;
    *face = r.face;
    out[0] = r.q;
    out[1] = r.x;
    out[2] = r.y;
    out[3] = r.ux;
    out[4] = r.uy;
    out[5] = r.s;
    *ncoll = r.ncoll;
    *event = r.event;
}

/*
 * Canonical-frame transmission with per-particle Philox ids and first
 * events; event_out[i] receives the next unused event counter.
 */
void orc_transmit_ids(int64_t n, const double *xi, const double *cos_in, const double *sin_in,
                      const double *tau, const double *c, int mode, uint64_t seed,
                      const uint64_t *ids, const uint32_t *events, int32_t *status, int32_t *face,
                      double *q, double *ux, double *uy, double *s, int64_t *ncoll,
                      uint32_t *event_out)
{
    for (int64_t i = 0; i < n; ++i) {
        orc_walk_result r;
        orc_walk_box(tau[i], c[i], mode, 0.0, xi[i] * tau[i], cos_in[i], sin_in[i], seed, ids[i],
                     events[i], &r);
        status[i] = r.status;
        face[i] = r.face;
        q[i] = r.q;
        ux[i] = r.ux;
        uy[i] = r.uy;
        s[i] = r.s;
        ncoll[i] = r.ncoll;
        event_out[i] = r.event;
    }
}

/*
 * The same walk in a rectangular cell (the geometry variant with unequal
 * sides): optical width tx along x, height ty along y; exits report q along
 * the face normalized to [0,1) (counter-clockwise, as for the square), so
 * p = face + q stays in [0,4). tx = ty = tau is exactly orc_walk_box.
 */
static void exit_point_rect(double tx, double ty, int face, double x, double y,
                            orc_walk_result *res)
{
    double q;
    switch (face) {
    case 0: q = x / tx; y = 0.0; break;
    case 1: q = y / ty; x = tx; break;
    case 2: q = (tx - x) / tx; y = ty; break;
    default: q = (ty - y) / ty; x = 0.0; break;
    }
    if (q < 0.0) q = 0.0;
    if (q > 1.0) q = 1.0;
    res->face = face;
    res->q = q;
    res->x = x;
    res->y = y;
}

void orc_walk_rect(double tx, double ty, double c, int mode, double x, double y, double ux,
                   double uy, uint64_t seed, uint64_t id, uint32_t event0, orc_walk_result *res)
{
    const double rate = (mode == ORC_MODE_IMPLICIT) ? c : 1.0;
    uint32_t event = event0;
    double s = 0.0;
    int64_t ncoll = 0;
    for (;;) {
        double u[4];
        orc_uniform4(seed, id, event, ORC_TAG_WALK, u);
        ++event;
        double d = (rate > 0.0) ? -log(u[0]) / rate : INFINITY;
        double dbx = INFINITY, dby = INFINITY;
        if (ux > 0.0) dbx = (tx - x) / ux;
        else if (ux < 0.0) dbx = -x / ux;
        if (uy > 0.0) dby = (ty - y) / uy;
        else if (uy < 0.0) dby = -y / uy;
        double db = dbx <= dby ? dbx : dby;
        if (d >= db) {
            s += db;
            double xe = x + db * ux, ye = y + db * uy;
            int face = (dbx <= dby) ? (ux > 0.0 ? 1 : 3) : (uy > 0.0 ? 2 : 0);
            exit_point_rect(tx, ty, face, xe, ye, res);
            res->status = ORC_EXITED;
            res->ux = ux;
            res->uy = uy;
            break;
        }
        s += d;
        x += d * ux;
        y += d * uy;
        ++ncoll;
        if (mode == ORC_MODE_ANALOG && u[1] > c) {
            res->status = ORC_ABSORBED;
            res->face = -1;
            res->q = 0.0;
            res->x = x;
            res->y = y;
            res->ux = ux;
            res->uy = uy;
            break;
        }
        double phi = ORC_TWO_PI * u[2];
        ux = cos(phi);
        uy = sin(phi);
    }
    res->s = s;
    res->ncoll = ncoll;
    res->event = event;
}

/* Canonical-frame transmission through rectangles: particle i enters the
   left face at y = xi[i]*ty[i]; otherwise as orc_transmit_ids. */
void orc_transmit_rect_ids(int64_t n, const double *xi, const double *cos_in,
                           const double *sin_in, const double *tx, const double *ty,
                           const double *c, int mode, uint64_t seed, const uint64_t *ids,
                           const uint32_t *events, int32_t *status, int32_t *face, double *q,
                           double *ux, double *uy, double *s, int64_t *ncoll, uint32_t *event_out)
{
    for (int64_t i = 0; i < n; ++i) {
        orc_walk_result r;
        orc_walk_rect(tx[i], ty[i], c[i], mode, 0.0, xi[i] * ty[i], cos_in[i], sin_in[i], seed,
                      ids[i], events[i], &r);
        status[i] = r.status;
        face[i] = r.face;
        q[i] = r.q;
        ux[i] = r.ux;
        uy[i] = r.uy;
        s[i] = r.s;
        ncoll[i] = r.ncoll;
        event_out[i] = r.event;
    }
}

/*
 * The walk in x-y geometry (the geometry variant in which the cell is the
 * cross-section of an infinite prism and directions are 3-D; the paper
 * encodes them by their projection on the unit disk): the direction is the
 * unit vector (ux, uy, uz), the particle's position moves in the plane by
 * d (ux, uy) over a flight of 3-D length d, and the track length s is 3-D.
 * Faces, q and the flight draws are those of orc_walk_rect. A scattering
 * draws the new direction isotropically on the sphere: azimuth 2 pi u2 and
 * polar cosine uz = 2 u3 - 1 (u3 is the fourth uniform of the flight's draw);
 * with sphere = 0 it stays on the circle (uz = 0) and the walk is
 * orc_walk_rect draw for draw.
 */
void orc_walk_xy(double tx, double ty, double c, int mode, int sphere, double x, double y,
                 double ux, double uy, double uz, uint64_t seed, uint64_t id, uint32_t event0,
                 orc_walk_result *res, double *uz_out)
{
    const double rate = (mode == ORC_MODE_IMPLICIT) ? c : 1.0;
    uint32_t event = event0;
    double s = 0.0;
    int64_t ncoll = 0;
    for (;;) {
        double u[4];
        orc_uniform4(seed, id, event, ORC_TAG_WALK, u);
        ++event;
        double d = (rate > 0.0) ? -log(u[0]) / rate : INFINITY;
        double dbx = INFINITY, dby = INFINITY;
        if (ux > 0.0) dbx = (tx - x) / ux;
        else if (ux < 0.0) dbx = -x / ux;
        if (uy > 0.0) dby = (ty - y) / uy;
        else if (uy < 0.0) dby = -y / uy;
        double db = dbx <= dby ? dbx : dby;
        if (d >= db) {
            s += db;
            double xe = x + db * ux, ye = y + db * uy;
            int face = (dbx <= dby) ? (ux > 0.0 ? 1 : 3) : (uy > 0.0 ? 2 : 0);
            exit_point_rect(tx, ty, face, xe, ye, res);
            res->status = ORC_EXITED;
            break;
        }
        s += d;
        x += d * ux;
        y += d * uy;
        ++ncoll;
        if (mode == ORC_MODE_ANALOG && u[1] > c) {
            res->status = ORC_ABSORBED;
            res->face = -1;
            res->q = 0.0;
            res->x = x;
            res->y = y;
            break;
        }
        double phi = ORC_TWO_PI * u[2];
        double r = 1.0;
        uz = 0.0;
        if (sphere) {
            uz = 2.0 * u[3] - 1.0;
            r = sqrt(1.0 - uz * uz);
        }
        ux = r * cos(phi);
        uy = r * sin(phi);
    }
    res->ux = ux;
    res->uy = uy;
    res->s = s;
    res->ncoll = ncoll;
    res->event = event;
    *uz_out = uz;
}

/* Canonical-frame transmission in x-y geometry: particle i enters the left
   face at y = xi[i]*ty[i] with the 3-D direction (ux_in, uy_in, uz_in)[i]. */
void orc_transmit_xy_ids(int64_t n, const double *xi, const double *ux_in, const double *uy_in,
                         const double *uz_in, const double *tx, const double *ty,
                         const double *c, int mode, int sphere, uint64_t seed,
                         const uint64_t *ids, const uint32_t *events, int32_t *status,
                         int32_t *face, double *q, double *ux, double *uy, double *uz, double *s,
                         int64_t *ncoll, uint32_t *event_out)
{
    for (int64_t i = 0; i < n; ++i) {
        orc_walk_result r;
        orc_walk_xy(tx[i], ty[i], c[i], mode, sphere, 0.0, xi[i] * ty[i], ux_in[i], uy_in[i],
                    uz_in[i], seed, ids[i], events[i], &r, &uz[i]);
        status[i] = r.status;
        face[i] = r.face;
        q[i] = r.q;
        ux[i] = r.ux;
        uy[i] = r.uy;
        s[i] = r.s;
        ncoll[i] = r.ncoll;
        event_out[i] = r.event;
    }
}
