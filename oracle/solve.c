/*
 * Oracle: standard Monte Carlo transport solve on a 2-D grid of square cells,
 * FP64, one history at a time (test infrastructure only).
 *
 * Follows the Monte Carlo method section of the paper with implicit capture:
 * a history is born from the source with weight 1, streams and scatters with
 * flights sampled from sigma_s (Eq. 4), and in each cell it crosses the total
 * track length Delta s_tot attenuates its weight (Eq. 5), deposits
 * Delta w (Eq. 6) and scores Delta w / (V sigma_a) into that cell's scalar
 * flux (Eq. 7). Vacuum boundaries end a history; a history whose weight drops
 * below the cutoff plays Russian roulette (the paper terminates below a
 * cutoff; roulette is its unbiased form).
 *
 * Units: every cell has physical side h = 1, so V = 1, sigma_t = tau,
 * sigma_s = c*tau, sigma_a = (1-c)*tau. Inside a cell the walk runs in
 * optical coordinates [0,tau]^2, where the track length s is in total mean
 * free paths and sigma_a * (s / tau) = (1-c) s.
 *
 * Source: cell k is chosen with probability src[k] / sum(src); the birth
 * point is uniform in that cell and the direction isotropic. Random numbers:
 * birth at (h, 0, TAG_BIRTH) -> u0 cell, u1,u2 position, u3 angle; flights at
 * (h, event, TAG_WALK) with one event counter per history; roulette at
 * (h, event, TAG_ROULETTE) with the event counter reached after the walk.
 *
 * The flux returned is per source particle per unit area.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include "oracle.h"

static const double TWO_PI = 6.283185307179586476925286766559;

/* Smallest k with cdf[k] >= target (cdf non-decreasing, cdf[n-1] >= target). */
static int64_t cdf_search(const double *cdf, int64_t n, double target)
{
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] >= target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

/* Deposit of one cell transmission with track length s (optical units). */
static double deposit(double w, double s, double tau, double c, double *flux_cell)
{
    double a = 1.0 - c;
    if (a > 0.0) {
        double dw = w * (-expm1(-a * s));         /* Eq. 6 */
        *flux_cell += dw / (a * tau);             /* Eq. 7, V = 1 */
        return dw;
    }
    *flux_cell += w * s / tau;                    /* sigma_a -> 0 limit of Eq. 7 */
    return 0.0;
}

/*
 * stats (nullable, length 6): [0] leaked weight, [1] absorbed weight,
 * [2] net roulette weight change, [3] cell transmissions, [4] collisions,
 * [5] roulette kills.
 */
int orc_solve_analog(int nx, int ny, const double *tau, const double *c, const double *src,
                     int64_t n_hist, uint64_t seed, double w_cut, double p_survive,
                     double *flux, double *stats)
{
    int64_t ncell = (int64_t)nx * ny;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)ncell);
    if (!cdf) return -1;
    double acc = 0.0;
    for (int64_t k = 0; k < ncell; ++k) {
        acc += src[k] > 0.0 ? src[k] : 0.0;
        cdf[k] = acc;
        flux[k] = 0.0;
    }
    if (!(acc > 0.0)) {
        free(cdf);
        return -2;
    }
    double st[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t h = 0; h < n_hist; ++h) {
        double u[4];
        orc_uniform4(seed, (uint64_t)h, 0u, ORC_TAG_BIRTH, u);
        int64_t k = cdf_search(cdf, ncell, u[0] * acc);
        int i = (int)(k % nx), j = (int)(k / nx);
        double t = tau[k];
        double x = u[1] * t, y = u[2] * t;
        double ux = cos(TWO_PI * u[3]), uy = sin(TWO_PI * u[3]);
        double w = 1.0;
        uint32_t event = 0;
        for (;;) {
            int64_t cell = (int64_t)j * nx + i;
            t = tau[cell];
            double cc = c[cell];
            orc_walk_result r;
            orc_walk_box(t, cc, ORC_MODE_IMPLICIT, x, y, ux, uy, seed, (uint64_t)h, event, &r);
            event = r.event;
            st[3] += 1.0;
            st[4] += (double)r.ncoll;
            double dw = deposit(w, r.s, t, cc, &flux[cell]);
            st[1] += dw;
            w -= dw;
            if (w < w_cut) {
                double ur[4];
                orc_uniform4(seed, (uint64_t)h, event, ORC_TAG_ROULETTE, ur);
                if (ur[0] <= p_survive) {
                    st[2] += w / p_survive - w;
                    w = w / p_survive;
                } else {
                    st[2] -= w;
                    st[5] += 1.0;
                    break;
                }
            }
            /* cross into the neighbour through the exit face */
            ux = r.ux;
            uy = r.uy;
            double X, Y; /* normalized exit point */
            switch (r.face) {
            case 0: X = r.q; Y = 0.0; break;
            case 1: X = 1.0; Y = r.q; break;
            case 2: X = 1.0 - r.q; Y = 1.0; break;
            default: X = 0.0; Y = 1.0 - r.q; break;
            }
            int ni = i, nj = j;
            if (r.face == 0) { nj = j - 1; Y = 1.0; }
            else if (r.face == 1) { ni = i + 1; X = 0.0; }
            else if (r.face == 2) { nj = j + 1; Y = 0.0; }
            else { ni = i - 1; X = 1.0; }
            if (ni < 0 || ni >= nx || nj < 0 || nj >= ny) {
                st[0] += w;
                break;
            }
            i = ni;
            j = nj;
            double tn = tau[(int64_t)j * nx + i];
            x = X * tn;
            y = Y * tn;
        }
    }
    for (int64_t k = 0; k < ncell; ++k) flux[k] /= (double)n_hist;
    if (stats)
        for (int m = 0; m < 6; ++m) stats[m] = st[m];
    free(cdf);
    return 0;
}
