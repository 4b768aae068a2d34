/*
 * gmc.h -- C ABI of the GB300 Generative Monte Carlo library (libgmc.so).
 *
 * Generative Monte Carlo replaces the collision-by-collision random walk
 * inside a mesh cell by a sample of the cell's exit state drawn from a
 * learned conditional distribution p(y | c) (section "Generative Monte Carlo
 * Sampler"): the exit state y = (p_exit, Omega_exit, s) (Eq. 11) is x(1) of
 * the flow ODE dx/dt = v_theta(x, t), x(0) ~ N(0, I) (Eq. 8), conditioned on
 * the entry state and the cell in optical coordinates (Eq. 10).
 *
 * Geometry and units used by every entry point:
 *  - A cell is the square [0,tau]^2 in optical coordinates (sigma_t = 1);
 *    tau is its optical side and c = sigma_s / sigma_t its scattering ratio.
 *    Directions are unit vectors of the plane (cos theta, sin theta).
 *  - Canonical frame (stage 1 of the transport algorithm): the particle
 *    enters the left face x = 0 at y = xi * tau, xi in [0,1], moving with
 *    cos theta > 0.
 *  - Faces are numbered counter-clockwise from the corner (0,0): 0 bottom,
 *    1 right, 2 top, 3 left. The unwrapped perimeter coordinate is
 *    p = face + q in [0,4) with q the counter-clockwise position on the face:
 *    bottom x = q tau, right y = q tau, top x = (1-q) tau, left y = (1-q) tau.
 *  - Path lengths s are in optical units (total mean free paths).
 *
 * Conventions:
 *  - Every call returns a gmc_status; nothing throws across the ABI. On error
 *    gmc_last_error(ctx) describes the failure (the returned string is the
 *    calling thread's copy, valid until its next gmc_last_error call).
 *  - Array arguments are structure-of-arrays, row k of an [m][n] array
 *    starting at element k*n. Unless a parameter says "host", array pointers
 *    may be device pointers (the call runs asynchronously on the context's
 *    stream) or host pointers (the call returns when results are on the
 *    host): page-locked host memory (cudaHostAlloc, cudaHostRegister) is
 *    read and written in place by the kernels over the CPU-GPU link; other
 *    host memory is copied in and out through context-owned device buffers.
 *    Device memory must belong to the context's GPU (or be managed memory):
 *    another GPU's memory gives GMC_EINVAL before any kernel runs.
 *    The caller owns every buffer it passes; the context owns its weights,
 *    particle banks and scratch.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with counter
 *    (id_lo, id_hi, event, tag) and key (seed_lo, seed_hi); tags: 1 walk
 *    flights, 2 flow-ODE noise, 3 roulette, 4 births, 5 training data,
 *    6 training batches. Uniforms lie in (0,1].
 */
#ifndef GMC_H
#define GMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gmc_status {
    GMC_OK = 0,
    GMC_EINVAL = -1,     /* bad argument (null pointer, size, range) */
    GMC_ENOMEM = -2,     /* device or host allocation failed */
    GMC_ECUDA = -3,      /* a CUDA runtime call failed */
    GMC_ETIMEOUT = -4,   /* a bounded device-side wait ran out */
    GMC_EFORMAT = -5,    /* malformed or unsupported weight file */
    GMC_ENOTIMPL = -6,   /* option not implemented */
    GMC_EBUSY = -7,      /* result not ready yet (serving) */
    GMC_ENOWEIGHTS = -8, /* a GMC call before gmc_load_weights */
    GMC_EIO = -9         /* file could not be read or written */
} gmc_status;

typedef enum gmc_precision { GMC_FP32 = 0, GMC_BF16 = 1, GMC_FP8 = 2 } gmc_precision;
/* Fixed-step integrators of Eq. 8 with h = 1/K, t_k = k h: explicit Euler,
   explicit midpoint, classical Runge-Kutta (four evaluations per step; the
   solver the paper times). */
typedef enum gmc_integrator { GMC_EULER = 0, GMC_MIDPOINT = 1, GMC_RK4 = 2 } gmc_integrator;
typedef enum gmc_absorb_mode { GMC_ABSORB_ANALOG = 0, GMC_ABSORB_IMPLICIT = 1 } gmc_absorb_mode;
typedef enum gmc_method { GMC_METHOD_ANALOG = 0, GMC_METHOD_GMC = 1 } gmc_method;
/* Kernel of the BF16 tensor-core sampler (results agree within the BF16
   bound; the FP8 path always uses the tile kernel): GMC_KERNEL_TILE, one
   CTA per SM running two M = 128 tiles with one accumulator; GMC_KERNEL_PAIR,
   clusters of two CTAs running M = 256 tiles (tcgen05 cta_group::2) with two
   accumulators per CTA. */
typedef enum gmc_sampler_kernel { GMC_KERNEL_TILE = 0, GMC_KERNEL_PAIR = 1 } gmc_sampler_kernel;

typedef struct gmc_ctx gmc_ctx;

/* Options of the GMC sampler and of transport solves (gmc_set_config). */
typedef struct gmc_config {
    int steps;             /* ODE steps K (Eq. 8), 1..256; default 16 */
    int integrator;        /* gmc_integrator; default GMC_EULER */
    int precision;         /* gmc_precision of the velocity network; default GMC_BF16 */
    double w_cut;          /* roulette threshold on the particle weight; default 1e-4 */
    double p_survive;      /* roulette survival probability; default 0.1 */
    int64_t bank_capacity; /* particles in flight per wave in transport_solve; default 2^21 */
    int flights_per_wave;  /* random-walk flights a particle takes per wave of transport_solve
                              before it waits for the next wave (births, and every walk of
                              GMC_METHOD_ANALOG); results do not depend on it; default 512 */
    double gmc_min_tau;    /* GMC solves only: cells with tau below this are crossed (and
                              their births walked) by the random walk instead of the
                              networks, so GMC runs where one network evaluation costs less
                              than the walk's flights; 0 (default) = every cell by GMC, as
                              in the paper */
    /* GMC solves: the box of (tau, c) the networks were trained on (both
       models; defaults [0.1, 1000] x [0.5, 0.999], the trainer's). The
       networks learn the implicit-capture walk, whose exits depend on the
       scattering thickness c tau alone and whose track lengths scale as 1/c
       (section "Monte Carlo Method", Eq. 4-5). A cell outside the box is
       sampled at the in-box condition (tau', c') with c' tau' = c tau (c'
       the value in [c_lo, c_hi] nearest c that keeps tau' in the box) and
       its sampled track length multiplied by c'/c; a cell whose c tau lies
       outside [c_lo tau_lo, c_hi tau_hi] (c = 0 included) has no such
       condition and is crossed, and its births walked, by the random walk.
       Need 0 < net_tau_lo <= net_tau_hi, 0 < net_c_lo <= net_c_hi <= 1. */
    double net_tau_lo, net_tau_hi;
    double net_c_lo, net_c_hi;
    int sampler_kernel;    /* gmc_sampler_kernel of BF16 sampling (gmc_transmit, solves,
                              gmc_transmit_noalloc); default GMC_KERNEL_TILE */
} gmc_config;

/* Per-solve counters (all weights per history-weight unit, not normalized). */
typedef struct gmc_solve_stats {
    double leaked;          /* weight that left the domain */
    double absorbed;        /* deposited weight, sum of Delta w (Eq. 6) */
    double roulette_net;    /* weight added (+) or removed (-) by roulette */
    int64_t transmissions;  /* cell transmissions, births included */
    int64_t collisions;     /* scatterings simulated by random walks */
    int64_t roulette_kills; /* histories ended by roulette */
    int64_t waves;          /* event waves of the particle loop while the solve was admitted */
    int64_t inward_fixes;   /* sampled exit directions that pointed into the cell */
    double seconds;         /* device time from admission to the last wave */
    double latency;         /* host wall time from submission to completion */
} gmc_solve_stats;

/* ---- context ------------------------------------------------------------ */

/*
 * Failure-path self-test (no counterpart in the paper): one device thread
 * waits on an mbarrier that nothing arrives at, using the bounded wait of the
 * tensor-core kernels, gives up after limit_ms (0 < limit_ms <= 2000) and sets
 * the device error word. Returns what every blocking call returns after a
 * wait gave up: GMC_ETIMEOUT, with the error word cleared and the context
 * usable. Blocking.
 */
gmc_status gmc_selftest_wait(gmc_ctx *ctx, double limit_ms);

/* Creates a context on CUDA device `device` with its own stream (a blocking
   stream: ordered with work on the legacy default stream, not with other
   non-blocking streams; pass those with gmc_set_stream). */
gmc_status gmc_create(gmc_ctx **out, int device);
/* Frees the context and every device buffer it owns. Null is accepted. */
gmc_status gmc_destroy(gmc_ctx *ctx);
/* Uses `cuda_stream` (a cudaStream_t, or null for the context's own stream)
   for every later call; the caller keeps ownership of a stream it passes. */
gmc_status gmc_set_stream(gmc_ctx *ctx, void *cuda_stream);
/* Waits until all work queued by the context has finished. */
gmc_status gmc_synchronize(gmc_ctx *ctx);
gmc_status gmc_get_config(const gmc_ctx *ctx, gmc_config *out);
/* Validates and applies `cfg` (steps in [1, 256], w_cut >= 0,
   p_survive in (0, 1], bank_capacity in [1024, 2^28]); GMC_EBUSY while the
   server (gmc_serve_start) runs. */
gmc_status gmc_set_config(gmc_ctx *ctx, const gmc_config *cfg);
const char *gmc_status_str(gmc_status s);
const char *gmc_last_error(const gmc_ctx *ctx);

/* ---- random numbers ------------------------------------------------------ */

/* Raw Philox4x32-10 blocks for ids id0 .. id0+n-1 at one (event, tag):
   out [n][4] u32. */
gmc_status gmc_philox(gmc_ctx *ctx, int64_t n, uint64_t seed, uint64_t id0, uint32_t event,
                      uint32_t tag, uint32_t *out);
/* Box-Muller normals from the same blocks: u = (x+1) 2^-32,
   z0,z1 = sqrt(-2 ln u0) (cos, sin)(2 pi u1), z2,z3 likewise from u2,u3.
   out [4][n] float. */
gmc_status gmc_normals(gmc_ctx *ctx, int64_t n, uint64_t seed, uint64_t id0, uint32_t event,
                       uint32_t tag, float *out);

/* ---- GMC sampler (stage 2 of the transport algorithm) --------------------- */

/*
 * Loads a velocity network from a "GMCW" version-1 file (host path):
 * magic "GMCW", u32 version = 1, u32 n_layers = 5, u32 dims[6] =
 * {25,256,256,256,256,4}, u32 n_cond = 5, n_state = 4, n_emb = 16, flags;
 * f32 cond_mean[5], cond_std[5], y_mean[4], y_std[4]; then per layer
 * f32 W[out][in], f32 b[out]. The network input is [standardized condition
 * (5), state x (4), emb(t) (16)] with emb(t) = [sin(2^j pi t)]_{j<8},
 * [cos(2^j pi t)]_{j<8}; hidden layers use SiLU. Returns GMC_EIO if the file
 * cannot be read, GMC_EFORMAT on any layout mismatch (the network loaded
 * before, if any, is then kept unchanged), GMC_EBUSY while the server runs.
 * The FP32 weights are kept and the BF16 / FP8 packed copies are derived
 * from them.
 * flags = 1 marks the residual-modulated network, a reading of the paper's
 * architecture (section "Network Architecture and Inputs": residual blocks
 * with adaptive modulation conditioned on the physical context): the file
 * continues with f32 M[3][256][5] and G[3][2][256], and hidden layers 2-4
 * become a_l = a_{l-1} + SiLU(g_l z_l) with z_l = W_l a_{l-1} + b_l + M_l c
 * and g_l = 1 + G_l[0] c_3 + G_l[1] c_4 (c standardized; c_3 = ln tau,
 * c_4 = c). It runs at GMC_FP32 and at GMC_BF16 with GMC_KERNEL_TILE;
 * GMC_FP8 and GMC_KERNEL_PAIR give GMC_EINVAL in gmc_transmit, solves and
 * serving. Other flag bits give GMC_EFORMAT.
 * n_cond = 6 with dims[0] = 26 is a network for rectangular cells (section
 * "Network Architecture and Inputs": the condition holds both optical
 * dimensions): the sixth condition component ln(tau_y / tau_x) enters as
 * input column 25, after the time embedding, and cond_mean / cond_std have 6
 * entries. It samples single cells (gmc_transmit with [6][n] conditions) at
 * GMC_FP32 and GMC_BF16 with GMC_KERNEL_TILE; solves, serving and
 * gmc_transmit_noalloc, whose cells are squares, refuse it with GMC_EINVAL,
 * and it cannot carry flag 1.
 */
gmc_status gmc_load_weights(gmc_ctx *ctx, const char *path);
/* Same, from a host buffer holding the file's bytes. */
gmc_status gmc_load_weights_buffer(gmc_ctx *ctx, const void *blob, size_t nbytes);

/*
 * Internal (volumetric-source) model: the second network of the method
 * (section "Network Architecture and Inputs": an internal model for particles
 * born inside a cell, a boundary model for particles crossing between cells).
 * Same GMCW layout; its condition is (X, Y, ln tau, c, d) for a birth at
 * (X, Y) in [0,1]^2 of the cell, d = min(X, Y, 1 - X, 1 - Y), and its state the
 * exit (p, cos, sin, ln s) in the cell's own frame. The birth direction is
 * isotropic and not a condition: the network samples the exit marginalized
 * over it. When loaded, GMC solves sample births with it (births otherwise
 * take the random walk). Errors as gmc_load_weights.
 */
gmc_status gmc_load_internal_weights(gmc_ctx *ctx, const char *path);
gmc_status gmc_load_internal_weights_buffer(gmc_ctx *ctx, const void *blob, size_t nbytes);

/*
 * Boundary model of x-y geometry (section "Network Architecture and Inputs":
 * 3-D directions encoded by their projection on the unit disk): same GMCW
 * layout and network shape, condition (xi, ux, uy, ln tau, c), state (p, ux,
 * uy, ln s); used by gmc_transmit_xy. Errors as gmc_load_weights.
 */
gmc_status gmc_load_xy_weights(gmc_ctx *ctx, const char *path);
gmc_status gmc_load_xy_weights_buffer(gmc_ctx *ctx, const void *blob, size_t nbytes);

/*
 * Internal model of x-y geometry: the internal model's condition (X, Y,
 * ln tau, c, d) for a birth inside a prism cell with an isotropic 3-D
 * direction, and its state the exit (p, ux, uy, ln s) with (ux, uy) the
 * projected exit direction (decoded into the unit disk) and s the 3-D track
 * length. When loaded, x-y GMC solves (transport_solve_xy) sample births
 * with it; gmc_sample_internal_xy samples it directly (arguments as
 * gmc_sample_internal). Errors as gmc_load_weights.
 */
gmc_status gmc_load_internal_xy_weights(gmc_ctx *ctx, const char *path);
gmc_status gmc_load_internal_xy_weights_buffer(gmc_ctx *ctx, const void *blob, size_t nbytes);
gmc_status gmc_sample_internal_xy(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                                  uint64_t seed, uint64_t id0, int steps, int integrator,
                                  int precision, float *y_raw, float *exit);

/*
 * Samples n exit states (Eq. 8, Eq. 11) with the loaded network.
 *  cond    [5][n] float: xi, cos theta_in, sin theta_in, ln tau, c (raw,
 *          standardized inside with the file's cond_mean / cond_std);
 *          [6][n] for a network of rectangular cells (its file has n_cond = 6):
 *          xi, cos, sin, ln tau_x, c, ln(tau_y / tau_x) for a cell of optical
 *          width tau_x and height tau_y entered on its left face.
 *  noise   [4][n] float x(0), or null: then x(0) is drawn as gmc_normals with
 *          ids id0+i, event 0, tag 2.
 *  steps   ODE steps K >= 1 (h = 1/K, t_k = k h); integrator gmc_integrator.
 *  precision gmc_precision: FP32 (SIMT, FP32 throughout), BF16 (tcgen05
 *          tensor cores, BF16 operands, FP32 accumulation and state), FP8
 *          (as BF16, but the three 256 x 256 layers take E4M3 weights with one
 *          FP32 scale per output channel and E4M3 inputs; the paper fixes no
 *          precision, this is a reduced-precision variant of Eq. 8's v_theta).
 *  y_raw   [4][n] float, nullable: standardized x(1).
 *  exit    [4][n] float, nullable: decoded exit state in the canonical frame:
 *          p in [0,4) (wrapped), exit direction (ux, uy) made unit and
 *          pointing out of face floor(p) (an inward normal component is
 *          reflected), s = max(exp(ln s), 1e-7).
 * At least one of y_raw / exit must be non-null. n = 0 is a no-op.
 */
gmc_status gmc_transmit(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                        uint64_t seed, uint64_t id0, int steps, int integrator, int precision,
                        float *y_raw, float *exit);
/* gmc_transmit with the internal model: cond [5][n] = (X, Y, ln tau, c, d) as
   above, exits in the cell's own frame; GMC_ENOWEIGHTS if none is loaded. */
gmc_status gmc_sample_internal(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                               uint64_t seed, uint64_t id0, int steps, int integrator,
                               int precision, float *y_raw, float *exit);
/*
 * gmc_transmit for x-y geometry (section "Network Architecture and Inputs",
 * the direction encoded on the unit disk) with the network loaded by
 * gmc_load_xy_weights (GMC_ENOWEIGHTS if none): cond [5][n] = (xi, ux, uy,
 * ln tau, c) with (ux, uy) the projection of the 3-D entry direction; the
 * decoded exit is (p, ux, uy, s) with the projected exit direction kept
 * inside the unit disk (scaled onto the circle only when it lies outside),
 * its normal component made outward (reflected, or the outward normal when
 * none is left) and s the 3-D track length.
 */
gmc_status gmc_transmit_xy(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                           uint64_t seed, uint64_t id0, int steps, int integrator, int precision,
                           float *y_raw, float *exit);

/*
 * gmc_transmit without any device allocation during the call (the paper has
 * no counterpart: this serves callers that cannot call cudaMalloc, such as
 * code under a framework that owns the device allocator, code inside a
 * latency-critical loop or graph-recording section, or hosts that allocate
 * only at start-up). Same arguments and results as gmc_transmit with
 * precision GMC_BF16, except:
 *  - every array must be device memory of the context's GPU, or managed
 *    memory (host pointers and other GPUs' memory give GMC_EINVAL);
 *  - steps must be in [1, 256] (Euler, midpoint) or [1, 128] (RK4): the
 *    layer-1 bias table lives in a static 512 KiB device array (512 network
 *    evaluations), held by every GPU that loads the library until the
 *    process exits; larger values give GMC_EINVAL;
 *  - the first call on a device resolves that array's address (and may load
 *    the library's device code); make it before any stream capture;
 *  - all calls on a device share the array: calls whose kernels overlap on
 *    the GPU race and must be serialized by the caller.
 * Asynchronous on the context's stream; a bounded-wait failure is reported
 * by the next gmc_synchronize.
 */
gmc_status gmc_transmit_noalloc(gmc_ctx *ctx, int64_t n, const float *cond, const float *noise,
                                uint64_t seed, uint64_t id0, int steps, int integrator,
                                float *y_raw, float *exit);

/* ---- analog random-walk transmission (the method GMC replaces) ------------ */

/*
 * Random-walk transmission through one cell per particle (section "Monte
 * Carlo Method", Eq. 4): free flights d = -ln(u)/sigma, step min(d_b, d),
 * isotropic scattering. mode GMC_ABSORB_ANALOG: sigma = 1 and each collision
 * survives with probability c (survive iff u1 <= c), otherwise the particle
 * is absorbed; GMC_ABSORB_IMPLICIT: sigma = c, no absorption (the weight
 * factor exp(-(1-c) s) of Eq. 5 is left to the caller).
 * Philox: flight j of particle i uses counter (id0+i, event0+j, tag 1):
 * u0 -> flight, u1 -> survival, u2 -> new angle 2 pi u2.
 *  xi, cos_in, sin_in, tau, c  [n] float (tau > 0, c in [0,1], cos_in > 0).
 *  status  [n] int32: 0 exited, 1 absorbed.
 *  exit    [4][n] float: p = face + q (-1 if absorbed), final direction
 *          (ux, uy), track length s in the cell.
 *  ncoll   [n] uint32, nullable: collisions (scatterings and absorption).
 */
gmc_status analog_transmit(gmc_ctx *ctx, int64_t n, const float *xi, const float *cos_in,
                           const float *sin_in, const float *tau, const float *c, int mode,
                           uint64_t seed, uint64_t id0, uint32_t event0, int32_t *status,
                           float *exit, uint32_t *ncoll);

/*
 * As analog_transmit for rectangular cells (the random walk of section "Monte
 * Carlo Method", Eq. 4, in the paper's cell of width W and height H, here with
 * unequal optical sides): cell i has optical width tau_x[i] along x and
 * height tau_y[i] along the entry face; the particle enters the left face at height
 * xi[i] * tau_y[i]. The exit position q is normalized along the exit face
 * (p = face + q in [0,4) as for the square cell), s is the track length in
 * optical units. tau_x = tau_y = tau is analog_transmit's walk.
 *  tau_x, tau_y  [n] float (> 0). Other arguments as analog_transmit.
 */
gmc_status analog_transmit_rect(gmc_ctx *ctx, int64_t n, const float *xi, const float *cos_in,
                                const float *sin_in, const float *tau_x, const float *tau_y,
                                const float *c, int mode, uint64_t seed, uint64_t id0,
                                uint32_t event0, int32_t *status, float *exit, uint32_t *ncoll);

/*
 * As analog_transmit_rect in x-y geometry (the paper's encoding of a
 * direction by its projection on the unit disk, section "Network
 * Architecture and Inputs"; the walk of section "Monte Carlo Method", Eq. 4):
 * the cell is the cross-section of an infinite prism and directions are 3-D
 * unit vectors, given and returned by their projection (ux, uy) on the
 * plane; a flight of 3-D length d moves the particle by d (ux, uy); a
 * scattering draws the direction isotropically on the sphere (azimuth
 * 2 pi u2, polar cosine 2 u3 - 1 from the flight's Philox block); s is the
 * 3-D track length. The out-of-plane component is +-sqrt(1 - ux^2 - uy^2);
 * its sign does not enter the walk.
 *  ux_in, uy_in  [n] float: entry direction's projection, ux_in > 0,
 *                ux_in^2 + uy_in^2 <= 1.
 *  exit          [4][n] float: p (or -1), projected exit direction ux, uy,
 *                s. Other arguments as analog_transmit_rect.
 */
gmc_status analog_transmit_xy(gmc_ctx *ctx, int64_t n, const float *xi, const float *ux_in,
                              const float *uy_in, const float *tau_x, const float *tau_y,
                              const float *c, int mode, uint64_t seed, uint64_t id0,
                              uint32_t event0, int32_t *status, float *exit, uint32_t *ncoll);

/* ---- transport solve (the four-stage transport algorithm) ----------------- */

/*
 * Scalar flux of a fixed-source problem on an nx x ny grid of unit cells
 * (cell (i,j) at element j*nx+i; physical side 1, so V = 1, sigma_t = tau,
 * sigma_a = (1-c) tau), vacuum boundaries, isotropic volumetric source
 * `source` (relative strengths, >= 0, not all zero; the birth cell is drawn
 * in proportion, the point uniformly, the direction isotropically).
 * Every cell crossing deposits Delta w = w (1 - exp(-sigma_a Delta s))
 * (Eq. 6) and scores Delta w / (V sigma_a) (Eq. 7) into the cell's FP64
 * tally; the weight is attenuated by exp(-sigma_a Delta s) (Eq. 5); below
 * w_cut the particle plays roulette (survive with p_survive, weight /=
 * p_survive). method GMC_METHOD_ANALOG walks every cell with implicit
 * capture; GMC_METHOD_GMC walks only the birth cell and samples every later
 * cell crossing with the network (config steps / integrator / precision).
 *  tau, c, source  host [ny*nx] float (tau > 0, c in [0,1]; for GMC,
 *                  tau in [0.05, 2000] and c in [0.4, 1]).
 *  flux            host [ny*nx] double: flux per source particle.
 *  stats           host, nullable.
 * Blocking: returns when the flux is on the host.
 */
gmc_status transport_solve(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                           const float *source, int64_t n_histories, int method, uint64_t seed,
                           double *flux, gmc_solve_stats *stats);

/*
 * As transport_solve with a surface source on the left boundary (x = 0)
 * instead of a volumetric one: history h (Philox draw (h, 0, tag 4) =
 * (u0, u1, u2, u3)) enters boundary row j, the first whose cumulative
 * strength reaches u0 * sum(wall), through the west face of cell (0, j) at
 * height j + u1, with sin(theta) = 2 u2 - 1 against the inward normal (the
 * cosine law of an isotropic radiance seen through the boundary), weight 1;
 * its first cell crossing is a transmission of the chosen method. This is the
 * boundary-source problem of the paper's experiments (a driven wall).
 *  wall  host [ny] float, relative strengths (>= 0, not all zero).
 * Other arguments, the result and blocking as for transport_solve.
 */
gmc_status transport_solve_wall(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                                const float *wall, int64_t n_histories, int method, uint64_t seed,
                                double *flux, gmc_solve_stats *stats);

/*
 * The two solves in x-y geometry (the geometry variant of section "Network
 * Architecture and Inputs": every cell is the cross-section of an infinite
 * prism, directions are 3-D and enter the networks by their projection on
 * the unit disk): a flight of 3-D length d moves the particle by d (ux, uy)
 * in the plane, the track length s of Eq. 5-7 is the 3-D one, and the walk
 * scatters isotropically on the sphere (azimuth 2 pi u2, polar cosine
 * 2 u3 - 1 of the flight's draw). Volumetric births take the azimuth of
 * transport_solve and the polar cosine 2 u - 1 from the first uniform of the
 * draw (h, 1, tag 4); wall entries take the 3-D cosine law, cosine to the
 * inward normal sqrt(u2) and azimuth about it 2 pi u3. GMC_METHOD_GMC samples
 * cell crossings with the x-y boundary network (gmc_load_xy_weights;
 * GMC_ENOWEIGHTS without it) and its births with the x-y internal model
 * when one is loaded (gmc_load_internal_xy_weights), else walks them. Other arguments, the
 * result and blocking as for transport_solve and transport_solve_wall.
 */
gmc_status transport_solve_xy(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                              const float *source, int64_t n_histories, int method, uint64_t seed,
                              double *flux, gmc_solve_stats *stats);
gmc_status transport_solve_wall_xy(gmc_ctx *ctx, int nx, int ny, const float *tau, const float *c,
                                   const float *wall, int64_t n_histories, int method,
                                   uint64_t seed, double *flux, gmc_solve_stats *stats);

/*
 * transport_solve on rectangular cells of physical size dx x dy (every cell
 * alike; the geometry variant of section "Network Architecture and Inputs"
 * with W != H): sigma [ny*nx] the cells' cross sections, so cell k has the
 * optical width sigma[k] dx and height sigma[k] dy. The walk crosses the
 * rectangle as in analog_transmit_rect; births are uniform in the cell and
 * walked. GMC_METHOD_GMC samples cell crossings with a network of
 * rectangular cells loaded by gmc_load_weights (n_cond 6; GMC_EINVAL
 * otherwise): in the canonical frame of the entry face the condition's
 * width is the depth behind it and the aspect the face's length over it (a
 * quarter turn exchanges the two sides). flux: per source particle per unit
 * area, Delta w / (sigma_a dx dy) (Eq. 7). A cell outside the networks' box
 * (gmc_config.net_*) is sampled at the equivalent condition that keeps both
 * optical sides in it: c' in [net_c_lo, net_c_hi] and in
 * [c max(tx, ty) / net_tau_hi, c min(tx, ty) / net_tau_lo] (nearest c),
 * tx' = c tx / c', ty' = c ty / c', track lengths times c'/c; a cell where
 * no such c' exists is crossed by the random walk. Volumetric sources only.
 * GMC_EINVAL as well for dx or dy not finite and > 0, dy / dx outside
 * [1e-37, 1e37], or a cell with sigma dy outside (0, 1e38] (the walk forms
 * the height in FP32). Other arguments, the result and blocking as for
 * transport_solve.
 */
gmc_status transport_solve_rect(gmc_ctx *ctx, int nx, int ny, const float *sigma, const float *c,
                                const float *source, float dx, float dy, int64_t n_histories,
                                int method, uint64_t seed, double *flux, gmc_solve_stats *stats);

/* ---- serving: continuous batching of transport solves ---------------------- */

/* One transport solve (arguments of transport_solve; arrays are host memory
   and are copied by gmc_submit, so the caller may free them afterwards). */
typedef struct gmc_solve_req {
    int nx, ny;
    const float *tau, *c, *source;
    int64_t n_histories;
    uint64_t seed;
} gmc_solve_req;

typedef struct gmc_serve_config {
    int method;           /* gmc_method used for every request */
    size_t memory_budget; /* device bytes for admitted requests' grids and
                             tallies: 37 B per cell (tau, c, the networks'
                             condition and track-length factor, the walk
                             flag, source CDF, FP64 tally; each array
                             rounded up to 256 B); >= 1 MiB */
} gmc_serve_config;

/*
 * Starts a worker thread that runs the wave engine of transport_solve over
 * every admitted request at once: requests share one particle bank
 * (bank_capacity from gmc_config), each new wave gives free bank slots to
 * the births of admitted requests in equal shares, and a request is admitted
 * (first come, first served) as soon as its grid, CDF and tally fit in the
 * memory budget and one of 64 request slots is free. Its result equals that
 * of transport_solve alone (same random numbers; only the order of FP64
 * additions differs). The server uses its own stream and buffers; loading
 * weights and gmc_set_config return GMC_EBUSY while it runs.
 */
gmc_status gmc_serve_start(gmc_ctx *ctx, const gmc_serve_config *cfg);
/* Queues a solve; *ticket identifies it. GMC_ENOMEM if the request alone
   exceeds the memory budget, GMC_EINVAL as transport_solve. */
gmc_status gmc_submit(gmc_ctx *ctx, const gmc_solve_req *req, uint64_t *ticket);
/* GMC_EBUSY while the request runs; GMC_OK once done, filling flux (host
   [ny*nx] double, flux per source particle) and stats (nullable); the ticket
   is then retired. */
gmc_status gmc_poll(gmc_ctx *ctx, uint64_t ticket, double *flux, gmc_solve_stats *stats);
/* As gmc_poll, blocking up to timeout_s seconds (GMC_ETIMEOUT after). */
gmc_status gmc_wait(gmc_ctx *ctx, uint64_t ticket, double timeout_s, double *flux,
                    gmc_solve_stats *stats);
/* Stops the worker; unfinished requests are dropped. */
gmc_status gmc_serve_stop(gmc_ctx *ctx);

/* ---- learning the sampler (conditional flow matching, Eq. 9) ------------ */

/* AdamW and batch options of gmc_train_begin. */
typedef struct gmc_train_config {
    int64_t batch;       /* rows per step, in [1, 2^20]; e.g. 8192 */
    double lr;           /* learning rate, > 0 and finite, e.g. 1e-3 */
    double beta1, beta2; /* each in [0, 1), e.g. 0.9, 0.999 */
    double eps;          /* > 0 and finite, e.g. 1e-8 */
    double weight_decay; /* decoupled weight decay, >= 0 and finite, e.g. 0.01 */
    uint64_t seed;       /* Philox key of the batch draws (tag 6) */
    int precision;       /* GMC_FP32: SIMT FP32 GEMMs, FP32 activations (the only
                            choice for the residual-modulated network and for a
                            network of rectangular cells); GMC_BF16: the
                            tcgen05 step (four kernels per step): BF16 activations,
                            SiLU' factors and input gradients between layers, FP32
                            accumulation, weight and bias gradients summed in FP32 in
                            a fixed order, FP32 master weights and AdamW moments */
} gmc_train_config;

/*
 * Training data (section "Network Architecture and Inputs": exit states of
 * pure-scattering Monte Carlo transmissions): for sample i, Philox block
 * (i, 0, tag 5) gives ln tau uniform in [ln tau_lo, ln tau_hi], c uniform in
 * [c_lo, c_hi], xi uniform, sin theta uniform in (-1, 1); the implicit-capture
 * walk (analog_transmit mode GMC_ABSORB_IMPLICIT, flights from event 1) runs
 * from the left face. cond [5][n] = (xi, cos, sin, ln tau, c) and
 * y [4][n] = (p, cos theta_out, sin theta_out, ln s): device memory.
 * GMC_EINVAL unless 0 < tau_lo <= tau_hi (finite) and 0 <= c_lo <= c_hi <= 1
 * (the same ranges for every training-data generator below; for
 * gmc_train_data_rect also 0 < aspect_lo <= aspect_hi, finite).
 */
gmc_status gmc_train_data(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo, float tau_hi,
                          float c_lo, float c_hi, float *cond, float *y);
/*
 * Training data of the internal model: for sample i, Philox block (i, 0, tag 7)
 * gives ln tau uniform in [ln tau_lo, ln tau_hi], c uniform in [c_lo, c_hi],
 * X and Y uniform; (i, 1, tag 7) the isotropic birth direction; the
 * implicit-capture walk from (X, Y) draws from event 2 on.
 * cond [5][n] = (X, Y, ln tau, c, min(X, Y, 1 - X, 1 - Y)), y [4][n] =
 * (p, cos, sin, ln s) in the cell's own frame: device memory.
 */
gmc_status gmc_train_data_internal(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo,
                                   float tau_hi, float c_lo, float c_hi, float *cond, float *y);
/*
 * Training data of the boundary model in x-y geometry (section "Network
 * Architecture and Inputs": the direction enters as its projection on the
 * unit disk; the cell is the cross-section of an infinite prism and
 * scattering is isotropic on the sphere, as analog_transmit_xy): for sample
 * i, Philox block (i, 0, tag 8) gives ln tau uniform in [ln tau_lo,
 * ln tau_hi], c uniform in [c_lo, c_hi], xi uniform and the cosine
 * mu = sqrt(u) of the entry direction to the face normal; (i, 1, tag 8) its
 * azimuth 2 pi u about the normal; the projected entry direction is
 * (mu, sqrt(1 - mu^2) cos phi). The implicit-capture walk runs from the left
 * face, flights from event 2. cond [5][n] = (xi, ux, uy, ln tau, c) and
 * y [4][n] = (p, ux_out, uy_out, ln s) with (ux_out, uy_out) the projected
 * exit direction and s the 3-D track length: device memory.
 */
gmc_status gmc_train_data_xy(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo, float tau_hi,
                             float c_lo, float c_hi, float *cond, float *y);
/*
 * Training data of the internal model in x-y geometry: for sample i, Philox
 * block (i, 0, tag 9) gives ln tau uniform in [ln tau_lo, ln tau_hi], c
 * uniform in [c_lo, c_hi], X and Y uniform; (i, 1, tag 9) the isotropic 3-D
 * birth direction, azimuth 2 pi u0 and polar cosine 2 u1 - 1; the
 * implicit-capture walk on the sphere from (X, Y) draws from event 2 on.
 * cond [5][n] = (X, Y, ln tau, c, min(X, Y, 1 - X, 1 - Y)), y [4][n] =
 * (p, ux, uy, ln s) in the cell's own frame (projected exit direction, 3-D
 * track length): device memory.
 */
gmc_status gmc_train_data_internal_xy(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo,
                                      float tau_hi, float c_lo, float c_hi, float *cond, float *y);
/*
 * Training data of the boundary model for rectangular cells (section
 * "Network Architecture and Inputs": the condition holds both optical
 * dimensions): for sample i, Philox block (i, 0, tag 10) gives ln tau_x
 * uniform in [ln tau_lo, ln tau_hi], c uniform in [c_lo, c_hi], xi uniform and
 * sin theta = 2 u - 1; (i, 1, tag 10) the aspect, ln(tau_y / tau_x) uniform in
 * [ln aspect_lo, ln aspect_hi]. The implicit-capture walk in the cell
 * [0, tau_x] x [0, tau_y] runs from (0, xi tau_y), flights from event 2.
 * cond [6][n] = (xi, cos, sin, ln tau_x, c, ln(tau_y / tau_x)), y [4][n] =
 * (p, cos, sin, ln s), q normalized per face: device memory. A network for
 * rectangular cells (n_cond 6) trains on it with precision GMC_FP32.
 */
gmc_status gmc_train_data_rect(gmc_ctx *ctx, int64_t n, uint64_t seed, float tau_lo, float tau_hi,
                               float aspect_lo, float aspect_hi, float c_lo, float c_hi, float *cond,
                               float *y);
/*
 * Starts training on the device dataset (cond, y as gmc_train_data writes;
 * the caller keeps them alive while training). Standardization statistics
 * (mean and standard deviation of the 5 condition and 4 target components)
 * are computed from the data; the FP32 master weights start from the loaded
 * network (gmc_load_weights must have been called); AdamW moments start at 0.
 * GMC_EINVAL for a configuration outside the ranges of gmc_train_config.
 */
gmc_status gmc_train_begin(gmc_ctx *ctx, int64_t n, const float *cond, const float *y,
                           const gmc_train_config *cfg);
/*
 * n_steps optimizer steps: batch rows from Philox (row r of step k uses
 * (k*batch + r, 0, tag 6): sample index, t in (0,1]; (.., 1, tag 6): x0),
 * x_t = (1-t) x0 + t x1, loss = mean_b ||v(x_t, t | c) - (x1 - x0)||^2
 * (Eq. 9), hand-written backward, AdamW:
 * p <- p (1 - lr wd) - lr m_hat / (sqrt(v_hat) + eps).
 * losses: host [n_steps] float, nullable (blocking when given).
 */
gmc_status gmc_train_steps(gmc_ctx *ctx, int64_t n_steps, float *losses);
/* Learning rate of later gmc_train_steps calls (a schedule is a sequence of
   calls); AdamW moments and the step count carry over. */
gmc_status gmc_train_set_lr(gmc_ctx *ctx, double lr);
/*
 * Loss and gradient of Eq. 9 at the current master weights for an explicit
 * batch (host arrays): cn [B][5] standardized conditions ([B][6] for a
 * network of rectangular cells), x1 [B][4] standardized targets, x0 [B][4]
 * noise, t [B]. grad: host array of gmc_train_param_count_ctx() floats in
 * the order W1 [256][32] (input columns 25..31 are padding; column 25 is the
 * aspect of a rectangular-cell network), b1, W2, b2, W3, b3, W4, b4,
 * W5 [4][256], b5, then the residual-modulated network's M and G.
 * B must not exceed the configured batch.
 */
gmc_status gmc_train_grad(gmc_ctx *ctx, int64_t B, const float *cn, const float *x1,
                          const float *x0, const float *t, double *loss, float *grad);
/* Copies the FP32 master weights (layout of gmc_train_grad) to host `out`. */
gmc_status gmc_train_params(gmc_ctx *ctx, float *out);
int64_t gmc_train_param_count(void);
/* Parameters of the network being trained (GMC_EINVAL before
   gmc_train_begin): gmc_train_param_count() for the MLP; for the
   residual-modulated network (weight-file flag 1) 5376 more, appended in the
   order M2..M4 [256][5] (condition shifts of hidden layers 2-4), then
   G2..G4 [2][256] (their channel scales). gmc_train_grad and
   gmc_train_params then read or write this many floats. */
gmc_status gmc_train_param_count_ctx(const gmc_ctx *ctx, int64_t *count);
/*
 * Training checkpoint (host memory): the FP32 master weights, AdamW's first
 * and second moments, the step count, the hyperparameters (learning rate as
 * last set, betas, eps, weight decay, seed) and the standardization
 * statistics. gmc_train_state_size gives the size in bytes (a header plus
 * 3 gmc_train_param_count_ctx() floats). gmc_train_save_state writes a
 * checkpoint into `blob` (exactly that many bytes). gmc_train_load_state
 * restores one into the training state of gmc_train_begin, which must have
 * been called on the same dataset with the same batch and precision
 * (GMC_EINVAL otherwise; GMC_EFORMAT for a blob that is not a checkpoint,
 * one of another network form: residual-modulated or not, square or
 * rectangular cells, or one whose statistics or hyperparameters are out of
 * range: a non-finite statistic, a standard deviation <= 0, lr <= 0, a beta
 * outside [0, 1), eps <= 0, a negative weight decay).
 * The checkpoint records the dataset's size and its standardization
 * statistics, which gmc_train_begin recomputes from the data: other data (a
 * different size, or statistics that differ in any bit) gives GMC_EINVAL.
 * Step k's batch is drawn from Philox at (seed, k), so steps after a restore
 * continue the saved run exactly.
 */
gmc_status gmc_train_state_size(const gmc_ctx *ctx, size_t *bytes);
gmc_status gmc_train_save_state(gmc_ctx *ctx, void *blob, size_t nbytes);
gmc_status gmc_train_load_state(gmc_ctx *ctx, const void *blob, size_t nbytes);
/* Makes the trained network (with its standardization) the sampler's
   network; also writes it as a GMCW file when `path` is not null.
   GMC_EBUSY, with nothing written, while the server runs. */
gmc_status gmc_train_commit(gmc_ctx *ctx, const char *path);

#ifdef __cplusplus
}
#endif
#endif /* GMC_H */
