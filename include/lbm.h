/*
 * lbm.h - C ABI of the GB300 (sm_103a) multiphase lattice Boltzmann library for contact angles
 * on curved wetting surfaces (Liu, Yao, Li, Wen, "Contact angle measurement on curved wetting
 * surface in multiphase lattice Boltzmann method", arXiv:2202.06516).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an lbm_status; nothing aborts, exits or traps. On failure the context
 *    keeps a message readable with lbm_last_error().
 *  - Host buffers passed in are borrowed for the duration of the call and never freed. Device
 *    memory is owned by the context and released by lbm_destroy().
 *  - Work is issued on the context's stream (lbm_params.stream, or a private non-blocking stream
 *    when NULL). Calls that return results to the host synchronise that stream.
 *  - Lattice: fluid-domain nodes (i, j), 0 <= i < nx periodic in x, 0 <= j < ny; rows j = -2, -1
 *    and j = ny, ny+1 are solid wall rows (the two wetting layers of Sec. 3.1). Node index
 *    n = j * nx + i. Row-major host arrays of the fluid domain have shape (ny, nx); arrays of the
 *    extended lattice have shape (ny + 4, nx) with row r holding j = r - 2.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque; owns the device state of one lattice */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,        /* invalid argument (message says which) */
    LBM_ERR_CUDA = 2,       /* a CUDA runtime call failed (message has the CUDA error) */
    LBM_ERR_STATE = 3,      /* call out of order, e.g. lbm_step before lbm_set_geometry */
    LBM_ERR_UNSTABLE = 4,   /* non-finite or non-positive density found by a reduction */
    LBM_ERR_NO_CONTACT = 5, /* a side has no interface points in the band near the substrate */
    LBM_ERR_TIMEOUT = 6     /* reserved for bounded device-side waits */
} lbm_status;

enum { LBM_FP32 = 0, LBM_FP64 = 1 };          /* storage and arithmetic type of the step */
enum { LBM_EOS_PR = 0, LBM_EOS_CS = 1 };      /* Peng-Robinson (Eq. 10) or Carnahan-Starling */
enum { LBM_MRT = 0, LBM_BGK = 1 };            /* collision of Eq. 1 or Eq. 3 */
enum { LBM_FLUID = 0, LBM_LAYER1 = 1, LBM_LAYER2 = 2, LBM_SOLID = 3 }; /* node classes */
enum { LBM_TILE_AUTO = -1 };                  /* lbm_params.tile_x: choose by autotuning */
enum { LBM_BB_HALFWAY = 0, LBM_BB_INTERP = 1 }; /* lbm_geometry.boundary: curved-wall scheme */

/* Model parameters (lattice units).
 *  k2, kappa: k^2 and kappa-hat of the mesh-space chemical potential, Eq. 12.
 *  tau: s_v = 1/tau (Sec. 2.1) and the BGK relaxation time (Eq. 3).
 *  s_e, s_eps, s_q: MRT rates of S = diag(0, s_e, s_eps, 0, s_q, 0, s_q, s_v, s_v) (Sec. 2.1).
 *  gx, gy: body acceleration; the force (rho - g_rho_ref) g acts on gas and liquid (Sec. 4).
 *  g_rho_ref: reference density of the body force. 0 (default): the full weight rho g. rho_g:
 *    the gas carries no load, which stands in for a closed container whose gas weight is
 *    borne by its hydrostatic pressure; needed when g points along the periodic x axis,
 *    where rho g on the gas would drive an unbounded channel flow.
 *  rho_g, rho_l: coexistence densities; <= 0 selects the library's Maxwell construction.
 *  tile_x, tile_y, min_blocks: step-kernel variant: tile shape and the CTAs per SM the register
 *    budget is fitted to (0 = no constraint); all three 0 selects 32x16/5 in FP32 and 32x16/0 in
 *    FP64. Supported (tile/min_blocks):
 *    FP32 32x8/0, 32x8/6, 32x16/0, 32x16/5, 32x16/6, 64x16/0, 32x32/0; FP64 32x8/0, 32x16/0.
 *    tile_x = LBM_TILE_AUTO: start with the default and let lbm_autotune pick the variant at the
 *    first lbm_step (for lbm_batch_create: lbm_batch_autotune at the first lbm_batch_run).
 *  stream: a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream) or NULL. */
typedef struct lbm_params {
    int32_t nx, ny;
    int32_t precision; /* LBM_FP32 or LBM_FP64 */
    int32_t eos;       /* LBM_EOS_PR or LBM_EOS_CS */
    int32_t collision; /* LBM_MRT or LBM_BGK */
    int32_t device;    /* CUDA device ordinal */
    int32_t tile_x, tile_y;
    int32_t min_blocks;
    double Tr, k2, kappa, tau, s_e, s_eps, s_q;
    double gx, gy;
    double rho_g, rho_l;
    void *stream;
    double g_rho_ref;  /* appended: positional initialisers of the older layout stay valid */
} lbm_params;

/* Geometry and initial state (Sec. 3.1, Fig. 1, Fig. 2, Fig. 9, Eq. 16).
 *  Circle: solid nodes are those with (i - cx)^2 + (j - cy)^2 <= R^2 (convex substrate, the
 *    default) or, with concave = 1, those with (i - cx)^2 + (j - cy)^2 > R^2 (a circular cavity:
 *    the concave substrate of Fig. 2b), evaluated exactly in doubled-integer coordinates, so cx,
 *    cy, R must be multiples of 1/2. In both cases the wall surface is taken at radius R + 1/2
 *    (half a link between the last fluid and the first solid node) for the measurement.
 *  Wall chemical potential of a wetting-layer node: mu_circle in the circle's solid (or, with stripes,
 *    alternating mu_circle / mu_stripe_b by arc length R*(phi - pi/2) in units of stripe_arc,
 *    phi = atan2(j - cy, i - cx)); mu_bottom below the domain; mu_top above it.
 *  Boundary scheme for populations whose source node is solid: LBM_BB_HALFWAY returns the
 *    population that left toward the wall (wall half a link out, exactly mass-conserving);
 *    LBM_BB_INTERP places the wall on the analytic surfaces (the circle of radius R + 1/2, the
 *    planes y = -1/2 and y = ny - 1/2) at the link fraction Delta (at least 1/10; 1/2 for a link
 *    that does not cross the circle within its length), interpolates linearly (between the
 *    node and its fluid neighbour behind it for Delta < 1/2, between the node's two opposite
 *    populations for Delta >= 1/2; the half-way value where no fluid neighbour lies behind) and
 *    adds the difference between the population that left and the one that returns to the
 *    node's rest population, so mass stays conserved. The first step after lbm_set_geometry pulls without
 *    interpolation (the initial populations are the rest-state equilibrium w_q rho0). Not
 *    available in batches (lbm_batch_set_geometry returns LBM_ERR_ARG).
 *  Initial density: rho0 (host, (ny, nx), read at fluid nodes) if non-NULL, else the Eq. 16 drop
 *    (drop_x, drop_y, drop_r, width drop_W); populations start at f = f_eq(rho, 0). */
typedef struct lbm_geometry {
    int32_t has_circle;
    int32_t stripes;
    double cx, cy, R;
    double mu_circle, stripe_arc, mu_stripe_b;
    double mu_bottom, mu_top;
    double drop_x, drop_y, drop_r, drop_W;
    const double *rho0;
    int32_t concave;   /* appended: 0 = solid disc (convex), 1 = solid outside the circle */
    int32_t boundary;  /* appended: LBM_BB_HALFWAY (default) or LBM_BB_INTERP */
} lbm_geometry;

/* One side of the contact-angle measurement (Sec. 3.2, Eq. 15, Fig. 1, Fig. 2). Angles in
 * degrees. theta is measured through the liquid between the line through p1 and p2 and the
 * substrate tangent at the contact point; alpha is the tangent's inclination to the horizontal;
 * beta = theta + alpha on the convex circle, theta - alpha on the concave one (Fig. 2), theta on
 * a flat wall. The left (out[0]) and right (out[1]) sides are seen from the liquid standing on
 * the wall: split by the sign of the cross product between the wall normal into the fluid at the
 * liquid centroid and the direction of the point from the circle centre. d1, d2: distances of p1, p2
 * from the substrate. link1, link2: (node index * 4 + slot) of the chosen liquid/gas links, slot
 * 0..3 = link to (i+1, j), (i, j+1), (i+1, j+1), (i-1, j+1). */
typedef struct lbm_angle {
    int32_t status; /* LBM_OK or LBM_ERR_NO_CONTACT */
    double theta_deg, alpha_deg, beta_deg;
    double contact_x, contact_y;
    double p1_x, p1_y, p2_x, p2_y;
    double d1, d2;
    int64_t link1, link2;
} lbm_angle;

typedef struct lbm_info {
    double rho_g, rho_l, p_sat, mu_sat; /* coexistence in use; mu_sat = psi'(rho_sat), k = 1 */
    double T;                           /* absolute temperature Tr * Tc */
    int64_t steps;                      /* time steps taken since lbm_set_geometry */
    int64_t n_fluid;                    /* fluid nodes */
    int32_t tile_x, tile_y;
    int32_t precision;
    int32_t min_blocks;
} lbm_info;

/* Maxwell equal-area coexistence of an EOS at reduced temperature Tr (Sec. 4, after Eq. 16),
 * computed on the host in FP64. out[4] = rho_g, rho_l, p_sat, mu_sat (mu at k = 1).
 * LBM_ERR_ARG above the critical temperature or for an unknown EOS. */
lbm_status lbm_coexistence(int32_t eos, double Tr, double out[4]);

/* Bulk equation of state at density rho (Eq. 10 for Peng-Robinson, or Carnahan-Starling),
 * evaluated on the host in FP64: out[0] = p0(rho), out[1] = psi'(rho), the bulk chemical
 * potential at k = 1 (Eq. 11). The model's pressure and chemical potential are k^2 times these
 * (Eq. 12). Used for Laplace-law surface tensions (Delta p = k^2 (p0(rho_in) - p0(rho_out))).
 * LBM_ERR_ARG for an unknown EOS, Tr outside (0, 1), or rho outside (0, rho_max). */
lbm_status lbm_eos_eval(int32_t eos, double Tr, double rho, double out[2]);

/* Allocate a lattice on p->device (2 x 9 population planes, 2 density planes, flags, wall
 * chemical potential, reduction and measurement scratch). *out receives the context; on failure
 * *out is NULL and nothing is leaked. */
lbm_status lbm_create(const lbm_params *p, lbm_ctx **out);

/* Build the geometry on the device (classification, wetting layers, wall chemical potential,
 * boundary-link masks) and set the initial state; resets the step counter. Copies g->rho0 from
 * the host when given. When every wall field (all but the drop and rho0) equals the current
 * geometry's, the walls already on the device are kept and only the state is set. Synchronous. */
lbm_status lbm_set_geometry(lbm_ctx *ctx, const lbm_geometry *g);

/* Advance nsteps time steps (Eq. 1-4 with Eq. 7, 12-14): one fused kernel per step, replayed
 * from a CUDA graph in chunks when the stream allows capture. Asynchronous; returns LBM_OK once
 * the work is queued (LBM_ERR_STATE before lbm_set_geometry, LBM_ERR_ARG for nsteps < 0). */
lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Measure the left (out[0]) and right (out[1]) contact angles on the current density field with
 * the on-device scheme of Sec. 3.2: liquid/gas links (a node is liquid when rho > rho_m, the
 * mean of rho_g and rho_l), Eq. 15 points, per side the points nearest to 1 and 2 lattice units
 * from the substrate within 0.5..2.5 (ties: smaller |d - target|, then smaller link id), the line
 * through them cut with the substrate (the circle at R + 1/2 if present, else the bottom wall
 * y = -1/2). Sides split by the liquid centroid. Synchronous. Returns LBM_ERR_NO_CONTACT if
 * either side failed (its status says so; the other side is still filled). */
lbm_status lbm_measure_contact_angle(lbm_ctx *ctx, lbm_angle out[2]);

/* Copy fields of the current state to caller buffers of n = nx * ny doubles each ((ny, nx),
 * zero at solid nodes). which: bit 0 density, bit 1 velocity v = u + F/(2 rho) (Sec. 2.2, below
 * Eq. 13; computes the force of the current state), bit 2 destinations are device pointers.
 * Any of rho, ux, uy may be NULL when its bit is clear. Synchronous. */
#define LBM_FIELD_RHO 1u
#define LBM_FIELD_VEL 2u
#define LBM_FIELD_DEVICE_DST 4u
lbm_status lbm_read_fields(lbm_ctx *ctx, uint32_t which, double *rho, double *ux, double *uy,
                           size_t n);

/* FP64 sums over fluid nodes (deterministic two-pass reduction): out[0] total mass, out[1]
 * number of liquid nodes (rho > rho_m), out[2], out[3] their centroid x, y. Returns
 * LBM_ERR_UNSTABLE if a density is non-finite or non-positive. Synchronous. */
lbm_status lbm_mass(lbm_ctx *ctx, double out[4]);

/* Geometry as built on the device: flags ((ny+4) x nx node classes), mu_w ((ny+4) x nx wall
 * chemical potential, 0 off the wetting layers) and the boundary links (fluid node n, direction
 * q with x + e_q solid) as codes n * 9 + q in ascending order. Any output may be NULL; links
 * holds at most cap codes, *n_links receives the total. D2Q9 directions q = 0..8: rest, (1,0),
 * (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1). Synchronous. */
lbm_status lbm_read_geometry(lbm_ctx *ctx, uint8_t *flags, double *mu_w, int64_t *links,
                             int64_t cap, int64_t *n_links);

/* Liquid/gas links of the current density field with their Eq. 15 points and substrate
 * distances, in ascending link id (node * 4 + slot): ids[k], pxyd[3k..3k+2] = px, py, d. Writes
 * at most cap entries; *n receives the total. Synchronous. */
lbm_status lbm_read_candidates(lbm_ctx *ctx, int64_t *ids, double *pxyd, int64_t cap,
                               int64_t *n);

lbm_status lbm_get_info(lbm_ctx *ctx, lbm_info *out);

/* One timed step-kernel variant: tile shape, register budget (CTAs per SM, 0 = none), the mean
 * device time of one step over the trial in microseconds, and (batched kernel only) the grid
 * mode: 0 = one CTA per tile, 1 = persistent CTAs looping over the tile table. */
typedef struct lbm_tune_entry {
    int32_t tile_x, tile_y, min_blocks;
    double us_per_step;
    int32_t persistent;
} lbm_tune_entry;

/* Step-kernel autotuner (no counterpart in the paper; it only picks among launch shapes that
 * compute the same step). Times every compiled variant of the lattice's precision over
 * trial_steps launches (after 2 untimed ones) with CUDA events on the lattice's stream, on the
 * lattice's own geometry and state, and keeps the fastest; later lbm_step calls (and their
 * captured graphs) use it. The trial launches read the current populations and write the other
 * ping-pong buffer without advancing, so the simulation state and step count are unchanged.
 * entries (may be NULL) receives up to max_entries timings in variant order, *n_out (may be NULL)
 * the number of variants timed. LBM_ERR_STATE before lbm_set_geometry, LBM_ERR_ARG for
 * trial_steps < 1. Synchronous. */
lbm_status lbm_autotune(lbm_ctx *ctx, int32_t trial_steps, lbm_tune_entry *entries,
                        int32_t max_entries, int32_t *n_out);

/* Allocation-free variant of lbm_mass for a caller-owned FP32 density field.
 * For callers that must not allocate device memory at this point: a framework that owns every
 * device byte through its own pool, code that cannot afford the implicit device synchronisation
 * of cudaMalloc/cudaFree, or a process that has budgeted the whole GPU. The paper has no
 * counterpart; this is a deployment convenience, not part of the method.
 *  rho:   device, rho[j * pitch + i] for 0 <= j < ny, 0 <= i < nx (fluid-domain rows).
 *  flags: device, same layout; a node is summed when its flag is 0 (LBM_FLUID).
 *  out:   device, 5 doubles: total mass, number of liquid nodes (rho > rho_m), their centroid
 *         x and y, and the number of non-finite or non-positive densities.
 *  stream: cudaStream_t or NULL; work is queued asynchronously on the calling thread's current
 *         device, which must hold the three arrays.
 * It calls no cudaMalloc, cudaFree or allocating library routine. Its scratch is a fixed device
 * array inside the library image of LBM_NOALLOC_MAX_ROWS x 8 doubles (256 KiB), which every GPU
 * that loads the library holds until the process exits; ny > LBM_NOALLOC_MAX_ROWS is rejected
 * with LBM_ERR_ARG. The first call on a device looks up the array's device address (a one-time
 * set-up per device); make that first call before any stream capture. The address is kept for
 * the life of the process: after a cudaDeviceReset of that device it is stale, so do not call
 * this entry point on a device that was reset after its first call. Calls overwrite every
 * scratch entry they read, so no clearing is needed, but calls that overlap on the GPU share the
 * array and race. Errors: LBM_ERR_ARG (NULL pointer, nx or ny <= 0, pitch < nx, ny too large),
 * LBM_ERR_CUDA (no current device, set-up or launch failure); the message is available from
 * lbm_last_error(NULL). */
#define LBM_NOALLOC_MAX_ROWS 4096
lbm_status lbm_mass_noalloc(const float *rho, const uint8_t *flags, int32_t nx, int32_t ny,
                            int32_t pitch, double rho_m, double *out, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Batched sweeps: independent lattices of uneven size (drop radius, cylinder curvature and
 * wettability sweeps, Sec. 4.1-4.2) advanced together by one kernel launch per step over a
 * device table of (instance, tile) pairs (one CTA per tile, or persistent CTAs looping over the
 * table), replayed from a CUDA graph, with per-instance convergence.
 * ------------------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch; /* opaque; owns n lattices, their stream and tile tables */

/* Create n lattices of sizes nx[i] x ny[i] sharing the model parameters (model->nx, ny, tile_y,
 * min_blocks and stream are ignored; precision must be LBM_FP32; model->tile_x = LBM_TILE_AUTO
 * autotunes the batch kernel at the first lbm_batch_run, any other value starts with the
 * default 32x16 tiles, one CTA per tile). Every instance is an lbm_ctx on the batch's private
 * stream. On failure
 * *out is NULL and nothing is leaked. */
lbm_status lbm_batch_create(const lbm_params *model, int32_t n, const int32_t *nx,
                            const int32_t *ny, lbm_batch **out);

/* Geometry and initial state of instance i (as lbm_set_geometry); marks it runnable. */
lbm_status lbm_batch_set_geometry(lbm_batch *b, int32_t i, const lbm_geometry *g);

/* Advance every runnable instance, check_every steps per graph replay (even, >= 2), until it
 * converges or max_steps have been taken. Converged at a check: the residual
 * sum|rho(t) - rho(t - check_every)| / sum rho over fluid nodes (FP64, deterministic) is below
 * tol, or (angle_tol > 0) both contact angles (Sec. 3.2 measurement) moved by at most angle_tol
 * degrees since the previous check at two consecutive checks. Converged or unstable instances
 * leave the tile table at the check. Outputs (each n entries, may be NULL): steps taken,
 * converged flag, last residual (-1 if never checked). Synchronous. */
lbm_status lbm_batch_run(lbm_batch *b, int64_t max_steps, int32_t check_every, double tol,
                         double angle_tol, int64_t *steps_out, int32_t *converged_out,
                         double *residual_out);

/* Autotuner of the batched kernel: times each compiled tile variant (FP32 32x8, 32x16, 64x16,
 * 32x32, each with its register budget) in both grid modes (one CTA per tile, then persistent;
 * entries in that order, 2 per variant) over trial_steps launches on
 * the tile table of the instances that have geometry (those sharing the parity of the first), and
 * keeps the fastest for later lbm_batch_run calls. As in lbm_autotune the trial launches do not
 * advance any instance. entries / n_out as in lbm_autotune. LBM_ERR_STATE if no instance has
 * geometry. Synchronous. */
lbm_status lbm_batch_autotune(lbm_batch *b, int32_t trial_steps, lbm_tune_entry *entries,
                              int32_t max_entries, int32_t *n_out);

/* Contact angles of every instance (out[2 i], out[2 i + 1] = left, right), as
 * lbm_measure_contact_angle. Returns LBM_ERR_NO_CONTACT if any side of any instance failed. */
lbm_status lbm_batch_measure(lbm_batch *b, lbm_angle *out);

/* Borrow the context of instance i (read fields, mass, geometry); owned by the batch. */
lbm_status lbm_batch_instance(lbm_batch *b, int32_t i, lbm_ctx **ctx);

const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* ---------------------------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper; it replaces part of the relaxation from the
 * Eq. 16 flat-cap start): a U-Net on an H x W lattice mapping (solid mask, wall-wetting map,
 * drop-volume plane) to phi = (rho - rho_g) / (rho_l - rho_g), trained on solver-equilibrated
 * fields. BF16 activations and weight copies, FP32 master weights, FP32 accumulation on tensor
 * cores. Architecture: encoder levels with base, 2, 4, 8 x base channels (two 3x3 conv + leaky
 * ReLU (slope 0.1) each, 2x2 average pooling between), decoder levels of a 3x3 conv on the 2x
 * nearest-upsampled
 * coarser output and two 3x3 convs on [that | skip], 1x1 sigmoid head. Parameters: one FP32
 * vector, per convolution in forward order weight [c_out][ky][kx][c_in] then bias [c_out], then
 * head weight [base] and bias [1].
 * ------------------------------------------------------------------------------------------- */
typedef struct lbm_surrogate lbm_surrogate;

/* H, W multiples of 8; base in {8, 16, 32}; buffers for up to max_batch samples. Weights start
 * at zero: call lbm_surrogate_set_weights. */
lbm_status lbm_surrogate_create(int32_t H, int32_t W, int32_t base, int32_t max_batch,
                                int32_t device, lbm_surrogate **out);
int64_t lbm_surrogate_num_params(const lbm_surrogate *s);
/* Copy FP32 master weights from the host (resets the Adam moments and step count). */
lbm_status lbm_surrogate_set_weights(lbm_surrogate *s, const float *host, int64_t n);
/* Copy the FP32 master weights (grads = 0) or the last step's gradients (grads = 1) to host. */
lbm_status lbm_surrogate_get_weights(lbm_surrogate *s, float *host, int64_t n, int32_t grads);
/* x: device BF16 inputs (B, H, W, 8) NHWC; phi_out: device FP32 (B, H, W). Synchronous. */
lbm_status lbm_surrogate_forward(lbm_surrogate *s, const void *x, int32_t B, float *phi_out);
/* Forward, loss = sum mask (phi - target)^2 / sum mask, backward into the gradient vector and,
 * for lr > 0, one Adam step (beta 0.9 / 0.999, eps 1e-8). target: device FP32 (B, H, W); mask:
 * device uint8 (B, H, W). *loss receives the loss. Synchronous. */
lbm_status lbm_surrogate_train_step(lbm_surrogate *s, const void *x, const float *target,
                                    const uint8_t *mask, int32_t B, float lr, double *loss);
/* Copy the last training step's phi (B, H, W) to the host. */
lbm_status lbm_surrogate_phi(lbm_surrogate *s, float *host_phi, int32_t B);
const char *lbm_surrogate_last_error(const lbm_surrogate *s);
void lbm_surrogate_destroy(lbm_surrogate *s);

/* The surrogate's tensor-core GEMM on its own: C = A B, BF16 device operands, FP32 device
 * output C[m * ldc + n]. a_kmajor: A stored A[m * lda + k] (else A[k * lda + m]); b_kmajor: B
 * stored B[n * ldb + k] (else B[k * ldb + n]). K-major operands need K and ld multiples of 8,
 * MN-major ones M (N) and ld multiples of 8. Asynchronous on stream. */
lbm_status lbm_sg_gemm(const void *A, const void *B, int32_t M, int32_t N, int32_t K,
                       int32_t a_kmajor, int32_t b_kmajor, int32_t lda, int32_t ldb, float *C,
                       int32_t ldc, void *stream);

/* Failure-path test hook (no counterpart in the paper): latch, from the host, the flag that a
 * tensor-core GEMM sets when one of its bounded device waits runs out. The next
 * lbm_surrogate_forward, lbm_surrogate_train_step or lbm_sg_gemm call then returns
 * LBM_ERR_TIMEOUT (its message says a wait timed out) and clears the flag, exactly as after a
 * real expiry. Nothing is launched and no GPU state changes. LBM_ERR_CUDA if the mapped host
 * flag could not be allocated. */
lbm_status lbm_sg_inject_timeout(void);

/* Checkpoint and restart (no counterpart in the paper): the dynamic state of a lattice, i.e. the
 * current populations and densities exactly as stored on the device (padded planes, the
 * context's precision) and the step counter, behind a small header (magic, version, nx, ny,
 * element size, steps, plane size). The geometry is not part of it: restore by creating a
 * context with the same parameters, calling lbm_set_geometry with the same geometry, then
 * lbm_load_state; stepping on is then bit-identical to the uninterrupted run.
 * lbm_state_bytes: the checkpoint's size for this context (0 for NULL).
 * lbm_save_state: writes it into a caller-owned host buffer of exactly that size; synchronous.
 *   LBM_ERR_STATE before lbm_set_geometry, LBM_ERR_ARG for a NULL buffer or another size.
 * lbm_load_state: reads it back; LBM_ERR_STATE before lbm_set_geometry, LBM_ERR_ARG for a
 *   buffer that is not a checkpoint of this version or belongs to another nx, ny or precision
 *   (the context is then unchanged). Synchronous. */
size_t lbm_state_bytes(const lbm_ctx *ctx);
lbm_status lbm_save_state(lbm_ctx *ctx, void *host, size_t bytes);
lbm_status lbm_load_state(lbm_ctx *ctx, const void *host, size_t bytes);

/* Wait for the context's stream. */
lbm_status lbm_synchronize(lbm_ctx *ctx);

/* Release all device memory, graphs and the private stream. NULL is ignored. */
void lbm_destroy(lbm_ctx *ctx);

/* Message of the last failed call on ctx ("" if none); for ctx == NULL, of the last failed
 * lbm_create or lbm_coexistence in this process. */
const char *lbm_last_error(const lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
