/*
 * spfm.h -- C ABI of the GB300 library for the explicit time step of the
 * sharp phase-field method (SPFM) and of the conventional finite-difference
 * (CF) phase-field model, after Fleck, Schleifer, Zimbrod, "Frictionless
 * motion of diffuse interfaces by sharp phase-field modeling"
 * (arXiv:1910.05180).
 *
 * Model (Sec. 2.1).  On a cubic grid of spacing dx the field phi_p evolves by
 * the Allen-Cahn relaxation of Eq. 2, 3 lambda Gamma dphi/dt = -2 M dF/dphi,
 * of the discrete free energy of Eq. 1, summed over the 3, 9 or 13 grid
 * directions of Tab. 1 (6, 18 or 26 neighbours).  Per cell and step:
 *
 *   R_p = sum_k c_k (phi_{p+r_k} + phi_{p-r_k} - 2 phi_p)
 *         - q s sum_k 4 c_k A_k / (1 - A_k s^2)        (TI, Eqs. 5-6)
 *           or  - (D/lambda^2)(16/3) sum_k w_k q s    (CF, Tab. 2)
 *         - (4 M dF / (lambda Gamma)) q                 (h3 driving term)
 *   phi_p <- phi_p + dt R_p                             (explicit Euler)
 *
 * with q = phi(1-phi), s = 1-2phi, D = 2M/(3 C_Gamma), w_k = gamma_j nu_j,
 * nu_j = 3/m_j, c_k = D w_k / |r_k|^2 and A_k = tanh^2(2 r_k.n / lambda).
 *
 * Conventions shared by every call:
 *  - Every call returns an spfm_status; nothing is thrown across the ABI.
 *    On failure spfm_last_error() holds a one-line message.
 *  - Device memory is owned by the caller (e.g. allocated through PyTorch).
 *    The library owns only its opaque host objects and never frees caller
 *    buffers.  Pointers named `field`, `scratch` and `dst`/`src` with
 *    *_on_host == 0 are device pointers of the current CUDA device.
 *  - Field layout in HBM: x fastest, with a one-cell ghost layer on every
 *    face.  Interior cell (i, j, k), 0 <= i < nx etc., is
 *      field[((k + 1) * (ny + 2) + (j + 1)) * pitch_x + x_off + i],
 *    ghost cells sit at i = -1, nx, j = -1, ny, k = -1, nz.  x_off is 32 bytes
 *    worth of elements (4 FP64, 8 FP32, 16 BF16), pitch_x a 32-byte multiple
 *    >= x_off + nx + 1, so every interior row starts on a 32-byte boundary
 *    relative to the base pointer.  The base pointer must be 16-byte aligned
 *    (256-byte alignment, as cudaMalloc gives, keeps whole 32-byte sectors).
 *    The elements left of x_off - 1 and right of x_off + nx are padding; the
 *    library may write them.  The library keeps the ghosts
 *    consistent with the boundary conditions; use spfm_get_field /
 *    spfm_set_field to exchange dense interior arrays.
 *  - Launches are asynchronous on the grid's stream.  spfm_interface_stats,
 *    spfm_get_field (to host) and spfm_batch_stats synchronise that stream.
 */
#ifndef SPFM_H
#define SPFM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int spfm_status;
#define SPFM_OK 0
#define SPFM_EINVAL (-1)     /* bad argument: sizes, lambda <= 0, |n| != 1, stencil */
#define SPFM_EUNSTABLE (-2)  /* dt above the explicit-Euler stability bound */
#define SPFM_EPHASE (-3)     /* CF driving force beyond phase stability, Sec. 3.1 */
#define SPFM_ECUDA (-4)      /* a CUDA runtime call failed */
#define SPFM_ENONFINITE (-5) /* the field holds NaN/Inf (reported by the stats) */
#define SPFM_ETIMEOUT (-6)   /* a bounded device-side wait gave up */
#define SPFM_ENOMEM (-7)     /* caller-provided scratch is too small */

enum { SPFM_F64 = 0, SPFM_F32 = 1, SPFM_BF16 = 2 };              /* storage type */
enum { SPFM_PERIODIC = 0, SPFM_NOFLUX = 1, SPFM_CONTACT = 2 };   /* boundary kinds */
/* schemes: TI with one global direction, TI_n (local normal), and the CF
 * (conventional finite-difference) models of Tab. 2 with the interpolation
 * functions h3 = phi^2 (3 - 2 phi), h5 = phi^3 (10 - 15 phi + 6 phi^2) and
 * h_Abel = phi^2 / (phi^2 + (1 - phi)^2) */
enum { SPFM_TI_GLOBAL = 0, SPFM_TI_LOCAL = 1, SPFM_FD = 2, SPFM_FD_H5 = 3, SPFM_FD_HABEL = 4 };
enum { SPFM_STATS_ENERGY = 1 };                                  /* stats flags */
enum { SPFM_ROUND_NEAREST = 0, SPFM_ROUND_STOCHASTIC = 1 };      /* update rounding */

typedef struct spfm_grid spfm_grid;
typedef struct spfm_batch spfm_batch;

typedef struct {
    int nx, ny, nz;          /* interior cells, each >= 1 */
    int dtype;               /* SPFM_F64 | SPFM_F32 | SPFM_BF16 (BF16 = storage only) */
    int bc[6];               /* per face x-, x+, y-, y+, z-, z+; PERIODIC must be paired */
    double n[3];             /* unit interface normal: the CONTACT boundary (Eq. 7), the
                                planar position estimator and, unless u is given, the
                                TI_<hkl> coupling direction */
    double gamma[3];         /* shell ponderations gamma_1..3; all 0 selects defaults:
                                (1,0,0), (1/3,2/3,0), (1/2,1/3,1/6) for 6/18/26 */
    double C_gamma;          /* interface-energy calibration; 0 selects 2/3 */
    double center[3];        /* centre of the radial position estimator */
    void *field[2];          /* caller-owned device buffers (ping-pong), field_bytes each */
    void *scratch;           /* caller-owned device scratch, scratch_bytes (spfm_layout) */
    size_t scratch_bytes;
    void *stream;            /* cudaStream_t; NULL = legacy default stream */
    double u[3];             /* TI_<hkl> coupling direction of Eq. 5, a_k = tanh(2 r_k.u /
                                lambda), when it differs from n (Tab. 2: u || <hkl>);
                                all 0 selects u = n; else |u| = 1 */
} spfm_grid_desc;

typedef struct {
    double volume;      /* sum phi dx^3 */
    double S_w;         /* sum q over the band 1e-6 < phi < 1-1e-6 */
    double S_c;         /* sum q (p.n - (lambda/2) artanh(1-2phi)) over the band */
    double S_r;         /* sum q (|p-center| + (lambda/2) artanh(1-2phi)) over the band */
    double phi_min, phi_max;
    double nonfinite;   /* number of NaN/Inf cells */
    double position;    /* S_c / S_w: planar interface position along n (Sec. 2.3) */
    double radius;      /* S_r / S_w: radius of a grain with phi = 0 inside */
    double energy;      /* interface energy F_int of Eq. 1 at dF = 0 (SPFM_STATS_ENERGY) */
    double steps;       /* steps taken since the last init/set_field */
    double time;        /* simulated time since the last init/set_field */
} spfm_stats;

/* Per-grid step parameters of a batch (same meaning as in spfm_step). */
typedef struct {
    double M, Gamma, lambda, dx, dt, dF;
    int stencil, scheme;
} spfm_step_args;

/* Layout of a grid: pitch_x and x_off (elements), bytes of ONE field buffer
 * and bytes of scratch the caller must provide.  Any output pointer may be NULL.
 * The scratch holds the stats reduction and a device error word that the step
 * kernels set when a bounded wait gives up (reported by spfm_interface_stats
 * as SPFM_ETIMEOUT). */
spfm_status spfm_layout(const spfm_grid_desc *desc, size_t *pitch_x, size_t *x_off,
                        size_t *field_bytes, size_t *scratch_bytes);

/* Validate desc and create the host handle.  The handle borrows the buffers. */
spfm_status spfm_create_grid(const spfm_grid_desc *desc, spfm_grid **out);
spfm_status spfm_destroy_grid(spfm_grid *g);
spfm_status spfm_set_stream(spfm_grid *g, void *stream);

/* Rounding of the explicit update phi + dt R (Eq. 2) to the storage type.
 * SPFM_ROUND_NEAREST (the default) rounds to nearest.  SPFM_ROUND_STOCHASTIC
 * rounds up or down with probabilities proportional to the distances (the
 * expected stored value is the exact update; an exactly representable update
 * is stored as is): with FP32 or BF16 storage, a slow interface moves by less
 * than half a unit in the last place of phi near phi = 1 each step, and
 * round-to-nearest drops those increments, which biases its velocity (about
 * 2e-4 relative at dF = 3e-4 and 3e-3 at dF = 1e-4 in FP32, lambda = 2..6,
 * dt = 0.05).  The random bits are a hash of the padded cell index and a key
 * of (seed, the grid's step count), so a run is reproducible and a grid
 * draws the same bits alone and in a batch.  FP64 grids: SPFM_EINVAL (their
 * increments are not lost).  Takes effect at the next step; all grids of a
 * batch must share the mode.  Costs about 11 instructions per cell update. */
spfm_status spfm_set_rounding(spfm_grid *g, int mode, unsigned long long seed);

/* Planes of the z-march each CTA of a step launch takes (a tuning knob; the
 * paper has no counterpart).  0 (the default) chooses per launch from the
 * kernel's occupancy and the grid's shape; a value above nz acts as nz.  The
 * field is bit for bit the same for every choice.  SPFM_EINVAL for
 * zchunk < 0.  Takes effect at the next step (spfm_step and
 * spfm_step_conserving; a batch uses its own depth). */
spfm_status spfm_set_zchunk(spfm_grid *g, int zchunk);

/* Planes per CTA of the grid's last step launch (0 before the first step;
 * -1 for a NULL grid). */
int spfm_last_zchunk(const spfm_grid *g);

/* Test hook (the paper has no counterpart): the chunk length the automatic
 * choice gives a launch of `tiles` xy tiles over nz planes, for a kernel of
 * per_sm resident CTAs per SM on sms SMs, with `target` CTAs for grids of many
 * rounds.  Host only, no device call.  -1 for an argument below 1. */
int spfm_debug_pick_zchunk(int tiles, int nz, int per_sm, int sms, int target);

/* Test hook of the failure reporting (the paper has no counterpart): the next
 * spfm_step launch skips the copy of one plane in its first CTA, whose bounded
 * waits (about 2 s each) then give up; the kernel returns without writing that
 * tile, and the next spfm_interface_stats reports SPFM_ETIMEOUT.  The field is
 * invalid afterwards: re-initialise it (init or set_field clears the error).
 * One-shot; no effect on batches. */
spfm_status spfm_debug_skip_copy(spfm_grid *g);

/* Ideal planar profile of Eq. 3, phi = (1 - tanh(2 (p.n - c)/lambda))/2 at
 * p = dx (i, j, k), with the desc's n.  Computed in FP64, stored in dtype. */
spfm_status spfm_init_planar(spfm_grid *g, double c, double lambda, double dx);
/* Radial ideal profile of a grain with phi = 0 inside:
 * phi = (1 - tanh(2 (R - |p - ctr|)/lambda))/2.  Also sets desc center = ctr. */
spfm_status spfm_init_sphere(spfm_grid *g, const double ctr[3], double R, double lambda,
                             double dx);

/* Cubic particle with phi = 0 inside, half side `half` around ctr: phi = 1 -
 * prod_a (1 - tanh(2 (|p_a - ctr_a| - half)/lambda))/2, the start of the
 * shape relaxation of Sec. 3.3 (the paper gives no cube profile; this product
 * is the 1D ideal profile across each face away from edges and corners).  Also
 * sets desc center = ctr. */
spfm_status spfm_init_cube(spfm_grid *g, const double ctr[3], double half, double lambda, double dx);

/* n_steps explicit steps (Eq. 2 with Eq. 1; TI per Eqs. 5-6, TI_n with the
 * local normal, or CF).  stencil in {6, 18, 26}.  Validates first:
 * SPFM_EINVAL, SPFM_EUNSTABLE (dt above 2 / bound of the Jacobian's spectral
 * radius), SPFM_EPHASE (CF and |dF dx/Gamma| >= 8/(3 C_Gamma lambda/dx),
 * Sec. 3.1).  Asynchronous on the grid's stream: one kernel launch per step
 * when the step kernel writes the ghost layer itself, else two (see
 * spfm_kernels_per_step). */
spfm_status spfm_step(spfm_grid *g, int n_steps, double M, double Gamma, double lambda,
                      double dx, double dt, double dF, int stencil, int scheme);

/* n_steps constant-volume steps (Sec. 3.3: a homogeneous, time-dependent
 * driving force keeps the particle volume fixed).  Each step is spfm_step at
 * dF = 0, then the one homogeneous dF for which the step leaves sum_p phi_p
 * unchanged: with phi* the result at dF = 0, every cell loses alpha q(phi_p),
 * alpha = sum_p (phi*_p - phi_p) / sum_p q(phi_p) (FP64 sums in a fixed order),
 * which is dF = alpha lambda Gamma / (4 M dt) in the driving term of Eq. 2.
 * Validation as spfm_step at dF = 0 (the phase-stability check of Sec. 3.1
 * cannot see a dF decided during the run); schemes with h3 only (SPFM_EINVAL
 * for SPFM_FD_H5 and SPFM_FD_HABEL).  Uses the grid's scratch.  The step
 * rounds as spfm_set_rounding sets; the correction rounds to nearest.
 * dF_last (host pointer or NULL) receives the last step's dF; a non-NULL
 * dF_last synchronises the stream. */
spfm_status spfm_step_conserving(spfm_grid *g, int n_steps, double M, double Gamma, double lambda,
                                 double dx, double dt, int stencil, int scheme, double *dF_last);

/* FP64 interface diagnostics of the current field (Sec. 2.3 inversion of the
 * ideal profile); flags may include SPFM_STATS_ENERGY.  Uses the model of the
 * last spfm_step (or lambda/dx of the last init).  Synchronises the stream.
 * Returns SPFM_ETIMEOUT if a step kernel's bounded wait gave up since the last
 * init/set_field, else SPFM_ENONFINITE (with *out filled) if the field holds
 * NaN/Inf. */
spfm_status spfm_interface_stats(spfm_grid *g, int flags, spfm_stats *out);

/* The diagnostics above without any device allocation or caller scratch, for
 * callers that cannot allocate device memory (their device memory belongs to
 * another framework's pool, or they only borrow the field they measure).  The
 * paper has no counterpart: this is a deployment variant of the stats pass.
 * desc gives sizes, dtype, n and center (bc, buffers, scratch are not used);
 * field is a device buffer in the ghosted layout of spfm_layout; lambda and dx
 * define the profile inversion.  out->energy is NaN, steps and time are 0.
 * The reduction partials sit in a fixed array inside the library, sized for
 * nz <= 1024 (96 KiB, held by every GPU that loads the library until exit):
 * larger nz returns SPFM_EINVAL, as do the extent limits of spfm_create_grid
 * and |n| != 1.  The first call on a device looks up the array's address for
 * the current device; make it before any stream capture.  desc->stream must
 * belong to the current device (else SPFM_EINVAL).  Calls share the array, so
 * calls that overlap on the GPU race.  Synchronises desc->stream. */
spfm_status spfm_interface_stats_static(const spfm_grid_desc *desc, const void *field, double lambda,
                                        double dx, spfm_stats *out);

/* Residual anisotropy of a particle (Sec. 3.3): the phi = 1/2 contour points on
 * the grid edges (nonlinear interpolation of Sec. 2.3, Eqs. 8-10), their
 * distances R_i from the particle's barycentre (cells weighted by their
 * particle-phase fraction; the particle is phase inside_phase, 0 or 1), and
 * out[0] eps_eff = (R_max - R_min)/(2 R_mean), out[1] R_mean, out[2] R_min,
 * out[3] R_max, out[4] number of contour points, out[5..7] barycentre.  FP64,
 * uses the grid's scratch, synchronises the stream. */
spfm_status spfm_sphericity(spfm_grid *g, int inside_phase, double *out8);

/* Moving frame of the 1D friction study (Sec. 3.1: the system is moved back by
 * one grid point whenever the favoured phase fills half of it): the current
 * field shifted along x, phi_i <- phi_{i+cells}, the cells that open up taking
 * the value of the row's end cell; written to the other buffer, which becomes
 * current.  Ghosts are rebuilt when a model is known.  Asynchronous. */
spfm_status spfm_shift_x(spfm_grid *g, int cells);
/* The largest dt that spfm_step accepts for these parameters: 2 over the bound
 * of the Euler Jacobian's spectral radius (the same validation, SPFM_EPHASE
 * included).  No launch. */
spfm_status spfm_max_dt(spfm_grid *g, double M, double Gamma, double lambda, double dx, double dF,
                        int stencil, int scheme, double *dt_max);

/* Copy the interior of the current field to/from a dense (nz, ny, nx) array of
 * the storage type; *_on_host selects a host or a device pointer.  set_field
 * resets the step count and rebuilds the ghost layer (at the next step when no
 * lambda is known yet). */
spfm_status spfm_get_field(spfm_grid *g, void *dst, int dst_on_host);
spfm_status spfm_set_field(spfm_grid *g, const void *src, int src_on_host);
/* Index (0 or 1) of the buffer holding the current field. */
int spfm_current(const spfm_grid *g);
/* Kernel launches of one spfm_step step on g: 1 when every face is periodic,
 * nx is a whole number (>= 2) of 32-byte sectors and ny >= 2 (the step kernel
 * then writes the periodic ghost images of its new cells itself), else 2 (the
 * step kernel and the ghost-face refresh); -1 for NULL. */
int spfm_kernels_per_step(const spfm_grid *g);

/* Message of the last failure on g (or of this thread when g is NULL). */
const char *spfm_last_error(const spfm_grid *g);

/* ---- batches: many grids of one dtype advanced by one launch per step over
 * a packed tile work-list.  No counterpart in the paper, which advances one
 * grid at a time; each grid's result is the same as with spfm_step. */
spfm_status spfm_batch_scratch_bytes(spfm_grid *const *grids, int n, size_t *bytes);
spfm_status spfm_batch_create(spfm_grid *const *grids, int n, void *scratch,
                              size_t scratch_bytes, void *stream, spfm_batch **out);
/* n_steps steps of every grid with its own args[i]; all grids must share stencil and
 * scheme.  Replays a captured CUDA graph of the per-step launches. */
spfm_status spfm_batch_step(spfm_batch *b, int n_steps, const spfm_step_args *args);
/* Tile policies of a batch's work-list: the xy tile shape of each grid's items.
 * FP32 batches have two shapes, 64 x 16 cells (the single-grid tile) and 32 x 32
 * (for grids narrower than 64 cells or padded by the wide tile); FP64 and BF16
 * batches have the first only and accept every policy.
 *   SPFM_TILES_WIDE    every grid on 64 x 16 tiles
 *   SPFM_TILES_SQUARE  every grid on 32 x 32 tiles
 *   SPFM_TILES_FIT     each grid on the shape that pads its nx x ny extent least,
 *                      ties to 64 x 16 (the default; the two shapes then run as
 *                      two persistent launches per step) */
enum { SPFM_TILES_WIDE = 0, SPFM_TILES_SQUARE = 1, SPFM_TILES_FIT = 2 };
/* Autotuner of the batch's work-list: first the tile policy (FP32 batches: the
 * three above, at the current depth), then the z-march depth of its items
 * (planes per item: 8, 12, 16, 24, 32, 48 or 64).  Each candidate is timed with
 * CUDA events over steps_per_trial steps (a multiple of 16, at least 16) after a
 * 16-step warm-up, all of them real steps of every grid with args, exactly as
 * spfm_batch_step would take them: the grids advance by (3 + 7) * (16 +
 * steps_per_trial) steps in all for FP32 (7 * (...) otherwise), and their fields
 * do not depend on the policy or depth chosen.  The fastest policy and depth are
 * kept for later steps (spfm_batch_tiles reports them).  Needs a non-default
 * stream (graphs).  out_depth (may be NULL) receives the depth chosen, out_ms
 * (may be NULL, else 7 doubles) the milliseconds per step of each depth in the
 * order above.  Synchronises the stream.  No counterpart in the paper. */
spfm_status spfm_batch_autotune(spfm_batch *b, const spfm_step_args *args, int steps_per_trial,
                                int *out_depth, double *out_ms);
/* Set the tile policy of the batch's work-list (one of SPFM_TILES_*), keeping
 * its depth; the fields do not depend on it.  Synchronises the stream. */
spfm_status spfm_batch_set_tiles(spfm_batch *b, int policy);
/* The batch's current tile policy and z-march depth (either may be NULL). */
spfm_status spfm_batch_tiles(const spfm_batch *b, int *policy, int *depth);
/* Diagnostics of every grid in one pass; out has n entries.  Synchronises. */
spfm_status spfm_batch_stats(spfm_batch *b, int flags, spfm_stats *out);
spfm_status spfm_batch_destroy(spfm_batch *b);

#ifdef __cplusplus
}
#endif
#endif
