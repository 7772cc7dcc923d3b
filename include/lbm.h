/*
 * lbm.h -- C ABI of liblbm, a GB300 (sm_103a) implementation of the
 * single-component pseudo-potential D2Q9 lattice Boltzmann model analysed by
 * Hu, Li & Uddin, "Force Method in a Pseudo-potential Lattice Boltzmann
 * Model" (arXiv:1412.5170).
 *
 * One time step (Sec. 2, Eq. 1; Sec. 4.4.2, Eq. 36) on a periodic nx x ny
 * lattice, fused into one kernel:
 *   rho, u        Eq. 3 moments of the pulled populations
 *   psi           Eq. 7 with G = -1 from the K-scaled Carnahan-Starling
 *                 EOS, Eqs. 29-30 (a = 1, b = 4, R = 1): psi^2 = 2(rho/3 - p)
 *   F             Kupershtokh's hybrid force, Eq. 6, weights w(1) = 1/3,
 *                 w(2) = 1/12 (Eq. 4), U = G psi^2/2
 *   v             u + F/(2 rho) (Sec. 3.2)
 *   collision     BGK (Eq. 1) with Guo (Eq. 23), exact-difference (Eq. 22)
 *                 or Shan-Chen velocity-shift (Eqs. 20-21) forcing, or MRT
 *                 with Guo's source in moment space (Eqs. 34-35); and Li et
 *                 al.'s model for comparison (Sec. 4.3, Eqs. 31-32: BGK,
 *                 Eq. 4 force, Guo's source with a shifted velocity)
 *   streaming     pull, periodic in x and y (Eq. 1 / Eq. 36)
 *
 * Conventions shared by every entry point:
 *   - Lattice fields are row-major [ny][nx] (x fastest); populations are
 *     [9][ny][nx] with the velocity order e0 = (0,0), e1..e4 = (1,0), (0,1),
 *     (-1,0), (0,-1), e5..e8 = (1,1), (-1,1), (-1,-1), (1,-1).
 *   - A is the weight of Eq. 6 exactly as printed there (eps = -2A,
 *     Table 1).  T_over_Tc is the reduced temperature with Tc taken from the
 *     constants of Eq. 29.
 *   - Every function returns an int status (LBM_OK = 0 or an LBM_E_* code)
 *     and never throws; lbm_strerror() names a status.  After an error the
 *     context stays valid unless the error was LBM_E_CUDA.
 *   - Pointers named *_host are host memory owned by the caller; pointers
 *     named *_dev are device memory owned by the caller.  Memory the library
 *     allocates it also frees (lbm_destroy / lbm_batch_destroy).
 *   - Work is queued on the stream given at creation; calls that return
 *     results in host memory synchronise that stream, others are
 *     asynchronous.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LBM_OK 0
#define LBM_E_INVALID 1        /* bad argument (tau <= 1/2, T/Tc outside (0,1), K <= 0, size ...) */
#define LBM_E_CUDA 2           /* a CUDA call failed; the context should be destroyed */
#define LBM_E_NONFINITE 3      /* a population, density or velocity became NaN/Inf */
#define LBM_E_EOS_DOMAIN 4     /* rho outside (0,1) or rho/3 - p < 0: psi undefined (Eq. 7) */
#define LBM_E_TIMEOUT 5        /* a bounded device-side wait gave up */
#define LBM_E_NOT_CONVERGED 6  /* run-to-steady reached max_steps */
#define LBM_E_IO 7             /* checkpoint file could not be read or written / is corrupt */
#define LBM_E_UNSUPPORTED 8    /* valid request this build does not support */

typedef enum { LBM_BGK = 0, LBM_MRT = 1 } lbm_collision;            /* Eq. 1 / Eq. 34 */
/* Eq. 23 / Eq. 22 / Eq. 21 / Li et al.'s model, Eq. 31 (Sec. 4.3) */
typedef enum { LBM_GUO = 0, LBM_EDM = 1, LBM_SC = 2, LBM_LI = 3 } lbm_forcing;
typedef enum { LBM_FP64 = 0, LBM_FP32_DEV = 1 } lbm_precision;
typedef enum { LBM_SLAB = 0, LBM_DROPLET = 1, LBM_BUBBLE = 2, LBM_DROPLET_ARRAY = 3 } lbm_preset;

/* Model and lattice parameters.
 *   nx, ny        periodic lattice size, each >= 1 (nodes)
 *   T_over_Tc     reduced temperature, 0 < T/Tc < 1 (Eq. 29)
 *   tau           BGK relaxation time / MRT viscous time tau_nu, > 1/2
 *   A             Eq. 6 weight (paper convention), any real
 *   K             Eq. 30 EOS scale, > 0
 *   s_e, s_eps, s_q   MRT rates of the e, eps and q moments (Eq. 35); the
 *                 viscous rate is 1/tau and s_rho = s_j = 1 (they drop out
 *                 under Guo forcing).  Ignored for BGK.
 *   precision     LBM_FP64: populations and arithmetic in double.
 *                 LBM_FP32_DEV: populations stored in float as deviations
 *                 f_a - w_a rho_ref, arithmetic in float; reductions in double.
 *   rho_ref       reference density of LBM_FP32_DEV (use the vapour density);
 *                 ignored for LBM_FP64.
 *   sigma         LBM_LI only (Sec. 4.3, Eqs. 31-32): Guo's source with v
 *                 replaced by v' = v + sigma F / ((tau - 1/2) psi^2) in its
 *                 second-order term, which sets eps = 16 sigma for the Eq. 4
 *                 force; LBM_LI requires BGK and A = 0 (Eq. 6 with A = 0 is
 *                 Eq. 4) and sigma >= 0.  Must be 0 for the other forcings. */
typedef struct {
    int32_t nx, ny;
    int32_t collision;   /* lbm_collision */
    int32_t forcing;     /* lbm_forcing; MRT supports LBM_GUO only */
    int32_t precision;   /* lbm_precision */
    int32_t reserved;    /* must be 0 */
    double T_over_Tc, tau, A, K;
    double s_e, s_eps, s_q;
    double rho_ref;
    double sigma;
} lbm_params;

/* Whole-lattice observables at the current time t (FP64 reductions).
 *   mass        sum of rho over the lattice
 *   max_v       max |v|, v = u + F/(2 rho): the spurious-velocity magnitude Us_max
 *   max_dv      max |v(t) - v(t_snap)| against the snapshot taken by the
 *               previous lbm_stats(..., snapshot = 1) call; -1 if none
 *   rho_min, rho_max   extremes of rho
 *   rho_center  rho at node (nx/2, ny/2); rho_corner: rho at node (0, 0)
 *   rho_row_mid mean of rho over row y = ny/2; rho_row0: over row y = 0
 *   steps       time steps taken since the last initialisation
 *   status      LBM_OK, or the first error code seen since the last check */
typedef struct {
    double mass, max_v, max_dv, rho_min, rho_max;
    double rho_center, rho_corner, rho_row_mid, rho_row0;
    int64_t steps;
    int32_t status;
    int32_t reserved;
} lbm_stats_t;

typedef struct lbm_ctx lbm_ctx;

/* ---- library ---- */
const char *lbm_strerror(int status);
int lbm_version(void);   /* (major << 16) | minor */

/* Critical temperature implied by Eq. 29's constants with a = 1, b = 4, R = 1. */
double lbm_tc(void);

/* Maxwell equal-area coexistence densities of the Eq. 29/30 EOS at T/Tc
 * (Sec. 3.1, Eq. 19); K-independent (Sec. 4.1).  Host FP64.  Writes the
 * vapour and liquid densities; LBM_E_INVALID if T/Tc is outside (0, 1). */
int lbm_maxwell(double T_over_Tc, double *rho_v, double *rho_l);

/* Mechanical-stability coexistence densities (Sec. 3.1, Eq. 18) of the
 * Eq. 29/30 EOS scaled by K, with psi^2 = 2 (rho/3 - p0) (Eq. 7, G = -1) and
 * exponent eps (eps = -2A for Eq. 6's force, 16 sigma for Li et al.'s model,
 * Eq. 32): p0(rho_v) = p0(rho_l) = p_c and the integral of (p_c - p0)
 * psi'/psi^(1+eps) from rho_v to rho_l vanishes.  Host FP64 (bisection on p_c,
 * Gauss-Legendre quadrature in log rho).  LBM_E_INVALID if T/Tc is outside
 * (0, 1), K <= 0, or no root is bracketed. */
int lbm_mechanical(double T_over_Tc, double K, double eps, double *rho_v, double *rho_l);

/* Fused multiply-add throughput of the current GPU in TFLOP/s (2 flops per
 * FMA), FP64 (precision = LBM_FP64) or FP32 (LBM_FP32_DEV), from a kernel of
 * independent FMA chains timed with CUDA events (best of five launches).
 * The roofline of the FP64 step, which is bound by double-precision
 * arithmetic on this GPU; measurement only, the paper has no counterpart.
 * Synchronises the device. */
int lbm_fma_peak(int precision, double *tflops);

/* ---- single-lattice context ---- */

/* Device bytes a context needs for p (populations x2, moment and snapshot
 * buffers, reduction scratch).  Pass a block of at least this size to
 * lbm_create to make the library use caller-owned device memory. */
int lbm_workspace_bytes(const lbm_params *p, size_t *bytes);

/* Create a context on the current CUDA device.
 *   cuda_stream     cudaStream_t all work is queued on (NULL = default stream)
 *   workspace_dev   NULL: the library allocates its device memory; else a
 *                   caller-owned device block of workspace_bytes >= the value
 *                   of lbm_workspace_bytes, 256-byte aligned, which must
 *                   outlive the context
 * The state is undefined until an lbm_init_* call. */
int lbm_create(const lbm_params *p, void *cuda_stream, void *workspace_dev,
               size_t workspace_bytes, lbm_ctx **out);
void lbm_destroy(lbm_ctx *ctx);

/* f_a(x, 0) = w_a rho0(x), the equilibrium at rest (initial condition; the
 * paper does not state one).  rho0_host: ny*nx doubles. Resets the step count. */
int lbm_init_density(lbm_ctx *ctx, const double *rho0_host);

/* Same, from a density field already on the device (ny*nx doubles). */
int lbm_init_density_dev(lbm_ctx *ctx, const double *rho0_dev);

/* Built-in initial fields: rho0 = rho_v + (rho_l - rho_v) (1 - tanh(2 d/width))/2
 * + noise_amp (2 xi - 1), xi = (SplitMix64(seed ^ (y nx + x)) >> 11) 2^-53, d the
 * signed distance to the liquid (slab |y - ny/2| - size; droplet r - size
 * about (nx/2, ny/2); bubble: phases swapped; droplet array: r - size about the
 * centre of each cell of side 'cell').  rho_l, rho_v <= 0 select the Maxwell
 * densities at the context's T/Tc. */
int lbm_init_preset(lbm_ctx *ctx, int kind, double size, double width, double rho_l,
                    double rho_v, int32_t cell, uint64_t seed, double noise_amp);

/* Advance nsteps time steps (asynchronous).  Errors seen by the kernels
 * (LBM_E_NONFINITE, LBM_E_EOS_DOMAIN) are latched and reported by
 * lbm_stats / lbm_run_to_steady. */
int lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Observables at the current time (synchronises).  snapshot != 0 also stores
 * v(t) for the next max_dv. */
int lbm_stats(lbm_ctx *ctx, int snapshot, lbm_stats_t *out);

/* Step until max|v(t) - v(t - check_every)| < tol, checking every
 * check_every steps, or until max_steps.  steps_done (may be NULL) receives
 * the steps taken by this call.  Returns LBM_OK when converged,
 * LBM_E_NOT_CONVERGED at max_steps, or the latched kernel error. */
int lbm_run_to_steady(lbm_ctx *ctx, double tol, int64_t check_every, int64_t max_steps,
                      int64_t *steps_done);

/* rho, vx, vy at the current time into caller host buffers of ny*nx doubles
 * each (any may be NULL).  v = u + F/(2 rho).  Synchronises. */
int lbm_read_moments(lbm_ctx *ctx, double *rho_host, double *vx_host, double *vy_host);

/* Asynchronous host I/O: the copies run on two copy streams of the context
 * (one per direction) and overlap the steps queued around them.
 *   lbm_init_density_async: as lbm_init_density; the copy of rho0_host into a
 *     device staging array starts at once (after the previous asynchronous
 *     init has read that array), and the init kernels follow it on the
 *     context's stream.
 *   lbm_read_moments_async: rho, vx, vy of the state reached by the work
 *     queued so far (as lbm_read_moments) are written into one of two device
 *     slots, alternately, and copied into the host buffers on the copy
 *     stream.  A read into a slot whose previous copy is still in flight
 *     waits for it on the device, not on the host.
 *   lbm_wait_io: returns when every copy queued by these calls is done.
 * Host buffers (ny*nx doubles each; page-locked, or the copies do not
 * overlap) stay owned by the caller and must stay valid, and unread or
 * unchanged, until lbm_wait_io returns.  The first call allocates the copy
 * streams and 7*ny*nx device doubles (also for a context on a caller's
 * workspace); lbm_destroy releases them.  None of the three synchronises
 * the context's stream. */
int lbm_init_density_async(lbm_ctx *ctx, const double *rho0_host);
int lbm_read_moments_async(lbm_ctx *ctx, double *rho_host, double *vx_host, double *vy_host);
int lbm_wait_io(lbm_ctx *ctx);

/* Post-streaming populations f_a(x, t) (the distribution at the current time,
 * before collision) as 9*ny*nx doubles, and the inverse.  Synchronises. */
int lbm_read_populations(lbm_ctx *ctx, double *f_host);
int lbm_write_populations(lbm_ctx *ctx, const double *f_host);

/* Rows [y0, y0 + nrows) of the stored state -- the post-collision
 * populations of the previous step, pulled by the next one (Eq. 1) -- copied
 * out of the lattice into a device buffer the caller owns (to_lattice = 0)
 * or from it into the lattice (to_lattice = 1).  Buffer layout [9][nrows][nx]
 * in the storage type: double for LBM_FP64, float deviations f - w rho_ref
 * for LBM_FP32_DEV.  The copies are queued on the context's stream, in order
 * with its steps, without synchronising.  This is the y-slab halo exchange
 * of one lattice split over ranks: a node's update reads the stored rows
 * within two of it (the pull one row, the psi of Eq. 6's stencil one row
 * further), so each rank steps its rows plus two halo rows per side and
 * refreshes those from its neighbours after every step.  LBM_E_INVALID for
 * rows outside [0, ny) or a null buffer. */
int lbm_copy_rows(lbm_ctx *ctx, int y0, int nrows, void *buf_dev, int to_lattice);

/* Checkpoint: header (magic, version, params, steps), the raw population
 * buffer and an FNV-1a checksum.  lbm_load needs a context created with the
 * same params; it restores the state bit for bit. */
int lbm_save(lbm_ctx *ctx, const char *path);
int lbm_load(lbm_ctx *ctx, const char *path);

/* Failure detection of the staged kernels (no paper counterpart).  Every
 * shared-memory stage wait of the strip kernels is bounded: a row copy that
 * does not land within the poll limit makes the kernel flag a timeout, wait
 * (again bounded) for the copies it has issued, and return, so that the
 * context stays usable and lbm_stats / lbm_run_to_steady report
 * LBM_E_TIMEOUT.  lbm_inject_stage_timeout makes that path run without a
 * stuck copy: in the next time step only, the first stage wait of every CTA
 * gives up at once.  The step then leaves its output undefined and latches
 * LBM_E_TIMEOUT; re-initialise the state (lbm_init_*, lbm_load,
 * lbm_write_populations) to go on.  LBM_E_UNSUPPORTED if the context runs
 * the generic kernel (configuration 0), which stages nothing. */
int lbm_inject_stage_timeout(lbm_ctx *ctx);

/* Kernel variant in use: 0 = generic tiled kernel (any nx), 1 = pipelined
 * strip kernel (nx % 4 == 0).  lbm_set_variant forces one (1 selects the
 * first strip configuration; LBM_E_UNSUPPORTED if the lattice does not
 * allow it); -1 restores the automatic choice: the strip kernel where it
 * applies (for FP32 lattices at least 1024 wide its 256-thread, two-stage
 * configuration) and its strips and row chunks can give every SM a CTA,
 * else the generic kernel.  lbm_autotune picks by timing. */
int lbm_get_variant(lbm_ctx *ctx, int *variant);
int lbm_set_variant(lbm_ctx *ctx, int variant);

/* Kernel configurations for a parameter set: id 0 is the generic kernel, ids
 * 1..count-1 the strip kernel with the tile shapes lbm_config_describe
 * reports (threads per CTA, shared-memory row stages, lattice nodes per
 * thread).  Pure host queries. */
int lbm_config_count(const lbm_params *p, int *count);
int lbm_config_describe(const lbm_params *p, int config, int *threads, int *stages, int *nodes_per_thread);
int lbm_get_config(lbm_ctx *ctx, int *config);
int lbm_set_config(lbm_ctx *ctx, int config);

/* Autotuner: times every configuration for trial_steps fused steps on this
 * context's lattice (CUDA events on the context stream; the trials write the
 * spare population buffer, so the state is not advanced) and selects the
 * fastest.  config / ms_per_step (may be NULL) receive the choice and its
 * time per step.  Synchronises. */
int lbm_autotune(lbm_ctx *ctx, int trial_steps, int *config, double *ms_per_step);

/* ---- batched instances ----
 * Many independent periodic lattices with their own size, T/Tc, tau, A, K and
 * initial field (the paper's tau, T/Tc and EOS-scale sweeps, Secs. 4.2-4.4)
 * advanced together: one kernel launch per time step covers every running
 * instance through a table of (instance, column strip, row chunk) work
 * items, each check interval is one CUDA graph, and convergence or failure is
 * decided per instance on the device.  Populations are FP32 deviations
 * (precision must be LBM_FP32_DEV; rho_ref = the instance's Maxwell vapour
 * density); every nx must be a multiple of 4.  All batch calls are
 * synchronous; the batch owns its device memory and its CUDA stream. */
typedef struct {
    int32_t collision;   /* lbm_collision */
    int32_t forcing;     /* lbm_forcing (MRT: Guo only) */
    int32_t precision;   /* LBM_FP32_DEV */
    int32_t reserved;    /* 0 */
    double s_e, s_eps, s_q;   /* MRT rates shared by all instances */
    double sigma;        /* LBM_LI: Li et al.'s sigma shared by all instances
                            (every instance then needs A = 0, Eq. 4's force;
                            see lbm_params); 0 for the other forcings */
} lbm_batch_params;

/* One instance: lattice, model parameters (as in lbm_params) and its initial
 * field (as in lbm_init_preset: kind, size = radius or half-width, tanh width,
 * rho_l / rho_v <= 0 for the Maxwell densities, droplet-array cell, noise). */
typedef struct {
    int32_t nx, ny, kind, cell;
    double T_over_Tc, tau, A, K;
    double size, width, rho_l, rho_v, noise_amp;
    uint64_t seed;
} lbm_instance;

/* Per-instance observables returned by lbm_batch_results, in this order. */
#define LBM_BATCH_NOBS 10  /* mass, max_v, max_dv, max_drho, rho_min, rho_max,
                              rho_center, rho_corner, rho_row_mid, rho_row0 */
#define LBM_RUNNING 0
#define LBM_CONVERGED 1
#define LBM_FAILED 2

typedef struct lbm_batch lbm_batch;

int lbm_batch_create(const lbm_batch_params *bp, const lbm_instance *inst, int n, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);

/* Initial state of every instance from its preset (computed on the device):
 * f_a = w_a rho0, the plain method's start at rest.  Resets steps, states
 * and snapshots. */
int lbm_batch_init(lbm_batch *b);

/* Where the nb samples of an instance's radial density profile sit: sample k
 * at distance r_k = |centre + spacing (k - (nb - 1)/2)| from the lattice
 * centre (droplet, bubble) or from the mid-row y = ny/2 (slab), so the grid
 * can be centred on the interface (centre = the radius or half-width) with a
 * spacing in lattice units.  use = 0 skips the instance (lbm_batch_init_profiles
 * gives it its preset). */
typedef struct {
    int32_t use, reserved;
    double centre, spacing;
} lbm_profile_geom;

#define LBM_INIT_REST 1   /* populations at rest: f_a = f_a^eq(rho0, -F/(2 rho0)) */

/* Initial state of the instances with geom_host[i].use != 0 from a density
 * profile (the learned warm start): profiles_dev is a device array [n][nb] of
 * densities on the grids geom_host[i], interpolated linearly in r and held
 * at the end values beyond them; the other instances get their preset.
 * flags & LBM_INIT_REST: the profile instances start from the equilibrium at
 * the velocity u = -F/(2 rho0), so that v = u + F/(2 rho) is zero and the
 * Guo (Eq. 23) forcing meets a fluid at rest; F is the Eq. 6 force of rho0,
 * computed as in the time step.  Otherwise f_a = w_a rho0.  Resets steps,
 * states and snapshots. */
int lbm_batch_init_profiles(lbm_batch *b, const double *profiles_dev, int nb, const lbm_profile_geom *geom_host,
                            int flags);

/* nsteps time steps of every running instance (no convergence checks). */
int lbm_batch_step(lbm_batch *b, int64_t nsteps);

/* Step every running instance, checking each every check_every steps: an
 * instance converges when max|v(t) - v(t - check_every)| < tol_v, when
 * max|rho(t) - rho(t - check_every)|/rho < tol_rho, or when both of its
 * coexistence densities (liquid and vapour probe: centre and corner node of
 * a droplet or bubble, mid and edge row of a slab) changed by less than
 * tol_coex relative since the previous check (a tolerance <= 0 is ignored);
 * it fails when a kernel flags a non-finite or out-of-domain value.  Either
 * way it stops stepping while the others go on.  Returns LBM_OK when no
 * instance is left running, LBM_E_NOT_CONVERGED at max_steps. */
int lbm_batch_run_to_steady(lbm_batch *b, double tol_v, double tol_rho, double tol_coex, int64_t check_every,
                            int64_t max_steps, int64_t *steps_done);

/* How lbm_batch_run_to_steady judges the coexistence probes against
 * tol_coex (a stopping rule of the measurement; the paper fixes none):
 *   LBM_COEX_CHANGE  the relative change of each probe since the previous
 *                    check (the default);
 *   LBM_COEX_TAIL    also the estimated change still to come: two
 *                    successive changes d and d' of a probe taken as a
 *                    geometric series of ratio r = d/d' (Aitken's
 *                    extrapolation) give |d| r/(1-r) for 0 <= r < 1 and |d|
 *                    for r < 0; the estimate from the last pair of changes
 *                    and from the pair before must both be below the
 *                    tolerance.  While the changes do not shrink (r >= 1),
 *                    or before four checks, the instance does not stop.  A
 *                    run that creeps towards its steady state by small,
 *                    slowly shrinking changes then runs on until what is
 *                    left is below the tolerance.
 * Applies from the next check on; LBM_E_INVALID for another value. */
#define LBM_COEX_CHANGE 0
#define LBM_COEX_TAIL 1
int lbm_batch_set_coex_rule(lbm_batch *b, int rule);

/* Recompute the observables of every instance (no convergence decisions, no
 * snapshot change).  A running instance that a kernel flagged (non-finite or
 * out-of-domain value) is marked LBM_FAILED with its code, as a check of
 * lbm_batch_run_to_steady would. */
int lbm_batch_observe(lbm_batch *b);

/* Host arrays of n entries (any may be NULL): state (LBM_RUNNING /
 * LBM_CONVERGED / LBM_FAILED), failure code (LBM_E_*), steps taken, and
 * n * LBM_BATCH_NOBS observables from the last check or observe. */
int lbm_batch_results(lbm_batch *b, int32_t *state, int32_t *code, int64_t *steps, double *obs);

/* FP64 density field of instance i (ny*nx, host). */
int lbm_batch_read_density(lbm_batch *b, int i, double *rho_host);

/* Radial density profiles of every instance, host array [n][nb], on the
 * sample grids geom_host[i] (see lbm_profile_geom; every entry is used): at
 * r_k the mean over 64 directions of the bilinearly interpolated density at
 * distance r_k from the lattice centre (droplet, bubble), or the mean over x
 * and both sides of y = ny/2 +- r_k (slab); r_k is held at most half the
 * period minus one (min(nx, ny)/2 - 1, or ny/2 - 1 for a slab), so samples
 * past it repeat the farthest point rather than wrap onto the next image. */
int lbm_batch_profiles(lbm_batch *b, int nb, const lbm_profile_geom *geom_host, double *prof_host);

/* Tile shape of the batched step: the strip width of a work item, its row
 * stages, rows per work item, and whether a row's pulled populations stay in
 * registers from its psi pass to its collision (carry = 1: every stage in
 * flight) or are re-read from the stage (carry = 0).
 *   columns 128: one warp walks a strip; stages 3 or 4 (carry 0), 2 or 3 (carry 1).
 *   columns 256: a 64-thread CTA walks a strip; stages 3, carry 1 only.
 *   columns 512: a 128-thread CTA walks a strip; stages 2 or 3, carry 1 only.
 * Other combinations return LBM_E_INVALID.  lbm_batch_autotune times the
 * seven (columns, stages, carry) candidates x rows 32, 64, 128, 256 for trial_steps
 * steps each without advancing the state and keeps the fastest; any output
 * pointer may be NULL. */
int lbm_batch_set_tuning(lbm_batch *b, int columns, int stages, int rows_per_item, int carry);
int lbm_batch_autotune(lbm_batch *b, int trial_steps, int *columns, int *stages, int *rows_per_item, int *carry,
                       double *ms_per_step);

/* Total lattice nodes of the batch (-1 if b is NULL). */
int64_t lbm_batch_nodes(lbm_batch *b);

/* ---- learned warm start ----
 * The paper has no learned component; this network serves the batched
 * solver.  A tanh multilayer perceptron n_in -> n_hidden (x hidden_layers) ->
 * n_out, FP32, trained and evaluated by the library's own CUDA kernels
 * (forward, backward, Adam).  For the warm start the inputs are (T/Tc, tau,
 * A, K, radius) and the outputs log-density samples of the converged profile
 * (see lbm_batch_profiles).  Inputs and targets are standardised inside the
 * model with the affine scalings of lbm_ws_set_scaling.  Parameters are
 * flattened layer by layer as [W (out x in, row-major), b], hidden layers
 * first.  Host arrays are row-major [n][n_in] / [n][n_out] floats; all calls
 * synchronise. */
typedef struct {
    int32_t n_in, n_hidden, hidden_layers, n_out;
    uint64_t seed;      /* Glorot-uniform initial weights from SplitMix64(seed) */
} lbm_ws_cfg;

typedef struct lbm_ws lbm_ws;

int lbm_ws_create(const lbm_ws_cfg *cfg, lbm_ws **out);
void lbm_ws_destroy(lbm_ws *w);
int lbm_ws_num_params(lbm_ws *w, int64_t *n);
int lbm_ws_set_scaling(lbm_ws *w, const float *x_mean, const float *x_std, const float *y_mean, const float *y_std);
int lbm_ws_get_params(lbm_ws *w, float *params_host);
int lbm_ws_set_params(lbm_ws *w, const float *params_host);   /* also resets the Adam state */

/* Mean squared error in standardised output units over n samples and its
 * gradient with respect to the flattened parameters (grad_host may be NULL). */
int lbm_ws_loss_grad(lbm_ws *w, const float *X_host, const float *Y_host, int n, float *loss, float *grad_host);

/* Adam (beta1 0.9, beta2 0.999, eps 1e-8) on minibatches of the MSE, epochs
 * passes over a per-epoch SplitMix64(seed) shuffle; final_loss (may be NULL)
 * receives the loss over all n samples afterwards. */
int lbm_ws_train(lbm_ws *w, const float *X_host, const float *Y_host, int n, int epochs, int batch, float lr,
                 uint64_t seed, float *final_loss);

/* Network outputs (in target units) for n input rows. */
int lbm_ws_predict(lbm_ws *w, const float *X_host, int n, float *Y_host);

/* ---- observables without allocation ----
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: code inside a host application whose memory
 * pool owns the device and forbids cudaMalloc/cudaFree, or loops that must
 * not stall on an allocation (both calls may synchronise the device).
 *
 * lbm_stats_noalloc computes what lbm_stats(ctx, 0, out) computes, from a
 * population buffer the caller owns, and allocates nothing: its scratch is a
 * fixed array of LBM_NOALLOC_MAX_TILES 64-byte records (4 MiB) compiled into
 * the library, which every GPU that loads the library keeps until the
 * process exits.
 *   p         parameters of the lattice (as for lbm_create)
 *   f_dev     device buffer of 9*ny*nx values in the library's stored layout:
 *             double (LBM_FP64) or float (LBM_FP32_DEV) post-collision
 *             populations of the previous step in the pull convention,
 *             f*_a(x) = f_a(x + e_a, t) - w_a rho_ref (rho_ref = 0 for FP64)
 *   cuda_stream  stream the work is queued on; the call synchronises it
 *   out       host struct; max_dv = -1 and steps = 0 (no context history)
 * Limits and behaviour:
 *   - lattices needing more than LBM_NOALLOC_MAX_TILES tiles of 32 x 8 nodes
 *     (ceil(nx/32) * ceil(ny/8); any lattice up to 4096 x 4096 fits) are
 *     rejected with LBM_E_UNSUPPORTED and a message on stderr;
 *   - every call shares the one scratch array and leaves its contents
 *     behind, so calls that overlap on the GPU (other threads or streams)
 *     race and must be serialised by the caller;
 *   - the first call on each device does a one-time set-up (it looks up the
 *     scratch array's device address with that device current), and so does
 *     the first call in each further CUDA context on it (the address belongs
 *     to the context: after cudaDeviceReset, or in a context the caller
 *     created, it is looked up again); make that first call before any
 *     stream capture;
 *   - each call waits for its stream (the result is read back into host
 *     memory before it returns). */
#define LBM_NOALLOC_MAX_TILES 65536
int lbm_stats_noalloc(const lbm_params *p, const void *f_dev, void *cuda_stream, lbm_stats_t *out);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
