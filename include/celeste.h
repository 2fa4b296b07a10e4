/*
 * celeste.h - C ABI of the GB300 (sm_103a) Celeste per-source ELBO / Newton library.
 *
 * The operations follow "Learning an Astronomical Catalog of the Visible Universe through
 * Scalable Bayesian Inference" (Regier et al.):
 *   - Sec. "The Celeste Model": images with fixed metadata Lambda_n (PSF, sky, calibration,
 *     pixel<->sky map) whose pixel counts are Poisson with a rate set by the catalog;
 *   - Sec. "Variational Inference", Eq. (1)-(3): the ELBO and the factorised q;
 *     each source's parameters are optimised with its neighbours held fixed, by Newton's
 *     method with a trust region and the exact gradient and dense Hessian.
 *
 * Conventions (all calls):
 *   - 27 free variational parameters per source, float64, row-major [S][27]:
 *       0,1 world position u; 2 logit fracDev; 3 logit axis ratio; 4 angle (rad);
 *       5 log half-light radius; 6 logit P(galaxy);
 *       7,8 star mean / log variance of log r-band flux; 9,10 the same for galaxies;
 *       11-14 star colour means; 15-18 star colour log variances;
 *       19-22 galaxy colour means; 23-26 galaxy colour log variances.
 *   - Pixel (row i, col j) of an image has its centre at pixel coordinates (x, y) = (j, i);
 *     world -> pixel map p = A u + o with wcs = {A00, A01, A10, A11, o0, o1}.
 *   - "device" pointers are CUDA device memory of the current device; "host" pointers are
 *     ordinary host memory.  The library never frees caller memory.
 *   - Calls taking a stream are asynchronous on it, except where stated.
 *   - Return value: CELESTE_OK or a CELESTE_ERR_* code; celeste_strerror() describes it and
 *     celeste_last_error_detail() gives the message of the last failure on this thread.
 */
#ifndef CELESTE_H
#define CELESTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CELESTE_NPARAM 27
#define CELESTE_NPSF 3
#define CELESTE_NEXP 6
#define CELESTE_NDEV 8
#define CELESTE_MAX_RADIUS 64

typedef struct CUstream_st* celeste_stream_t; /* identical to cudaStream_t */

enum {
  CELESTE_OK = 0,
  CELESTE_ERR_INVALID_ARG = 1, /* a descriptor or argument failed validation; nothing launched */
  CELESTE_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  CELESTE_ERR_TIMEOUT = 3,     /* a bounded device-side wait ran out */
  CELESTE_ERR_WORKSPACE = 4,   /* workspace missing, too small or misaligned */
  CELESTE_ERR_STATE = 5        /* call order violated (e.g. elbo before bind) */
};

/* Per-source outcome of celeste_newton_batch. */
enum {
  CELESTE_STATUS_CONVERGED = 0,
  CELESTE_STATUS_MAX_ITER = 1,
  CELESTE_STATUS_NONFINITE = 2,
  CELESTE_STATUS_RADIUS_COLLAPSE = 3
};

/* Bits of `want` in celeste_elbo_batch. */
#define CELESTE_WANT_ELBO 1u
#define CELESTE_WANT_GRAD 2u
#define CELESTE_WANT_HESS 4u

/* One image and its metadata Lambda_n (Sec. "The Celeste Model").
 *   pixels: device, float32 row-major [height][width] photon counts (>= 0, finite);
 *           must stay valid while the problem is bound.
 *   band:   0..4 = u,g,r,i,z; reference band is r (2).
 *   sky:    expected background counts per pixel (> 0).
 *   iota:   calibration, counts per nanomaggy (> 0).
 *   psf:    3 Gaussian components x 6 parameters {weight logit, mean x, mean y,
 *           log sigma x, log sigma y, atanh correlation}, each a quadratic polynomial in
 *           (xh, yh) = (2x/(width-1)-1, 2y/(height-1)-1) with coefficients for
 *           {1, xh, yh, xh^2, xh*yh, yh^2}; weights are the softmax of the logits. */
typedef struct {
  int32_t height, width, band;
  const float* pixels;
  double sky, iota;
  double wcs[6];
  double psf[CELESTE_NPSF][6][6];
} celeste_image_desc;

/* The problem: images, the catalog locations that anchor each source's patches, priors
 * and the galaxy-profile mixture tables (all host memory, copied by celeste_problem_create).
 *   u0:     host [S][2] catalog world positions.  Source s's patch in image n is the
 *           (2R+1)^2 pixel square centred on round(A_n u0_s + o_n), present when that centre
 *           lies inside image n, clipped to the image; the PSF of (s, n) is evaluated at
 *           A_n u0_s + o_n and held fixed.
 *   radius: host [S] patch half-width R in 1..CELESTE_MAX_RADIUS.
 *   priors: {P(galaxy), mean of log r, variance of log r, colour mean, colour variance}.
 *   exp_* / dev_*: unit-flux circular mixtures sum_j nu_j N(0, tau_j I) (nu > 0, tau > 0)
 *           for the exponential and de Vaucouleurs profiles.
 *   tile_pixels: pixels per work tile (128, 256, 512 or 1024; 0 = default 128).
 *   hessian_mode: how the pixel kernel forms the Hessian's Jacobian cross-product
 *           sum_m Y_m^T C_m Y_m (the per-tile SYRK; everything else is unchanged):
 *           CELESTE_HESS_FP32 (0) float32 FMAs; on the tensor cores (mma.sync, float32
 *           accumulation): CELESTE_HESS_TF32 (1) TF32 operands; CELESTE_HESS_BF16X3 (2) BF16
 *           hi + lo split operands, hi*hi + hi*lo + lo*hi; CELESTE_HESS_BF16X6 (3) BF16
 *           hi + mid + lo split operands, the six products down to 2^-16 of the leading one;
 *           CELESTE_HESS_TF32X3 (4) TF32 big + small split operands, big*big + big*small +
 *           small*big.  Modes 1-4 need tile_pixels 128. */
typedef struct {
  int32_t n_images;
  const celeste_image_desc* images;
  int32_t n_sources;
  const double* u0;
  const int32_t* radius;
  double priors[5];
  double exp_nu[CELESTE_NEXP], exp_tau[CELESTE_NEXP];
  double dev_nu[CELESTE_NDEV], dev_tau[CELESTE_NDEV];
  int32_t tile_pixels;
  int32_t hessian_mode;
} celeste_problem_desc;

enum {
  CELESTE_HESS_FP32 = 0,
  CELESTE_HESS_TF32 = 1,
  CELESTE_HESS_BF16X3 = 2,
  CELESTE_HESS_BF16X6 = 3,
  CELESTE_HESS_TF32X3 = 4
};

typedef struct celeste_problem celeste_problem;

/* Trust-region Newton options (Sec. "Variational Inference": Newton with a trust region,
 * machine tolerance within 50 iterations).  Zero-initialised fields take the defaults shown. */
typedef struct {
  int32_t max_iter;   /* 50 */
  double ftol;        /* 1e-8: stop after an accepted step with |f_k - f_k+1| <= ftol |f_k+1|, when an
                         interior (full Newton) step predicts a decrease <= ftol |f|, or when a
                         rejected step had predicted a decrease <= ftol |f| */
  double gtol;        /* 1e-10: stop when max |grad| <= gtol */
  double delta0;      /* 1.0: initial radius (used where delta_inout[s] <= 0) */
  double delta_max;   /* 1e4 */
  double eta;         /* 0.1: acceptance threshold on actual/predicted reduction */
  double delta_min;   /* 1e-12: below this the source stops with RADIUS_COLLAPSE */
  int32_t graph_iters; /* 4: Newton iterations captured in one CUDA graph and run between two
                          host checks of the active count; 1: plain launches, one check per
                          iteration.  Iterations after the last source stops launch kernels
                          that find empty worklists and change nothing. */
  int32_t cta_sources; /* 0: twice the SM count.  An iteration that starts with at most this many
                          active sources solves each subproblem on four warps (one CTA, the SM's
                          four float64 pipes) instead of one; negative: always one warp.  Both
                          solve the same subproblem; their roundings differ. */
} celeste_newton_opts;

/* Validate the description and build the host-side layout (patches, neighbours, work
 * tiles).  Synchronous, host only, allocates no device memory.  On success *out owns copies
 * of every host array; free it with celeste_problem_destroy.
 * Errors: CELESTE_ERR_INVALID_ARG (non-finite or out-of-range metadata, radius outside
 * 1..64, non-SPD PSF covariance, bad mixture table, NULL pointers). */
int celeste_problem_create(const celeste_problem_desc* desc, celeste_problem** out);

/* Device workspace bytes needed by celeste_problem_bind (>0). */
size_t celeste_problem_workspace_bytes(const celeste_problem* p);

/* Counts of the layout: sources, patches, tiles, total patch pixels, neighbour entries. */
int celeste_problem_counts(const celeste_problem* p, int64_t counts[5]);

/* Bind a caller-owned device workspace (>= workspace_bytes, 256-byte aligned) and upload the
 * layout into it; evaluates each patch's PSF on the device.  The workspace must outlive
 * every later call on this problem.  Asynchronous on `stream`. */
int celeste_problem_bind(celeste_problem* p, void* workspace, size_t bytes, celeste_stream_t stream);

/* New pixel values in the same images (the device buffers given at create, same layout and catalog
 * positions): re-gathers every patch pixel's count and log-factorial term, as bind does, without
 * re-uploading the layout; clears the error words.  The background must be rendered again before the
 * next evaluation.  Asynchronous on `stream`. */
int celeste_problem_refresh_pixels(celeste_problem* p, celeste_stream_t stream);

/* Fixed part of every patch pixel's rate: gathers the counts and renders the neighbours'
 * expected brightness and variance (Sec. "Variational Inference": neighbours held fixed).
 *   nbr_theta: device float64 [S][27], the parameters the neighbours are fixed at.
 * Must run after bind and again whenever the neighbours' parameters change. */
int celeste_render_background(celeste_problem* p, const double* nbr_theta, celeste_stream_t stream);

/* As celeste_render_background, with the neighbours' extent chosen by `mode`:
 *   CELESTE_NBR_FULL (0): each neighbour's full light on every pixel of the target's patch (the
 *     per-source objective, neighbours held fixed);
 *   CELESTE_NBR_WINDOW (1): each neighbour's light only on the pixels of its own window, as in
 *     the objective over all sources jointly (paper, concluding section: a stationary point of
 *     the objective over all light sources at once).  Rendered at nbr_theta = theta, the
 *     per-source gradient and Hessian of celeste_elbo_batch are then the joint objective's
 *     gradient and diagonal Hessian blocks.
 * Errors: CELESTE_ERR_INVALID_ARG for another mode or a NULL nbr_theta. */
int celeste_render_background_mode(celeste_problem* p, const double* nbr_theta, int mode, celeste_stream_t stream);

enum { CELESTE_NBR_FULL = 0, CELESTE_NBR_WINDOW = 1 };

/* Joint objective over all sources (every pixel of the union of the windows counted once, each
 * source's light on its own window):
 *   J(theta) = sum_n sum_{m in U_n} l(x_m, E_m, V_m) - sum_s KL_s,
 *   E_m = sky + iota sum_{s: m in W_s} E[G_s](m),  V_m = iota^2 sum_{s: m in W_s} Var[G_s](m).
 * Its cross-source Hessian block of two sources whose windows overlap is
 *   d2J / dtheta_s dtheta_t = sum_{m in W_s cap W_t} l_EE dE/ds dE/dt^T + l_EV (dE/ds dV/dt^T + dV/ds dE/dt^T).
 *
 * celeste_joint_pairs: the pairs (s, t), s < t, of sources whose windows overlap in some image,
 * in the order celeste_joint_cross_hessian writes their blocks.
 *   pairs:    host int32 [capacity][2], or NULL to query the count only;
 *   capacity: number of pairs `pairs` can hold; n_pairs: host, receives the number of pairs.
 * Host only (no device memory, usable before bind): the pair list and the overlap tiles are built
 * from the layout on the first call and kept on the problem; the first device call uploads them.
 * Errors: CELESTE_ERR_INVALID_ARG when capacity is too small or n_pairs is NULL. */
int celeste_joint_pairs(celeste_problem* p, int32_t* pairs, int64_t capacity, int64_t* n_pairs);

/* Device memory of the joint calls (celeste_joint_cross_hessian, _newton, _value): the overlap
 * lists and tiles, the cross-tile sums and the joint Newton state (about 12 KB per source plus
 * 12 bytes per patch pixel).  celeste_joint_workspace_bytes: bytes needed (host only; builds the
 * overlap lists on first use; 0 for a NULL problem).  celeste_joint_bind: bind a caller-owned
 * device buffer of at least that size, 256-byte aligned, after celeste_problem_bind, and upload the
 * lists into it (asynchronous on `stream`; the problem keeps the host copies).  The library
 * allocates nothing for the joint calls; they return CELESTE_ERR_STATE until a workspace is bound.
 * The buffer must outlive every later joint call on the problem.
 * Errors: CELESTE_ERR_STATE before celeste_problem_bind; CELESTE_ERR_WORKSPACE when the buffer is
 * missing, too small or misaligned. */
size_t celeste_joint_workspace_bytes(celeste_problem* p);
int celeste_joint_bind(celeste_problem* p, void* workspace, size_t bytes, celeste_stream_t stream);

/* Cross-source Hessian blocks of J at theta, one per pair of celeste_joint_pairs:
 *   theta:  device float64 [S][27], the parameters of every source;
 *   blocks: device float64 [n_pairs][27][27]; block k row i, column j = d2J/dtheta_{s,i} dtheta_{t,j}
 *           for pair k = (s, t).
 * The background must have been rendered with CELESTE_NBR_WINDOW at nbr_theta = theta (the pixel
 * rates E_m, V_m include every source's light); the call checks the mode, not the parameters.
 * Per-pixel Jacobian rows of both sources in float32, per-tile sums in float32, the cross-tile
 * sum and the lift to the 27 parameters in float64.  Asynchronous on `stream`.
 * Errors: CELESTE_ERR_STATE when the background was not rendered in window mode. */
int celeste_joint_cross_hessian(celeste_problem* p, const double* theta, double* blocks, celeste_stream_t stream);

/* Trust-region Newton on the joint objective J over all sources at once (paper, concluding
 * section), with the per-source solve's rules (Nocedal & Wright Alg. 4.1: eta, the radius update
 * by 1/4 and 2, ftol on accepted changes, on the Newton decrement and on the prediction of a
 * rejected step, gtol on max |grad|).  The
 * subproblem is solved by preconditioned conjugate gradients with Steihaug's stopping rules
 * (Nocedal & Wright Alg. 7.2) over the block-sparse Hessian (celeste_elbo_batch's per-source
 * blocks in window mode and celeste_joint_cross_hessian's cross blocks); the preconditioner is
 * blockdiag(-H_ss + mu_s I), mu_s the first shift of {0, 1e-8, 1e-6, 1e-4, 1e-2, 1} x max|H_ii|
 * that makes the block positive definite, and the radius is measured in its norm, starting at the
 * norm of the block-diagonal Newton step and capped at opts->delta_max times that.  J's change at
 * a trial point is summed per pixel against the stored rates at the current point (float32 per
 * pixel, float64 across tiles and sources), each pixel weighted by 1 / (windows holding it).
 *   theta:  device float64 [S][27], start on entry, result on return;
 *   opts:   NULL or the per-source solve's options (graph_iters unused; delta0 unused: see above);
 *   max_cg: conjugate-gradient iterations per subproblem (<= 0: 100); a subproblem stops early
 *           once the residual is below 1e-2 |g|;
 *   iters_out, status_out, J_out, cg_iters_out (may be NULL): host; outer iterations, one
 *           CELESTE_STATUS_* for the whole solve, J at the result, total CG iterations.
 * Synchronous (reads a few scalars back every iteration); leaves the background rendered in
 * window mode at the result.  Its state lives in the joint workspace (celeste_joint_bind). */
int celeste_joint_newton(celeste_problem* p, double* theta, const celeste_newton_opts* opts, int32_t max_cg,
                         int32_t* iters_out, int32_t* status_out, double* J_out, int32_t* cg_iters_out,
                         celeste_stream_t stream);

/* The joint objective J at theta (device float64 [S][27]) into *J_out (host): the window-mode
 * background at theta, each patch pixel's term weighted by 1 / (windows holding it), float32 per
 * pixel and float64 across tiles and sources, minus every source's KL.  Synchronous; leaves the
 * background rendered in window mode at theta. */
int celeste_joint_value(celeste_problem* p, const double* theta, double* J_out, celeste_stream_t stream);

/* ELBO of every source's subproblem and, on request, its exact gradient and dense Hessian
 * w.r.t. the 27 free parameters (Eq. (1)-(2) restricted to the source's patches, minus its KL).
 *   theta: device float64 [S][27].
 *   want:  OR of CELESTE_WANT_*; outputs not wanted may be NULL.
 *   elbo:  device float64 [S]; grad: device float64 [S][27]; hess: device float64 [S][27][27].
 * Pixel arithmetic is float32; the cross-pixel sums and the assembly are float64.
 * Asynchronous: errors found on the device are not in the return value.  The call first clears
 * the problem's timeout word; a pixel kernel whose bounded wait on a tile's bulk copies runs out
 * sets it, leaves that CTA's remaining tiles unevaluated and writes NaN for the tile it waited
 * on, so the outputs are undefined.  celeste_problem_check reports it. */
int celeste_elbo_batch(celeste_problem* p, const double* theta, unsigned want,
                       double* elbo, double* grad, double* hess, celeste_stream_t stream);

/* Waits for `stream` and reports what the device recorded since the problem's last evaluating
 * call started (celeste_elbo_batch, celeste_elbo_batch_noalloc, celeste_newton_batch,
 * celeste_covariance_batch, the joint calls), and since bind for the pixel counts:
 *   CELESTE_ERR_TIMEOUT       a pixel kernel's bounded wait on its bulk copies ran out;
 *   CELESTE_ERR_INVALID_ARG   an image holds negative or non-finite counts (found at bind);
 *   CELESTE_OK                neither.
 * Synchronous.  celeste_newton_batch and the joint calls return these codes themselves. */
int celeste_problem_check(celeste_problem* p, celeste_stream_t stream);

/* Budget, in SM clock cycles, of the pixel kernels' first wait on each tile's bulk copies
 * (default ~2 s: 0 restores it).  A negative budget makes every such wait give up at once,
 * without waiting: the timeout path runs (error word set, a full-budget wait for the copies
 * already in flight so that none lands after the CTA exits, NaN tile sums, early exit) on a
 * healthy device, which is how the tests exercise it.  Takes effect on the next call. */
int celeste_problem_set_wait_budget(celeste_problem* p, long long cycles);

/* Trust-region Newton on every source's subproblem, all sources in one batch.
 *   theta_inout: device float64 [S][27], start in, optimum out.
 *   delta_inout: device float64 [S] trust radius (<= 0 means opts->delta0); the final radius
 *                is written back, so a later call resumes where this one stopped.
 *   iters_out, status_out: device int32 [S]; elbo_out: device float64 [S] (may be NULL).
 * The iterations run as CUDA graphs of opts->graph_iters iterations (captured on a stream private
 * to the problem, launched on `stream`, kept for later calls with the same arguments); the host
 * waits on `stream` after each graph to test whether any source is still active. */
int celeste_newton_batch(celeste_problem* p, double* theta_inout, const celeste_newton_opts* opts,
                         double* delta_inout, int32_t* iters_out, int32_t* status_out,
                         double* elbo_out, celeste_stream_t stream);

/* Linear-response covariance of every source's variational parameters at theta (normally the
 * optimum from celeste_newton_batch): cov_s = (-H_s)^-1, H_s the exact ELBO Hessian w.r.t. the 27
 * free parameters (Sec. "Variational Inference", the Newton solver's curvature reused).
 *   theta: device float64 [S][27]; cov: device float64 [S][27][27] out; ok: device int32 [S] out,
 *   1 where -H_s is positive definite (else cov_s is NaN).  Uses the problem's Newton workspace;
 *   the background must be rendered. */
int celeste_covariance_batch(celeste_problem* p, const double* theta, double* cov, int32_t* ok,
                             celeste_stream_t stream);

/* The trust-region subproblem of celeste_newton_batch on its own, for n independent problems
 * (Sec. "Variational Inference": Newton's method with a trust region):
 *     p = argmin g.p + p.B.p/2  subject to |p| <= delta.
 *   B: device float64 [n][27][27] symmetric; g: device [n][27]; delta: device [n] (> 0).
 *   p: device [n][27] out; pred: device [n] out, -(g.p + p.B.p/2) (may be NULL);
 *   hard: device int32 [n] out, 1 where the hard case (g orthogonal to the eigenvector of the
 *   smallest eigenvalue) was taken (may be NULL).  Solved in float64 (tridiagonal reduction,
 *   Sturm multisection for the smallest eigenvalue, safeguarded Newton on 1/|p| - 1/delta). */
int celeste_tr_solve_batch(const double* B, const double* g, const double* delta, int n, double* p,
                           double* pred, int32_t* hard, celeste_stream_t stream);

/* celeste_tr_solve_batch with the solver's two layouts and its multiplier hint exposed, for tests:
 *   warps:    1 (one warp per problem, the layout of iterations with many active sources) or 4 (one
 *             CTA of four warps per problem, the layout celeste_newton_batch uses when few are left);
 *   lam_hint: device float64 [n] or NULL; a multiplier near the solution's (negative: none), used
 *             to place the first pass of the multiplier search (the Newton iteration passes each
 *             source's previous multiplier); the solution does not depend on it beyond rounding;
 *   lam:      device float64 [n] out or NULL: the multiplier found (0 for an interior step,
 *             negative after the hard case).
 * The other arguments are celeste_tr_solve_batch's.  Errors: CELESTE_ERR_INVALID_ARG for warps
 * other than 1 or 4, n < 0, or a required pointer NULL with n > 0. */
int celeste_tr_solve_batch_ex(const double* B, const double* g, const double* delta, int n, int warps,
                              const double* lam_hint, double* p, double* pred, int32_t* hard, double* lam,
                              celeste_stream_t stream);

/* The float64 reciprocal the subproblem solver divides with (its recurrences divide once per row),
 * applied elementwise, so that its error bound can be tested: r[i] ~ 1 / x[i] from the PTX
 * approximate reciprocal refined by two Newton-Raphson steps (no counterpart in the paper; an
 * implementation detail of the float64 solve).  x, r: device float64 [n] (r may alias x).  For
 * normal x, |r - 1/x| is within 2 units in the last place of 1/x; x = 0 or |x| < 2^-1022 gives NaN,
 * |x| > 2^1022 gives 0.  Returns CELESTE_ERR_INVALID_ARG for n < 0 or a null pointer with n > 0. */
int celeste_tr_reciprocal(const double* x, double* r, int n, celeste_stream_t stream);

/* Device-time accounting of the library's own kernels, for benchmarks.
 *   celeste_profile_start: reset and start recording.  While recording, every launch of the
 *     ELBO+gradient+Hessian pixel kernel, of the value-only pixel kernel and of the trust-region
 *     step kernel is bracketed by CUDA events recorded on the stream it is launched on.
 *   celeste_profile_stop: stop recording, wait for the recorded events and fill *out.
 * Not part of the numerical path; the counters cost one atomic per pixel-kernel CTA. */
typedef struct {
  double full_ms;             /* summed duration of ELBO+gradient+Hessian pixel-kernel launches */
  double value_ms;            /* summed duration of value-only pixel-kernel launches */
  int64_t full_launches, value_launches;
  int64_t full_pixels;        /* pixel evaluations with value, gradient and Hessian */
  int64_t value_pixels;       /* pixel evaluations with value only */
  int64_t kernel_launches;    /* every kernel launched by the library while recording */
  int64_t newton_iterations;  /* trust-region iterations run by celeste_newton_batch */
  double tr_ms;               /* summed duration of trust-region step launches (celeste_newton_batch) */
  int64_t tr_launches;
} celeste_profile_stats;

int celeste_profile_start(celeste_problem* p);
int celeste_profile_stop(celeste_problem* p, celeste_profile_stats* out);

/* Measured rate of one arithmetic pipe of the current device, the denominators of the benchmark's
 * rooflines (not part of the method):
 *   kind 0: FP32 fused multiply-add, in flop/s (2 per FMA) - the pixel kernels' bound;
 *   kind 1: the special-function unit's base-2 exponential (ex2.approx), in operations/s;
 *   kind 2: FP64 fused multiply-add, in flop/s - the trust-region step's pipe;
 *   kind 3: FP32 fused multiply-add issued two lanes wide (packed FP32), in flop/s - the form the
 *           pixel kernels' galaxy components use.
 * Runs independent FMA (or ex2) chains on every SM, grown until a launch lasts ~25 ms, and reports
 * the best of three launches timed by CUDA events on `stream`; *seconds (may be NULL) gets that
 * launch's duration.  Synchronous; allocates and frees a few MB of device memory. */
int celeste_measure_peak(int kind, double* ops_per_s, double* seconds, celeste_stream_t stream);

/* The same evaluation as celeste_elbo_batch with want = ELBO | GRAD | HESS, for callers that may
 * not allocate device memory when they evaluate (a pre-sized arena, an allocator owned by another
 * framework, a request path that must not allocate).  The call allocates nothing: the kernels'
 * scratch (per-patch tables, per-pixel source moments, per-tile partial sums, per-source flags and
 * brightness constants, worklists) lives in one fixed 8 MiB device array inside this library,
 * which every GPU that loads the library keeps until the process exits.
 * The paper has no counterpart; it is a deployment variant of the evaluation above.
 *   p must be bound and have its background rendered; theta, elbo, grad, hess as in
 *   celeste_elbo_batch (all four required).
 *   Limit: 432 * n_tiles, 4 * n_sources, 8224 * n_patches, 8 * n_pixels,
 *   4 * (n_tiles + n_patches + n_sources) and 340 * n_sources bytes, each rounded up to 256, plus
 *   256 must fit in 8 MiB (e.g. ~700 patches of 17 x 17 pixels); larger problems get
 *   CELESTE_ERR_INVALID_ARG before any launch.
 *   The error words and the profiling counters stay in the bound workspace: the call clears the
 *   timeout word first, a timed-out bulk-copy wait sets it there (celeste_problem_check reports
 *   it), and celeste_profile_start/stop count this call's pixel-kernel launches and pixels.
 *   The first call on a device looks up the array's device address with that device current;
 *   make that first call before any stream capture.
 *   Every call shares the one array: calls that overlap on the GPU (different streams, threads
 *   or problems without ordering between them) race and corrupt each other's results. */
int celeste_elbo_batch_noalloc(celeste_problem* p, const double* theta, double* elbo, double* grad,
                               double* hess, celeste_stream_t stream);

/* ---------------------------------------------------------------- learned warm start
 * A small CNN maps a source's 5-band 32 x 32 patch to initial variational parameters; Newton
 * (celeste_newton_batch) then runs from that start to the same tolerance as from any other, so
 * the network only changes where the solve begins.  The paper's model has no such network; it is
 * the warm start of the workload's learned-part configuration.
 * Network: conv3x3 5->32 (stride 1), 32->64, 64->64, 64->64 (stride 2 each), padding 1, ReLU ->
 * 4 x 4 x 64 = 1024 -> fully connected 256, ReLU -> 27.  Activations NHWC BF16 (uint16_t bit
 * patterns), products on the tensor cores with FP32 accumulation, FP32 master parameters.
 * Parameter vector (FP32, celeste_cnn_param_count() entries, and a BF16 copy of the same length):
 *   W1 [32][3][3][5], b1 [32], W2 [64][3][3][32], b2 [64], W3 [64][3][3][64], b3 [64],
 *   W4 [64][3][3][64], b4 [64], W5 [256][1024] (input index (h * 4 + w) * 64 + c), b5 [256],
 *   W6 [27][256], b6 [27].
 * All pointers are device memory owned by the caller; all calls are asynchronous on `stream`. */
int64_t celeste_cnn_param_count(void);

/* Activation workspace for a batch (bytes; the buffer must be 256-byte aligned). */
size_t celeste_cnn_workspace_bytes(int batch);

/* He-normal weights (std sqrt(2 / fan_in); the last layer times 0.1) from a counter-based
 * generator seeded by `seed`, zero biases; writes both copies. */
int celeste_cnn_init(float* params, uint16_t* params_bf16, uint64_t seed, celeste_stream_t stream);

/* y [batch][27] = network(x [batch][32][32][5]); with out_scale / out_shift (both or neither,
 * [27]) the output is y * scale + shift.  Keeps the activations in ws for celeste_cnn_backward.
 * Runs on the tcgen05 tensor cores (celeste_cnn_forward_ex with CELESTE_CNN_TCGEN05). */
int celeste_cnn_forward(const float* params, const uint16_t* params_bf16, const uint16_t* x, int batch,
                        const float* out_scale, const float* out_shift, float* y, void* ws, size_t ws_bytes,
                        celeste_stream_t stream);

/* The same forward pass on a chosen engine:
 *   CELESTE_CNN_MMA_SYNC (0): one implicit-GEMM kernel per layer, warp-level mma.sync m16n8k16;
 *   CELESTE_CNN_TCGEN05 (1): per layer a GEMM on the fifth-generation tensor cores, 128-row tiles,
 *     operands gathered into 128-byte-swizzled shared memory, tcgen05.mma into a tensor-memory
 *     accumulator, tcgen05.ld epilogue (bias, ReLU).  Waits are bounded: a product that does not
 *     complete sets an error word that celeste_cnn_status reports.
 * Both use BF16 operands and FP32 accumulation; their outputs differ only in summation order. */
enum { CELESTE_CNN_MMA_SYNC = 0, CELESTE_CNN_TCGEN05 = 1 };
int celeste_cnn_forward_ex(const float* params, const uint16_t* params_bf16, const uint16_t* x, int batch,
                           const float* out_scale, const float* out_shift, float* y, void* ws, size_t ws_bytes,
                           int engine, celeste_stream_t stream);

/* CELESTE_ERR_TIMEOUT (and clears it) if a tensor-core product of the network's forward pass did not
 * complete within its wait budget since the last call; CELESTE_OK otherwise.  Synchronous (reads a
 * device word of the current device). */
int celeste_cnn_status(void);

/* grad [param_count] += d loss / d params given dy = d loss / d y [batch][27], after a forward
 * call on the same x, ws and parameters (without scale / shift). */
int celeste_cnn_backward(const float* params, const uint16_t* params_bf16, const uint16_t* x, const float* dy,
                         int batch, float* grad, void* ws, size_t ws_bytes, celeste_stream_t stream);

/* loss (one double, accumulated) += mean over [batch][27] of weight_j (y - target)^2 and
 * dy = its gradient; weight [27] may be NULL (all ones). */
int celeste_cnn_mse(const float* y, const float* target, const float* weight, int batch, float* dy, double* loss,
                    celeste_stream_t stream);

/* One AdamW step (bias-corrected; decoupled weight decay) on the FP32 parameters, refreshing the
 * BF16 copy; m, v: FP32 moment buffers of param_count entries; step >= 1. */
int celeste_cnn_adamw(float* params, uint16_t* params_bf16, float* m, float* v, const float* grad, float lr,
                      float beta1, float beta2, float eps, float weight_decay, int step, celeste_stream_t stream);

/* Network input of every source of a bound problem: x [S][32][32][5] (BF16), band b taken from
 * the source's first patch in an image of band b, centred on its patch centre, pixel value
 * asinh((count - sky) / sqrt(sky)), zero where the band is missing or outside the image. */
int celeste_extract_patches(celeste_problem* p, uint16_t* x, celeste_stream_t stream);

/* Release the problem (not the caller's workspace).  NULL is ignored. */
void celeste_problem_destroy(celeste_problem* p);

const char* celeste_strerror(int code);
const char* celeste_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* CELESTE_H */
