/* lasp.h -- C-ABI of the GB300 grouped spectral-fitting library (liblasp.so).
 *
 * The library fits many observed spectra at once with the LASP-Adam method of
 * arXiv 2512.24840 (section 2.2): each spectrum's model is a polynomial
 * interpolator in (Teff, log g, [Fe/H]) (Eq. 1), broadened and shifted by a
 * sampled Gaussian kernel on a ln-lambda grid (Eq. 5), multiplied by a
 * Legendre continuum solved by weighted least squares (Eq. 6); the
 * inverse-variance-weighted residual (Eq. 7) gives a per-spectrum RMS loss
 * (Eq. 9) that Adam minimises until each spectrum meets one of the three stop
 * rules (stage 8).  Parameter errors come from linear error propagation
 * (stage 9).
 *
 * Conventions
 *  - Every call returns LASP_OK (0) or a negative LASP_E* code; calls never
 *    abort and never print.  lasp_strerror() names a code.
 *  - Array arguments documented "device" must be CUDA device pointers on the
 *    current device; "host" ones are host memory.  The caller owns every
 *    batch, result and output buffer.  The library owns the interpolator
 *    handle (its table copies), and any scratch it allocates per call on the
 *    given stream (stream-ordered, released before the call's work ends).
 *  - Calls taking `stream` (a cudaStream_t, NULL = legacy default stream)
 *    enqueue their work on it and return without synchronising, except where
 *    noted.  Arguments are validated on the host before anything is enqueued.
 *  - Row-major layouts.  Physical parameters theta are ordered
 *    (Teff [K], log g [dex], [Fe/H] [dex], RV [km/s], sigma_v [km/s]).
 *  - Per-spectrum outcomes are reported in status bits, not return codes.
 *  - Bounded waits.  The tensor-core kernels wait on memory barriers for their
 *    bulk copies and MMAs; every such wait gives up after a fixed number of
 *    polls (far longer than any correct wait), sets a device flag, lets its
 *    copies and MMAs in flight complete and returns.  Where the flag is read
 *    back is stated per call; it surfaces as LASP_ETIMEOUT, and fits stepped
 *    after it get LASP_ST_TIMEOUT instead of a converged status.
 */
#ifndef LASP_H
#define LASP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define LASP_OK        0
#define LASP_EINVAL   (-1)   /* bad argument (NULL, size, degree, option)     */
#define LASP_ENOMEM   (-2)   /* device allocation failed                       */
#define LASP_ECUDA    (-3)   /* a CUDA runtime call or launch failed           */
#define LASP_ETIMEOUT (-4)   /* a bounded device wait gave up                  */
#define LASP_EGRID    (-5)   /* grid/table mismatch: pad too small for the box */
#define LASP_ENODEV   (-6)   /* no usable sm_103 device                        */
#define LASP_EBUSY    (-7)   /* a server ring is full: retry after a tick      */

/* ---- per-spectrum status bits (lasp_result.status) ---- */
#define LASP_ST_CONV_TOL   1u   /* |l_t - l_{t-window}| < tol (stage 8 rule 2)        */
#define LASP_ST_CONV_RISE  2u   /* loss rose on `window` consecutive steps (rule 3)   */
#define LASP_ST_MAXSTEPS   4u   /* max_steps updates taken (rule 1)                   */
#define LASP_ST_NONPOS     8u   /* continuum P b <= 0 on a used pixel at the result   */
#define LASP_ST_NONFINITE 16u   /* loss or gradient not finite; fit stopped           */
#define LASP_ST_SINGULAR  32u   /* continuum normal equations not positive definite  */
#define LASP_ST_NODATA    64u   /* fewer than D+1+5 usable pixels, or weight <= 0    */
#define LASP_ST_RUNNING  128u   /* (slot state only) fit not finished yet             */
#define LASP_ST_TIMEOUT  256u   /* a bounded device wait gave up while this fit was
                                   stepped: the fit ended there, its result is not
                                   valid (theta = the last parameters, loss NaN)     */

/* ---- arithmetic of the interpolator contraction and the normal equations ---- */
#define LASP_PREC_FP32   0   /* FP32 CUDA-core contraction, FP32 normal equations      */
#define LASP_PREC_TF32   1   /* tcgen05 TF32 contraction, FP32 accumulate               */
#define LASP_PREC_BF16   2   /* tcgen05 BF16 contraction, FP32 accumulate               */
#define LASP_PREC_TF32X3 3   /* tcgen05 3-pass split TF32 (about FP32 accurate)         */

/* ---- precision of the per-spectrum normal equations (lasp_fit_opts.fp64_normal_eq) ----
 * Each thread forms the products of its own pixels in FP32 and sums them in
 * FP32 (16 pixels a thread); the options differ in how those partial sums are
 * added across the CTA and how the (D+1)x(D+1) system is solved. */
#define LASP_NE_FP32 0   /* FP32 sums, FP32 Cholesky solve                          */
#define LASP_NE_FF   1   /* float-float: warps added in exact two-sums (~48 bits);
                            FP32 Cholesky refined once with a float-float residual */
#define LASP_NE_FP64 2   /* FP64: the partial sums widened to double, added by
                            double shuffles, Cholesky solve in double            */

/* Interpolator description (Eq. 1 with one polynomial regime; see
 * lasp_piecewise_desc for Teff regimes).
 * The model grid is the observed ln-lambda grid extended by `pad` pixels on
 * each side: n_model = n_pix + 2 pad.  The basis variables
 * v = (log10 Teff, log g, [Fe/H]) are mapped onto [-1, 1] by
 * u = 2 (v - basis_lo) / (basis_hi - basis_lo) - 1 and
 * phi_k = u_T^a u_g^b u_f^c with (a, b, c) = exps[k].
 * box_lo/box_hi bound the physical parameters; the fit works on x in [-1,1]^5
 * mapped linearly onto the box (stage 8 rescaling). */
typedef struct {
    int K;                  /* basis terms, 1..32                                 */
    int n_pix;              /* observed pixels p >= 16, with the model grid
                               n_pix + 2 pad <= 8192 (16 model pixels a thread
                               of a 512-thread CTA); larger is LASP_EINVAL       */
    int pad;                /* H >= ceil(max|mu| + 5 max sigma) over the box,
                               at most 47 (2H+1 <= 95 taps)                      */
    double dln;             /* ln-lambda step of the grid (> 0)                   */
    const int8_t* exps;     /* host, K x 3 non-negative exponents (<= 8)          */
    double basis_lo[3], basis_hi[3];
    double box_lo[5], box_hi[5];
} lasp_interp_desc;

typedef struct lasp_interp_s* lasp_interp;   /* opaque, library-owned */

/* Upload the interpolator table (Eq. 1) and build its device images.
 * coeff: host, K x n_model float32 row-major (C_k,m).  Builds the FP32 table,
 * the TF32 hi/lo and BF16 tile images used by the tensor-core contraction.
 * Synchronous: returns once the table is on the device, so the handle may be
 * used on any stream.  Errors: LASP_EINVAL (bad desc), LASP_EGRID (pad smaller than
 * the widest kernel reachable in the box), LASP_ENOMEM, LASP_ECUDA,
 * LASP_ENODEV.  On success *out owns device memory until lasp_free_interp. */
int lasp_init_interp(const lasp_interp_desc* desc, const float* coeff, lasp_interp* out);
void lasp_free_interp(lasp_interp h);

/* Piecewise interpolator (Eq. 1 with Teff regimes; sec. 3.1): n_reg
 * polynomial regimes ordered by Teff, coolest first (the paper's emulator has
 * cold, warm and hot models with 25, 26 and 19 terms).  Regime r has K[r]
 * terms, its own exponents and its own basis box.  Regimes r and r+1 overlap
 * on (teff_blend[2r], teff_blend[2r+1]]: there the model is the linear blend
 * in Teff, (1 - t) F_r + t F_{r+1} with t = (Teff - teff_blend[2r]) /
 * (teff_blend[2r+1] - teff_blend[2r]); elsewhere it is the one regime whose
 * range holds Teff (Teff <= teff_blend[0]: regime 0; (teff_blend[2r-1],
 * teff_blend[2r]]: regime r; above the last bound: the last regime).  The
 * paper's five ranges are teff_blend = {4000, 4550, 7000, 9000}.  The model is
 * continuous in Teff; its Teff derivative jumps at the bounds.
 * coeff: host, (K[0] + ... + K[n_reg-1]) x n_model float32, the regimes'
 * tables stacked in order.  exps: host, the same rows x 3.  At most 96 rows
 * in all.  Handles made here serve every entry point that takes a handle:
 * the tensor-core paths stack the regimes' rows into up to three K blocks of
 * 32 terms (the rows of regimes inactive at a spectrum's Teff enter with zero
 * weight, a masked grouped contraction).  Errors as lasp_init_interp, plus
 * LASP_EINVAL for n_reg outside 1..3, a regime without terms, or bounds not
 * strictly increasing. */
typedef struct {
    int n_reg;              /* 1..3                                            */
    int K[3];               /* terms per regime, each >= 1, sum <= 96          */
    int n_pix;              /* p >= 16 with p + 2 pad <= 8192                  */
    int pad;                /* H, as lasp_interp_desc                          */
    double dln;             /* ln-lambda step of the grid (> 0)                */
    const int8_t* exps;     /* host, (sum K) x 3 non-negative exponents (<= 8) */
    double basis_lo[3][3], basis_hi[3][3];   /* per regime, as lasp_interp_desc */
    double teff_blend[4];   /* 2 (n_reg - 1) strictly increasing Teff bounds   */
    double box_lo[5], box_hi[5];
} lasp_piecewise_desc;

int lasp_init_interp_piecewise(const lasp_piecewise_desc* desc, const float* coeff,
                               lasp_interp* out);

/* A batch of N observed spectra on the interpolator's grid (device, row-major
 * N x n_pix).  good: 1 = pixel used (the mask A of Eq. 8), 0 = masked.
 * Pixels with good = 0, ivar <= 0 or non-finite values are not used.
 * theta0: device, N x 5 physical initial parameters (clipped to the box). */
typedef struct {
    int N;
    int n_pix;              /* must equal the descriptor's n_pix */
    const float* flux;
    const float* ivar;
    const uint8_t* good;
    const float* theta0;
} lasp_batch;

/* Fit options.  lasp_default_opts() gives the paper's settings: lr 0.1, Adam
 * betas (0.9, 0.999), eps 1e-8, tol 1e-5 over a window of 50 steps, at most
 * 5000 steps (stage 8), median weight (quantile 0.5, section 3.3), Legendre
 * degree 6, no edge pixels dropped, FP32 arithmetic, No Clean (Clean: mask
 * updates every 30 steps, at most 11).
 * Clean (stage 6): after evaluating step t = every, 2 every, ... (at most
 * clean_max updates) the mask is recomputed from the weighted residual
 * sqrt(W) eps and model sqrt(W) c F'' at x_t (f_shift 0.5 on the first
 * update, 0.2 after; see lasp_clean_mask) starting from the pixels in use,
 * and applies from step t + 1. */
typedef struct {
    float lr, beta1, beta2, eps, tol;
    int window;             /* 1..64                                   */
    int max_steps;          /* 0..1000000                              */
    int legendre_deg;       /* D, one of 2, 4, 6, 8                    */
    int edge_px;            /* pixels at each end left out of the loss */
    float quantile;         /* w_i = this quantile of the used flux    */
    int precision;          /* LASP_PREC_*                              */
    int fp64_normal_eq;     /* precision of the continuum normal equations (Eq. 6) and
                               of the stage-9 sums, LASP_NE_*: FP32 (0), float-float
                               (1, about 48 bits without FP64 instructions) or FP64
                               (2).  The name is kept for the ABI; only
                               LASP_NE_FP64 issues FP64 instructions. */
    int clean;              /* 1: Clean outlier masking (stage 6, Eq. 8); Adam
                               fits with the separable loss, every precision */
    int clean_every;        /* mask update every this many steps (30)   */
    int clean_max;          /* at most this many updates (11)           */
    int optimizer;          /* LASP_OPT_ADAM (stage 8) or LASP_OPT_LM    */
    int loss_mode;          /* LASP_LOSS_SEPARABLE or LASP_LOSS_JOINT    */
} lasp_fit_opts;

/* Optimisers.  LASP_OPT_ADAM: the paper's Adam with the three stop rules.
 * LASP_OPT_LM: the curvature-aware step of the paper's outlook (sec. 4.5):
 * Levenberg-Marquardt on x for S = sum W eps^2 with the continuum re-solved,
 * the Jacobian of sqrt(W) eps taken analytically (as for stage 9), FP64
 * normal equations; parameters held on a bound by the gradient are frozen;
 * Nielsen's damping rule.  The fit ends with status LASP_ST_CONV_TOL when the
 * Gauss-Newton predicted decrease g^T A^-1 g falls to tol * S (1e-10 suits
 * FP32 model values; the Adam default 1e-5 stops far too early) or when ten
 * damped trials in a row fail, and with LASP_ST_MAXSTEPS after max_steps
 * accepted steps (steps = accepted steps).  FP32 precision only; no Clean. */
#define LASP_OPT_ADAM 0
#define LASP_OPT_LM   1

/* Loss modes.  LASP_LOSS_SEPARABLE (default): each spectrum minimises its own
 * l_i = sqrt(sum_j W eps^2 / p) with its own stop rules, so its result does
 * not depend on the batch.  LASP_LOSS_JOINT: Eq. 9 read literally, one RMS
 * over the group L = sqrt(sum_i S_i / (N p)); spectrum i steps on dL/dx_i =
 * (l_i / (N L)) dl_i/dx_i, and the stop rules run on L: every spectrum still
 * in the group stops at the same step with the same status (spectra whose
 * normal equations fail leave the group at that step).  JOINT needs a step
 * over all spectra at once: it runs on the grouped tensor-core pipeline
 * (precision != LASP_PREC_FP32, Adam, no Clean), else LASP_EINVAL. */
#define LASP_LOSS_SEPARABLE 0
#define LASP_LOSS_JOINT     1

void lasp_default_opts(lasp_fit_opts* o);

/* Results (device, caller-owned).  theta N x 5 physical, loss N (Eq. 9 per
 * spectrum), steps N (updates taken), status N (LASP_ST_* bits).
 * cont_coeff: N x (D+1) continuum coefficients b for the normalised flux
 * y = flux / w, or NULL.  weight: N values of w, or NULL. */
typedef struct {
    float* theta;
    float* loss;
    int32_t* steps;
    uint32_t* status;
    float* cont_coeff;
    float* weight;
} lasp_result;

/* Fit every spectrum of the batch to convergence (stage 8).  At
 * LASP_PREC_FP32 a preprocessing kernel prepares every spectrum, then one
 * fused persistent kernel runs all Adam steps with four spectra per CTA
 * (each table value loaded once for the four); each spectrum stops on its own
 * rule and its place goes to the next spectrum at once.  Device workspace of
 * about 8 n_pix bytes a spectrum comes from the stream's memory pool for the
 * call.  Asynchronous on `stream` at LASP_PREC_FP32.  At a tensor-core
 * precision the steps run as replays of a captured graph of 8 steps, and the
 * call reads the active count (and the timeout flag) after each replay, so
 * it returns when the fit is done; LASP_ETIMEOUT when a bounded wait gave up
 * (the fits stepped from then on carry LASP_ST_TIMEOUT). */
int lasp_fit_batch(lasp_interp h, const lasp_batch* batch, const lasp_fit_opts* opts,
                   lasp_result* result, void* stream);

/* Resumable fit slots, the device side of continuous batching (stage 8 run
 * in chunks).  A slot pool owns, on the device, n_slots observation buffers
 * (flux, ivar, good: n_pix each, theta0), the Adam state of each slot and its
 * results, so a fit keeps its optimiser state resident between launches and a
 * slot whose spectrum stops is refilled with the next one.  A fit split over
 * several lasp_slots_step launches performs exactly the arithmetic of
 * lasp_fit_batch: its result is bitwise the same and does not depend on the
 * other slots.  Status of a slot: LASP_ST_RUNNING while fitting, the final
 * LASP_ST_* bits once stopped, 0 when never used. */
typedef struct lasp_slots_s* lasp_slots;          /* opaque, library-owned */

/* Allocates the pool (device memory ~ n_slots x (9 n_pix + 480) bytes plus a
 * staging copy of the observation buffers).  opts are copied.  Synchronous:
 * returns once the pool's device memory is initialised, so the first admit
 * may go on any stream, a non-blocking one included.
 * opts->precision LASP_PREC_FP32: the fused FP32 fit kernel steps the slots,
 * four per CTA; each slot also keeps its preprocessed y, W rows (8 bytes a
 * pixel, n_pix rounded up to 16), written when the slot is admitted.
 * A tensor-core precision: the grouped pipeline runs over the slots (served
 * mixed precision; Legendre degree 6, FP32 or float-float normal equations;
 * about 50 n_pix more bytes per slot); its steps go in chunks of 8, so a step
 * call's budget is rounded up to a multiple of 8.  Clean: each slot keeps its Clean mask in
 * device memory between steps (in its W row), so the updates fall on the same
 * steps as in a one-shot fit at the same precision.  The joint loss:
 * LASP_EINVAL. */
int lasp_slots_create(lasp_interp h, int n_slots, const lasp_fit_opts* opts, lasp_slots* out);
void lasp_slots_free(lasp_slots s);

/* Admit `count` spectra into the given slot indices (host int32, distinct,
 * 0 <= idx < n_slots).  flux, ivar: host count x n_pix float32; good: host
 * count x n_pix uint8; theta0: host count x 5 float32.  The rows are copied
 * host -> device on `stream` (pinned host memory makes the copy asynchronous)
 * and scattered into the slots, which become LASP_ST_RUNNING; an FP32 pool
 * also preprocesses them there (a spectrum with too few usable pixels gets its
 * final LASP_ST_NODATA result at once).  The host buffers must stay unchanged
 * until the stream passes this call. */
int lasp_slots_admit(lasp_slots s, int count, const int32_t* slot_idx, const float* flux,
                     const float* ivar, const uint8_t* good, const float* theta0, void* stream);

/* Run at most `budget` (>= 1) Adam steps on every running slot (one launch of
 * the fused fit kernel, whose lanes take the running slots in turn; slots that
 * stop write their results). */
int lasp_slots_step(lasp_slots s, int budget, void* stream);

/* As lasp_slots_step, with the caller's count of running slots: the launch is
 * sized to it, so a lightly used pool leaves the other SMs free (for another
 * pool's step on another stream).  Any n_running >= 1 gives the same results;
 * the true count gives the best schedule.  LASP_EINVAL for n_running < 1. */
int lasp_slots_step_running(lasp_slots s, int budget, int n_running, void* stream);

/* Copy every slot's theta (n_slots x 5), loss, steps, status and weight to
 * host buffers (any may be NULL) on `stream`.  In a tensor-core pool a
 * bounded wait that gave up during a step call ends every fit that call
 * stepped with status LASP_ST_TIMEOUT (the flag is cleared at the start of
 * each step call). */
int lasp_slots_fetch(lasp_slots s, float* theta, float* loss, int32_t* steps, uint32_t* status,
                     float* weight, void* stream);

/* ---- continuous-batching server: a native scheduler over slot pools ----
 * One lane per interpolator (one wavelength grid): a slot pool, a CUDA stream
 * and a pinned submission ring of `ring` requests.  lasp_server_submit copies
 * one request (host arrays) into its lane's ring and may be called from any
 * thread, also while another thread is inside lasp_server_tick.
 * lasp_server_tick runs one scheduling tick: on every lane it admits waiting
 * requests (FIFO) into free slots, runs at most `chunk` Adam steps on the
 * running slots (the lanes' streams overlap on the GPU), fetches status and
 * results, waits for its lanes, and moves the finished fits to the result
 * queue, freeing their slots.  Call tick from one thread at a time.
 * lasp_server_poll pops up to `max` finished results.  A fit split into
 * chunks does exactly the arithmetic of a one-shot lasp_fit_batch, so a
 * served result is bitwise the one the same spectrum gets alone.  Times are
 * steady-clock nanoseconds (submit and the end of the retiring tick).  The
 * paper fits fixed groups; this request loop has no counterpart there. */
typedef struct lasp_server_s* lasp_server;   /* opaque, library-owned */

typedef struct {
    int64_t tag;            /* the caller's tag given to lasp_server_submit */
    int lane;
    float theta[5];         /* physical parameters                       */
    float loss;
    int32_t steps;
    uint32_t status;        /* LASP_ST_* */
    int64_t t_submit_ns, t_done_ns;
} lasp_served;

/* n_lanes (1..8) lanes: interps[l] (handles stay owned by the caller and must
 * outlive the server), n_slots[l] >= 1 slots and ring[l] >= 1 pinned request
 * entries each; opts and chunk (>= 1 Adam steps per tick) apply to every
 * lane.  Synchronous.  Errors: LASP_EINVAL, LASP_ENOMEM, LASP_ECUDA. */
int lasp_server_create(int n_lanes, const lasp_interp* interps, const int* n_slots, const int* ring,
                       const lasp_fit_opts* opts, int chunk, lasp_server* out);
void lasp_server_destroy(lasp_server s);

/* Copy one request into lane `lane`'s ring: flux, ivar (n_pix float32), good
 * (n_pix uint8), theta0 (5 float32 physical), all host memory that may be
 * reused on return.  `tag` is returned with the result.  LASP_EBUSY when the
 * ring is full (nothing is copied). */
int lasp_server_submit(lasp_server s, int lane, const float* flux, const float* ivar,
                       const uint8_t* good, const float* theta0, int64_t tag);

/* Copy n requests (rows of n x n_pix flux, ivar float32, n x n_pix good uint8,
 * n x 5 theta0 float32, all host memory that may be reused on return; tags[n])
 * into lane `lane`'s ring in row order, under one lock and with one submit
 * time.  Takes as many rows as the ring has room for, from the first:
 * *n_taken receives that count.  Returns LASP_OK when all n were taken,
 * LASP_EBUSY when fewer were (the rest were not copied), LASP_EINVAL for a
 * bad handle, lane, n < 0 or a NULL pointer (n_taken always; the arrays when
 * n > 0).  Equivalent to n lasp_server_submit calls. */
int lasp_server_submit_n(lasp_server s, int lane, int n, const float* flux, const float* ivar,
                         const uint8_t* good, const float* theta0, const int64_t* tags, int* n_taken);

/* One scheduling tick (see above); *n_finished (may be NULL) receives the
 * number of fits retired in it.  Blocks until the tick's GPU work is done.
 * Returns LASP_ETIMEOUT when a fit retired in this tick carries
 * LASP_ST_TIMEOUT (its result is still queued, with that status). */
int lasp_server_tick(lasp_server s, int* n_finished);

/* Pop up to max finished results into out (host); *n receives the count. */
int lasp_server_poll(lasp_server s, lasp_served* out, int max, int* n);

/* Requests submitted and not yet retired (waiting in rings or running). */
int lasp_server_pending(lasp_server s, int64_t* n);

/* Stage 9 parameter uncertainties at theta (device, N x 5 physical, e.g. the
 * fitted values): Jacobian J of the weighted residual sqrt(W) eps w.r.t. the
 * physical parameters with the continuum re-solved (variable projection),
 * cov = (r.r / (n - 5)) (J^T J)^{-1} with n the used pixels.  The sums (the
 * normal equations, J^T J, r.r) are added across the CTA in float-float, or
 * in FP64 when opts->fp64_normal_eq is LASP_NE_FP64; the 5x5 inverse and the
 * scale are computed in FP64.  sigma: device N x 5 = sqrt(diag cov).
 * cov: device N x 25 FP64 or NULL.  status: device N or NULL (LASP_ST_*). */
int lasp_errors(lasp_interp h, const lasp_batch* batch, const lasp_fit_opts* opts,
                const float* theta, float* sigma, double* cov, uint32_t* status,
                void* stream);

/* Forward model of Eqs. 1, 5, 6 without the fit: model = (P b) * (G (x) phi C).
 * theta: device N x 5 physical; b: device N x (deg+1); model: device N x n_pix. */
int lasp_forward(lasp_interp h, int N, const float* theta, const float* b, int deg,
                 float* model, void* stream);

/* Vector-Jacobian product of lasp_forward (the hand-written adjoint): given
 * gmodel = dL/dmodel (device N x n_pix) returns gtheta (device N x 5, physical
 * units) and gb (device N x (deg+1)). */
int lasp_backward(lasp_interp h, int N, const float* theta, const float* b, int deg,
                  const float* gmodel, float* gtheta, float* gb, void* stream);

/* The interpolator contraction alone (Eq. 1): Fp = phi(theta) C, device
 * N x n_model output, with the arithmetic of `precision` (LASP_PREC_*).
 * At LASP_PREC_FP32 asynchronous.  At a tensor-core precision synchronous:
 * the call waits for its kernel and returns LASP_ETIMEOUT when a bounded
 * wait gave up; the outputs of the tiles not computed are then NaN. */
int lasp_interp_eval(lasp_interp h, int N, const float* theta, float* Fp, int precision,
                     void* stream);

/* Allocation-free form of lasp_interp_eval for the tensor-core precisions
 * (LASP_PREC_TF32, LASP_PREC_BF16, LASP_PREC_TF32X3).  The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * device memory -- for example code running inside a framework that owns all
 * device memory through its own pool, or a serving loop with a fixed memory
 * budget, where a cudaMalloc would break the budget or stall other streams
 * (cudaMalloc can synchronise the device).  It needs no lasp_interp handle
 * (creating one allocates) and calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * desc: host, as for lasp_init_interp.  coeff: device, K x n_model FP32 table
 * (caller-owned input).  theta: device N x 5 physical.  Fp: device N x n_model
 * output.  The swizzled table images and the kernel's wait-timeout flag live
 * in one static device array of LASP_STATIC_MAX_MODEL_PIX / 128 tiles
 * (3 MiB + 256 B per GPU that loads the library, held until exit); n_model
 * above LASP_STATIC_MAX_MODEL_PIX is rejected with LASP_EINVAL.
 *
 * The first call on a device looks up the array's device address (with that
 * device current) and zeroes its timeout flag; make that first call before
 * any stream capture.  Every call shares the array and rewrites it: calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads on one device) race and must be serialised by the caller.
 * A bounded wait that gives up writes NaN into the outputs of the tiles it
 * did not compute and leaves the flag set; the next call made outside stream
 * capture reads the flag after the work already on `stream` (a host wait on
 * that stream), clears it and returns LASP_ETIMEOUT without doing its own
 * work.  Errors: LASP_EINVAL, LASP_EGRID, LASP_ENODEV, LASP_ECUDA,
 * LASP_ETIMEOUT.  Its kernels run asynchronously on `stream`. */
#define LASP_STATIC_MAX_MODEL_PIX 8192
int lasp_interp_eval_static(const lasp_interp_desc* desc, const float* coeff, int N,
                            const float* theta, float* Fp, int precision, void* stream);

/* Flux-conserving resampling of an interpolator table from a linear
 * wavelength grid onto the library's ln-lambda grid (section 2.2 stage 3,
 * Eqs. 2-4).  The operation is linear in the flux and does not depend on
 * theta, so it is applied once to every table row and the resampled table is
 * then passed to lasp_init_interp (zero cost per Adam step).
 * coeff_lin: device K x q float32, model pixel k centred at lam1 + k dlam
 * (Angstrom) with edges at +- dlam/2.  coeff_out: device K x n_out float32,
 * output pixel i centred at exp(ln_lam0 + i dln) with edges at
 * exp(ln_lam0 + (i +- 1/2) dln).  Each output is the mean flux of the
 * piecewise-constant model over its bin -- exactly the difference of the
 * cumulative integral interpolated at the bin edges (Eqs. 2-4) -- computed as
 * overlap integrals in FP64; no flux outside the model range.  Asynchronous. */
int lasp_resample_linear(int K, int q, double lam1, double dlam, const float* coeff_lin, int n_out,
                         double ln_lam0, double dln, float* coeff_out, void* stream);

/* Clean outlier mask (stage 6, Eq. 8) of N spectra from their weighted
 * residual r = sqrt(W) eps and weighted model m = sqrt(W) c F'' (device
 * N x p float32) and the pixels in use (device N x p uint8, 1 = used):
 * sigma = std of r over used pixels; G_j = max |m_j - m_{j+-1}| (existing
 * neighbours); B: |r| - fshift G > k sigma, k = 3 relaxed to 4, 5, 7 while
 * more than 3% of the used pixels are flagged; C: neighbours of B outliers
 * with |r| - fshift G > 2 sigma; D: neighbours j' of flagged pixels j with
 * r_j r_j' > 0, |r_j'| <= |r_j| and |r_j'| - fshift G_j' > sigma' (std over
 * used pixels not in B or C), repeated until unchanged, at most 20 passes.
 * keep: device N x p uint8 = used and not flagged; k_used: device N int32
 * (the k of B) or NULL.  p <= 8192.  Asynchronous. */
int lasp_clean_mask(int N, int p, const float* r, const float* m, const uint8_t* used, float fshift,
                    uint8_t* keep, int32_t* k_used, void* stream);

/* Number of kernels the last call on this thread enqueued (for accounting). */
int lasp_last_launches(void);

/* Per-kernel device time, for measurement.  lasp_profile(1) switches it on
 * (process-wide; 0 switches it off).  While it is on, lasp_fit_batch,
 * lasp_errors and the curvature-aware fit bracket each kernel they launch
 * with CUDA events on their stream and wait for it, so every kernel is timed
 * on its own (the tensor-core fit then launches its steps one by one instead
 * of replaying the step graph); calls become synchronous.  The slot calls
 * time their kernels too, and their host-device copies as the entries
 * "slots_admit_h2d" (one per lasp_slots_admit) and "slots_fetch_d2h" (one
 * per lasp_slots_fetch).  lasp_profile_read
 * copies up to `max` entries (one per kernel name: launches and total device
 * milliseconds since the last read) into out, *n the count, and clears the
 * table. */
typedef struct {
    char name[48];
    int32_t launches;
    double ms;
} lasp_kernel_time;
int lasp_profile(int on);
int lasp_profile_read(lasp_kernel_time* out, int max, int* n);

/* Testing hook for the timeout path: with polls >= 0 the first table-copy
 * wait of every CTA of the tensor-core kernels launched (or captured) from
 * then on gives up after `polls` polls -- a wait issued before any MMA, whose
 * copy is then drained under the normal limit before the CTA exits; polls < 0
 * restores the normal limits.  Process-wide.  Always LASP_OK. */
int lasp_test_wait_limit(int polls);

const char* lasp_strerror(int code);
int lasp_version(void);

#ifdef __cplusplus
}
#endif
#endif
