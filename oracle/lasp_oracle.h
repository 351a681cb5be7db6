/* FP64 CPU oracle of the grouped spectral fit (test infrastructure only).
 *
 * This library is the slow, plain reference that the CUDA path is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the product path never does.  It shares no code, header or
 * table with the CUDA library.
 *
 * Every function follows the method of arXiv 2512.24840, section 2.2:
 *   basis + interpolator (Eq. 1), Gaussian broadening and shift (Eq. 5),
 *   multiplicative Legendre continuum by weighted least squares (Eq. 6),
 *   residual (Eq. 7), loss (Eq. 9, per-spectrum separable form), Adam with the
 *   three stop rules (stage 8) and the finite-difference covariance (stage 9).
 * Readings where the paper is silent are listed beside each function.
 */
#ifndef LASP_ORACLE_H
#define LASP_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_ST_CONV_TOL   1u   /* |l_t - l_{t-50}| < tol            */
#define ORC_ST_CONV_RISE  2u   /* loss rose on 50 consecutive steps */
#define ORC_ST_MAXSTEPS   4u   /* max_steps updates taken           */
#define ORC_ST_NONPOS     8u   /* continuum P b <= 0 on a used pixel */
#define ORC_ST_NONFINITE 16u   /* non-finite loss or gradient       */
#define ORC_ST_SINGULAR  32u   /* normal equations not positive definite */
#define ORC_ST_NODATA    64u   /* too few usable pixels             */

typedef struct {
    int K;                     /* number of basis terms                      */
    const signed char* exps;   /* K x 3 exponents of (u_T, u_g, u_f)          */
    double blo[3], bhi[3];     /* basis box: log10 Teff, log g, [Fe/H]       */
    double plo[5], phi[5];     /* parameter box (Teff, logg, FeH, RV, sigma)  */
    double dln;                /* ln-lambda step of the grid                 */
    int pad;                   /* H: model pixels beyond each observed end   */
    int n_pix;                 /* p: observed pixels                         */
    int deg;                   /* Legendre degree D (D+1 coefficients)       */
    const double* C;           /* K x (n_pix + 2 pad) coefficient table      */
    /* Piecewise emulator (Eq. 1 with Teff regimes f1..f5, sec. 3.1).  n_reg <= 1:
     * one regime with the basis box blo/bhi.  n_reg = 2 or 3: the rows of C
     * and exps are regime 0's reg_K[0] rows, then regime 1's, ...; regime r
     * uses the basis box rblo[r]/rbhi[r]; regimes r and r+1 blend linearly in
     * Teff on (tblend[2r], tblend[2r+1]]. */
    int n_reg;
    int reg_K[3];
    double rblo[3][3], rbhi[3][3];
    double tblend[4];
} orc_model;

typedef struct {
    double lr, beta1, beta2, eps, tol;
    int window, max_steps, edge_px;
    double quantile;
    int clean;          /* 1: Clean masking (Eq. 8) during the fit            */
    int clean_every;    /* mask updates at t = every, 2 every, ... (30)       */
    int clean_max;      /* at most this many updates (11)                     */
} orc_opts;

/* x in [-1,1]^5 -> physical parameters (linear box map). */
void orc_phys_from_x(const orc_model* M, const double* x, double* th);
void orc_x_from_phys(const orc_model* M, const double* th, double* x);

/* phi_k(theta) and d phi_k / d(Teff, logg, FeH) (K x 3, may be NULL).  For a
 * piecewise emulator each row is its regime's weight w_r(Teff) times its
 * monomial, so the Teff derivative includes the weight's slope. */
void orc_basis(const orc_model* M, const double* th, double* phi, double* dphi);

/* Sampled Gaussian kernel of Eq. 5 on s = -H..H (zero for |s| > h).
 * g, dg_dmu, dg_dsig have 2H+1 entries (s = -H at index 0).  Returns h. */
int orc_kernel(double mu, double sig, int H, double* g, double* dg_dmu, double* dg_dsig);

/* Legendre P_0..P_D at the nodes x_j = -1 + 2 j / p (Eq. 6); out p x (D+1). */
void orc_legendre(int p, int D, double* out);

/* F' = phi C (n_model), F'' (n_pix), continuum c = P b and model c * F''. */
void orc_model_flux(const orc_model* M, const double* th, const double* b,
                    double* Fp, double* Fpp, double* cont, double* model);

/* Vector-Jacobian product of model = (P b) * (G(mu,sigma) (x) phi(theta) C)
 * with respect to theta (physical, 5) and b (D+1), given gm = dL/dmodel. */
void orc_model_vjp(const orc_model* M, const double* th, const double* b,
                   const double* gm, double* gth, double* gb);

/* Median-type weight and weights (section 3.3 step 2; stage 7):
 * w = quantile of the flux over used pixels (linear interpolation between
 * order statistics); y = flux / w; W = A ivar / mean(ivar over used pixels),
 * zero on masked and edge pixels.  Returns the count of used pixels. */
int orc_prep(int n_pix, const float* flux, const float* ivar, const unsigned char* good,
             double quantile, int edge_px, double* y, double* W, double* w_out);

/* Loss l = sqrt(sum_j W_j eps_j^2 / p) with the continuum b solved by WLS
 * (Eqs. 6, 7, 9), and dl/dx (5) by the envelope theorem and the chain rule.
 * b_out (D+1), eps_out (p), cont_out (p) may be NULL.  Returns status bits. */
unsigned orc_eval(const orc_model* M, const double* y, const double* W, const double* x,
                  double* loss, double* grad_x, double* b_out, double* eps_out,
                  double* cont_out);

/* One Adam update (PyTorch semantics, bias-corrected) of n values at step
 * number t (1-based), followed by the box projection when clamp != 0. */
void orc_adam_update(int n, double* x, double* m, double* v, const double* g, int t,
                     double lr, double b1, double b2, double eps, int clamp);

/* Stop test after recording loss l_t (t = updates taken so far).
 * hist: the losses l_0..l_t.  Returns the ORC_ST_* bit that stops, or 0. */
unsigned orc_stop_rule(const double* hist, int t, int window, double tol, int max_steps);

/* Fit n spectra (rows of length n_pix) from theta0 (n x 5 physical).
 * Outputs theta (n x 5), loss (n), steps (n), status (n), b (n x (D+1)) or NULL.
 * Spectra are independent; OpenMP threads split them when threads > 1. */
void orc_fit(const orc_model* M, const orc_opts* O, int n, const float* flux,
             const float* ivar, const unsigned char* good, const double* theta0,
             double* theta, double* loss, int* steps, unsigned* status, double* b,
             int threads);

/* PAPER_JOINT reading of Eq. 9 (kept for comparison with the separable
 * default): one RMS over the group, L = sqrt(sum_i S_i / (N p)) with S_i =
 * sum_j W_ij eps_ij^2 over the N spectra still in the group.  Every
 * spectrum's parameters take Adam steps on dL/dx_i = (l_i / (N L)) dl_i/dx_i
 * (l_i the spectrum's own loss), and the stop rules run on L for the whole
 * group: one step count and one stop status for every spectrum that is still
 * in it.  A spectrum without data, or whose normal equations fail or whose
 * loss or gradient is not finite, leaves the group with its own status at
 * that step.  loss[i] = l_i at the stop; *loss_group = L at the stop.  The
 * spectra are evaluated in parallel, L is summed in index order. */
void orc_fit_joint(const orc_model* M, const orc_opts* O, int n, const float* flux,
                   const float* ivar, const unsigned char* good, const double* theta0,
                   double* theta, double* loss, int* steps, unsigned* status, double* loss_group,
                   int threads);

/* One spectrum: loss and gradient trajectory for a fixed number of steps with
 * the stop rules off (trajectory parity).  x_traj ((nsteps+1) x 5), loss_traj
 * (nsteps+1). */
void orc_fit_trajectory(const orc_model* M, const orc_opts* O, const float* flux,
                        const float* ivar, const unsigned char* good, const double* theta0,
                        int nsteps, double* x_traj, double* loss_traj);

/* Stage 9: central-difference Jacobian of the weighted residual sqrt(W) eps
 * w.r.t. physical theta (b re-solved at each probe; step 1e-4 of the half box
 * width), cov = (r.r / (n - 5)) (J^T J)^{-1}, sigma = sqrt(diag cov).
 * jac_out (n_pix x 5) may be NULL.  Returns status bits. */
unsigned orc_errors(const orc_model* M, const orc_opts* O, const float* flux,
                    const float* ivar, const unsigned char* good, const double* theta,
                    double* sigma, double* cov, double* jac_out);

/* Flux-conserving resampling (section 2.2 stage 3, Eqs. 2-4) of a spectrum F
 * on a linear grid lam_k = lam1 + k dlam (k = 0..q-1, pixel edges at
 * lam_k -+ dlam/2) onto the ln grid ln(lam_i) = ln_lam0 + i dln (i = 0..n_out-1,
 * bin edges at exp(ln_lam0 + (i -+ 1/2) dln)): cumulative integral of F at the
 * model edges (Eq. 2), linear interpolation of it at the target edges (Eq. 3),
 * difference over the edge spacing (Eq. 4).  Outside the model range the
 * cumulative integral is held constant (no flux). */
void orc_resample(int q, double lam1, double dlam, const double* F, int n_out, double ln_lam0,
                  double dln, double* out);

/* Clean outlier mask (stage 6, Eq. 8) from the weighted residual r_j =
 * sqrt(W_j) eps_j and the weighted model m_j = sqrt(W_j) c_j F''_j of one
 * spectrum.  used[j] = 1 for pixels currently used (predefined mask and the
 * previous Clean mask).  sigma = std of r over used pixels;
 * G_j = max(|m_j - m_{j-1}|, |m_j - m_{j+1}|) (existing neighbours only);
 * B: |r_j| - fshift G_j > k sigma, k = 3, relaxed to 4, 5, 7 while more than
 * 3% of the used pixels are flagged; C: neighbours of B outliers with
 * |r| - fshift G > 2 sigma; D: neighbours j' of flagged pixels j (B, C or D)
 * with r_j r_j' > 0, |r_j'| <= |r_j| and |r_j'| - fshift G_j' > sigma', sigma'
 * the std over used pixels not in B or C, repeated until unchanged (at most
 * 20 passes).  keep[j] = used[j] and not flagged.  Every quantity and every
 * comparison is in double precision.  Returns the k used. */
int orc_clean_mask(int p, const double* r, const double* m, const unsigned char* used, double fshift,
                   unsigned char* keep);

/* Curvature-aware fit (the paper's outlook, sec. 4.5): Levenberg-Marquardt
 * on x in [-1,1]^5 minimising S(x) = sum_j W_j eps_j^2 with the continuum
 * re-solved at every point (the same objective as Eq. 9).  At each iterate:
 * r = sqrt(W) eps, the Jacobian J of r w.r.t. x by central differences (step
 * 1e-4, as stage 9), A = J^T J, g = J^T r; parameters held at a bound by the
 * gradient are frozen; pred0 = g^T A^-1 g (the Gauss-Newton predicted
 * decrease).  Converged (status 1) when pred0 <= rtol S.  Otherwise trial
 * steps solve (A + lambda diag A) d = -g, x_t = clamp(x + d).  The gain ratio
 * rho of a trial is (S - S(x_t)) / pred when the step's predicted decrease
 * pred is at least 1e-6 S; below that S differences are not trusted and rho
 * compares pred0(x_t) with the merit the model predicts (requiring also
 * S(x_t) <= S(1 + 1e-6)).  rho > 0 accepts and scales lambda by
 * max(1/3, 1 - (2 rho - 1)^3) (floor 1e-12), nu = 2; otherwise lambda x nu,
 * nu x 2 (Nielsen's damping rule).  Ten rejections in a row stop (status 1);
 * max_iter accepted steps stop (status 4).  Outputs as orc_fit (iters =
 * accepted steps). */
void orc_fit_lm(const orc_model* M, const orc_opts* O, int n, const float* flux, const float* ivar,
                const unsigned char* good, const double* theta0, int max_iter, double rtol,
                double* theta, double* loss, int* iters, unsigned* status, int threads);

int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
