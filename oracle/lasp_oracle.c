/* FP64 CPU oracle of the grouped spectral fit -- test infrastructure only.
 *
 * Plain loops in double precision, written for a reader to check against
 * arXiv 2512.24840 section 2.2 by eye.  No blocking, fusion or reordering
 * beyond what the equations state.  Loaded only by the tests, the smoke check
 * and the benchmark's CPU-baseline leg; it shares nothing with the CUDA path.
 *
 * Readings of the paper used here (each also listed in the design notes):
 *  - loss: per spectrum l_i = sqrt(sum_j W_ij eps_ij^2 / p) (Eq. 9 with N = 1);
 *    the group objective is sum_i l_i, so Adam (elementwise) runs per spectrum.
 *  - W = A ivar / mean(ivar over used pixels); uniform ivar gives Eq. 9 exactly.
 *  - kernel (Eq. 5): F''_j = sum_{s=-h..h} g_s F'_{j+H-s}, g_s the sampled
 *    Gaussian exp(-(s-mu)^2 / 2 sigma^2) normalised to unit sum,
 *    h = ceil(|mu| + 5 sigma); mu = RV / (c dln), sigma = sigma_v / (c dln).
 *  - the model grid extends the observed one by H = pad pixels each side.
 *  - Legendre nodes x_j = -1 + 2 j / p, j = 0..p-1 (Eq. 6 as printed).
 *  - WLS weights of the continuum fit are the loss weights W.
 *  - stop rules (stage 8): after evaluating l_t: |l_t - l_{t-50}| < tol, or 50
 *    consecutive rises, or t = max_steps; the parameters returned are x_t.
 */
#include "lasp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define C_KMS 299792.458
#define NB_MAX 9               /* Legendre continuum terms supported: degree <= 8 */

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_phys_from_x(const orc_model* M, const double* x, double* th) {
    for (int k = 0; k < 5; ++k) th[k] = M->plo[k] + 0.5 * (x[k] + 1.0) * (M->phi[k] - M->plo[k]);
}

void orc_x_from_phys(const orc_model* M, const double* th, double* x) {
    for (int k = 0; k < 5; ++k) x[k] = 2.0 * (th[k] - M->plo[k]) / (M->phi[k] - M->plo[k]) - 1.0;
}

static double ipow(double u, int a) {
    double r = 1.0;
    for (int i = 0; i < a; ++i) r *= u;
    return r;
}

/* Weight of regime r of the piecewise emulator at Teff T (Eq. 1: f1 = cold,
 * f2 = cold-warm blend, f3 = warm, f4 = warm-hot blend, f5 = hot for three
 * regimes) and its slope dw/dT.  The weight rises linearly from 0 to 1 across
 * the blend interval shared with the cooler neighbour, is 1 up to the blend
 * interval shared with the hotter neighbour, falls linearly to 0 across it,
 * and is 0 beyond.  Intervals are open below and closed above. */
static void regime_weight(const orc_model* M, int r, double T, double* w, double* dw) {
    const double* tb = M->tblend;
    *w = 0.0;
    *dw = 0.0;
    if (r > 0) {
        double lo = tb[2 * r - 2], hi = tb[2 * r - 1];
        if (T <= lo) return;
        if (T <= hi) {
            *w = (T - lo) / (hi - lo);
            *dw = 1.0 / (hi - lo);
            return;
        }
    }
    if (r == M->n_reg - 1) {
        *w = 1.0;
        return;
    }
    double lo = tb[2 * r], hi = tb[2 * r + 1];
    if (T <= lo) {
        *w = 1.0;
    } else if (T <= hi) {
        *w = (hi - T) / (hi - lo);
        *dw = -1.0 / (hi - lo);
    }
}

/* Eq. 1: phi_k = w_r(Teff) u_T^a u_g^b u_f^c for row k of regime r, the u's
 * the basis variables (log10 Teff, log g, [Fe/H]) mapped linearly onto
 * [-1, 1] by the regime's box (one regime: w = 1, box blo/bhi). */
void orc_basis(const orc_model* M, const double* th, double* phi, double* dphi) {
    int n_reg = M->n_reg > 1 ? M->n_reg : 1;
    double v[3] = {log10(th[0]), th[1], th[2]};
    int k = 0;
    for (int r = 0; r < n_reg; ++r) {
        const double* lo = n_reg > 1 ? M->rblo[r] : M->blo;
        const double* hi = n_reg > 1 ? M->rbhi[r] : M->bhi;
        int Kr = n_reg > 1 ? M->reg_K[r] : M->K;
        double w = 1.0, dw = 0.0;
        if (n_reg > 1) regime_weight(M, r, th[0], &w, &dw);
        double u[3], du[3];
        for (int i = 0; i < 3; ++i) {
            u[i] = 2.0 * (v[i] - lo[i]) / (hi[i] - lo[i]) - 1.0;
            du[i] = 2.0 / (hi[i] - lo[i]);
        }
        du[0] /= th[0] * log(10.0);           /* d log10(Teff) / d Teff */
        for (int q = 0; q < Kr; ++q, ++k) {
            int a = M->exps[3 * k], b = M->exps[3 * k + 1], c = M->exps[3 * k + 2];
            double mono = ipow(u[0], a) * ipow(u[1], b) * ipow(u[2], c);
            phi[k] = w * mono;
            if (dphi) {
                double d0 = a ? a * ipow(u[0], a - 1) * ipow(u[1], b) * ipow(u[2], c) * du[0] : 0.0;
                dphi[3 * k + 0] = w * d0 + dw * mono;
                dphi[3 * k + 1] = b ? w * b * ipow(u[0], a) * ipow(u[1], b - 1) * ipow(u[2], c) * du[1] : 0.0;
                dphi[3 * k + 2] = c ? w * c * ipow(u[0], a) * ipow(u[1], b) * ipow(u[2], c - 1) * du[2] : 0.0;
            }
        }
    }
}

/* Eq. 5 kernel G(mu, sigma) of length 2 ceil(|mu| + 5 sigma) + 1. */
int orc_kernel(double mu, double sig, int H, double* g, double* dg_dmu, double* dg_dsig) {
    int h = (int)ceil(fabs(mu) + 5.0 * sig);
    if (h > H) h = H;
    if (h < 0) h = 0;
    int n = 2 * H + 1;
    double Z = 0.0, md = 0.0, mq = 0.0;
    for (int i = 0; i < n; ++i) {
        int s = i - H;
        g[i] = 0.0;
        if (s < -h || s > h) continue;
        g[i] = exp(-(s - mu) * (s - mu) / (2.0 * sig * sig));
        Z += g[i];
    }
    for (int i = 0; i < n; ++i) g[i] /= Z;
    for (int i = 0; i < n; ++i) {
        int s = i - H;
        md += g[i] * (s - mu) / (sig * sig);
        mq += g[i] * (s - mu) * (s - mu) / (sig * sig * sig);
    }
    for (int i = 0; i < n; ++i) {
        int s = i - H;
        if (dg_dmu) dg_dmu[i] = g[i] * ((s - mu) / (sig * sig) - md);
        if (dg_dsig) dg_dsig[i] = g[i] * ((s - mu) * (s - mu) / (sig * sig * sig) - mq);
    }
    return h;
}

/* Legendre polynomials by Bonnet's recursion at x_j = -1 + 2 j / p. */
void orc_legendre(int p, int D, double* out) {
    for (int j = 0; j < p; ++j) {
        double x = -1.0 + 2.0 * j / p;
        double* P = out + (size_t)j * (D + 1);
        P[0] = 1.0;
        if (D >= 1) P[1] = x;
        for (int n = 1; n < D; ++n) P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1);
    }
}

static void interp_and_broaden(const orc_model* M, const double* th, double* Fp, double* Fpp,
                               double* g, double* dgm, double* dgs, double* phi, double* dphi) {
    int H = M->pad, p = M->n_pix, nm = p + 2 * H;
    orc_basis(M, th, phi, dphi);
    for (int m = 0; m < nm; ++m) {                     /* Eq. 1: F' = phi C */
        double acc = 0.0;
        for (int k = 0; k < M->K; ++k) acc += phi[k] * M->C[(size_t)k * nm + m];
        Fp[m] = acc;
    }
    double mu = th[3] / (C_KMS * M->dln), sig = th[4] / (C_KMS * M->dln);
    orc_kernel(mu, sig, H, g, dgm, dgs);
    for (int j = 0; j < p; ++j) {                      /* Eq. 5: F'' = F' (x) G */
        double acc = 0.0;
        for (int s = -H; s <= H; ++s) acc += g[s + H] * Fp[j + H - s];
        Fpp[j] = acc;
    }
}

void orc_model_flux(const orc_model* M, const double* th, const double* b, double* Fp,
                    double* Fpp, double* cont, double* model) {
    int H = M->pad, p = M->n_pix, D = M->deg;
    double* g = malloc(sizeof(double) * (2 * H + 1));
    double* phi = malloc(sizeof(double) * M->K);
    double* P = malloc(sizeof(double) * (size_t)p * (D + 1));
    interp_and_broaden(M, th, Fp, Fpp, g, NULL, NULL, phi, NULL);
    orc_legendre(p, D, P);
    for (int j = 0; j < p; ++j) {                      /* Eq. 6: (P b) * F'' */
        double c = 0.0;
        for (int d = 0; d <= D; ++d) c += b[d] * P[(size_t)j * (D + 1) + d];
        if (cont) cont[j] = c;
        if (model) model[j] = c * Fpp[j];
    }
    free(g); free(phi); free(P);
}

/* Backward through the broadening and the interpolator, given dL/dF''.
 * Adds to gth[0..4] (physical parameters). */
static void backprop_fpp(const orc_model* M, const double* Fp,
                         const double* gFpp, const double* dgm, const double* dgs,
                         const double* g, const double* dphi, double* gth) {
    int H = M->pad, p = M->n_pix, nm = p + 2 * H;
    double gmu = 0.0, gsig = 0.0;
    for (int j = 0; j < p; ++j) {
        for (int s = -H; s <= H; ++s) {
            gmu += gFpp[j] * dgm[s + H] * Fp[j + H - s];
            gsig += gFpp[j] * dgs[s + H] * Fp[j + H - s];
        }
    }
    double* gFp = calloc(nm, sizeof(double));
    for (int j = 0; j < p; ++j)
        for (int s = -H; s <= H; ++s) gFp[j + H - s] += gFpp[j] * g[s + H];
    for (int k = 0; k < M->K; ++k) {
        double gphi = 0.0;
        for (int m = 0; m < nm; ++m) gphi += gFp[m] * M->C[(size_t)k * nm + m];
        for (int i = 0; i < 3; ++i) gth[i] += gphi * dphi[3 * k + i];
    }
    gth[3] += gmu / (C_KMS * M->dln);
    gth[4] += gsig / (C_KMS * M->dln);
    free(gFp);
}

void orc_model_vjp(const orc_model* M, const double* th, const double* b, const double* gm,
                   double* gth, double* gb) {
    int H = M->pad, p = M->n_pix, nm = p + 2 * H, D = M->deg;
    double* Fp = malloc(sizeof(double) * nm);
    double* Fpp = malloc(sizeof(double) * p);
    double* g = malloc(sizeof(double) * (2 * H + 1));
    double* dgm = malloc(sizeof(double) * (2 * H + 1));
    double* dgs = malloc(sizeof(double) * (2 * H + 1));
    double* phi = malloc(sizeof(double) * M->K);
    double* dphi = malloc(sizeof(double) * 3 * M->K);
    double* P = malloc(sizeof(double) * (size_t)p * (D + 1));
    double* gFpp = malloc(sizeof(double) * p);
    interp_and_broaden(M, th, Fp, Fpp, g, dgm, dgs, phi, dphi);
    orc_legendre(p, D, P);
    for (int d = 0; d <= D; ++d) gb[d] = 0.0;
    for (int j = 0; j < p; ++j) {
        double c = 0.0;
        for (int d = 0; d <= D; ++d) c += b[d] * P[(size_t)j * (D + 1) + d];
        for (int d = 0; d <= D; ++d) gb[d] += gm[j] * Fpp[j] * P[(size_t)j * (D + 1) + d];
        gFpp[j] = gm[j] * c;
    }
    for (int k = 0; k < 5; ++k) gth[k] = 0.0;
    backprop_fpp(M, Fp, gFpp, dgm, dgs, g, dphi, gth);
    free(Fp); free(Fpp); free(g); free(dgm); free(dgs); free(phi); free(dphi); free(P); free(gFpp);
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

int orc_prep(int n_pix, const float* flux, const float* ivar, const unsigned char* good,
             double quantile, int edge_px, double* y, double* W, double* w_out) {
    double* v = malloc(sizeof(double) * n_pix);
    int n = 0;
    double isum = 0.0;
    for (int j = 0; j < n_pix; ++j) {
        int use = good[j] && ivar[j] > 0.0f && isfinite(flux[j]) && isfinite(ivar[j]);
        if (use) { v[n++] = flux[j]; isum += ivar[j]; }
    }
    double w = NAN;
    if (n > 0) {
        qsort(v, n, sizeof(double), cmp_double);
        double pos = quantile * (n - 1);
        int lo = (int)floor(pos);
        if (lo >= n - 1) w = v[n - 1];
        else w = v[lo] + (pos - lo) * (v[lo + 1] - v[lo]);
    }
    double imean = n > 0 ? isum / n : 0.0;
    int n_obj = 0;
    for (int j = 0; j < n_pix; ++j) {
        int use = good[j] && ivar[j] > 0.0f && isfinite(flux[j]) && isfinite(ivar[j]);
        int edge = j < edge_px || j >= n_pix - edge_px;
        if (use && !edge && w > 0.0) {
            y[j] = flux[j] / w;
            W[j] = ivar[j] / imean;
            ++n_obj;
        } else {
            y[j] = 0.0;
            W[j] = 0.0;
        }
    }
    *w_out = w;
    free(v);
    return n_obj;
}

/* Cholesky solve of the (n x n) SPD system A z = r.  Returns 0 if A is not
 * numerically positive definite. */
static int chol_solve(int n, const double* A, const double* r, double* z) {
    double L[NB_MAX * NB_MAX], t[NB_MAX];
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return 0;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * t[k];
        t[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = t[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * z[k];
        z[i] = s / L[i * n + i];
    }
    return 1;
}

/* Eq. 6 by weighted least squares: minimise sum_j W_j (y_j - (P b)_j F''_j)^2. */
static int solve_continuum(int p, int D, const double* P, const double* Fpp, const double* y,
                           const double* W, double* b) {
    int n = D + 1;
    double G[NB_MAX * NB_MAX], r[NB_MAX];
    for (int a = 0; a < n; ++a) {
        r[a] = 0.0;
        for (int c = 0; c < n; ++c) G[a * n + c] = 0.0;
    }
    for (int j = 0; j < p; ++j) {
        const double* Pj = P + (size_t)j * n;
        for (int a = 0; a < n; ++a) {
            r[a] += W[j] * Fpp[j] * y[j] * Pj[a];
            for (int c = 0; c < n; ++c) G[a * n + c] += W[j] * Fpp[j] * Fpp[j] * Pj[a] * Pj[c];
        }
    }
    return chol_solve(n, G, r, b);
}

unsigned orc_eval(const orc_model* M, const double* y, const double* W, const double* x,
                  double* loss, double* grad_x, double* b_out, double* eps_out, double* cont_out) {
    int H = M->pad, p = M->n_pix, nm = p + 2 * H, D = M->deg;
    unsigned st = 0;
    double th[5], b[NB_MAX];
    for (int d = 0; d < NB_MAX; ++d) b[d] = NAN;
    double* Fp = malloc(sizeof(double) * nm);
    double* Fpp = malloc(sizeof(double) * p);
    double* g = malloc(sizeof(double) * (2 * H + 1));
    double* dgm = malloc(sizeof(double) * (2 * H + 1));
    double* dgs = malloc(sizeof(double) * (2 * H + 1));
    double* phi = malloc(sizeof(double) * M->K);
    double* dphi = malloc(sizeof(double) * 3 * M->K);
    double* P = malloc(sizeof(double) * (size_t)p * (D + 1));
    double* gFpp = malloc(sizeof(double) * p);
    orc_phys_from_x(M, x, th);
    interp_and_broaden(M, th, Fp, Fpp, g, dgm, dgs, phi, dphi);
    orc_legendre(p, D, P);
    if (!solve_continuum(p, D, P, Fpp, y, W, b)) {
        st |= ORC_ST_SINGULAR;
        *loss = NAN;
        for (int k = 0; k < 5; ++k) grad_x[k] = 0.0;
        goto done;
    }
    double S = 0.0;
    for (int j = 0; j < p; ++j) {                      /* Eq. 7 residual */
        double c = 0.0;
        for (int d = 0; d <= D; ++d) c += b[d] * P[(size_t)j * (D + 1) + d];
        double e = y[j] - c * Fpp[j];
        S += W[j] * e * e;
        if (W[j] > 0.0 && c <= 0.0) st |= ORC_ST_NONPOS;
        if (eps_out) eps_out[j] = e;
        if (cont_out) cont_out[j] = c;
        gFpp[j] = -W[j] * e * c;                       /* d(S/2)/dF''_j, b held at b* */
    }
    double l = sqrt(S / p);                            /* Eq. 9, one spectrum */
    *loss = l;
    double scale = l > 0.0 ? 1.0 / (p * l) : 0.0;      /* dl/dS = 1 / (2 p l) */
    for (int j = 0; j < p; ++j) gFpp[j] *= scale;
    double gth[5] = {0, 0, 0, 0, 0};
    backprop_fpp(M, Fp, gFpp, dgm, dgs, g, dphi, gth);
    for (int k = 0; k < 5; ++k) grad_x[k] = gth[k] * 0.5 * (M->phi[k] - M->plo[k]);
    if (!isfinite(l)) st |= ORC_ST_NONFINITE;
    for (int k = 0; k < 5; ++k) if (!isfinite(grad_x[k])) st |= ORC_ST_NONFINITE;
done:
    if (b_out) for (int d = 0; d <= D; ++d) b_out[d] = b[d];
    free(Fp); free(Fpp); free(g); free(dgm); free(dgs); free(phi); free(dphi); free(P); free(gFpp);
    return st;
}

/* torch.optim.Adam update with default options except lr, then projection
 * onto the box [-1, 1] (the parameters are normalised to that range). */
void orc_adam_update(int n, double* x, double* m, double* v, const double* g, int t, double lr,
                     double b1, double b2, double eps, int clamp) {
    double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
    for (int i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double denom = sqrt(v[i]) / sqrt(bc2) + eps;
        x[i] -= (lr / bc1) * m[i] / denom;
        if (clamp) {
            if (x[i] < -1.0) x[i] = -1.0;
            if (x[i] > 1.0) x[i] = 1.0;
        }
    }
}

unsigned orc_stop_rule(const double* hist, int t, int window, double tol, int max_steps) {
    if (t >= window) {
        if (fabs(hist[t] - hist[t - window]) < tol) return ORC_ST_CONV_TOL;
        int rising = 1;
        for (int i = t - window + 1; i <= t; ++i)
            if (!(hist[i] > hist[i - 1])) { rising = 0; break; }
        if (rising) return ORC_ST_CONV_RISE;
    }
    if (t >= max_steps) return ORC_ST_MAXSTEPS;
    return 0;
}

/* Clean update after evaluating at x_t (stage 6 schedule of stage 8): from
 * the residual eps at x_t, the new mask takes effect from step t + 1.  The
 * weighted residual and model enter the mask rules in double precision. */
static void clean_update(int p, const double* y, const double* Wb, const double* eps, int update,
                         unsigned char* keep, double* W) {
    double* r = malloc(sizeof(double) * p);
    double* m = malloc(sizeof(double) * p);
    unsigned char* used = malloc(p);
    for (int j = 0; j < p; ++j) {
        double s = sqrt(Wb[j]);
        r[j] = s * eps[j];
        m[j] = s * (y[j] - eps[j]);
        used[j] = Wb[j] > 0.0 && keep[j];
    }
    orc_clean_mask(p, r, m, used, update == 1 ? 0.5 : 0.2, keep);
    for (int j = 0; j < p; ++j) W[j] = keep[j] ? Wb[j] : 0.0;
    free(r); free(m); free(used);
}

static void fit_one(const orc_model* M, const orc_opts* O, const float* flux, const float* ivar,
                    const unsigned char* good, const double* theta0, double* theta, double* loss,
                    int* steps, unsigned* status, double* b_out) {
    int p = M->n_pix, D = M->deg;
    double* y = malloc(sizeof(double) * p);
    double* W = malloc(sizeof(double) * p);
    double* Wb = malloc(sizeof(double) * p);
    double* eps = malloc(sizeof(double) * p);
    unsigned char* keep = malloc(p);
    double* hist = malloc(sizeof(double) * (O->max_steps + 1));
    double w, x[5], m[5] = {0}, v[5] = {0}, g[5], b[NB_MAX];
    int n_obj = orc_prep(p, flux, ivar, good, O->quantile, O->edge_px, y, W, &w);
    for (int k = 0; k < 5; ++k) theta[k] = theta0[k];
    *loss = NAN;
    *steps = 0;
    if (n_obj < D + 1 + 5 || !(w > 0.0) || !isfinite(w)) {
        *status = ORC_ST_NODATA;
        goto out;
    }
    orc_x_from_phys(M, theta0, x);
    for (int k = 0; k < 5; ++k) x[k] = x[k] < -1.0 ? -1.0 : (x[k] > 1.0 ? 1.0 : x[k]);
    for (int j = 0; j < p; ++j) {
        Wb[j] = W[j];
        keep[j] = 1;
    }
    for (int t = 0;; ++t) {
        double l;
        unsigned st = orc_eval(M, y, W, x, &l, g, b, eps, NULL);
        if (st & (ORC_ST_SINGULAR | ORC_ST_NONFINITE)) {
            *status = st;
            *loss = l;
            *steps = t;
            orc_phys_from_x(M, x, theta);
            break;
        }
        hist[t] = l;
        unsigned stop = orc_stop_rule(hist, t, O->window, O->tol, O->max_steps);
        if (stop) {
            *status = stop | (st & ORC_ST_NONPOS);
            *loss = l;
            *steps = t;
            orc_phys_from_x(M, x, theta);
            if (b_out) for (int d = 0; d <= D; ++d) b_out[d] = b[d];
            break;
        }
        orc_adam_update(5, x, m, v, g, t + 1, O->lr, O->beta1, O->beta2, O->eps, 1);
        if (O->clean && t > 0 && O->clean_every > 0 && t % O->clean_every == 0 &&
            t / O->clean_every <= O->clean_max)
            clean_update(p, y, Wb, eps, t / O->clean_every, keep, W);
    }
out:
    free(y); free(W); free(Wb); free(eps); free(keep); free(hist);
}

void orc_fit(const orc_model* M, const orc_opts* O, int n, const float* flux, const float* ivar,
             const unsigned char* good, const double* theta0, double* theta, double* loss,
             int* steps, unsigned* status, double* b, int threads) {
    int p = M->n_pix, nb = M->deg + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int i = 0; i < n; ++i) {
        fit_one(M, O, flux + (size_t)i * p, ivar + (size_t)i * p, good + (size_t)i * p,
                theta0 + 5 * i, theta + 5 * i, loss + i, steps + i, status + i,
                b ? b + (size_t)i * nb : NULL);
    }
}

void orc_fit_joint(const orc_model* M, const orc_opts* O, int n, const float* flux, const float* ivar,
                   const unsigned char* good, const double* theta0, double* theta, double* loss,
                   int* steps, unsigned* status, double* loss_group, int threads) {
    int p = M->n_pix, D = M->deg;
    double* y = malloc(sizeof(double) * (size_t)n * p);
    double* W = malloc(sizeof(double) * (size_t)n * p);
    double* x = calloc((size_t)n * 5, sizeof(double));
    double* m = calloc((size_t)n * 5, sizeof(double));
    double* v = calloc((size_t)n * 5, sizeof(double));
    double* g = calloc((size_t)n * 5, sizeof(double));
    double* l = calloc((size_t)n, sizeof(double));
    unsigned* st = calloc((size_t)n, sizeof(unsigned));
    int* active = calloc((size_t)n, sizeof(int));
    double* hist = malloc(sizeof(double) * (O->max_steps + 1));
    *loss_group = NAN;
    for (int i = 0; i < n; ++i) {
        double w;
        int n_obj = orc_prep(p, flux + (size_t)i * p, ivar + (size_t)i * p, good + (size_t)i * p,
                             O->quantile, O->edge_px, y + (size_t)i * p, W + (size_t)i * p, &w);
        for (int k = 0; k < 5; ++k) theta[5 * i + k] = theta0[5 * i + k];
        loss[i] = NAN;
        steps[i] = 0;
        status[i] = 0;
        if (n_obj < D + 1 + 5 || !(w > 0.0) || !isfinite(w)) {
            status[i] = ORC_ST_NODATA;
            continue;
        }
        orc_x_from_phys(M, theta0 + 5 * i, x + 5 * i);
        for (int k = 0; k < 5; ++k) x[5 * i + k] = x[5 * i + k] < -1.0 ? -1.0 : (x[5 * i + k] > 1.0 ? 1.0 : x[5 * i + k]);
        active[i] = 1;
    }
    for (int t = 0;; ++t) {
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads > 0 ? threads : 1)
        for (int i = 0; i < n; ++i)
            if (active[i])
                st[i] = orc_eval(M, y + (size_t)i * p, W + (size_t)i * p, x + 5 * i, l + i, g + 5 * i, NULL,
                                 NULL, NULL);
        int na = 0;
        double ssum = 0.0;
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            if (st[i] & (ORC_ST_SINGULAR | ORC_ST_NONFINITE)) {
                status[i] = st[i];
                loss[i] = l[i];
                steps[i] = t;
                orc_phys_from_x(M, x + 5 * i, theta + 5 * i);
                active[i] = 0;
                continue;
            }
            ++na;
            ssum += (double)p * l[i] * l[i];
        }
        if (na == 0) break;
        const double L = sqrt(ssum / ((double)na * p));
        hist[t] = L;
        unsigned stop = orc_stop_rule(hist, t, O->window, O->tol, O->max_steps);
        if (stop) {
            for (int i = 0; i < n; ++i) {
                if (!active[i]) continue;
                status[i] = stop | (st[i] & ORC_ST_NONPOS);
                loss[i] = l[i];
                steps[i] = t;
                orc_phys_from_x(M, x + 5 * i, theta + 5 * i);
            }
            *loss_group = L;
            break;
        }
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            double gj[5];
            const double c = l[i] / ((double)na * L);
            for (int k = 0; k < 5; ++k) gj[k] = c * g[5 * i + k];
            orc_adam_update(5, x + 5 * i, m + 5 * i, v + 5 * i, gj, t + 1, O->lr, O->beta1, O->beta2,
                            O->eps, 1);
        }
    }
    free(y); free(W); free(x); free(m); free(v); free(g); free(l); free(st); free(active); free(hist);
}

void orc_fit_trajectory(const orc_model* M, const orc_opts* O, const float* flux,
                        const float* ivar, const unsigned char* good, const double* theta0,
                        int nsteps, double* x_traj, double* loss_traj) {
    int p = M->n_pix;
    double* y = malloc(sizeof(double) * p);
    double* W = malloc(sizeof(double) * p);
    double w, x[5], m[5] = {0}, v[5] = {0}, g[5];
    orc_prep(p, flux, ivar, good, O->quantile, O->edge_px, y, W, &w);
    orc_x_from_phys(M, theta0, x);
    for (int k = 0; k < 5; ++k) x[k] = x[k] < -1.0 ? -1.0 : (x[k] > 1.0 ? 1.0 : x[k]);
    for (int t = 0; t <= nsteps; ++t) {
        double l;
        orc_eval(M, y, W, x, &l, g, NULL, NULL, NULL);
        for (int k = 0; k < 5; ++k) x_traj[5 * t + k] = x[k];
        loss_traj[t] = l;
        if (t < nsteps) orc_adam_update(5, x, m, v, g, t + 1, O->lr, O->beta1, O->beta2, O->eps, 1);
    }
    free(y); free(W);
}

/* Weighted residual r = sqrt(W) eps at physical theta with b re-solved. */
static int weighted_resid(const orc_model* M, const double* y, const double* W,
                          const double* th, double* r) {
    double x[5], l, g[5], b[NB_MAX];
    int p = M->n_pix;
    double* eps = malloc(sizeof(double) * p);
    orc_x_from_phys(M, th, x);
    unsigned st = orc_eval(M, y, W, x, &l, g, b, eps, NULL);
    for (int j = 0; j < p; ++j) r[j] = sqrt(W[j]) * eps[j];
    free(eps);
    return !(st & ORC_ST_SINGULAR);
}

/* Gauss-Jordan inverse with partial pivoting of a 5 x 5 matrix. */
static int inv5(const double* A, double* Ai) {
    double a[5][10];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 10; ++j) a[i][j] = j < 5 ? A[i * 5 + j] : (j - 5 == i ? 1.0 : 0.0);
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        for (int i = c + 1; i < 5; ++i) if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
        if (!(fabs(a[piv][c]) > 0.0)) return 0;
        if (piv != c)
            for (int j = 0; j < 10; ++j) { double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
        double d = a[c][c];
        for (int j = 0; j < 10; ++j) a[c][j] /= d;
        for (int i = 0; i < 5; ++i) {
            if (i == c) continue;
            double f = a[i][c];
            for (int j = 0; j < 10; ++j) a[i][j] -= f * a[c][j];
        }
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) Ai[i * 5 + j] = a[i][j + 5];
    return 1;
}

unsigned orc_errors(const orc_model* M, const orc_opts* O, const float* flux, const float* ivar,
                    const unsigned char* good, const double* theta, double* sigma, double* cov,
                    double* jac_out) {
    int p = M->n_pix;
    unsigned st = 0;
    double* y = malloc(sizeof(double) * p);
    double* W = malloc(sizeof(double) * p);
    double* r0 = malloc(sizeof(double) * p);
    double* rp = malloc(sizeof(double) * p);
    double* rm = malloc(sizeof(double) * p);
    double* J = malloc(sizeof(double) * (size_t)p * 5);
    double w;
    int n_obj = orc_prep(p, flux, ivar, good, O->quantile, O->edge_px, y, W, &w);
    for (int k = 0; k < 5; ++k) sigma[k] = NAN;
    for (int k = 0; k < 25; ++k) cov[k] = NAN;
    if (n_obj <= 5 || !(w > 0.0)) { st |= ORC_ST_NODATA; goto out; }
    if (!weighted_resid(M, y, W, theta, r0)) { st |= ORC_ST_SINGULAR; goto out; }
    for (int k = 0; k < 5; ++k) {
        double h = 1e-4 * 0.5 * (M->phi[k] - M->plo[k]);
        double tp[5], tm[5];
        for (int i = 0; i < 5; ++i) tp[i] = tm[i] = theta[i];
        tp[k] += h;
        tm[k] -= h;
        if (!weighted_resid(M, y, W, tp, rp) || !weighted_resid(M, y, W, tm, rm)) {
            st |= ORC_ST_SINGULAR;
            goto out;
        }
        for (int j = 0; j < p; ++j) J[(size_t)j * 5 + k] = (rp[j] - rm[j]) / (2.0 * h);
    }
    double rr = 0.0, JtJ[25], inv[25];
    for (int j = 0; j < p; ++j) rr += r0[j] * r0[j];
    for (int a = 0; a < 5; ++a)
        for (int c = 0; c < 5; ++c) {
            double s = 0.0;
            for (int j = 0; j < p; ++j) s += J[(size_t)j * 5 + a] * J[(size_t)j * 5 + c];
            JtJ[a * 5 + c] = s;
        }
    if (!inv5(JtJ, inv)) { st |= ORC_ST_SINGULAR; goto out; }
    double s2 = rr / (n_obj - 5);
    for (int k = 0; k < 25; ++k) cov[k] = s2 * inv[k];
    for (int k = 0; k < 5; ++k) sigma[k] = sqrt(cov[k * 5 + k]);
    if (jac_out) memcpy(jac_out, J, sizeof(double) * (size_t)p * 5);
out:
    free(y); free(W); free(r0); free(rp); free(rm); free(J);
    return st;
}

void orc_resample(int q, double lam1, double dlam, const double* F, int n_out, double ln_lam0,
                  double dln, double* out) {
    /* Eq. 2: cumulative integral at the q + 1 model edges */
    double* cum = malloc(sizeof(double) * (q + 1));
    cum[0] = 0.0;
    for (int k = 0; k < q; ++k) cum[k + 1] = cum[k] + F[k] * dlam;
    double e0 = lam1 - 0.5 * dlam;
    /* Eq. 3: linear interpolation of the cumulative integral at a target edge */
    double* edge_val = malloc(sizeof(double) * (n_out + 1));
    double* edge = malloc(sizeof(double) * (n_out + 1));
    for (int i = 0; i <= n_out; ++i) {
        double x = exp(ln_lam0 + (i - 0.5) * dln);
        edge[i] = x;
        double u = (x - e0) / dlam;            /* position in model-edge units */
        if (u <= 0.0) edge_val[i] = cum[0];
        else if (u >= q) edge_val[i] = cum[q];
        else {
            int k = (int)floor(u);
            if (k >= q) k = q - 1;
            double f = u - k;
            edge_val[i] = cum[k] + f * (cum[k + 1] - cum[k]);
        }
    }
    /* Eq. 4: difference over the edge spacing */
    for (int i = 0; i < n_out; ++i) out[i] = (edge_val[i + 1] - edge_val[i]) / (edge[i + 1] - edge[i]);
    free(cum);
    free(edge_val);
    free(edge);
}

/* Population standard deviation of r over the pixels with sel[j] != 0
 * (double precision throughout). */
static double std_sel(int p, const double* r, const unsigned char* sel) {
    double s1 = 0.0, s2 = 0.0;
    int n = 0;
    for (int j = 0; j < p; ++j)
        if (sel[j]) { s1 += r[j]; s2 += r[j] * r[j]; ++n; }
    if (n == 0) return 0.0;
    double mean = s1 / n, var = s2 / n - mean * mean;
    return sqrt(var > 0.0 ? var : 0.0);
}

/* Clean mask of stage 6 (Eq. 8), every quantity and comparison in double
 * precision.  B: |r_j| - f G_j > k sigma with G_j the larger model jump to an
 * existing neighbour, k = 3 raised to 4, 5, 7 while more than 3% of the used
 * pixels are flagged; C: used neighbours of B pixels above 2 sigma; D:
 * same-sign neighbours with no larger |r| above sigma' (the std over used
 * pixels in neither B nor C), grown until unchanged, at most 20 passes. */
int orc_clean_mask(int p, const double* r, const double* m, const unsigned char* used, double fshift,
                   unsigned char* keep) {
    double* G = malloc(sizeof(double) * p);
    double* lhs = malloc(sizeof(double) * p);
    unsigned char* B = calloc(p, 1);
    unsigned char* flag = calloc(p, 1);
    unsigned char* sel = malloc(p);
    for (int j = 0; j < p; ++j) {
        double g = 0.0;
        if (j > 0) g = fabs(m[j] - m[j - 1]);
        if (j < p - 1 && fabs(m[j] - m[j + 1]) > g) g = fabs(m[j] - m[j + 1]);
        G[j] = g;
        lhs[j] = fabs(r[j]) - fshift * G[j];
    }
    int n_used = 0;
    for (int j = 0; j < p; ++j) n_used += used[j] ? 1 : 0;
    const double sigma = std_sel(p, r, used);
    /* B with k = 3, relaxed while more than 3% of the used pixels are flagged */
    const double ks[4] = {3.0, 4.0, 5.0, 7.0};
    int kk = 0;
    for (; kk < 4; ++kk) {
        int nb = 0;
        for (int j = 0; j < p; ++j) {
            B[j] = used[j] && lhs[j] > ks[kk] * sigma;
            nb += B[j];
        }
        if (!(nb > 0.03 * n_used)) break;
    }
    if (kk == 4) kk = 3;
    /* C: neighbours of B outliers */
    for (int j = 0; j < p; ++j) flag[j] = B[j];
    for (int j = 0; j < p; ++j) {
        if (!used[j] || B[j]) continue;
        int nbB = (j > 0 && B[j - 1]) || (j < p - 1 && B[j + 1]);
        if (nbB && lhs[j] > 2.0 * sigma) flag[j] = 1;
    }
    /* sigma' over used pixels not in B or C */
    for (int j = 0; j < p; ++j) sel[j] = used[j] && !flag[j];
    const double sigp = std_sel(p, r, sel);
    /* D: grow along same-sign, non-increasing residuals above sigma' */
    unsigned char* nxt = malloc(p);
    for (int it = 0; it < 20; ++it) {
        int changed = 0;
        for (int j = 0; j < p; ++j) {
            nxt[j] = flag[j];
            if (flag[j] || !used[j]) continue;
            for (int d = -1; d <= 1; d += 2) {
                int i = j + d;
                if (i < 0 || i >= p || !flag[i]) continue;
                if (r[i] * r[j] > 0.0 && fabs(r[j]) <= fabs(r[i]) && lhs[j] > sigp) {
                    nxt[j] = 1;
                    changed = 1;
                }
            }
        }
        for (int j = 0; j < p; ++j) flag[j] = nxt[j];
        if (!changed) break;
    }
    for (int j = 0; j < p; ++j) keep[j] = used[j] && !flag[j];
    free(G); free(lhs); free(B); free(flag); free(sel); free(nxt);
    return (int)ks[kk];
}

/* S(x) and the weighted residual r = sqrt(W) eps at x (continuum re-solved). */
static int lm_eval(const orc_model* M, const double* y, const double* W, const double* x, double* S,
                   double* r) {
    double l, g[5], b[NB_MAX];
    int p = M->n_pix;
    double* eps = malloc(sizeof(double) * p);
    unsigned st = orc_eval(M, y, W, x, &l, g, b, eps, NULL);
    double s = 0.0;
    for (int j = 0; j < p; ++j) {
        double rj = sqrt(W[j]) * eps[j];
        if (r) r[j] = rj;
        s += rj * rj;
    }
    free(eps);
    *S = s;
    return !(st & ORC_ST_SINGULAR) && isfinite(s);
}

/* Gauss-Newton quantities at x: S, r, the central-difference Jacobian J of r
 * w.r.t. x (step 1e-4), and the reduced system (Ar, gr) in which parameters
 * held at a bound of the box by the gradient (x = -1 with g > 0, x = +1 with
 * g < 0) are frozen (unit row and column, zero gradient).  pred0 = g^T A^-1 g
 * is the decrease of S that the undamped Gauss-Newton step predicts
 * (infinite when A is not positive definite).  Returns 0 when an evaluation
 * fails. */
static int lm_full(const orc_model* M, const double* y, const double* W, const double* x, double* r,
                   double* rp, double* rm, double* J, double* S, double* Ar, double* gr, double* pred0) {
    int p = M->n_pix;
    if (!lm_eval(M, y, W, x, S, r)) return 0;
    for (int k = 0; k < 5; ++k) {
        double xp[5], xm[5], Sp, Sm, h = 1e-4;
        for (int q = 0; q < 5; ++q) xp[q] = xm[q] = x[q];
        xp[k] += h;
        xm[k] -= h;
        if (!lm_eval(M, y, W, xp, &Sp, rp) || !lm_eval(M, y, W, xm, &Sm, rm)) return 0;
        for (int j = 0; j < p; ++j) J[(size_t)j * 5 + k] = (rp[j] - rm[j]) / (2.0 * h);
    }
    double A[25], g[5], d0[5];
    int fr[5];
    for (int a = 0; a < 5; ++a) {
        g[a] = 0.0;
        for (int j = 0; j < p; ++j) g[a] += J[(size_t)j * 5 + a] * r[j];
        for (int c = 0; c < 5; ++c) {
            double s = 0.0;
            for (int j = 0; j < p; ++j) s += J[(size_t)j * 5 + a] * J[(size_t)j * 5 + c];
            A[a * 5 + c] = s;
        }
    }
    for (int a = 0; a < 5; ++a) fr[a] = !((x[a] <= -1.0 && g[a] > 0.0) || (x[a] >= 1.0 && g[a] < 0.0));
    for (int a = 0; a < 5; ++a) {
        gr[a] = fr[a] ? g[a] : 0.0;
        for (int c = 0; c < 5; ++c) Ar[a * 5 + c] = (fr[a] && fr[c]) ? A[a * 5 + c] : (a == c ? 1.0 : 0.0);
    }
    double mg[5];
    for (int a = 0; a < 5; ++a) mg[a] = -gr[a];
    if (chol_solve(5, Ar, mg, d0)) {
        double s = 0.0;
        for (int a = 0; a < 5; ++a) s -= gr[a] * d0[a];
        *pred0 = s;
    } else {
        *pred0 = INFINITY;
    }
    return 1;
}

static void lm_one(const orc_model* M, const orc_opts* O, const float* flux, const float* ivar,
                   const unsigned char* good, const double* theta0, int max_iter, double rtol,
                   double* theta, double* loss, int* iters, unsigned* status) {
    /* S differences below this fraction of S are not trusted: there the
     * trial is judged by the Gauss-Newton merit pred0 instead. */
    const double eta = 1e-6;
    int p = M->n_pix;
    double* y = malloc(sizeof(double) * p);
    double* W = malloc(sizeof(double) * p);
    double* r = malloc(sizeof(double) * p);
    double* rp = malloc(sizeof(double) * p);
    double* rm = malloc(sizeof(double) * p);
    double* J = malloc(sizeof(double) * (size_t)p * 5);
    double w, x[5], S, Ar[25], gr[5], pred0, lam = 1e-3, nu = 2.0;
    int n_obj = orc_prep(p, flux, ivar, good, O->quantile, O->edge_px, y, W, &w);
    for (int k = 0; k < 5; ++k) theta[k] = theta0[k];
    *loss = NAN;
    *iters = 0;
    *status = 0;
    if (n_obj < M->deg + 1 + 5 || !(w > 0.0) || !isfinite(w)) {
        *status = ORC_ST_NODATA;
        goto out;
    }
    orc_x_from_phys(M, theta0, x);
    for (int k = 0; k < 5; ++k) x[k] = x[k] < -1.0 ? -1.0 : (x[k] > 1.0 ? 1.0 : x[k]);
    if (!lm_full(M, y, W, x, r, rp, rm, J, &S, Ar, gr, &pred0)) { *status = ORC_ST_SINGULAR; goto done; }
    for (int it = 0;; ++it) {
        *iters = it;
        if (pred0 <= rtol * S) { *status = ORC_ST_CONV_TOL; break; }
        if (it >= max_iter) { *status = ORC_ST_MAXSTEPS; break; }
        int accepted = 0, have_full = 0;
        double xn[5], Sn = S, An[25], gn[5], pn = pred0;
        for (int trial = 0; trial < 10 && !accepted; ++trial) {
            double Ad[25], rhs[5], d[5], rho = -1.0;
            for (int q = 0; q < 25; ++q) Ad[q] = Ar[q];
            for (int a = 0; a < 5; ++a) {
                Ad[a * 5 + a] += lam * Ar[a * 5 + a];
                rhs[a] = -gr[a];
            }
            if (chol_solve(5, Ad, rhs, d)) {
                /* predicted decrease of S for d: -(2 g.d + d^T A d) */
                double pred = 0.0;
                for (int a = 0; a < 5; ++a) {
                    double Adv = 0.0;
                    for (int c = 0; c < 5; ++c) Adv += Ar[a * 5 + c] * d[c];
                    pred -= 2.0 * gr[a] * d[a] + d[a] * Adv;
                }
                for (int q = 0; q < 5; ++q) {
                    xn[q] = x[q] + d[q];
                    xn[q] = xn[q] < -1.0 ? -1.0 : (xn[q] > 1.0 ? 1.0 : xn[q]);
                }
                if (pred >= eta * S) {
                    /* gain ratio of S */
                    double St;
                    have_full = 0;
                    if (lm_eval(M, y, W, xn, &St, NULL)) rho = (S - St) / pred;
                } else {
                    /* gain ratio of the merit pred0: the model's gradient after
                     * the step is g + A d = lambda diag(A) d */
                    have_full = 1;
                    if (lm_full(M, y, W, xn, r, rp, rm, J, &Sn, An, gn, &pn) && Sn <= S * (1.0 + eta)) {
                        double gm[5], z[5], pm = 0.0;
                        for (int a = 0; a < 5; ++a) gm[a] = lam * Ar[a * 5 + a] * d[a];
                        if (chol_solve(5, Ar, gm, z))
                            for (int a = 0; a < 5; ++a) pm += gm[a] * z[a];
                        double den = pred0 - pm > 0.0 ? pred0 - pm : pred0;
                        rho = (pred0 - pn) / den;
                    }
                }
            }
            if (rho > 0.0) {
                /* Nielsen's damping update */
                double t = 2.0 * rho - 1.0, f = 1.0 - t * t * t;
                lam *= f > 1.0 / 3.0 ? f : 1.0 / 3.0;
                if (lam < 1e-12) lam = 1e-12;
                nu = 2.0;
                accepted = 1;
            } else {
                lam *= nu;
                nu *= 2.0;
            }
        }
        if (!accepted) { *status = ORC_ST_CONV_TOL; break; }
        for (int q = 0; q < 5; ++q) x[q] = xn[q];
        if (have_full) {
            S = Sn;
            pred0 = pn;
            for (int q = 0; q < 25; ++q) Ar[q] = An[q];
            for (int a = 0; a < 5; ++a) gr[a] = gn[a];
        } else if (!lm_full(M, y, W, x, r, rp, rm, J, &S, Ar, gr, &pred0)) {
            *status = ORC_ST_SINGULAR;
            *iters = it + 1;
            break;
        }
    }
done:
    orc_phys_from_x(M, x, theta);
    *loss = sqrt(S / p);
out:
    free(y); free(W); free(r); free(rp); free(rm); free(J);
}

void orc_fit_lm(const orc_model* M, const orc_opts* O, int n, const float* flux, const float* ivar,
                const unsigned char* good, const double* theta0, int max_iter, double rtol,
                double* theta, double* loss, int* iters, unsigned* status, int threads) {
    int p = M->n_pix;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int i = 0; i < n; ++i)
        lm_one(M, O, flux + (size_t)i * p, ivar + (size_t)i * p, good + (size_t)i * p, theta0 + 5 * i,
               max_iter, rtol, theta + 5 * i, loss + i, iters + i, status + i);
}
