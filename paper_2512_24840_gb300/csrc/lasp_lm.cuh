// Curvature-aware fit (the paper's outlook, sec. 4.5): Levenberg-Marquardt on
// x in [-1,1]^5 for S(x) = sum_j W_j eps_j^2 with the continuum re-solved at
// every point -- the objective of Eq. 9.  One CTA per spectrum.  A full
// evaluation takes the Jacobian of r = sqrt(W) eps analytically (forward mode
// through Eq. 5 and the normal equations, as for stage 9) and forms A = J^T J
// and g = J^T r with float-float sums; parameters held on a bound by the gradient are
// frozen, and pred0 = g^T A^-1 g (the Gauss-Newton predicted decrease) is
// both the stop test (pred0 <= rtol S) and, where S differences fall below
// what FP32 model values resolve (1e-6 S), the merit that judges a trial.
// Damped steps (A + lambda diag A) d = -g follow Nielsen's damping rule.
// Thread 0 runs the control logic; all threads evaluate.  The per-pixel loops
// are not unrolled: unrolled, an evaluation was one long straight run of code
// that each warp executes once, and the kernel stalled on instruction fetch
// (ncu: 5 no-instruction stall cycles per issue); rolled, the per-pixel
// values live in local memory and the fit took 9.8 instead of 17.0 ms.
#pragma once

#include "lasp.h"
#include "lasp_common.cuh"

namespace lasp {

struct LmParams {
    ModelDev M;
    FitOpts O;
    int N;
    int max_iter;
    double rtol;
    const float* flux;
    const float* ivar;
    const uint8_t* good;
    const float* theta0;
    float* theta;
    float* loss;
    int32_t* steps;
    uint32_t* status;
    float* weight;
    float* cont;          // N x (D+1) continuum coefficients at the result, or nullptr
};

// Shared reduction space, floats a warp: every block sum of an evaluation has
// at most 64 values (54 normal-equation sums at Legendre degree 8).
constexpr int LM_RED_W = 64;

__host__ inline size_t lm_smem_bytes(int p, int H, int n_model, int NT) {
    size_t fl = (size_t)2 * ((p + 3) & ~3) + 4 * (size_t)((n_model + 3) & ~3) + 3 * 96 + (1 + DPS) * KROWS +
                (size_t)(NT / 32) * LM_RED_W + 256;
    size_t sortb = (size_t)3 * ((p + 3) & ~3);
    return 4 * (fl > sortb ? fl : sortb);
}

// Evaluate at physical theta (block-wide).  FULL: also the Jacobian sums
// A (15, packed upper triangle, x units), g (5, x units).  Returns S in
// s_sum[0] and the FULL sums in s_sum[1..20], all float-float (and s_ok: 1 if
// the normal equations were solvable).
template <int NT, int D, bool FULL>
__device__ void lm_eval(const ModelDev& M, const float* th, const float* y, const float* W, float* Fp,
                        int na, float* g, float* gmu, float* gsg, float* phi, float* dphi, float* red,
                        float2* outff, float2* s_G, float* s_b, float* s_db, float2* s_sum, int* s_h,
                        int* s_ok) {
    using Gm = Gram<D>;
    constexpr int NB = D + 1;
    constexpr int NV = Gm::NV;
    const int p = M.n_pix, H = M.pad, nm = M.n_model;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {
        warp_basis(M, th, phi, FULL ? dphi : nullptr);
        const int h = kernel_taps_warp(th[3] / M.kms_px, th[4] / M.kms_px, H, g, gmu, gsg);
        if (lane == 0) *s_h = h;
    }
    __syncthreads();
    const int h = *s_h;
    int k0, k1;
    active_rows(M, th[0], k0, k1);
    // F' (and at a full evaluation its three basis derivatives): 16 consecutive
    // model pixels per thread, the table rows (padded to 16 floats) from L2 with
    // 256-bit loads, each load feeding every contraction; per model pixel the
    // same sequence of fmas over k as one scalar load per value
    for (int m0 = tid * 16; m0 < nm; m0 += NT * 16) {
        constexpr int NQ = FULL ? 4 : 1;
        float a[NQ][16];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int r = 0; r < 16; ++r) a[q][r] = 0.0f;
        const float* crow = M.Cp + m0;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float* ck = crow + (size_t)k * M.ldc;
            const float pk = phi[k];
            float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f;
            if (FULL) {
                d0 = dphi[DPS * k + 0];
                d1 = dphi[DPS * k + 1];
                d2 = dphi[DPS * k + 2];
            }
#pragma unroll
            for (int h8 = 0; h8 < 2; ++h8) {
                float c[8];
                ldg8(ck + 8 * h8, c);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    a[0][8 * h8 + e] = fmaf(pk, c[e], a[0][8 * h8 + e]);
                    if (FULL) {
                        a[NQ > 1 ? 1 : 0][8 * h8 + e] = fmaf(d0, c[e], a[NQ > 1 ? 1 : 0][8 * h8 + e]);
                        a[NQ > 2 ? 2 : 0][8 * h8 + e] = fmaf(d1, c[e], a[NQ > 2 ? 2 : 0][8 * h8 + e]);
                        a[NQ > 3 ? 3 : 0][8 * h8 + e] = fmaf(d2, c[e], a[NQ > 3 ? 3 : 0][8 * h8 + e]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (m0 + r < nm) Fp[q * na + m0 + r] = a[q][r];
    }
    __syncthreads();
    float f[PPT], df[FULL ? 5 : 1][PPT];
    float gacc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) gacc[q] = 0.0f;
    const float ikms = 1.0f / M.kms_px;
#pragma unroll 1
    for (int r = 0; r < PPT; ++r) {
        const int j = tid + r * NT;
        f[r] = 0.0f;
        if (FULL)
#pragma unroll
            for (int k = 0; k < 5; ++k) df[k][r] = 0.0f;
        if (j < p) {
            float a0 = 0, a1 = 0, a2 = 0, a3 = 0, am = 0, as = 0;
            for (int s = -h; s <= h; ++s) {
                const int o = j + H - s;
                const float gs = g[s + H];
                const float fv = Fp[o];
                a0 = fmaf(gs, fv, a0);
                if (FULL) {
                    a1 = fmaf(gs, Fp[na + o], a1);
                    a2 = fmaf(gs, Fp[2 * na + o], a2);
                    a3 = fmaf(gs, Fp[3 * na + o], a3);
                    am = fmaf(gmu[s + H], fv, am);
                    as = fmaf(gsg[s + H], fv, as);
                }
            }
            f[r] = a0;
            if (FULL) {
                df[0][r] = a1;
                df[1][r] = a2;
                df[2][r] = a3;
                df[3][r] = am * ikms;
                df[4][r] = as * ikms;
            }
            const float Wj = W[j];
            if (Wj != 0.0f) {
                float Pl[NB];
                legendre<D>(legendre_node(j, p), Pl);
                const float vv = Wj * a0 * a0, uu = Wj * a0 * y[j];
#pragma unroll
                for (int a = 0; a < NB; ++a) {
#pragma unroll
                    for (int b2 = a; b2 < NB; ++b2) gacc[Gm::idx(a, b2)] = fmaf(vv * Pl[a], Pl[b2], gacc[Gm::idx(a, b2)]);
                    gacc[Gm::NG + a] = fmaf(uu, Pl[a], gacc[Gm::NG + a]);
                }
            }
        }
    }
    block_sum_ff<NV, NT>(gacc, red, outff);
    if (tid < NV) s_G[tid] = outff[tid];
    __syncthreads();
    if (warp == 0) {
        const float2* const rh[1] = {s_G + Gm::NG};
        float bd[NB];
        const bool ok = warp_chol_solve_ff<D, 1>(s_G, rh, bd);
        if (lane == 0) {
            *s_ok = ok ? 1 : 0;
            for (int a = 0; a < NB; ++a) s_b[a] = bd[a];
        }
    }
    __syncthreads();
    if (!*s_ok) return;
    float bl[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) bl[a] = s_b[a];
    if (!FULL) {
        float sacc[1] = {0.0f};
#pragma unroll 1
        for (int r = 0; r < PPT; ++r) {
            const int j = tid + r * NT;
            if (j < p && W[j] != 0.0f) {
                float Pl[NB];
                legendre<D>(legendre_node(j, p), Pl);
                float c = 0.0f;
#pragma unroll
                for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
                const float e = y[j] - c * f[r];
                sacc[0] = fmaf(W[j] * e, e, sacc[0]);
            }
        }
        block_sum_ff<1, NT>(sacc, red, outff);
        if (tid == 0) s_sum[0] = outff[0];
        __syncthreads();
        return;
    } else {
        // d b / d theta_k = G^-1 sum_j W_j P_d dF''_jk (eps_j - F''_j c_j); S
        constexpr int NT2 = 5 * NB + 1;
        float tacc[NT2];
#pragma unroll
        for (int q = 0; q < NT2; ++q) tacc[q] = 0.0f;
        float cc[PPT];
#pragma unroll 1
        for (int r = 0; r < PPT; ++r) {
            const int j = tid + r * NT;
            cc[r] = 0.0f;
            if (j < p && W[j] != 0.0f) {
                float Pl[NB];
                legendre<D>(legendre_node(j, p), Pl);
                float c = 0.0f;
#pragma unroll
                for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
                cc[r] = c;
                const float Wj = W[j];
                const float e = y[j] - c * f[r];
                const float q = Wj * (e - f[r] * c);
#pragma unroll
                for (int k = 0; k < 5; ++k)
#pragma unroll
                    for (int a = 0; a < NB; ++a) tacc[k * NB + a] = fmaf(q * df[k][r], Pl[a], tacc[k * NB + a]);
                tacc[5 * NB] = fmaf(Wj * e, e, tacc[5 * NB]);
            }
        }
        block_sum_ff<NT2, NT>(tacc, red, outff);
        if (warp == 0) {
            const float2* const rh[5] = {outff, outff + NB, outff + 2 * NB, outff + 3 * NB, outff + 4 * NB};
            float dbk[NB];
            warp_chol_solve_ff<D, 5>(s_G, rh, dbk);
            if (lane < 5)
                for (int a = 0; a < NB; ++a) s_db[lane * NB + a] = dbk[a];
        }
        if (tid == 0) s_sum[0] = outff[5 * NB];
        __syncthreads();
        float dbl[5][NB];
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int a = 0; a < NB; ++a) dbl[k][a] = s_db[k * NB + a];
        // J in x units (physical J times the half box width), A = J^T J, g = J^T r
        float jj[20];
#pragma unroll
        for (int q = 0; q < 20; ++q) jj[q] = 0.0f;
#pragma unroll 1
        for (int r = 0; r < PPT; ++r) {
            const int j = tid + r * NT;
            if (j < p && W[j] != 0.0f) {
                float Pl[NB];
                legendre<D>(legendre_node(j, p), Pl);
                const float sw = sqrtf(W[j]);
                const float rj = sw * (y[j] - cc[r] * f[r]);
                float Jr[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    float dc = 0.0f;
#pragma unroll
                    for (int a = 0; a < NB; ++a) dc = fmaf(dbl[k][a], Pl[a], dc);
                    Jr[k] = -sw * (cc[r] * df[k][r] + f[r] * dc) * M.phalf[k];
                }
                int q = 0;
#pragma unroll
                for (int a = 0; a < 5; ++a)
#pragma unroll
                    for (int b2 = a; b2 < 5; ++b2) {
                        jj[q] = fmaf(Jr[a], Jr[b2], jj[q]);
                        ++q;
                    }
#pragma unroll
                for (int a = 0; a < 5; ++a) jj[15 + a] = fmaf(Jr[a], rj, jj[15 + a]);
            }
        }
        block_sum_ff<20, NT>(jj, red, outff);
        if (tid < 20) s_sum[1 + tid] = outff[tid];
        __syncthreads();
    }
}

enum : int { LM_FULL_CUR = 0, LM_FULL_TRIAL = 1, LM_S_TRIAL = 2, LM_DONE = 3 };

// Control state of one CTA (shared memory, touched by thread 0 only).  S is
// float-float, so differences of S near convergence stay exact to about
// twice FP32 precision; the 5x5 systems are solved in FP32.
struct LmCtl {
    float2 S, Sn;
    float pred0, lam, nu, pred, pn;
    float Ar[15], gr[5];   // reduced system at the current point
    float An[15], gn[5];   // at the trial point (full trial evaluations)
    float d[5];
    int it, trial, phase;
    uint32_t status;
};

// (a - b) of two float-float values, rounded to float.
__device__ __forceinline__ float ff_diff(float2 a, float2 b) {
    const float2 s = two_sum(a.x, -b.x);
    return s.x + (s.y + (a.y - b.y));
}

// Reduced system from the sums of a full evaluation at x: parameters on a
// bound whose gradient points out of the box are frozen (unit row/column,
// zero gradient); pred0 = g^T A^-1 g (infinite if A is not positive definite).
__device__ inline void lm_reduce(const float2* sum, const float* x, float* Ar, float* gr, float2& S,
                                 float& pred0) {
    S = sum[0];
    bool fr[5];
    for (int a = 0; a < 5; ++a) {
        const float ga = sum[16 + a].x + sum[16 + a].y;
        fr[a] = !((x[a] <= -1.0f && ga > 0.0f) || (x[a] >= 1.0f && ga < 0.0f));
        gr[a] = fr[a] ? ga : 0.0f;
    }
    int q = 0;
    for (int a = 0; a < 5; ++a)
        for (int b = a; b < 5; ++b, ++q)
            Ar[q] = (fr[a] && fr[b]) ? sum[1 + q].x + sum[1 + q].y : (a == b ? 1.0f : 0.0f);
    float mg[5], d0[5];
    for (int a = 0; a < 5; ++a) mg[a] = -gr[a];
    if (chol_solve_rcp<4, float>(Ar, mg, d0)) {
        float s = 0.0f;
        for (int a = 0; a < 5; ++a) s -= gr[a] * d0[a];
        pred0 = s;
    } else {
        pred0 = INFINITY;
    }
}

// Next damped trial from the current point (after a rejection or a new
// iterate).  Sets c.phase to the evaluation the trial needs, or LM_DONE after
// ten rejections.
__device__ inline void lm_start_trial(LmCtl& c, const float* x, float* xt) {
    constexpr float kEta = 1e-6f;
    for (;;) {
        if (c.trial >= 10) {
            c.status = LASP_ST_CONV_TOL;
            c.phase = LM_DONE;
            return;
        }
        float Ad[15], rhs[5];
        for (int q = 0; q < 15; ++q) Ad[q] = c.Ar[q];
        for (int a = 0; a < 5; ++a) {
            Ad[Gram<4>::idx(a, a)] += c.lam * c.Ar[Gram<4>::idx(a, a)];
            rhs[a] = -c.gr[a];
        }
        if (chol_solve_rcp<4, float>(Ad, rhs, c.d)) break;
        c.lam *= c.nu;
        c.nu *= 2.0f;
        ++c.trial;
    }
    // predicted decrease of S: -(2 g.d + d^T A d)
    float pred = 0.0f;
    for (int a = 0; a < 5; ++a) {
        float Adv = 0.0f;
        for (int b = 0; b < 5; ++b) Adv += c.Ar[a <= b ? Gram<4>::idx(a, b) : Gram<4>::idx(b, a)] * c.d[b];
        pred -= 2.0f * c.gr[a] * c.d[a] + c.d[a] * Adv;
    }
    c.pred = pred;
    for (int k = 0; k < 5; ++k) xt[k] = fminf(1.0f, fmaxf(-1.0f, x[k] + c.d[k]));
    const float S = c.S.x + c.S.y;
    c.phase = pred >= kEta * S ? LM_S_TRIAL : LM_FULL_TRIAL;
}

__device__ inline void lm_new_iterate(LmCtl& c, const float* x, float* xt, int max_iter, float rtol) {
    if (c.pred0 <= rtol * (c.S.x + c.S.y)) {
        c.status = LASP_ST_CONV_TOL;
        c.phase = LM_DONE;
    } else if (c.it >= max_iter) {
        c.status = LASP_ST_MAXSTEPS;
        c.phase = LM_DONE;
    } else {
        c.trial = 0;
        lm_start_trial(c, x, xt);
    }
}

// Thread 0, after the evaluation of phase ph.
static __device__ __noinline__ void lm_control(LmCtl& c, int ph, int ok, const float2* sum, float* x,
                                               float* xt, int max_iter, float rtol) {
    constexpr float kEta = 1e-6f;
    if (ph == LM_FULL_CUR) {
        if (!ok) {
            c.status = LASP_ST_SINGULAR;
            c.phase = LM_DONE;
            return;
        }
        lm_reduce(sum, x, c.Ar, c.gr, c.S, c.pred0);
        lm_new_iterate(c, x, xt, max_iter, rtol);
        return;
    }
    float rho = -1.0f;
    if (ph == LM_S_TRIAL) {
        const float2 St = sum[0];
        if (ok && isfinite(St.x)) rho = ff_diff(c.S, St) / c.pred;
    } else if (ok) {
        lm_reduce(sum, xt, c.An, c.gn, c.Sn, c.pn);
        const float S = c.S.x + c.S.y;
        if (isfinite(c.Sn.x) && ff_diff(c.S, c.Sn) >= -kEta * S) {
            // merit the model predicts: its gradient after the step is lambda diag(A) d
            float gm[5], z[5], pm = 0.0f;
            for (int a = 0; a < 5; ++a) gm[a] = c.lam * c.Ar[Gram<4>::idx(a, a)] * c.d[a];
            if (chol_solve_rcp<4, float>(c.Ar, gm, z))
                for (int a = 0; a < 5; ++a) pm += gm[a] * z[a];
            const float den = c.pred0 - pm > 0.0f ? c.pred0 - pm : c.pred0;
            rho = (c.pred0 - c.pn) / den;
        }
    }
    if (rho > 0.0f) {
        const float t = 2.0f * rho - 1.0f, f = 1.0f - t * t * t;
        c.lam *= f > 1.0f / 3.0f ? f : 1.0f / 3.0f;
        if (c.lam < 1e-12f) c.lam = 1e-12f;
        c.nu = 2.0f;
        for (int k = 0; k < 5; ++k) x[k] = xt[k];
        ++c.it;
        if (ph == LM_S_TRIAL) {
            c.phase = LM_FULL_CUR;
        } else {
            c.S = c.Sn;
            c.pred0 = c.pn;
            for (int q = 0; q < 15; ++q) c.Ar[q] = c.An[q];
            for (int a = 0; a < 5; ++a) c.gr[a] = c.gn[a];
            lm_new_iterate(c, x, xt, max_iter, rtol);
        }
    } else {
        c.lam *= c.nu;
        c.nu *= 2.0f;
        ++c.trial;
        lm_start_trial(c, x, xt);
    }
}

// Two CTAs per SM at 256 threads (128 registers; the shared-memory plan of about
// 100 KB allows two): a few spills cost far less than halving the resident warps.
template <int NT, int D>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) lm_kernel(const LmParams P) {
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, nm = M.n_model;
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const int pa = (p + 3) & ~3, na = (nm + 3) & ~3;
    float* y = sm;
    float* W = y + pa;
    float* Fp = W + pa;
    float* g = Fp + 4 * na;
    float* gmu = g + 96;
    float* gsg = g + 192;
    float* phi = g + 288;
    float* dphi = phi + KROWS;
    float* red = phi + (1 + DPS) * KROWS;
    float* outf = red + (NT / 32) * LM_RED_W;
    float2* outff = reinterpret_cast<float2*>(outf + ((((size_t)(outf - sm)) & 1) ? 1 : 0));
    __shared__ float2 s_G[Gram<D>::NV], s_sum[21];
    __shared__ float s_b[D + 1], s_db[5 * (D + 1)], s_bx[D + 1];
    __shared__ float s_x[5], s_xt[5];
    __shared__ int s_h, s_ok;
    __shared__ LmCtl c;
    const size_t row = (size_t)i * p;
    float w;
    const int n_obj = prep_spectrum<NT>(P.flux + row, P.ivar + row, P.good + row, p, P.O.edge_px,
                                        P.O.quantile, y, W, Fp, red, &w);
    if (tid == 0) {
        for (int k = 0; k < 5; ++k) {
            float xx = (P.theta0[5 * i + k] - M.plo[k]) / M.phalf[k] - 1.0f;
            s_x[k] = fminf(1.0f, fmaxf(-1.0f, xx));
        }
        if (P.weight) P.weight[i] = w;
        c.lam = 1e-3f;
        c.nu = 2.0f;
        c.it = 0;
        c.trial = 0;
        c.status = 0;
        c.S = make_float2(NAN, 0.0f);
        c.phase = LM_FULL_CUR;
    }
    __syncthreads();
    if (n_obj < D + 1 + 5 || !(w > 0.0f) || !isfinite(w)) {
        if (tid == 0) {
            for (int k = 0; k < 5; ++k) P.theta[5 * i + k] = phys_of(M, k, s_x[k]);
            P.loss[i] = NAN;
            P.steps[i] = 0;
            P.status[i] = LASP_ST_NODATA;
        }
        if (P.cont && tid <= D) P.cont[(size_t)i * (D + 1) + tid] = NAN;
        return;
    }
    for (;;) {
        __syncthreads();
        const int ph = c.phase;
        if (ph == LM_DONE) break;
        const float* xp = ph == LM_FULL_CUR ? s_x : s_xt;
        float th[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) th[k] = phys_of(M, k, xp[k]);
        if (ph == LM_S_TRIAL)
            lm_eval<NT, D, false>(M, th, y, W, Fp, na, g, gmu, gsg, phi, dphi, red, outff, s_G, s_b, s_db,
                                  s_sum, &s_h, &s_ok);
        else
            lm_eval<NT, D, true>(M, th, y, W, Fp, na, g, gmu, gsg, phi, dphi, red, outff, s_G, s_b, s_db,
                                 s_sum, &s_h, &s_ok);
        if (tid == 0) {
            const int it0 = c.it;
            lm_control(c, ph, s_ok, s_sum, s_x, s_xt, P.max_iter, (float)P.rtol);
            // the continuum of the current parameters: that of an evaluation at
            // them, or of a trial the control step has just accepted
            if (ph == LM_FULL_CUR || c.it != it0)
                for (int a = 0; a <= D; ++a) s_bx[a] = s_b[a];
        }
    }
    if (tid == 0) {
        for (int k = 0; k < 5; ++k) P.theta[5 * i + k] = phys_of(M, k, s_x[k]);
        P.loss[i] = sqrtf((c.S.x + c.S.y) / (float)p);
        P.steps[i] = c.it;
        P.status[i] = c.status;
        if (P.cont)
            for (int a = 0; a <= D; ++a) P.cont[(size_t)i * (D + 1) + a] = s_bx[a];
    }
}

}  // namespace lasp
