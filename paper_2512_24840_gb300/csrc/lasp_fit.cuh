// Fused grouped-Adam fit kernel (FP32 CUDA-core form) -- sm_103a.
//
// One CTA fits one spectrum from its initial guess to its stop rule: every
// Adam step (stage 8 of section 2.2) evaluates Eq. 1 (basis contraction with
// the table, read from L2), Eq. 5 (broadening), Eq. 6 (weighted least-squares
// continuum), Eqs. 7 and 9 (residual, loss) and the hand-written adjoint of
// that chain, then applies Adam with the box projection and the three stop
// rules.  The observed spectrum is read from HBM once per fit; between steps
// everything stays in shared memory and registers.  A finished spectrum frees
// its CTA slot at once, which the hardware refills with the next spectrum, so
// spectra that converge early cost no idle steps.
#pragma once

#include "lasp_common.cuh"

namespace lasp {

struct FitParams {
    ModelDev M;
    FitOpts O;
    int N;
    const float* flux;
    const float* ivar;
    const uint8_t* good;
    const float* theta0;
    float* theta;
    float* loss;
    int32_t* steps;
    uint32_t* status;
    float* cont;      // N x (D+1) or nullptr
    float* weight;    // N or nullptr
};

// Shared-memory plan of the fit kernel (floats), in order.
struct FitSmem {
    int y, W, Fp, Db, g, gmu, gsg, phi, dphi, red, out, ring, total;
    __host__ __device__ FitSmem(int p, int H, int n_model, int NT, int D) {
        int NB = D + 1, NV = NB * (NB + 1) / 2 + NB;
        int nv_max = NV > (KMAX + 2) ? NV : (KMAX + 2);
        int o = 0;
        y = o;    o += (p + 3) & ~3;
        W = o;    o += (p + 3) & ~3;
        Fp = o;   o += (n_model + 3) & ~3;
        Db = o;   o += (p + 4 * H + 3) & ~3;
        g = o;    o += 96;
        gmu = o;  o += 96;
        gsg = o;  o += 96;
        phi = o;  o += KMAX;
        dphi = o; o += 3 * KMAX;
        red = o;  o += (NT / 32) * nv_max;
        out = o;  o += 2 * nv_max + 16;   // FP32 sums, or FP64 sums (2 floats each)
        ring = o; o += WINMAX;
        total = o;
    }
};

__host__ inline size_t fit_smem_bytes(int p, int H, int n_model, int NT, int D) {
    FitSmem s(p, H, n_model, NT, D);
    size_t sortb = (size_t)next_pow2(p);
    // the sort buffer of the preprocessing aliases Fp and Db (>= next_pow2(p))
    size_t need = (size_t)s.total;
    size_t sort_end = (size_t)s.Fp + sortb;
    return 4 * (need > sort_end ? need : sort_end);
}

template <int NT, int D>
__global__ void __launch_bounds__(NT) fit_kernel(const FitParams P) {
    using Gm = Gram<D>;
    constexpr int NB = D + 1;
    constexpr int NV = Gm::NV;
    constexpr int PPT = 16;                       // pixels per thread supported
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, H = M.pad, nm = M.n_model, K = M.K;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i = blockIdx.x;
    FitSmem L(p, H, nm, NT, D);
    float* y = sm + L.y;
    float* W = sm + L.W;
    float* Fp = sm + L.Fp;
    float* Db = sm + L.Db;
    float* g = sm + L.g;
    float* gmu = sm + L.gmu;
    float* gsg = sm + L.gsg;
    float* phi = sm + L.phi;
    float* dphi = sm + L.dphi;
    float* red = sm + L.red;
    float* out = sm + L.out;
    double* outd = reinterpret_cast<double*>(sm + ((L.out + 1) & ~1));
    float* ring = sm + L.ring;
    __shared__ float s_x[5], s_b[NB], s_scal[8];
    __shared__ int s_h, s_stop;

    const size_t row = (size_t)i * p;
    float w;
    const int n_obj = prep_spectrum<NT>(P.flux + row, P.ivar + row, P.good + row, p,
                                        P.O.edge_px, P.O.quantile, y, W, Fp, red, &w);
    // delta buffer: zero halo; interior rewritten every step
    for (int j = tid; j < p + 4 * H; j += NT) Db[j] = 0.0f;

    // Adam state lives in thread 0's registers.
    float x[5], m[5], v[5], prev = 0.0f;
    int rise = 0;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float xx = 2.0f * (P.theta0[5 * i + k] - M.plo[k]) / (2.0f * M.phalf[k]) - 1.0f;
            xx = fminf(1.0f, fmaxf(-1.0f, xx));
            x[k] = xx;
            s_x[k] = xx;
            m[k] = 0.0f;
            v[k] = 0.0f;
        }
        s_stop = 0;
        if (n_obj < NB + 5 || !(w > 0.0f) || !isfinite(w)) s_stop = (int)0x40;  // NODATA
    }
    __syncthreads();
    if (s_stop) {
        if (tid == 0) {
            for (int k = 0; k < 5; ++k) P.theta[5 * i + k] = phys_of(M, k, s_x[k]);
            P.loss[i] = NAN;
            P.steps[i] = 0;
            P.status[i] = 0x40u;
            if (P.weight) P.weight[i] = w;
        }
        if (P.cont && tid < NB) P.cont[(size_t)i * NB + tid] = NAN;
        return;
    }

    const float inv_p = 1.0f / (float)p;
    float fpp[PPT];

    for (int t = 0;; ++t) {
        // ---- a1/a2: parameters, basis, kernel taps (warp 0)
        if (warp == 0) {
            float th[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) th[k] = phys_of(M, k, s_x[k]);
            if (lane < K) basis_term(M, lane, th, phi, dphi);
            float mu = th[3] / M.kms_px, sig = th[4] / M.kms_px;
            int h = kernel_taps_warp(mu, sig, H, g, gmu, gsg);
            if (lane == 0) s_h = h;
        }
        __syncthreads();
        const int h = s_h;

        // ---- a3: F' = phi C  (Eq. 1), table from L2
        for (int mm = tid; mm < nm; mm += NT) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) acc = fmaf(phi[k], __ldg(M.C + (size_t)k * nm + mm), acc);
            Fp[mm] = acc;
        }
        __syncthreads();

        // ---- a4 + a5: F'' = F' (x) G (Eq. 5); normal equations of Eq. 6
        float gacc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) gacc[q] = 0.0f;
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int j = tid + r * NT;
            fpp[r] = 0.0f;
            if (j < p) {
                const float* src = Fp + j + H;
                float f = 0.0f;
                for (int s = -h; s <= h; ++s) f = fmaf(g[s + H], src[-s], f);
                fpp[r] = f;
                const float Wj = W[j];
                if (Wj != 0.0f) {
                    float Pl[NB];
                    legendre<D>(legendre_node(j, p), Pl);
                    const float vv = Wj * f * f, uu = Wj * f * y[j];
#pragma unroll
                    for (int a = 0; a < NB; ++a) {
                        const float va = vv * Pl[a];
#pragma unroll
                        for (int b2 = a; b2 < NB; ++b2) gacc[Gm::idx(a, b2)] = fmaf(va, Pl[b2], gacc[Gm::idx(a, b2)]);
                        gacc[Gm::NG + a] = fmaf(uu, Pl[a], gacc[Gm::NG + a]);
                    }
                }
            }
        }
        bool solved;
        if (P.O.fp64_ne) {
            block_sum_f64<NV, NT>(gacc, red, outd);
            if (tid == 0) {
                double bd[NB];
                solved = chol_solve_packed<D, double>(outd, outd + Gm::NG, bd);
                for (int a = 0; a < NB; ++a) s_b[a] = (float)bd[a];
                s_scal[0] = solved ? 1.0f : 0.0f;
            }
        } else {
            block_sum<NV, NT>(gacc, red, out);
            if (tid == 0) {
                float bf[NB];
                solved = chol_solve_packed<D, float>(out, out + Gm::NG, bf);
                for (int a = 0; a < NB; ++a) s_b[a] = bf[a];
                s_scal[0] = solved ? 1.0f : 0.0f;
            }
        }
        __syncthreads();

        // ---- a6: residual (Eq. 7), loss (Eq. 9); delta = W eps c for the adjoint
        float racc[2] = {0.0f, 0.0f};
        float bl[NB];
#pragma unroll
        for (int a = 0; a < NB; ++a) bl[a] = s_b[a];
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int j = tid + r * NT;
            if (j < p) {
                const float Wj = W[j];
                float dlt = 0.0f;
                if (Wj != 0.0f) {
                    float Pl[NB];
                    legendre<D>(legendre_node(j, p), Pl);
                    float c = 0.0f;
#pragma unroll
                    for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
                    const float e = y[j] - c * fpp[r];
                    racc[0] = fmaf(Wj * e, e, racc[0]);
                    if (c <= 0.0f) racc[1] = 1.0f;
                    dlt = Wj * e * c;
                }
                fpp[r] = dlt;                  // register now holds delta_j (unscaled)
                Db[j + 2 * H] = dlt;
            }
        }
        block_sum<2, NT>(racc, red, out);
        const float S = out[0];
        const bool nonpos = out[1] > 0.0f;
        const float l = sqrtf(S * inv_p);
        // dl/dF''_j = -W eps c / (p l) with b held at its optimum (envelope theorem)
        const float kappa = l > 0.0f ? -1.0f / ((float)p * l) : 0.0f;

        // ---- a7: adjoint through broadening and the basis contraction
        float bacc[2 + KMAX];
#pragma unroll
        for (int q = 0; q < 2 + KMAX; ++q) bacc[q] = 0.0f;
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int j = tid + r * NT;
            if (j < p && fpp[r] != 0.0f) {
                const float* src = Fp + j + H;
                float am = 0.0f, as = 0.0f;
                for (int s = -h; s <= h; ++s) {
                    const float fv = src[-s];
                    am = fmaf(gmu[s + H], fv, am);
                    as = fmaf(gsg[s + H], fv, as);
                }
                bacc[0] = fmaf(fpp[r], am, bacc[0]);
                bacc[1] = fmaf(fpp[r], as, bacc[1]);
            }
        }
        for (int mm = tid; mm < nm; mm += NT) {
            const float* src = Db + mm + H;
            float d = 0.0f;
            for (int s = -h; s <= h; ++s) d = fmaf(g[s + H], src[s], d);
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) bacc[2 + k] = fmaf(d, __ldg(M.C + (size_t)k * nm + mm), bacc[2 + k]);
        }
        block_sum<2 + KMAX, NT>(bacc, red, out);

        // ---- a8: chain rule to x, stop rules, Adam (thread 0)
        if (tid == 0) {
            float gx[5];
            float gth[3] = {0.0f, 0.0f, 0.0f};
            for (int k = 0; k < K; ++k) {
                gth[0] = fmaf(out[2 + k], dphi[3 * k + 0], gth[0]);
                gth[1] = fmaf(out[2 + k], dphi[3 * k + 1], gth[1]);
                gth[2] = fmaf(out[2 + k], dphi[3 * k + 2], gth[2]);
            }
            gx[0] = kappa * gth[0] * M.phalf[0];
            gx[1] = kappa * gth[1] * M.phalf[1];
            gx[2] = kappa * gth[2] * M.phalf[2];
            gx[3] = kappa * out[0] / M.kms_px * M.phalf[3];
            gx[4] = kappa * out[1] / M.kms_px * M.phalf[4];
            uint32_t stop = 0;
            if (!solved) stop = 32u;
            else {
                bool fin = isfinite(l);
#pragma unroll
                for (int k = 0; k < 5; ++k) fin = fin && isfinite(gx[k]);
                if (!fin) stop = 16u;
            }
            if (!stop) {
                const int Wn = P.O.window;
                if (t >= Wn && fabsf(l - ring[t % Wn]) < P.O.tol) stop = 1u;
                rise = (t >= 1 && l > prev) ? rise + 1 : 0;
                if (!stop && rise >= Wn) stop = 2u;
                if (!stop && t >= P.O.max_steps) stop = 4u;
                ring[t % Wn] = l;
                prev = l;
            }
            if (stop) {
                if (stop <= 4u && nonpos) stop |= 8u;
                for (int k = 0; k < 5; ++k) P.theta[5 * i + k] = phys_of(M, k, x[k]);
                P.loss[i] = l;
                P.steps[i] = t;
                P.status[i] = stop;
                if (P.weight) P.weight[i] = w;
                s_stop = 1;
            } else {
                const float tt = (float)(t + 1);
                const float bc1 = 1.0f - powf(P.O.beta1, tt);
                const float bc2 = 1.0f - powf(P.O.beta2, tt);
                const float step = P.O.lr / bc1, rbc2 = rsqrtf(bc2);
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    m[k] = P.O.beta1 * m[k] + (1.0f - P.O.beta1) * gx[k];
                    v[k] = P.O.beta2 * v[k] + (1.0f - P.O.beta2) * gx[k] * gx[k];
                    const float denom = sqrtf(v[k]) * rbc2 + P.O.eps;
                    x[k] = fminf(1.0f, fmaxf(-1.0f, x[k] - step * m[k] / denom));
                    s_x[k] = x[k];
                }
            }
        }
        __syncthreads();
        if (s_stop) break;
    }
    if (P.cont && tid < NB) P.cont[(size_t)i * NB + tid] = s_b[tid];
}

}  // namespace lasp
