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
//
// Work layout: thread t owns 16 consecutive pixels (and 16 consecutive model
// pixels).  Arrays read across threads live in shared memory in skewed rows
// (element i at i + i/16), so the stride-16 accesses of a warp hit 32 distinct
// banks.  Correlations run over blocks of 8 taps against a 23-value register
// window (128 FMAs per 31 shared loads).  The adjoint of the kernel
// parameters goes through the per-tap sums a_s = sum_j delta_j F'_{j+H-s}.
#pragma once

#include "lasp_clean.cuh"
#include "lasp_common.cuh"

namespace lasp {

constexpr int TB = 12;       // taps per block
constexpr int TAPBUF = 128; // tap buffer (>= 2 HMAX + 2 TB + 1)
// the correlations read taps in whole blocks of TB past the widest kernel (2 HMAX + 1 taps)
static_assert(TAPBUF >= 2 * HMAX + 2 * TB + 1, "tap buffer shorter than the widest kernel in blocks");
static_assert(MODEL_PIX_MAX == PPT * 512, "the largest model grid is one run of PPT pixels per thread of 512");
constexpr int NADJ = 7;     // end-of-step sums: S, nonpos, d/dmu, d/dsigma, d/d(Teff, logg, FeH)

// Device-resident fit state of resumable slots (struct of arrays, S slots).
// A launch in slot mode runs at most `budget` Adam steps per slot and saves
// the state of slots that have not stopped; t = -1 marks a freshly admitted
// slot (preprocessing and initial guess still to do).
struct SlotState {
    float* x;          // S x 5
    float* m;          // S x 5
    float* v;          // S x 5
    float* ring;       // S x WINMAX
    float* prev;       // S
    int* rise;         // S
    int* t;            // S
    double* b12;       // S x 2: beta1^t, beta2^t (the running products of the bias corrections)
    float* w;          // S  (weight, set at the first launch)
    float* imean;      // S  (mean inverse variance)
    uint16_t* cmask;   // S x ceil(p / 16) zero-weight bits of each thread's 16 pixels (Clean), or nullptr
    int budget;
};

struct FitParams {
    ModelDev M;
    FitOpts O;
    int N;
    SlotState S;       // S.x == nullptr: one launch fits every spectrum to its stop
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


// Shared-memory plan (floats).  Fp holds model pixels m in [-16, n_model+16)
// at skew(m + 16); Db holds delta_j for j in [-(2H+8), p + 2H + 24) at
// skew(j + 2H + 8), zero outside [0, p).
struct FitSmem {
    int y, W, Fp, Db, g, gmu, gsg, phi, dphi, red, out, ring, total, dofs;
    __host__ __device__ FitSmem(int p, int H, int n_model, int NT, int D, int K) {
        const int NB = D + 1, NV = NB * (NB + 1) / 2 + NB;
        const int nv_max = round32(NV > NADJ ? NV : NADJ);
        dofs = 2 * H + 8;
        int o = 0;
        y = o;    o += skew_size(p);
        W = o;    o += skew_size(p);
        Fp = o;   o += skew_size(n_model + 32);
        Db = o;   o += skew_size(p + 4 * H + 40);
        g = o;    o += TAPBUF;
        gmu = o;  o += TAPBUF;
        gsg = o;  o += TAPBUF;
        phi = o;  o += round32(K);          // sized by the table: the SM's L1 keeps the rest
        dphi = o; o += DPS * round32(K);
        const int red_n = (NT / 32) * (nv_max > 2 * round32(NV) ? nv_max : 2 * round32(NV));
        red = o;  o += red_n > PREP_RED ? red_n : PREP_RED;
        out = o;  o += 2 * nv_max + 16;
        ring = o; o += WINMAX;
        total = o;
    }
};

__host__ inline size_t fit_smem_bytes(int p, int H, int n_model, int NT, int D, int K) {
    FitSmem s(p, H, n_model, NT, D, K);
    size_t sort_end = (size_t)s.Fp + p;         // the preprocessing's select buffer
    return 4 * ((size_t)s.total > sort_end ? (size_t)s.total : sort_end);
}

// Reduce NV per-thread values over the CTA; the sums end in out[0..NV) and
// are visible to warp 0 only (after __syncwarp), with one CTA barrier.  Each
// warp reduce-scatters groups of 32 values, then warp 0 adds the warps in a
// fixed order, so the result depends only on this CTA's data.  red holds
// (NT/32) x round32(NV) floats.
template <int NV, int NT>
__device__ __forceinline__ void reduce_to_warp0(float (&v)[NV], float* red, float* out) {
    constexpr int NP = round32(NV);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < NP / 32; ++g) red[warp * NP + 32 * g + lane] = warp_sums_group<NV>(v, g);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int g = 0; g < NP / 32; ++g) {
            const int i = 32 * g + lane;
            float s = 0.0f;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) s += red[w * NP + i];
            if (i < NV) out[i] = s;
        }
        __syncwarp();
    }
}

// As reduce_to_warp0, with the warps added in float-float (exact two-sums):
// out[i] = (hi, lo).
template <int NV, int NT>
__device__ __forceinline__ void reduce_to_warp0_ff(float (&v)[NV], float* red, float2* outff) {
    constexpr int NP = round32(NV);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < NP / 32; ++g) red[warp * NP + 32 * g + lane] = warp_sums_group<NV>(v, g);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int g = 0; g < NP / 32; ++g) {
            const int i = 32 * g + lane;
            float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) s = ff_add(s, red[w * NP + i]);
            if (i < NV) outff[i] = s;
        }
        __syncwarp();
    }
}

// As reduce_to_warp0 with every partial sum in FP64: each thread's FP32 sum
// over its own pixels is widened to double, the warp reduce-scatters in double
// and warp 0 adds the warps in double.  redd: (NT/32) round32(NV) doubles;
// outd[i] is visible to warp 0 on return.
template <int NV, int NT>
__device__ __forceinline__ void reduce_to_warp0_f64(const float (&v)[NV], double* redd, double* outd) {
    constexpr int NP = round32(NV);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < NP / 32; ++g) redd[warp * NP + 32 * g + lane] = warp_sums_group_f64<NV>(v, g);
    __syncthreads();
    if (warp == 0) {
        for (int i = lane; i < NV; i += 32) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) s += redd[w * NP + i];
            outd[i] = s;
        }
        __syncwarp();
    }
}

// Continuum coefficients b of Eq. 6 from each thread's FP32 partial sums of
// the normal equations (packed upper triangle of G, then r), in the precision
// the fit options ask for: FP32 (sums and solve in FP32), float-float (warps
// added in exact two-sums, FP32 Cholesky refined once with a float-float
// residual), or FP64 (every partial sum beyond the thread's own pixels and the
// Cholesky solve in double).  sb[a] is b_a, or NaN where G is not positive
// definite, visible to every thread after the closing barrier.  red: the
// shared reduction buffer (2 (NT/32) round32(NV) floats), out: 2 NV floats,
// both 8-byte aligned.
// F64: whether the FP64 form is compiled in (kernels whose register budget is
// tight leave it out and are not launched with LASP_NE_FP64).
template <int D, int NT, bool F64 = true>
__device__ __forceinline__ void solve_continuum(float (&gacc)[Gram<D>::NV], int prec, float* red, float* out,
                                                float* sb) {
    using Gm = Gram<D>;
    constexpr int NB = D + 1, NV = Gm::NV;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (F64 && prec == LASP_NE_FP64) {
        double* outd = reinterpret_cast<double*>(out);
        reduce_to_warp0_f64<NV, NT>(gacc, reinterpret_cast<double*>(red), outd);
        if (tid == 0) {
            double bd[NB];
            const bool ok = chol_solve_rcp<D, double>(outd, outd + Gm::NG, bd);
#pragma unroll
            for (int a = 0; a < NB; ++a) sb[a] = ok ? (float)bd[a] : NAN;
        }
    } else if (prec == LASP_NE_FF) {
        float2* outff = reinterpret_cast<float2*>(out);
        reduce_to_warp0_ff<NV, NT>(gacc, red, outff);
        if (warp == 0) {
            const float2* const rh[1] = {outff + Gm::NG};
            float bf[NB];
            const bool ok = warp_chol_solve_ff<D, 1>(outff, rh, bf);
            if (lane == 0)
#pragma unroll
                for (int a = 0; a < NB; ++a) sb[a] = ok ? bf[a] : NAN;
        }
    } else {
        reduce_to_warp0<NV, NT>(gacc, red, out);
        if (tid == 0) {
            float bf[NB];
            const bool ok = chol_solve_rcp<D, float>(out, out + Gm::NG, bf);
#pragma unroll
            for (int a = 0; a < NB; ++a) sb[a] = ok ? bf[a] : NAN;
        }
    }
    __syncthreads();
}

// Basis, its derivatives, the active table rows (s_k[0..1]) and the kernel
// taps for normalised x (warp 0).  Taps are written for s + H in
// [0, TAPBUF), zero outside |s| <= h.
__device__ __forceinline__ int warp_prepare_step(const ModelDev& M, const float* x, float* phi,
                                                 float* dphi, float* g, float* gmu, float* gsg,
                                                 int* s_k) {
    const int lane = threadIdx.x & 31;
    float th[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) th[k] = phys_of(M, k, x[k]);
    warp_basis(M, th, phi, dphi);
    if (lane == 0) active_rows(M, th[0], s_k[0], s_k[1]);
    for (int i = 2 * M.pad + 1 + lane; i < TAPBUF; i += 32) {
        g[i] = 0.0f;
        gmu[i] = 0.0f;
        gsg[i] = 0.0f;
    }
    return kernel_taps_warp(th[3] / M.kms_px, th[4] / M.kms_px, M.pad, g, gmu, gsg);
}

// Clean mask update after evaluating step t (stage 6 schedule): t = every,
// 2 every, ..., at most clean_max updates.
__device__ __forceinline__ bool clean_step(const FitOpts& O, int t) {
    return O.clean && t > 0 && t % O.clean_every == 0 && t / O.clean_every <= O.clean_max;
}

template <int NT, int D>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 1) fit_kernel(const FitParams P) {
    using Gm = Gram<D>;
    constexpr int NB = D + 1;
    constexpr int NV = Gm::NV;
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, H = M.pad, nm = M.n_model;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i = blockIdx.x;
    const FitSmem L(p, H, nm, NT, D, M.K);
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
    float* out = sm + L.out;           // even offset: 8-byte aligned for the FP64 solve
    float* ring = sm + L.ring;
    __shared__ float s_x[5], s_b[NB];
    __shared__ int s_h, s_stop, s_k[2];
    __shared__ float s_w, s_imean;
    __shared__ double s_redd[3 * (NT / 32)], s_tot[3];

    const bool slots = P.S.x != nullptr;
    int t0 = 0;
    if (slots) {
        if (P.status[i] != 128u) return;          // slot not running (uniform per CTA)
        t0 = P.S.t[i];
    }
    const bool fresh = !slots || t0 < 0;
    if (t0 < 0) t0 = 0;

    // ---- preprocessing (section 3.3 step 2): y, W into skewed rows
    {
        const size_t row = (size_t)i * p;
        float w, imean;
        int n_obj;
        if (fresh) {
            n_obj = prep_spectrum<NT>(P.flux + row, P.ivar + row, P.good + row, p, P.O.edge_px,
                                      P.O.quantile, y, W, Fp, red, &w, &imean);
        } else {
            w = P.S.w[i];
            imean = P.S.imean[i];
            n_obj = refill_spectrum<NT>(P.flux + row, P.ivar + row, P.good + row, p, P.O.edge_px, w,
                                        imean, y, W, red);
        }
        __syncthreads();
        // re-layout y and W (written linearly) into skewed rows in place:
        // copy out to registers, barrier, copy back skewed.
        float ty[PPT], tw[PPT];
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int j = tid * PPT + r;
            ty[r] = j < p ? y[j] : 0.0f;
            tw[r] = j < p ? W[j] : 0.0f;
        }
        __syncthreads();
        // a resumed Clean fit keeps the pixels its mask updates removed
        const uint32_t cm = (!fresh && P.S.cmask && tid * PPT < p)
                                ? P.S.cmask[(size_t)i * ((p + PPT - 1) / PPT) + tid] : 0u;
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int j = tid * PPT + r;
            if (j < p) {
                y[skew(j)] = ty[r];
                W[skew(j)] = ((cm >> r) & 1u) ? 0.0f : tw[r];
            }
        }
        if (tid == 0) {
            s_w = w;
            s_imean = imean;
            s_stop = (fresh && (n_obj < NB + 5 || !(w > 0.0f) || !isfinite(w))) ? 1 : 0;
            if (slots && fresh) {
                P.S.w[i] = w;
                P.S.imean[i] = imean;
            }
        }
    }
    // zero the padded F' and delta buffers (their pads stay zero)
    for (int q = tid; q < skew_size(nm + 32); q += NT) Fp[q] = 0.0f;
    for (int q = tid; q < skew_size(p + 4 * H + 40); q += NT) Db[q] = 0.0f;

    // Adam state: parameter k lives in registers of lane k of warp 0 (k < 5);
    // lane 0 also keeps the stop-rule state.  beta^t are running products in
    // FP64 (the bias corrections are taken in double, as PyTorch does).
    float xk = 0.0f, mk = 0.0f, vk = 0.0f, prev = 0.0f;
    int rise = 0, ri = t0 % P.O.window;   // ring slot of step t
    double b1t = 1.0, b2t = 1.0;
    if (warp == 0) {
        if (t0 > 0) {                       // the products saved with the slot, exactly
            b1t = P.S.b12[2 * i];
            b2t = P.S.b12[2 * i + 1];
        }
        if (lane < 5) {
            if (fresh) {
                const float xx = (P.theta0[5 * i + lane] - M.plo[lane]) / M.phalf[lane] - 1.0f;
                xk = fminf(1.0f, fmaxf(-1.0f, xx));
            } else {
                xk = P.S.x[5 * i + lane];
                mk = P.S.m[5 * i + lane];
                vk = P.S.v[5 * i + lane];
            }
            s_x[lane] = xk;
        }
        if (lane == 0 && !fresh) {
            prev = P.S.prev[i];
            rise = P.S.rise[i];
        }
    }
    if (slots && !fresh)
        for (int q = tid; q < WINMAX; q += NT) ring[q] = P.S.ring[(size_t)i * WINMAX + q];
    __syncthreads();
    if (s_stop) {
        if (tid == 0) {
            for (int k = 0; k < 5; ++k) P.theta[5 * i + k] = phys_of(M, k, s_x[k]);
            P.loss[i] = NAN;
            P.steps[i] = 0;
            P.status[i] = 64u;
            if (P.weight) P.weight[i] = s_w;
        }
        if (P.cont && tid < NB) P.cont[(size_t)i * NB + tid] = NAN;
        return;
    }
    if (warp == 0) {
        int h = warp_prepare_step(M, s_x, phi, dphi, g, gmu, gsg, s_k);
        if (lane == 0) s_h = h;
    }
    __syncthreads();

    const float inv_p = 1.0f / (float)p;
    const int j0 = tid * PPT;              // first owned pixel / model pixel
    const bool own_pix = j0 < p;
    const bool own_mod = j0 < nm;
    const float xstep = 2.0f / (float)p;

    for (int t = t0;; ++t) {
        const int h = s_h;
        const int nblk = (2 * h + 1 + TB - 1) / TB;
        const int k0 = s_k[0], k1 = s_k[1];

        // ---- a3: F' = phi C (Eq. 1), 16 model pixels per thread, table from L2
        if (own_mod) {
            float acc[PPT];
#pragma unroll
            for (int r = 0; r < PPT; ++r) acc[r] = 0.0f;
            // rows are padded to 16 floats and j0 is a multiple of 16: 32-byte aligned
            const float* crow = M.Cp + j0;
#pragma unroll 2
            for (int k = k0; k < k1; ++k) {
                const float pk = phi[k];
                const float* ck = crow + (size_t)k * M.ldc;
#pragma unroll
                for (int q = 0; q < PPT / 8; ++q) {
                    float c[8];
                    ldg8(ck + 8 * q, c);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[8 * q + e] = fmaf(pk, c[e], acc[8 * q + e]);
                }
            }
#pragma unroll
            for (int r = 0; r < PPT; ++r)
                if (j0 + r < nm) Fp[skew(j0 + r + 16)] = acc[r];
        }
        __syncthreads();

        // ---- a4: F''_j = sum_s g_s F'_{j+H-s} (Eq. 5), 8-tap blocks
        float fpp[PPT];
#pragma unroll
        for (int r = 0; r < PPT; ++r) fpp[r] = 0.0f;
        if (own_pix) {
            for (int bk = 0; bk < nblk; ++bk) {
                const int s0 = -h + bk * TB;
                float gg[TB], win[PPT + TB - 1];
#pragma unroll
                for (int e = 0; e < TB; ++e) gg[e] = g[s0 + e + H];
                // win[q] = F'[j0 + H - s0 - 7 + q]
                const int base = j0 + H - s0 - (TB - 1) + 16;
#pragma unroll
                for (int q = 0; q < PPT + TB - 1; ++q) win[q] = Fp[skew(base + q)];
#pragma unroll
                for (int e = 0; e < TB; ++e)
#pragma unroll
                    for (int r = 0; r < PPT; ++r) fpp[r] = fmaf(gg[e], win[r - e + TB - 1], fpp[r]);
            }
        }

        // ---- a5: normal equations of Eq. 6
        float gacc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) gacc[q] = 0.0f;
        if (own_pix) {
#pragma unroll
            for (int r = 0; r < PPT; ++r) {
                const int j = j0 + r;
                const float Wj = j < p ? W[skew(j)] : 0.0f;
                if (Wj != 0.0f) {
                    float Pl[NB];
                    legendre<D>(fmaf((float)j, xstep, -1.0f), Pl);
                    const float f = fpp[r];
                    const float vv = Wj * f * f, uu = Wj * f * y[skew(j)];
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
        solve_continuum<D, NT>(gacc, P.O.fp64_ne, red, out, s_b);

        // ---- a6: residual (Eq. 7), loss (Eq. 9); delta = W eps c (unscaled)
        float racc[2] = {0.0f, 0.0f};
        {
            float bl[NB];
#pragma unroll
            for (int a = 0; a < NB; ++a) bl[a] = s_b[a];
            const bool solved = isfinite(bl[0]);
            if (own_pix && solved) {
#pragma unroll
                for (int r = 0; r < PPT; ++r) {
                    const int j = j0 + r;
                    float dlt = 0.0f;
                    const float Wj = j < p ? W[skew(j)] : 0.0f;
                    if (Wj != 0.0f) {
                        float Pl[NB];
                        legendre<D>(fmaf((float)j, xstep, -1.0f), Pl);
                        float c = 0.0f;
#pragma unroll
                        for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
                        const float e = y[skew(j)] - c * fpp[r];
                        racc[0] = fmaf(Wj * e, e, racc[0]);
                        if (c <= 0.0f) racc[1] = 1.0f;
                        dlt = Wj * e * c;
                    }
                    fpp[r] = dlt;     // the register now holds delta_j (unscaled)
                    if (j < p) Db[skew(j + L.dofs)] = dlt;
                }
            }
            if (!solved) racc[0] = NAN;
        }
        __syncthreads();     // delta buffer complete

        // ---- a7: adjoint, unscaled (dl/dF'' = kappa * delta with kappa = -1/(p l)
        // applied after the reduction).  (i) a_s = sum_j delta_j F'_{j+H-s};
        // d l/d mu = kappa sum_s gmu_s a_s.  bacc = [S, nonpos, mu, sigma, Teff, logg, FeH]
        float bacc[NADJ];
        bacc[0] = racc[0];
        bacc[1] = racc[1];
#pragma unroll
        for (int q = 2; q < NADJ; ++q) bacc[q] = 0.0f;
        if (own_pix) {
            for (int bk = 0; bk < nblk; ++bk) {
                const int s0 = -h + bk * TB;
                float win[PPT + TB - 1];
                const int base = j0 + H - s0 - (TB - 1) + 16;
#pragma unroll
                for (int q = 0; q < PPT + TB - 1; ++q) win[q] = Fp[skew(base + q)];
                float a[TB];
#pragma unroll
                for (int e = 0; e < TB; ++e) a[e] = 0.0f;
#pragma unroll
                for (int r = 0; r < PPT; ++r)
#pragma unroll
                    for (int e = 0; e < TB; ++e) a[e] = fmaf(fpp[r], win[r - e + TB - 1], a[e]);
#pragma unroll
                for (int e = 0; e < TB; ++e) {
                    bacc[2] = fmaf(gmu[s0 + e + H], a[e], bacc[2]);
                    bacc[3] = fmaf(gsg[s0 + e + H], a[e], bacc[3]);
                }
            }
        }
        // (ii) dF'_m = sum_s g_s delta_{m-H+s}; d l/d phi_k = kappa sum_m dF'_m C_km,
        // folded into the three basis derivatives per thread (sum over k of
        // dphi_k times the thread's partial sum), so the CTA reduces 3 values
        // instead of one per row.
        if (own_mod) {
            float dfp[PPT];
#pragma unroll
            for (int r = 0; r < PPT; ++r) dfp[r] = 0.0f;
            for (int bk = 0; bk < nblk; ++bk) {
                const int s0 = -h + bk * TB;
                float gg[TB], win[PPT + TB - 1];
#pragma unroll
                for (int e = 0; e < TB; ++e) gg[e] = g[s0 + e + H];
                // win[q] = delta[j0 - H + s0 + q]
                const int base = j0 - H + s0 + L.dofs;
#pragma unroll
                for (int q = 0; q < PPT + TB - 1; ++q) win[q] = Db[skew(base + q)];
#pragma unroll
                for (int e = 0; e < TB; ++e)
#pragma unroll
                    for (int r = 0; r < PPT; ++r) dfp[r] = fmaf(gg[e], win[r + e], dfp[r]);
            }
            const float* crow = M.Cp + j0;
#pragma unroll 2
            for (int k = k0; k < k1; ++k) {
                const float* ck = crow + (size_t)k * M.ldc;
                float a = 0.0f;
#pragma unroll
                for (int q = 0; q < PPT / 8; ++q) {
                    float c[8];
                    ldg8(ck + 8 * q, c);
#pragma unroll
                    for (int e = 0; e < 8; ++e) a = fmaf(dfp[8 * q + e], c[e], a);
                }
                const float4 dk = reinterpret_cast<const float4*>(dphi)[k];
                bacc[4] = fmaf(dk.x, a, bacc[4]);
                bacc[5] = fmaf(dk.y, a, bacc[5]);
                bacc[6] = fmaf(dk.z, a, bacc[6]);
            }
        }
        reduce_to_warp0<NADJ, NT>(bacc, red, out);

        // ---- a8: chain rule to x, stop rules, Adam; next step's basis + taps (warp 0)
        if (warp == 0) {
            // dl/dF''_j = -W eps c / (p l) with b held at its optimum (envelope theorem)
            const float l = sqrtf(out[0] * inv_p);
            const bool nonpos = out[1] > 0.0f;
            const float kappa = l > 0.0f ? -1.0f / ((float)p * l) : 0.0f;
            // lane k < 5: dl/dx_k (Teff, logg, FeH from the basis sums; mu, sigma from the taps)
            float gk = 0.0f;
            if (lane < 5) {
                const float src = lane < 3 ? out[4 + lane] : out[lane - 1] / M.kms_px;
                gk = kappa * src * M.phalf[lane];
            }
            const bool fin = __all_sync(0xffffffffu, lane >= 5 || isfinite(gk));
            uint32_t st = 0;
            if (lane == 0) {
                if (!isfinite(s_b[0])) st = 32u;
                else if (!(fin && isfinite(l))) st = 16u;
                if (!st) {
                    const int Wn = P.O.window;
                    if (t >= Wn && fabsf(l - ring[ri]) < P.O.tol) st = 1u;
                    rise = (t >= 1 && l > prev) ? rise + 1 : 0;
                    if (!st && rise >= Wn) st = 2u;
                    if (!st && t >= P.O.max_steps) st = 4u;
                    ring[ri] = l;
                    ri = ri + 1 == Wn ? 0 : ri + 1;      // = (t + 1) mod window
                    prev = l;
                }
                if (st && st <= 4u && nonpos) st |= 8u;
            }
            st = __shfl_sync(0xffffffffu, st, 0);
            int stop = 0;
            if (st) {
                if (lane < 5) P.theta[5 * i + lane] = phys_of(M, lane, xk);
                if (lane == 0) {
                    P.loss[i] = l;
                    P.steps[i] = t;
                    P.status[i] = st;
                    if (P.weight) P.weight[i] = s_w;
                }
                stop = 1;
            } else {
                b1t *= (double)P.O.beta1;
                b2t *= (double)P.O.beta2;
                // 1 - beta^t in double (beta2^t is close to 1 early on), the rest in float
                const float step = P.O.lr / (float)(1.0 - b1t);
                const float bc2s = sqrtf((float)(1.0 - b2t));
                if (lane < 5) {
                    mk = P.O.beta1 * mk + (1.0f - P.O.beta1) * gk;
                    vk = P.O.beta2 * vk + (1.0f - P.O.beta2) * gk * gk;
                    const float denom = sqrtf(vk) / bc2s + P.O.eps;
                    xk = fminf(1.0f, fmaxf(-1.0f, xk - step * mk / denom));
                    s_x[lane] = xk;
                }
                if (slots && t + 1 - t0 >= P.S.budget) {
                    // suspend: save the slot state; the slot stays running
                    if (lane < 5) {
                        P.S.x[5 * i + lane] = xk;
                        P.S.m[5 * i + lane] = mk;
                        P.S.v[5 * i + lane] = vk;
                    }
                    if (lane == 0) {
                        P.S.prev[i] = prev;
                        P.S.rise[i] = rise;
                        P.S.t[i] = t + 1;
                        P.S.b12[2 * i] = b1t;
                        P.S.b12[2 * i + 1] = b2t;
                    }
                    stop = 2;
                }
            }
            if (lane == 0) s_stop = stop;
            __syncwarp();
            if (!stop && !clean_step(P.O, t)) {
                int hn = warp_prepare_step(M, s_x, phi, dphi, g, gmu, gsg, s_k);
                if (lane == 0) s_h = hn;
            }
        }
        __syncthreads();
        if (s_stop == 1) break;
        // a chunk that suspends on a Clean step still applies that step's mask update,
        // as the one-shot fit does
        if (clean_step(P.O, t)) {
            // ---- stage 6 Clean update from the residual at x_t (taps g and F' still of x_t)
            const int upd = t / P.O.clean_every;
#pragma unroll
            for (int r = 0; r < PPT; ++r) fpp[r] = 0.0f;
            if (own_pix) {
                for (int bk = 0; bk < nblk; ++bk) {
                    const int s0 = -h + bk * TB;
                    float gg[TB], win[PPT + TB - 1];
#pragma unroll
                    for (int e = 0; e < TB; ++e) gg[e] = g[s0 + e + H];
                    const int base = j0 + H - s0 - (TB - 1) + 16;
#pragma unroll
                    for (int q = 0; q < PPT + TB - 1; ++q) win[q] = Fp[skew(base + q)];
#pragma unroll
                    for (int e = 0; e < TB; ++e)
#pragma unroll
                        for (int r = 0; r < PPT; ++r) fpp[r] = fmaf(gg[e], win[r - e + TB - 1], fpp[r]);
                }
            }
            float mm[PPT], wbv[PPT];
            uint32_t used = 0;
            {
                float bl[NB];
#pragma unroll
                for (int a = 0; a < NB; ++a) bl[a] = s_b[a];
                const size_t row = (size_t)i * p;
#pragma unroll
                for (int r = 0; r < PPT; ++r) {
                    const int j = j0 + r;
                    mm[r] = 0.0f;
                    wbv[r] = 0.0f;
                    if (j < p) {
                        const float f = P.flux[row + j], iv = P.ivar[row + j];
                        const bool use = P.good[row + j] && iv > 0.0f && isfinite(f) && isfinite(iv);
                        const bool edge = j < P.O.edge_px || j >= p - P.O.edge_px;
                        const float wb = (use && !edge && s_w > 0.0f) ? iv / s_imean : 0.0f;
                        float Pl[NB];
                        legendre<D>(fmaf((float)j, xstep, -1.0f), Pl);
                        float c = 0.0f;
#pragma unroll
                        for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
                        const float model = c * fpp[r];
                        const float sw = sqrtf(wb);
                        Db[skew(j + L.dofs)] = sw * (y[skew(j)] - model);
                        mm[r] = sw * model;
                        wbv[r] = wb;
                        if (W[skew(j)] > 0.0f) used |= 1u << r;
                    }
                }
            }
            __syncthreads();          // every thread is done reading F'
#pragma unroll
            for (int r = 0; r < PPT; ++r)
                if (j0 + r < p) Fp[skew(j0 + r + 16)] = mm[r];
            __syncthreads();
            const uint32_t keep = cta_clean_mask<NT, PPT>(p, j0, Db, L.dofs, Fp, 16, used,
                                                          upd == 1 ? 0.5f : 0.2f, reinterpret_cast<uint8_t*>(Fp),
                                                          s_redd, s_tot, nullptr);
#pragma unroll
            for (int r = 0; r < PPT; ++r)
                if (j0 + r < p) W[skew(j0 + r)] = ((keep >> r) & 1u) ? wbv[r] : 0.0f;
            // F' pads were overwritten by the mask scratch: zero them again
            for (int q = tid; q < 32; q += NT) {
                const int mq = q < 16 ? q - 16 : nm + q - 16;
                Fp[skew(mq + 16)] = 0.0f;
            }
            // the delta buffer pads are outside [0, p) and untouched
            if (warp == 0) {
                int hn = warp_prepare_step(M, s_x, phi, dphi, g, gmu, gsg, s_k);
                if (lane == 0) s_h = hn;
            }
            __syncthreads();
        }
        if (s_stop) break;
    }
    if (s_stop == 2) {
        for (int q = tid; q < WINMAX; q += NT) P.S.ring[(size_t)i * WINMAX + q] = ring[q];
        if (P.S.cmask && j0 < p) {
            uint32_t bits = 0;
#pragma unroll
            for (int r = 0; r < PPT; ++r)
                if (j0 + r < p && W[skew(j0 + r)] == 0.0f) bits |= 1u << r;
            P.S.cmask[(size_t)i * ((p + PPT - 1) / PPT) + tid] = (uint16_t)bits;
        }
        return;
    }
    if (P.cont && tid < NB) P.cont[(size_t)i * NB + tid] = s_b[tid];
}

}  // namespace lasp
