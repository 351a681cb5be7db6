// Forward model, its adjoint, the stage-9 Jacobian and the standalone basis
// contraction (FP32 CUDA-core forms) -- sm_103a.
#pragma once

#include "lasp_common.cuh"

namespace lasp {

struct ModelParams {
    ModelDev M;
    int N, D;
    const float* theta;   // N x 5 physical
    const float* b;       // N x (D+1)
    float* model;         // N x n_pix              (forward)
    const float* gmodel;  // N x n_pix              (backward)
    float* gtheta;        // N x 5                  (backward)
    float* gb;            // N x (D+1)              (backward)
};

__host__ inline size_t model_smem_bytes(int p, int H, int n_model) {
    return 4 * (size_t)(((n_model + 3) & ~3) + ((p + 4 * H + 3) & ~3) + 3 * 96 + (1 + DPS) * KROWS + 16 * 64);
}

// Per-spectrum basis + taps + F' into shared memory (one CTA).
template <int NT>
__device__ __forceinline__ int cta_interp(const ModelDev& M, const float* th5, float* phi, float* dphi,
                                          float* g, float* gmu, float* gsg, float* Fp, int* s_h) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        float th[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) th[k] = th5[k];
        warp_basis(M, th, phi, dphi);
        int h = kernel_taps_warp(th[3] / M.kms_px, th[4] / M.kms_px, M.pad, g, gmu, gsg);
        if (lane == 0) *s_h = h;
    }
    __syncthreads();
    int k0, k1;
    active_rows(M, th5[0], k0, k1);
    for (int mm = threadIdx.x; mm < M.n_model; mm += NT) {
        float acc = 0.0f;
        for (int k = k0; k < k1; ++k) acc = fmaf(phi[k], __ldg(M.C + (size_t)k * M.n_model + mm), acc);
        Fp[mm] = acc;
    }
    __syncthreads();
    return *s_h;
}

// model = (P b) * (G (x) phi C)  (Eqs. 1, 5, 6); one CTA per spectrum.
template <int NT, int D>
__global__ void __launch_bounds__(NT) forward_kernel(const ModelParams P) {
    constexpr int NB = D + 1;
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, H = M.pad, i = blockIdx.x;
    float* Fp = sm;
    float* g = Fp + ((M.n_model + 3) & ~3) + ((p + 4 * H + 3) & ~3);
    float* phi = g + 3 * 96;
    __shared__ int s_h;
    float th[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) th[k] = P.theta[5 * i + k];
    const int h = cta_interp<NT>(M, th, phi, nullptr, g, nullptr, nullptr, Fp, &s_h);
    float bl[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) bl[a] = P.b[(size_t)i * NB + a];
    for (int j = threadIdx.x; j < p; j += NT) {
        const float* src = Fp + j + H;
        float f = 0.0f;
        for (int s = -h; s <= h; ++s) f = fmaf(g[s + H], src[-s], f);
        float Pl[NB];
        legendre<D>(legendre_node(j, p), Pl);
        float c = 0.0f;
#pragma unroll
        for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
        P.model[(size_t)i * p + j] = c * f;
    }
}

// Hand-written adjoint of forward_kernel: gtheta (physical), gb.
template <int NT, int D>
__global__ void __launch_bounds__(NT) backward_kernel(const ModelParams P) {
    constexpr int NB = D + 1;
    constexpr int NV = NB + 5;
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, H = M.pad, nm = M.n_model, i = blockIdx.x;
    float* Fp = sm;
    float* Db = Fp + ((nm + 3) & ~3);
    float* g = Db + ((p + 4 * H + 3) & ~3);
    float* gmu = g + 96;
    float* gsg = g + 192;
    float* phi = g + 3 * 96;
    float* dphi = phi + KROWS;
    float* red = phi + (1 + DPS) * KROWS;
    float* out = red + (NT / 32) * NV;
    __shared__ int s_h;
    float th[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) th[k] = P.theta[5 * i + k];
    for (int j = threadIdx.x; j < p + 4 * H; j += NT) Db[j] = 0.0f;
    const int h = cta_interp<NT>(M, th, phi, dphi, g, gmu, gsg, Fp, &s_h);
    float bl[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) bl[a] = P.b[(size_t)i * NB + a];
    float acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0f;
    // d model_j / d b_d = P_d F''_j ; dL/dF''_j = gm_j c_j
    for (int j = threadIdx.x; j < p; j += NT) {
        const float* src = Fp + j + H;
        float f = 0.0f, am = 0.0f, as = 0.0f;
        for (int s = -h; s <= h; ++s) {
            const float fv = src[-s];
            f = fmaf(g[s + H], fv, f);
            am = fmaf(gmu[s + H], fv, am);
            as = fmaf(gsg[s + H], fv, as);
        }
        float Pl[NB];
        legendre<D>(legendre_node(j, p), Pl);
        float c = 0.0f;
#pragma unroll
        for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
        const float gm = P.gmodel[(size_t)i * p + j];
#pragma unroll
        for (int a = 0; a < NB; ++a) acc[a] = fmaf(gm * f, Pl[a], acc[a]);
        const float d = gm * c;
        acc[NB] = fmaf(d, am, acc[NB]);
        acc[NB + 1] = fmaf(d, as, acc[NB + 1]);
        Db[j + 2 * H] = d;
    }
    __syncthreads();
    // dL/dtheta_c = sum_m dF'_m sum_k dphi_kc C_km (c = Teff, logg, FeH)
    int k0, k1;
    active_rows(M, th[0], k0, k1);
    for (int mm = threadIdx.x; mm < nm; mm += NT) {
        const float* src = Db + mm + H;
        float d = 0.0f;
        for (int s = -h; s <= h; ++s) d = fmaf(g[s + H], src[s], d);
        float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f;
        for (int k = k0; k < k1; ++k) {
            const float c = __ldg(M.C + (size_t)k * nm + mm);
            e0 = fmaf(dphi[DPS * k + 0], c, e0);
            e1 = fmaf(dphi[DPS * k + 1], c, e1);
            e2 = fmaf(dphi[DPS * k + 2], c, e2);
        }
        acc[NB + 2] = fmaf(d, e0, acc[NB + 2]);
        acc[NB + 3] = fmaf(d, e1, acc[NB + 3]);
        acc[NB + 4] = fmaf(d, e2, acc[NB + 4]);
    }
    block_sum<NV, NT>(acc, red, out);
    if (threadIdx.x < NB) P.gb[(size_t)i * NB + threadIdx.x] = out[threadIdx.x];
    if (threadIdx.x < 3) P.gtheta[5 * i + threadIdx.x] = out[NB + 2 + threadIdx.x];
    if (threadIdx.x == 3) P.gtheta[5 * i + 3] = out[NB] / M.kms_px;
    if (threadIdx.x == 4) P.gtheta[5 * i + 4] = out[NB + 1] / M.kms_px;
}

// Eq. 1 alone: Fp = phi(theta) C (N x n_model), FP32 CUDA cores.
template <int NT>
__global__ void __launch_bounds__(NT) interp_fp32_kernel(ModelDev M, const float* __restrict__ theta,
                                                         float* __restrict__ Fp) {
    __shared__ float phi[KROWS];
    const int i = blockIdx.x;
    float th[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) th[k] = theta[5 * i + k];
    if (threadIdx.x < 32) warp_basis(M, th, phi, nullptr);
    __syncthreads();
    int k0, k1;
    active_rows(M, th[0], k0, k1);
    const int mm = blockIdx.y * NT + threadIdx.x;
    if (mm < M.n_model) {
        float acc = 0.0f;
        for (int k = k0; k < k1; ++k) acc = fmaf(phi[k], __ldg(M.C + (size_t)k * M.n_model + mm), acc);
        Fp[(size_t)i * M.n_model + mm] = acc;
    }
}

// ---------------------------------------------------------------------------
// Stage 9 parameter errors.  J = d r / d theta of the weighted residual
// r = sqrt(W) eps with the continuum b re-solved (variable projection), taken
// analytically: dF''/dtheta from the basis derivatives and the kernel
// derivatives; db/dtheta from the normal equations,
//   db_k = G^-1 sum_j W_j P(x_j) dF''_jk (eps_j - F''_j c_j),
//   J_jk = -sqrt(W_j) (c_j dF''_jk + F''_j (P db_k)_j).
// cov = (r.r / (n - 5)) (J^T J)^-1: J^T J summed in float-float (or FP64 with
// the FP64 normal-equation option), its 5x5 inverse and the scale in FP64.

// Shared reduction space of the errors kernel, floats a warp: 64 doubles
// (every block sum there has at most 64 values for Legendre degrees <= 8).
constexpr int ERR_RED_W = 128;

struct ErrParams {
    ModelDev M;
    FitOpts O;
    int N;
    const float* flux;
    const float* ivar;
    const uint8_t* good;
    const float* theta;
    float* sigma;
    double* cov;
    uint32_t* status;
};

__host__ inline size_t err_smem_bytes(int p, int H, int n_model, int NT) {
    size_t fl = (size_t)2 * ((p + 3) & ~3) + 4 * (size_t)((n_model + 3) & ~3) + 3 * 96 + (1 + DPS) * KROWS +
                (size_t)(NT / 32) * ERR_RED_W + 256;
    size_t sortb = (size_t)3 * ((p + 3) & ~3);
    return 4 * (fl > sortb ? fl : sortb);
}

// Two CTAs per SM at 256 threads (128 registers; the shared-memory plan of about
// 100 KB allows two): a few spills cost far less than halving the resident warps.
// The per-pixel loops are not unrolled (the per-pixel values live in local
// memory): unrolled, the kernel is one long run of code executed once per warp
// and waits on instruction fetch (1.66 -> 1.30 ms rolled, 4096 x 3909).
// F64: the sums added across the CTA and the 7x7 solves in FP64 (the
// LASP_NE_FP64 option), else in float-float.
template <int NT, int D, bool F64>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) errors_kernel(const ErrParams P) {
    using Gm = Gram<D>;
    constexpr int NB = D + 1;
    constexpr int NV = Gm::NV;
    constexpr int PPT = 16;
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, H = M.pad, nm = M.n_model;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i = blockIdx.x;
    const int pa = (p + 3) & ~3, na = (nm + 3) & ~3;
    float* y = sm;
    float* W = y + pa;
    float* Fp = W + pa;              // F', dF'/dTeff, dF'/dlogg, dF'/dFeH
    float* g = Fp + 4 * na;
    float* gmu = g + 96;
    float* gsg = g + 192;
    float* phi = g + 288;
    float* dphi = phi + KROWS;
    float* red = phi + (1 + DPS) * KROWS;
    float* outf = red + (NT / 32) * ERR_RED_W;
    float2* outff = reinterpret_cast<float2*>(outf + ((((size_t)(outf - sm)) & 1) ? 1 : 0));
    __shared__ float2 s_G[Gm::NV];
    __shared__ double s_Gd[Gm::NV], s_JJ[16];
    double* outd = reinterpret_cast<double*>(outff);
    double* redd = reinterpret_cast<double*>(red);
    constexpr bool f64 = F64;
    __shared__ float s_b[NB], s_db[5 * NB];
    __shared__ int s_h, s_ok;

    const size_t row = (size_t)i * p;
    float w;
    const int n_obj = prep_spectrum<NT>(P.flux + row, P.ivar + row, P.good + row, p, P.O.edge_px,
                                        P.O.quantile, y, W, Fp, red, &w);
    if (n_obj <= 5 || !(w > 0.0f)) {
        if (tid < 5) P.sigma[5 * i + tid] = NAN;
        if (P.cov && tid < 25) P.cov[25 * (size_t)i + tid] = NAN;
        if (P.status && tid == 0) P.status[i] = 64u;
        return;
    }
    if (warp == 0) {
        float th[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) th[k] = P.theta[5 * i + k];
        warp_basis(M, th, phi, dphi);
        int h = kernel_taps_warp(th[3] / M.kms_px, th[4] / M.kms_px, H, g, gmu, gsg);
        if (lane == 0) s_h = h;
    }
    __syncthreads();
    const int h = s_h;
    int k0, k1;
    active_rows(M, P.theta[5 * i], k0, k1);
    // F' and its three basis derivatives: 16 consecutive model pixels per thread,
    // the table rows (padded to 16 floats) from L2 with 256-bit loads, two rows
    // in flight, each load feeding the four contractions
    for (int m0 = tid * 16; m0 < nm; m0 += NT * 16) {
        float a[4][16];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int r = 0; r < 16; ++r) a[q][r] = 0.0f;
        const float* crow = M.Cp + m0;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float* ck = crow + (size_t)k * M.ldc;
            const float pk = phi[k], d0 = dphi[DPS * k + 0], d1 = dphi[DPS * k + 1], d2 = dphi[DPS * k + 2];
#pragma unroll
            for (int h8 = 0; h8 < 2; ++h8) {
                float c[8];
                ldg8(ck + 8 * h8, c);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    a[0][8 * h8 + e] = fmaf(pk, c[e], a[0][8 * h8 + e]);
                    a[1][8 * h8 + e] = fmaf(d0, c[e], a[1][8 * h8 + e]);
                    a[2][8 * h8 + e] = fmaf(d1, c[e], a[2][8 * h8 + e]);
                    a[3][8 * h8 + e] = fmaf(d2, c[e], a[3][8 * h8 + e]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (m0 + r < nm) Fp[q * na + m0 + r] = a[q][r];
    }
    __syncthreads();
    // F'' and its five derivatives per owned pixel (registers)
    float f[PPT], df[5][PPT];
    float gacc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) gacc[q] = 0.0f;
    const float ikms = 1.0f / M.kms_px;
#pragma unroll 1
    for (int r = 0; r < PPT; ++r) {
        const int j = tid + r * NT;
        f[r] = 0.0f;
#pragma unroll
        for (int k = 0; k < 5; ++k) df[k][r] = 0.0f;
        if (j < p) {
            float a0 = 0, a1 = 0, a2 = 0, a3 = 0, am = 0, as = 0;
            for (int s = -h; s <= h; ++s) {
                const int o = j + H - s;
                const float gs = g[s + H];
                const float fv = Fp[o];
                a0 = fmaf(gs, fv, a0);
                a1 = fmaf(gs, Fp[na + o], a1);
                a2 = fmaf(gs, Fp[2 * na + o], a2);
                a3 = fmaf(gs, Fp[3 * na + o], a3);
                am = fmaf(gmu[s + H], fv, am);
                as = fmaf(gsg[s + H], fv, as);
            }
            f[r] = a0;
            df[0][r] = a1;
            df[1][r] = a2;
            df[2][r] = a3;
            df[3][r] = am * ikms;
            df[4][r] = as * ikms;
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
    // the continuum of Eq. 6 at theta: float-float sums and solve, or FP64
    if constexpr (f64) {
        block_sum_f64<NV, NT>(gacc, redd, outd);
        if (tid < NV) s_Gd[tid] = outd[tid];
        __syncthreads();
        if (tid == 0) {
            double bd[NB];
            const bool ok = chol_solve_rcp<D, double>(s_Gd, s_Gd + Gm::NG, bd);
            s_ok = ok ? 1 : 0;
            for (int a = 0; a < NB; ++a) s_b[a] = (float)bd[a];
        }
    } else {
        block_sum_ff<NV, NT>(gacc, red, outff);
        if (tid < NV) s_G[tid] = outff[tid];
        __syncthreads();
        if (warp == 0) {
            const float2* const rh[1] = {s_G + Gm::NG};
            float bd[NB];
            const bool ok = warp_chol_solve_ff<D, 1>(s_G, rh, bd);
            if (lane == 0) {
                s_ok = ok ? 1 : 0;
                for (int a = 0; a < NB; ++a) s_b[a] = bd[a];
            }
        }
    }
    __syncthreads();
    if (!s_ok) {
        if (tid < 5) P.sigma[5 * i + tid] = NAN;
        if (P.cov && tid < 25) P.cov[25 * (size_t)i + tid] = NAN;
        if (P.status && tid == 0) P.status[i] = 32u;
        return;
    }
    // t_k[d] = sum_j W_j P_d dF''_jk (eps_j - F''_j c_j), and r.r
    constexpr int NT2 = 5 * NB + 1;
    float tacc[NT2];
#pragma unroll
    for (int q = 0; q < NT2; ++q) tacc[q] = 0.0f;
    float bl[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) bl[a] = s_b[a];
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
    if constexpr (f64) {
        block_sum_f64<NT2, NT>(tacc, redd, outd);
        if (tid < 5) {
            // db_k = G^-1 t_k, system k on thread k
            double dbk[NB];
            chol_solve_rcp<D, double>(s_Gd, outd + tid * NB, dbk);
            for (int a = 0; a < NB; ++a) s_db[tid * NB + a] = (float)dbk[a];
        }
        if (tid == 0) s_JJ[15] = outd[5 * NB];
    } else {
        block_sum_ff<NT2, NT>(tacc, red, outff);
        if (warp == 0) {
            // db_k = G^-1 t_k, the five systems on lanes 0..4
            const float2* const rh[5] = {outff, outff + NB, outff + 2 * NB, outff + 3 * NB, outff + 4 * NB};
            float dbk[NB];
            warp_chol_solve_ff<D, 5>(s_G, rh, dbk);
            if (lane < 5)
                for (int a = 0; a < NB; ++a) s_db[lane * NB + a] = dbk[a];
        }
        if (tid == 0) s_JJ[15] = (double)outff[5 * NB].x + (double)outff[5 * NB].y;
    }
    __syncthreads();
    // J_jk and J^T J (15 sums: FP32 over the thread's 16 pixels, FP64 across threads)
    float dbl[5][NB];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int a = 0; a < NB; ++a) dbl[k][a] = s_db[k * NB + a];
    float jj[15];
#pragma unroll
    for (int q = 0; q < 15; ++q) jj[q] = 0.0f;
#pragma unroll 1
    for (int r = 0; r < PPT; ++r) {
        const int j = tid + r * NT;
        if (j < p && W[j] != 0.0f) {
            float Pl[NB];
            legendre<D>(legendre_node(j, p), Pl);
            const float sw = sqrtf(W[j]);
            float Jr[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                float dc = 0.0f;
#pragma unroll
                for (int a = 0; a < NB; ++a) dc = fmaf(dbl[k][a], Pl[a], dc);
                Jr[k] = -sw * (cc[r] * df[k][r] + f[r] * dc);
            }
            int q = 0;
#pragma unroll
            for (int a = 0; a < 5; ++a)
#pragma unroll
                for (int b2 = a; b2 < 5; ++b2) { jj[q] = fmaf(Jr[a], Jr[b2], jj[q]); ++q; }
        }
    }
    // the 15 sums: FP32 within each thread, then float-float or FP64 across threads
    __syncthreads();                     // the db solves are done reading outff
    if constexpr (f64) {
        block_sum_f64<15, NT>(jj, redd, outd);
        if (tid < 15) s_JJ[tid] = outd[tid];
    } else {
        block_sum_ff<15, NT>(jj, red, outff);
        if (tid < 15) s_JJ[tid] = (double)outff[tid].x + (double)outff[tid].y;
    }
    __syncthreads();
    if (tid == 0) {
        // cov = s^2 (J^T J)^-1: the 5x5 inverse and the scale in FP64
        double A[25], Ai[25];
        int q = 0;
        for (int a = 0; a < 5; ++a)
            for (int b2 = a; b2 < 5; ++b2) {
                A[a * 5 + b2] = s_JJ[q];
                A[b2 * 5 + a] = s_JJ[q];
                ++q;
            }
        const bool ok = inv_spd5_f64(A, Ai);
        const double s2 = s_JJ[15] / (double)(n_obj - 5);
        for (int k = 0; k < 5; ++k) P.sigma[5 * i + k] = ok ? (float)sqrt(s2 * Ai[k * 5 + k]) : NAN;
        if (P.cov)
            for (int k = 0; k < 25; ++k) P.cov[25 * (size_t)i + k] = ok ? s2 * Ai[k] : NAN;
        if (P.status) P.status[i] = ok ? 0u : 32u;
    }
}

}  // namespace lasp
