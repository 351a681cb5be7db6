// Shared device helpers of the grouped spectral fit (sm_103a).
//
// Per-spectrum work is done by one CTA.  Pixel j of a spectrum is owned by
// thread (j mod NT) of its CTA, so per-pixel state (F'', delta) stays in that
// thread's registers; arrays read across threads (F', the residual adjoint)
// live in shared memory, where consecutive threads touch consecutive words.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include <math.h>

#include "lasp.h"

namespace lasp {

constexpr int KMAX = 32;          // rows of one tensor-core K block (single-regime tables)
constexpr int KROWS = 96;         // interpolator rows over all regimes (CUDA-core paths)
constexpr int NREG = 3;           // Teff regimes of a piecewise interpolator
constexpr int DPS = 4;            // stride of a basis-derivative row (Teff, logg, FeH, 0)
constexpr int PPT = 16;           // pixels per thread of the per-spectrum kernels
constexpr int WINMAX = 64;        // stop-rule window supported
constexpr int HMAX = 47;          // kernel half width supported (2H+1 <= 96 taps)
constexpr int TAPS_MAX = 2 * HMAX + 1;
constexpr int MODEL_PIX_MAX = PPT * 512;   // model pixels n_pix + 2 pad of one spectrum

// Threads per CTA of the fit kernels (one-spectrum, multi-lane and the grouped
// step body): each thread owns one run of PPT model pixels and the observed
// pixels of the same indices, so the block covers the whole model grid.
inline int fit_threads(int n_model) { return n_model <= PPT * 256 ? 256 : 512; }

// Interpolator constants passed by value to every kernel.  A piecewise
// interpolator (Eq. 1 with Teff regimes) stacks the rows of its regimes,
// coolest first: regime r owns rows [reg_row[r], reg_row[r+1]) with its own
// basis box; regimes r and r+1 overlap on (tb[2r], tb[2r+1]] in Teff.
struct ModelDev {
    const float* C;          // K x n_model, row-major, FP32
    const float* Cp;         // K x ldc, rows zero-padded to a multiple of 16 floats
    int ldc;
    int K, n_pix, pad, n_model;
    float kms_px;            // c * dln: km/s per pixel
    int n_reg;               // 1..NREG
    int reg_row[NREG + 1];
    float rblo[NREG][3], rbscale[NREG][3];  // u = (v - rblo) * rbscale - 1 per regime
    float tb[2 * (NREG - 1)];               // blend bounds in Teff, increasing
    float plo[5], phalf[5];  // theta = plo + (x + 1) * phalf
    int8_t exps[KROWS * 3];
};

struct FitOpts {
    float lr, beta1, beta2, eps, tol;
    int window, max_steps, edge_px;
    float quantile;
    int fp64_ne;
    int clean, clean_every, clean_max;
    int joint;               // group RMS loss (grouped pipeline only)
};

// Skewed rows in shared memory: element i at i + i/16, so that the
// stride-16 accesses of a warp (one 16-pixel run per thread) hit 32 banks.
__host__ __device__ constexpr int skew(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int round32(int n) { return (n + 31) & ~31; }
__host__ __device__ constexpr int skew_size(int n) { return ((skew(n) + 4) + 3) & ~3; }

// u^a and u^(a-1) (0 for a = 0) for 0 <= a <= 8 without a data-dependent
// loop: eight predicated multiplies, so lanes with different exponents do not
// diverge.  The products are taken in order u * u * ... from 1.
__device__ __forceinline__ float pow_pair(float u, int a, float& am1) {
    float r = 1.0f, rm = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool take = i < a;
        rm = take ? r : rm;
        r = take ? r * u : r;
    }
    am1 = rm;
    return r;
}

// 256-bit read-only global load of 8 floats (address 32-byte aligned): one
// request per 32-byte sector instead of two 16-byte halves.  The table rows
// it reads are streamed from L2 and not reused from L1 within a CTA, so they
// are not allocated in L1 (measured 7% faster on the fused fit).
__device__ __forceinline__ void ldg8(const float* p, float (&v)[8]) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
                   "=f"(v[7])
                 : "l"(p));
}

// Physical parameters from normalised x (stage 8 rescaling).
__device__ __forceinline__ float phys_of(const ModelDev& M, int k, float x) {
    return fmaf(x + 1.0f, M.phalf[k], M.plo[k]);
}

// Teff segment of a piecewise interpolator: the number of blend bounds below
// Teff.  Even segment 2r: regime r alone; odd segment 2r+1: the blend of
// regimes r and r+1 on (tb[2r], tb[2r+1]].
__device__ __forceinline__ int teff_segment(const ModelDev& M, float teff) {
    int s = 0;
    for (int q = 0; q < 2 * (M.n_reg - 1); ++q) s += teff > M.tb[q] ? 1 : 0;
    return s;
}

// Rows with a non-zero weight at teff: [k0, k1).
__device__ __forceinline__ void active_rows(const ModelDev& M, float teff, int& k0, int& k1) {
    const int s = teff_segment(M, teff);
    const int r = s >> 1;
    k0 = M.reg_row[r];
    k1 = M.reg_row[(s & 1) ? r + 2 : r + 1];
}

// Monomial u_T^a u_g^b u_f^c of one row in a basis box (lo, scale) and its
// derivatives with respect to (Teff, logg, FeH).
__device__ __forceinline__ float monomial(const float* lo, const float* sc, const int8_t* e,
                                          const float th[3], float* d) {
    const float u0 = (log10f(th[0]) - lo[0]) * sc[0] - 1.0f;
    const float u1 = (th[1] - lo[1]) * sc[1] - 1.0f;
    const float u2 = (th[2] - lo[2]) * sc[2] - 1.0f;
    const int a = e[0], b = e[1], c = e[2];
    float qa, qb, qc;
    const float pa = pow_pair(u0, a, qa), pb = pow_pair(u1, b, qb), pc = pow_pair(u2, c, qc);
    if (d) {
        // d u_T / d Teff = scale / (Teff ln 10)
        const float du0 = sc[0] / (th[0] * 2.302585092994046f);
        d[0] = a ? (float)a * qa * pb * pc * du0 : 0.0f;
        d[1] = b ? (float)b * pa * qb * pc * sc[1] : 0.0f;
        d[2] = c ? (float)c * pa * pb * qc * sc[2] : 0.0f;
    }
    return pa * pb * pc;
}

// Row k of the basis of Eq. 1 with the regime weight folded in, and its
// derivatives d[0..2] with respect to (Teff, logg, FeH).  Row k of regime r is
// w_r(Teff) times its monomial in the regime's own basis box; w_r is 1 inside
// the regime, falls or rises linearly in Teff across a blend interval, and is
// 0 elsewhere, so d phi / d Teff carries the weight's slope.
__device__ __forceinline__ float basis_term_one(const ModelDev& M, int k, const float th[3], float (&d)[3]) {
    if (M.n_reg == 1) return monomial(M.rblo[0], M.rbscale[0], M.exps + 3 * k, th, d);
    int r = 0;
    while (r + 1 < M.n_reg && k >= M.reg_row[r + 1]) ++r;
    float w = 1.0f, dw = 0.0f;
    const int s = teff_segment(M, th[0]);
    if (s & 1) {
        const int q = s >> 1;                          // blend of regimes q and q+1
        const float lo = M.tb[s - 1], hi = M.tb[s];
        const float inv = 1.0f / (hi - lo);
        const float t = (th[0] - lo) * inv;
        if (r == q) {
            w = 1.0f - t;
            dw = -inv;
        } else if (r == q + 1) {
            w = t;
            dw = inv;
        } else {
            w = 0.0f;
        }
    } else if (r != (s >> 1)) {
        w = 0.0f;
    }
    if (w == 0.0f && dw == 0.0f) {
        d[0] = d[1] = d[2] = 0.0f;
        return 0.0f;
    }
    float dm[3];
    const float mono = monomial(M.rblo[r], M.rbscale[r], M.exps + 3 * k, th, dm);
    d[0] = fmaf(w, dm[0], dw * mono);
    d[1] = w * dm[1];
    d[2] = w * dm[2];
    return w * mono;
}

// Basis of Eq. 1: phi_k and d phi_k / d(Teff, logg, FeH) of row k (dphi row
// k at DPS k: Teff, logg, FeH, 0), with the regime weight folded in.
__device__ __forceinline__ void basis_term(const ModelDev& M, int k, const float th[3],
                                           float* phi, float* dphi) {
    if (!dphi) {
        // value only: the monomial without its derivatives
        if (M.n_reg == 1) {
            phi[k] = monomial(M.rblo[0], M.rbscale[0], M.exps + 3 * k, th, nullptr);
            return;
        }
        float d[3];
        phi[k] = basis_term_one(M, k, th, d);
        return;
    }
    float d[3];
    phi[k] = basis_term_one(M, k, th, d);
    dphi[DPS * k + 0] = d[0];
    dphi[DPS * k + 1] = d[1];
    dphi[DPS * k + 2] = d[2];
    dphi[DPS * k + 3] = 0.0f;
}

// Every row's basis term, spread over the lanes of one warp.
__device__ __forceinline__ void warp_basis(const ModelDev& M, const float th[3], float* phi,
                                           float* dphi) {
    for (int k = (threadIdx.x & 31); k < M.K; k += 32) basis_term(M, k, th, phi, dphi);
}

// Sampled Gaussian kernel of Eq. 5 on s = -H..H (index s + H), unit sum over
// |s| <= h = ceil(|mu| + 5 sigma), zero beyond; with d g / d mu and
// d g / d sigma.  Executed by one full warp; returns h (clamped to H).
__device__ __forceinline__ int kernel_taps_warp(float mu, float sig, int H, float* g,
                                                float* gmu, float* gsg) {
    const int lane = threadIdx.x & 31;
    int h = (int)ceilf(fabsf(mu) + 5.0f * sig);
    h = h > H ? H : (h < 0 ? 0 : h);
    const float is2 = 1.0f / (sig * sig), is3 = is2 / sig;
    const float inv2s2 = 0.5f * is2;
    float e[3], d[3], q[3];
    float Z = 0.0f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        int i = lane + 32 * r;
        int s = i - H;
        float ds = (float)s - mu;
        e[r] = (i <= 2 * H && s >= -h && s <= h) ? expf(-ds * ds * inv2s2) : 0.0f;
        d[r] = ds * is2;
        q[r] = ds * ds * is3;
        Z += e[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Z += __shfl_xor_sync(0xffffffffu, Z, o);
    float md = 0.0f, mq = 0.0f;
    const float iZ = 1.0f / Z;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        e[r] *= iZ;
        md += e[r] * d[r];
        mq += e[r] * q[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        md += __shfl_xor_sync(0xffffffffu, md, o);
        mq += __shfl_xor_sync(0xffffffffu, mq, o);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        int i = lane + 32 * r;
        if (i <= 2 * H) {
            g[i] = e[r];
            if (gmu) gmu[i] = e[r] * (d[r] - md);
            if (gsg) gsg[i] = e[r] * (q[r] - mq);
        }
    }
    return h;
}

// Legendre P_0..P_D at x (Bonnet recursion), Eq. 6 nodes x_j = -1 + 2 j / p.
template <int D>
__device__ __forceinline__ void legendre(float x, float (&P)[D + 1]) {
    P[0] = 1.0f;
    if (D >= 1) P[1] = x;
#pragma unroll
    for (int n = 1; n < D; ++n)
        P[n + 1] = ((float)(2 * n + 1) * x * P[n] - (float)n * P[n - 1]) * (1.0f / (float)(n + 1));
}

__device__ __forceinline__ float legendre_node(int j, int p) {
    return -1.0f + (2.0f * (float)j) / (float)p;
}

template <int D>
struct Gram {
    static constexpr int NB = D + 1;
    static constexpr int NG = NB * (NB + 1) / 2;
    static constexpr int NV = NG + NB;   // packed upper triangle + right-hand side
    __device__ static constexpr int idx(int a, int b) { return a * NB - a * (a - 1) / 2 + (b - a); }
};

// Normal-equation sums of Eq. 6 with the products of one diagonal of G paired
// into packed FMAs: entries (a, a + d) and (a + 1, a + 1 + d) share one
// __ffma2_rn, whose operands are then (v P_a, v P_a+1) and (P_a+d, P_a+d+1),
// both adjacent pairs of the basis.  Every sum receives the same fmas, in the
// same order, as the scalar triangle loop; unpack() returns them in Gram<D>'s
// packed order.  Even degrees only.
template <int D>
struct GramPairs {
    static_assert(D % 2 == 0 && D >= 2, "even Legendre degree");
    static constexpr int NB = D + 1, H2 = D / 2;
    __host__ __device__ static constexpr int pbase(int d) {
        int s = 0;
        for (int q = 0; q < d; ++q) s += (NB - q) / 2;
        return s;
    }
    __host__ __device__ static constexpr int sbase(int d) {
        int s = 0;
        for (int q = 0; q < d; ++q) s += (NB - q) & 1;
        return s;
    }
    static constexpr int NPAIR = pbase(NB), NSING = sbase(NB);
    float2 gp[NPAIR], rp[H2];
    float gs[NSING], rs;

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < NPAIR; ++i) gp[i] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < NSING; ++i) gs[i] = 0.0f;
#pragma unroll
        for (int k = 0; k < H2; ++k) rp[k] = make_float2(0.0f, 0.0f);
        rs = 0.0f;
    }

    // one pixel: G += vv P P^T, r += uu P
    __device__ __forceinline__ void add(float vv, float uu, const float (&Pl)[NB]) {
        float2 pe[H2], po[H2], va[H2];
#pragma unroll
        for (int k = 0; k < H2; ++k) {
            pe[k] = make_float2(Pl[2 * k], Pl[2 * k + 1]);
            po[k] = make_float2(Pl[2 * k + 1], Pl[2 * k + 2]);
        }
        const float2 v2 = make_float2(vv, vv);
#pragma unroll
        for (int k = 0; k < H2; ++k) va[k] = __fmul2_rn(v2, pe[k]);
        const float va_d = vv * Pl[D];
#pragma unroll
        for (int d = 0; d <= D; ++d) {
            const int n = NB - d;
#pragma unroll
            for (int a = 0; a + 1 < n; a += 2) {
                const float2 b2 = (d & 1) ? po[(a + d - 1) / 2] : pe[(a + d) / 2];
                gp[pbase(d) + a / 2] = __ffma2_rn(va[a / 2], b2, gp[pbase(d) + a / 2]);
            }
            if (n & 1) {
                const int a = n - 1;
                const float v = a == D ? va_d : va[a / 2].x;
                gs[sbase(d)] = fmaf(v, Pl[a + d], gs[sbase(d)]);
            }
        }
        const float2 u2 = make_float2(uu, uu);
#pragma unroll
        for (int k = 0; k < H2; ++k) rp[k] = __ffma2_rn(u2, pe[k], rp[k]);
        rs = fmaf(uu, Pl[D], rs);
    }

    __device__ __forceinline__ void unpack(float (&g)[Gram<D>::NV]) const {
        using Gm = Gram<D>;
#pragma unroll
        for (int d = 0; d <= D; ++d) {
            const int n = NB - d;
#pragma unroll
            for (int a = 0; a + 1 < n; a += 2) {
                g[Gm::idx(a, a + d)] = gp[pbase(d) + a / 2].x;
                g[Gm::idx(a + 1, a + 1 + d)] = gp[pbase(d) + a / 2].y;
            }
            if (n & 1) g[Gm::idx(n - 1, n - 1 + d)] = gs[sbase(d)];
        }
#pragma unroll
        for (int k = 0; k < H2; ++k) {
            g[Gm::NG + 2 * k] = rp[k].x;
            g[Gm::NG + 2 * k + 1] = rp[k].y;
        }
        g[Gm::NG + D] = rs;
    }
};

// Block-wide sum of NV floats per thread.  Partial sums per warp go to
// red[warp * NV + i]; thread i < NV adds the warps in a fixed order, so the
// result depends only on the data of this CTA.  out may alias nothing in red.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(float (&v)[NV], float* red, float* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float s = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp * NV + i] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += red[w * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Cholesky solve of the packed (D+1)x(D+1) SPD system; returns false when a
// pivot is not positive.  T = float or double.
template <int D, typename T>
__device__ bool chol_solve_packed(const T* packed, const T* rhs, T* b) {
    constexpr int n = D + 1;
    T L[n][n];
    T t[n];
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            T s = packed[Gram<D>::idx(j, i)];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > T(0))) return false;
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        T s = rhs[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * t[k];
        t[i] = s / L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        T s = t[i];
        for (int k = i + 1; k < n; ++k) s -= L[k][i] * b[k];
        b[i] = s / L[i][i];
    }
    return true;
}

// 1/sqrt(s) without a divide or a square root in T: the single-precision
// reciprocal square root, refined by Newton steps y <- y (3 - s y^2) / 2 in T
// (one step suffices for float, two give double accuracy from float).
template <typename T>
__device__ __forceinline__ T rsqrt_refined(T s) {
    T y = (T)rsqrtf((float)s);
    y = y * (T(1.5) - T(0.5) * s * y * y);
    if (sizeof(T) == 8) y = y * (T(1.5) - T(0.5) * s * y * y);
    return y;
}

// Cholesky solve with reciprocal pivots (one thread).  Returns false when a
// pivot is not positive.  Pivots use rsqrt_refined, so the double version
// needs no double-precision divide or square root.
template <int D, typename T>
__device__ __forceinline__ bool chol_solve_rcp(const T* packed, const T* rhs, T* b) {
    constexpr int n = D + 1;
    T L[n][n], id[n], t[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T s = packed[Gram<D>::idx(j, i)];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > T(0))) return false;
                id[i] = rsqrt_refined(s);
                L[i][i] = s * id[i];
            } else {
                L[i][j] = s * id[j];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < n; ++i) {
        T s = rhs[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[i][k] * t[k];
        t[i] = s * id[i];
    }
#pragma unroll
    for (int i = n - 1; i >= 0; --i) {
        T s = t[i];
#pragma unroll
        for (int k = i + 1; k < n; ++k) s -= L[k][i] * b[k];
        b[i] = s * id[i];
    }
    return true;
}

// ---- float-float (unevaluated sum hi + lo) arithmetic, for sums and
// residuals that need about twice FP32 precision without FP64 instructions.
// two_sum is Knuth's error-free addition; the product error uses one FMA.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = a + b;
    const float bp = s - a;
    const float ap = s - bp;
    return make_float2(s, (a - ap) + (b - bp));
}

// a + b for a float-float a and a float b.
__device__ __forceinline__ float2 ff_add(float2 a, float b) {
    const float2 s = two_sum(a.x, b);
    return two_sum(s.x, s.y + a.y);
}

// a + b for float-float a and b.
__device__ __forceinline__ float2 ff_add2(float2 a, float2 b) {
    const float2 s = two_sum(a.x, b.x);
    return two_sum(s.x, s.y + (a.y + b.y));
}

// a - g x for float-float a and g, float x.
__device__ __forceinline__ float2 ff_sub_mul(float2 a, float2 g, float x) {
    const float p = g.x * x;
    const float pe = fmaf(g.x, x, -p);       // g.x x = p + pe exactly
    const float2 s = two_sum(a.x, -p);
    return two_sum(s.x, s.y + a.y - pe - g.y * x);
}

// Solve of float-float normal equations (packed upper triangle) for NR
// right-hand sides by one warp (all 32 lanes call it; NR (D+1) <= 64): an
// FP32 Cholesky factor of the leading parts and one step of iterative
// refinement whose residual rhs - G x0 is taken in float-float.  For the
// Legendre Gram matrices of Eq. 6 this matches a double-precision solve of
// the same sums.  Every lane factors the leading parts in
// FP32 (the same work as one thread, so no extra latency); lane l < NR solves
// for right-hand side l; the float-float residual rows are spread over the
// lanes (row i of system l on lane l (D+1) + i, and 32 further), so the
// refinement costs one row instead of NR (D+1) rows of serial float-float
// work.  Lane l < NR returns system l's solution in b; returns false (in every
// lane) when a pivot is not positive.
template <int D, int NR>
__device__ __forceinline__ bool warp_chol_solve_ff(const float2* packed, const float2* const (&rhs)[NR],
                                                   float (&b)[D + 1]) {
    constexpr int n = D + 1;
    static_assert(NR * n <= 64, "two residual rows per lane at most");
    const int lane = threadIdx.x & 31;
    float L[n][n], id[n];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < n; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float s = packed[Gram<D>::idx(j, i)].x;
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                ok = ok && s > 0.0f;
                id[i] = rsqrt_refined(s > 0.0f ? s : 1.0f);
                L[i][i] = s * id[i];
            } else {
                L[i][j] = s * id[j];
            }
        }
    }
    if (!ok) return false;
    auto solve = [&](const float (&r)[n], float (&x)[n]) {
        float t[n];
#pragma unroll
        for (int i = 0; i < n; ++i) {
            float s = r[i];
#pragma unroll
            for (int k = 0; k < i; ++k) s -= L[i][k] * t[k];
            t[i] = s * id[i];
        }
#pragma unroll
        for (int i = n - 1; i >= 0; --i) {
            float s = t[i];
#pragma unroll
            for (int k = i + 1; k < n; ++k) s -= L[k][i] * x[k];
            x[i] = s * id[i];
        }
    };
    const int me = lane < NR ? lane : 0;          // right-hand side of this lane
    float rf[n], x0[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        float2 v = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int l = 0; l < NR; ++l)
            if (l == me) v = rhs[l][i];
        rf[i] = v.x + v.y;
    }
    solve(rf, x0);
    // residual rows: pair q = lane (+32): system q / n, row q % n
    float res[2] = {0.0f, 0.0f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = lane + 32 * h;
        const int l = q / n, i = q - (q / n) * n;
        float xl[n];
#pragma unroll
        for (int j = 0; j < n; ++j) xl[j] = __shfl_sync(0xffffffffu, x0[j], l < NR ? l : 0);
        if (q < NR * n) {
            float2 r = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int m = 0; m < NR; ++m)
                if (m == l) r = rhs[m][i];
#pragma unroll
            for (int j = 0; j < n; ++j) r = ff_sub_mul(r, packed[i <= j ? Gram<D>::idx(i, j) : Gram<D>::idx(j, i)], xl[j]);
            res[h] = r.x + r.y;
        }
    }
    // gather system me's residual rows: row i sits on lane (me n + i) mod 32, half (me n + i) / 32
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int q = me * n + i;
        const float r0 = __shfl_sync(0xffffffffu, res[0], q & 31);
        const float r1 = __shfl_sync(0xffffffffu, res[1], q & 31);
        rf[i] = q < 32 ? r0 : r1;
    }
    float dx[n];
    solve(rf, dx);
#pragma unroll
    for (int i = 0; i < n; ++i) b[i] = x0[i] + dx[i];
    return true;
}

// Warp reduce-scatter of 32 values (butterfly transpose): afterwards v[0] of
// lane l holds the warp sum of value l.  31 shuffles instead of 5 x 32.
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const float send = up ? v[i] : v[i + w];
            const float keep = up ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

// Warp sums of values 32 g .. 32 g + 31 of v (zero past NV): lane l returns the
// warp sum of value 32 g + l.  Eight values or fewer go through xor butterflies
// with the levels in the scatter's order (16, 8, 4, 2, 1), which pair the same
// lanes at every level, so the sums are bitwise those of the scatter.
template <int NV>
__device__ __forceinline__ float warp_sums_group(const float (&v)[NV], int g) {
    const int lane = threadIdx.x & 31;
    if (NV - 32 * g > 8) {
        float t[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) t[i] = (32 * g + i < NV) ? v[32 * g + i] : 0.0f;
        return warp_reduce_scatter32(t);
    }
    float mine = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (32 * g + i < NV) {
            float s = v[32 * g + i];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == i) mine = s;
        }
    return mine;
}

// Block-wide sum of NV floats per thread: FP32 within each warp (a
// reduce-scatter), the warps added in float-float (exact two-sums) by thread
// i < NV; red: (NT/32) round32(NV) floats; out[i] = (hi, lo),
// visible to every thread after the closing barrier.
template <int NV, int NT>
__device__ __forceinline__ void block_sum_ff(float (&v)[NV], float* red, float2* out) {
    constexpr int NP = (NV + 31) / 32 * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < NP / 32; ++g) red[warp * NP + 32 * g + lane] = warp_sums_group<NV>(v, g);
    __syncthreads();
    if (threadIdx.x < NV) {
        float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s = ff_add(s, red[w * NP + threadIdx.x]);
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Warp sums in double of values 32 g .. 32 g + 31 of v (zero past NV), each
// widened from float: lane l returns the sum of value 32 g + l.  More than
// eight values go through a reduce-scatter (a lane sends, at each level, the
// half of its sums that its partner keeps: 31 double additions a lane for the
// group, where an xor butterfly per value takes five a value); fewer go
// through one butterfly each.
template <int NV>
__device__ __forceinline__ double warp_sums_group_f64(const float (&v)[NV], int g) {
    const int lane = threadIdx.x & 31;
    if (NV - 32 * g > 8) {
        double t[16];
        const bool up16 = (lane & 16) != 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const double a = 32 * g + i < NV ? (double)v[32 * g + i] : 0.0;
            const double b = 32 * g + i + 16 < NV ? (double)v[32 * g + i + 16] : 0.0;
            t[i] = (up16 ? b : a) + __shfl_xor_sync(0xffffffffu, up16 ? a : b, 16);
        }
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1) {
            const bool up = (lane & w) != 0;
#pragma unroll
            for (int i = 0; i < w; ++i) {
                const double send = up ? t[i] : t[i + w];
                const double keep = up ? t[i + w] : t[i];
                t[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
            }
        }
        return t[0];
    }
    double mine = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (32 * g + i < NV) {
            double x = (double)v[32 * g + i];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == i) mine = x;
        }
    return mine;
}

// Block-wide sum of NV floats per thread with every addition in FP64: each
// thread's value is widened to double, the warp reduce-scatters in double,
// thread i < NV adds the warps in a fixed order.  redd: (NT/32) round32(NV)
// doubles; outd[i] is visible to every thread after the closing barrier.
template <int NV, int NT>
__device__ __forceinline__ void block_sum_f64(const float (&v)[NV], double* redd, double* outd) {
    constexpr int NP = (NV + 31) / 32 * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < NP / 32; ++g) redd[warp * NP + 32 * g + lane] = warp_sums_group_f64<NV>(v, g);
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += redd[w * NP + threadIdx.x];
        outd[threadIdx.x] = s;
    }
    __syncthreads();
}

// Inverse of a 5x5 symmetric positive definite matrix in FP64 (one thread):
// Cholesky factor A = L L^T, then X = L^-T L^-1 column by column.  Returns
// false when a pivot is not positive.
__device__ __forceinline__ bool inv_spd5_f64(const double (&A)[25], double (&X)[25]) {
    double L[5][5], id[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            double s = A[i * 5 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i][i] = sqrt(s);
                id[i] = 1.0 / L[i][i];
            } else {
                L[i][j] = s * id[j];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        double t[5], x[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            double s = i == c ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < i; ++k) s -= L[i][k] * t[k];
            t[i] = s * id[i];
        }
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            double s = t[i];
#pragma unroll
            for (int k = i + 1; k < 5; ++k) s -= L[k][i] * x[k];
            x[i] = s * id[i];
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) X[i * 5 + c] = x[i];
    }
    return true;
}

// Inverse of a 5x5 symmetric positive definite matrix given in float-float
// (row-major): X0 from an FP32 Cholesky factor of the leading parts, then one
// refinement X = X0 + X0 (I - A X0) with the residual in float-float.  One
// thread.  Returns false when a pivot is not positive.
__device__ __forceinline__ bool inv_spd5_ff(const float2 (&A)[25], float (&X)[25]) {
    float L[5][5], id[5], X0[25];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float s = A[i * 5 + j].x;
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0f)) return false;
                id[i] = rsqrt_refined(s);
                L[i][i] = s * id[i];
            } else {
                L[i][j] = s * id[j];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        float t[5], x[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float s = i == c ? 1.0f : 0.0f;
#pragma unroll
            for (int k = 0; k < i; ++k) s -= L[i][k] * t[k];
            t[i] = s * id[i];
        }
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            float s = t[i];
#pragma unroll
            for (int k = i + 1; k < 5; ++k) s -= L[k][i] * x[k];
            x[i] = s * id[i];
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) X0[i * 5 + c] = x[i];
    }
    float R[25];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            float2 r = make_float2(i == j ? 1.0f : 0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < 5; ++k) r = ff_sub_mul(r, A[i * 5 + k], X0[k * 5 + j]);
            R[i * 5 + j] = r.x + r.y;
        }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            float s = X0[i * 5 + j];
#pragma unroll
            for (int k = 0; k < 5; ++k) s = fmaf(X0[i * 5 + k], R[k * 5 + j], s);
            X[i * 5 + j] = s;
        }
    return true;
}

// Shared scratch prep_spectrum needs in `red` (floats): the select histogram.
constexpr int PREP_RED = 272;

// Order-preserving map of non-NaN floats to unsigned keys, and its inverse.
__device__ __forceinline__ uint32_t order_key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The k-th smallest (0-based) key of vals[0..n) by most-significant-digit
// radix select: four passes of 8-bit digit histograms in shared memory (hist:
// 258 ints), each counting only the keys that share the digits chosen so
// far.  Lanes of a warp with equal digits add their count in one atomic.
// Requires 0 <= k < n; every thread returns the key.
template <int NT>
__device__ uint32_t block_select_key(const float* vals, int n, int k, int* hist) {
    const int lane = threadIdx.x & 31;
    uint32_t prefix = 0, mask = 0;
    int kk = k;
#pragma unroll 1
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += NT) hist[b] = 0;
        __syncthreads();
        for (int j0 = threadIdx.x - lane; j0 < n; j0 += NT) {
            const int j = j0 + lane;
            int d = -1;
            if (j < n) {
                const uint32_t key = order_key(vals[j]);
                if ((key & mask) == prefix) d = (int)((key >> shift) & 255u);
            }
            const unsigned same = __match_any_sync(0xffffffffu, d);
            if (d >= 0 && lane == __ffs(same) - 1) atomicAdd(&hist[d], __popc(same));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            int c[8], tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = hist[8 * lane + q];
                tot += c[q];
            }
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            int run = incl - tot;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (run <= kk && kk < run + c[q]) {
                    hist[256] = 8 * lane + q;
                    hist[257] = kk - run;
                }
                run += c[q];
            }
        }
        __syncthreads();
        prefix |= (uint32_t)hist[256] << shift;
        mask |= 255u << shift;
        kk = hist[257];
    }
    return prefix;
}

// For a key K of vals[0..n): the count of keys <= K and the smallest key
// above K (0xffffffff if none), on every thread.  hist: 2 (NT/32) + 2 ints.
template <int NT>
__device__ void block_next_key(const float* vals, int n, uint32_t K, int* hist, int* cnt_le, uint32_t* next) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cnt = 0;
    uint32_t mn = 0xffffffffu;
    for (int j = threadIdx.x; j < n; j += NT) {
        const uint32_t key = order_key(vals[j]);
        cnt += key <= K ? 1 : 0;
        if (key > K && key < mn) mn = key;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        mn = min(mn, (uint32_t)__shfl_xor_sync(0xffffffffu, mn, o));
    }
    __syncthreads();                       // the select's last reads of hist are done
    if (lane == 0) {
        hist[2 * warp] = cnt;
        hist[2 * warp + 1] = (int)mn;
    }
    __syncthreads();
    int c = 0;
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        c += hist[2 * w];
        m = min(m, (uint32_t)hist[2 * w + 1]);
    }
    *cnt_le = c;
    *next = m;
}

// Per-spectrum preprocessing (section 3.3 step 2; Eq. 9 weights):
// w = quantile of the used flux (linear interpolation between order
// statistics), y = flux / w, W = ivar / mean(ivar over used pixels), both zero
// on masked, non-finite and edge pixels.  The two order statistics come from
// a radix select over sortbuf (p floats; unused pixels enter as +inf, above
// every used one), the same values a sort gives; red holds PREP_RED floats.
// Returns the count of pixels that enter the loss; *w_out is w.
template <int NT>
__device__ int prep_spectrum(const float* __restrict__ flux, const float* __restrict__ ivar,
                             const uint8_t* __restrict__ good, int p, int edge_px, float quantile,
                             float* y, float* W, float* sortbuf, float* red, float* w_out,
                             float* imean_out = nullptr) {
    float cnt = 0.0f, isum = 0.0f;
    for (int j = threadIdx.x; j < p; j += NT) {
        float v = INFINITY;
        float f = flux[j], iv = ivar[j];
        bool use = good[j] && iv > 0.0f && isfinite(f) && isfinite(iv);
        if (use) {
            v = f;
            cnt += 1.0f;
            isum += iv;
        }
        sortbuf[j] = v;
    }
    float acc[2] = {cnt, isum};
    float* tot = red + (NT / 32) * 2;
    block_sum<2, NT>(acc, red, tot);
    const int n = (int)tot[0];
    const float imean = n > 0 ? tot[1] / (float)n : 0.0f;
    __syncthreads();                       // tot is read: red becomes the select's scratch
    float w = NAN;
    if (n > 0) {
        int* hist = reinterpret_cast<int*>(red);
        const double pos = (double)quantile * (double)(n - 1);
        const int lo = (int)floor(pos);
        const uint32_t klo = block_select_key<NT>(sortbuf, p, lo, hist);
        const float vlo = key_value(klo);
        if (lo >= n - 1) {
            w = vlo;
        } else {
            int cle;
            uint32_t knext;
            block_next_key<NT>(sortbuf, p, klo, hist, &cle, &knext);
            const float vhi = cle >= lo + 2 ? vlo : key_value(knext);
            w = (float)((double)vlo + (pos - lo) * ((double)vhi - (double)vlo));
        }
    }
    __syncthreads();
    float nobj = 0.0f;
    for (int j = threadIdx.x; j < p; j += NT) {
        float f = flux[j], iv = ivar[j];
        bool use = good[j] && iv > 0.0f && isfinite(f) && isfinite(iv);
        bool edge = j < edge_px || j >= p - edge_px;
        if (use && !edge && w > 0.0f) {
            y[j] = f / w;
            W[j] = iv / imean;
            nobj += 1.0f;
        } else {
            y[j] = 0.0f;
            W[j] = 0.0f;
        }
    }
    float acc1[1] = {nobj};
    block_sum<1, NT>(acc1, red, tot);
    *w_out = w;
    if (imean_out) *imean_out = imean;
    return (int)tot[0];
}

// y and W from a known weight w and mean inverse variance (a resumed fit):
// the same arithmetic as prep_spectrum without the quantile.  Returns the
// count of pixels that enter the loss.
template <int NT>
__device__ int refill_spectrum(const float* __restrict__ flux, const float* __restrict__ ivar,
                               const uint8_t* __restrict__ good, int p, int edge_px, float w,
                               float imean, float* y, float* W, float* red) {
    float nobj = 0.0f;
    for (int j = threadIdx.x; j < p; j += NT) {
        float f = flux[j], iv = ivar[j];
        bool use = good[j] && iv > 0.0f && isfinite(f) && isfinite(iv);
        bool edge = j < edge_px || j >= p - edge_px;
        if (use && !edge && w > 0.0f) {
            y[j] = f / w;
            W[j] = iv / imean;
            nobj += 1.0f;
        } else {
            y[j] = 0.0f;
            W[j] = 0.0f;
        }
    }
    float acc1[1] = {nobj};
    float* tot = red + (NT / 32) * 2;
    block_sum<1, NT>(acc1, red, tot);
    return (int)tot[0];
}

}  // namespace lasp
