// Fused fit with S spectra per CTA (FP32 CUDA-core form) -- sm_103a.
//
// fit_kernel spends most of an Adam step streaming the table from L2 twice:
// once for F' = phi C (Eq. 1) and once for the adjoint contraction
// d l / d phi_k = sum_m dF'_m C_km.  Here one CTA carries S spectra ("lanes")
// through their steps side by side and loads each table value once for all S
// lanes, so the table traffic per spectrum-step falls by S.  Everything else
// runs lane after lane with fit_kernel's code, thread ownership and order of
// every sum, so each spectrum gets bitwise the result fit_kernel gives it
// (rows outside a lane's active range contribute exact zeros: its phi and
// dphi vanish there).
//
// The grid is persistent: a lane whose spectrum stops takes the next one from
// a global counter, so no lane idles while spectra remain.  The per-spectrum
// preprocessing (y, W and the weight quantile) runs before, in fit_prep_kernel
// at full occupancy, instead of stalling a CTA at each refill; it leaves y and
// W in a global workspace row per spectrum, which the fit reads from L2 each
// step instead of keeping it in shared memory.  Each lane's F' and delta share
// one buffer, so four lanes take 95 KB of shared memory at 3909 pixels; at two
// CTAs per SM (eight spectra in flight) the table traffic per spectrum-step is
// a quarter of fit_kernel's.  Measured on the 4096 x 3909 batch (fit_kernel:
// 30.8 ms): four lanes at two CTAs per SM 23.6 ms, three lanes 24.1 ms, two
// lanes at three CTAs per SM 24.6 ms (before the later refinements, which
// brought four lanes to 19.3 ms).
//
// Five variants (MODE): the plain batch fit (MULTI_PLAIN); the batch fit with
// the Clean update (MULTI_CLEAN; stage 6, a lane's mask lives in its W row) or
// with the FP64 normal equations (MULTI_NE64);
// resumable slots (MULTI_SLOTS: a lane resumes a running slot from its saved
// state, suspends it after the step budget, and takes the next one from a
// list of running slots); and MULTI_FULL, resumable slots plus the Clean
// update and the FP64 normal equations.  Each variant compiles only what it
// runs, so the lighter ones spill less.
#pragma once

#include "lasp_clean.cuh"
#include "lasp_fit.cuh"

namespace lasp {

struct MultiWs {
    float* yw;      // N rows of 2 ldw floats: y, then W; zero beyond p
    float* wq;      // N: the weight w of each spectrum, NaN where preprocessing decided the fit
    float* im;      // N: the mean inverse variance of each spectrum (Clean's base weights)
    int ldw;        // row stride: p rounded up to 16
    int* next;      // index of the next spectrum to take (starts at 0); with a
                    // slot list, next[1] is the list's length
    const int* list;  // resumable slots: the running slots of this step, else nullptr
};

// The running slots of a pool, compacted into list[0 .. next[1]) (any order;
// next[0..1] cleared before).  One thread per slot.
static __global__ void slots_running_list(int n, const uint32_t* __restrict__ status, int* list, int* next) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && status[i] == 128u) list[atomicAdd(&next[1], 1)] = i;
}

// Shared-memory plan (floats): per lane [B | g | gmu | gsg | phi | dphi | ring]
// at lane * lane_stride, then the CTA's reduction buffers.  B holds the lane's
// F' (model pixel m at skew(m + 16)) until the last F' window of a step is
// read, then its delta (pixel j at skew(j + dofs)); each step rewrites every
// position either layout reads, pads included.
struct MultiSmem {
    int Fp, Db, g, gmu, gsg, phi, dphi, ring, lane, part, red, out, total, dofs;
    // full: the FULL variant, whose FP64 normal equations need 2 NV floats a warp in red
    __host__ __device__ MultiSmem(int p, int H, int n_model, int NT, int D, int K, int S, bool full) {
        const int NB = D + 1, NV = NB * (NB + 1) / 2 + NB;
        const int nv_max = round32(NV > NADJ * S ? NV : NADJ * S);
        const int red_w = full && 2 * round32(NV) > nv_max ? 2 * round32(NV) : nv_max;   // floats a warp
        dofs = 2 * H + 8;
        int nb = skew_size(n_model + 32);
        if (skew_size(p + 4 * H + 40) > nb) nb = skew_size(p + 4 * H + 40);
        int o = 0;
        Fp = o;
        Db = o;   o += (nb + 3) & ~3;
        g = o;    o += TAPBUF;
        gmu = o;  o += TAPBUF;
        gsg = o;  o += TAPBUF;
        phi = o;  o += round32(K);
        dphi = o; o += DPS * round32(K);
        ring = o; o += WINMAX;
        lane = o;
        o *= S;
        part = o; o += 4 * S * NT;       // per-thread lane sums, [4 s + q][thread]
        red = o;  o += (NT / 32) * red_w;
        out = o;  o += 2 * nv_max + 16;
        total = o;
    }
};

__host__ inline size_t fit_multi_smem_bytes(int p, int H, int n_model, int NT, int D, int K, int S, bool full) {
    return 4 * (size_t)MultiSmem(p, H, n_model, NT, D, K, S, full).total;
}

// Preprocessing of every spectrum before the fit (section 3.3 step 2), one CTA
// per spectrum at full occupancy: y and W into the spectrum's workspace row,
// w into wq, and the final result of spectra with too few usable pixels
// (status LASP_ST_NODATA, as fit_kernel writes it).  Shared memory:
// fit_prep_smem_bytes.
__host__ __device__ inline int fit_prep_smem_floats(int p) { return ((p + 3) & ~3) + PREP_RED; }

template <int NT, int D>
__global__ void __launch_bounds__(NT) fit_prep_kernel(const FitParams P, const MultiWs Wk) {
    constexpr int NB = D + 1;
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, tid = threadIdx.x, i = blockIdx.x;
    float* yr = Wk.yw + (size_t)i * 2 * Wk.ldw;
    float* wr = yr + Wk.ldw;
    const size_t row = (size_t)i * p;
    float w, imean;
    const int n_obj = prep_spectrum<NT>(P.flux + row, P.ivar + row, P.good + row, p, P.O.edge_px,
                                        P.O.quantile, yr, wr, sm, sm + ((p + 3) & ~3), &w, &imean);
    for (int q = p + tid; q < Wk.ldw; q += NT) {
        yr[q] = 0.0f;
        wr[q] = 0.0f;
    }
    const bool nodata = n_obj < NB + 5 || !(w > 0.0f) || !isfinite(w);
    if (tid == 0) {
        Wk.wq[i] = nodata ? NAN : w;
        Wk.im[i] = imean;
    }
    if (!nodata) return;
    if (tid < 5) {
        const float xx = (P.theta0[5 * i + tid] - M.plo[tid]) / M.phalf[tid] - 1.0f;
        P.theta[5 * i + tid] = phys_of(M, tid, fminf(1.0f, fmaxf(-1.0f, xx)));
    }
    if (tid == 0) {
        P.loss[i] = NAN;
        P.steps[i] = 0;
        P.status[i] = 64u;
        if (P.weight) P.weight[i] = w;
    }
    if (P.cont && tid < NB) P.cont[(size_t)i * NB + tid] = NAN;
}

// Preprocessing of spectra admitted into resumable slots (idx: their slot
// indices): y and W into the slots' workspace rows, w and the mean ivar into
// the slot state, the initial Adam state, and the final result of spectra
// with too few usable pixels (status LASP_ST_NODATA).
template <int NT, int D>
__global__ void __launch_bounds__(NT) fit_prep_slots_kernel(const FitParams P, const MultiWs Wk,
                                                            const int32_t* __restrict__ idx) {
    constexpr int NB = D + 1;
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, tid = threadIdx.x, i = idx[blockIdx.x];
    float* yr = Wk.yw + (size_t)i * 2 * Wk.ldw;
    float* wr = yr + Wk.ldw;
    const size_t row = (size_t)i * p;
    float w, imean;
    const int n_obj = prep_spectrum<NT>(P.flux + row, P.ivar + row, P.good + row, p, P.O.edge_px,
                                        P.O.quantile, yr, wr, sm, sm + ((p + 3) & ~3), &w, &imean);
    for (int q = p + tid; q < Wk.ldw; q += NT) {
        yr[q] = 0.0f;
        wr[q] = 0.0f;
    }
    const bool nodata = n_obj < NB + 5 || !(w > 0.0f) || !isfinite(w);
    if (tid < 5) {
        const float xx = fminf(1.0f, fmaxf(-1.0f, (P.theta0[5 * i + tid] - M.plo[tid]) / M.phalf[tid] - 1.0f));
        if (nodata) {
            P.theta[5 * i + tid] = phys_of(M, tid, xx);
        } else {
            P.S.x[5 * i + tid] = xx;
            P.S.m[5 * i + tid] = 0.0f;
            P.S.v[5 * i + tid] = 0.0f;
        }
    }
    if (tid == 0) {
        P.S.w[i] = w;
        P.S.imean[i] = imean;
        if (nodata) {
            P.loss[i] = NAN;
            P.steps[i] = 0;
            P.status[i] = 64u;
            if (P.weight) P.weight[i] = w;
        } else {
            P.S.prev[i] = 0.0f;
            P.S.rise[i] = 0;
            P.S.t[i] = 0;
        }
    }
    if (nodata && P.cont && tid < NB) P.cont[(size_t)i * NB + tid] = NAN;
}

// Order in which the batch fit takes the spectra of a piecewise interpolator:
// grouped by the Teff segment (a regime alone, or the blend of two) of their
// starting parameters, so that a CTA's four lanes tend to need the same table
// rows and its table passes run over fewer of them.  A counting sort: segment
// and count per spectrum, offsets (one thread; it also sets the list length
// next[1] = N), scatter.  Each spectrum's fit does not depend on the order.
static __global__ void regime_count_kernel(const ModelDev M, int N, const float* __restrict__ theta0,
                                           int* __restrict__ seg, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float x = fminf(1.0f, fmaxf(-1.0f, (theta0[5 * i] - M.plo[0]) / M.phalf[0] - 1.0f));
    const int s = teff_segment(M, phys_of(M, 0, x));
    seg[i] = s;
    atomicAdd(&count[s], 1);
}
static __global__ void regime_offsets_kernel(int N, int n_seg, int* count, int* next) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int o = 0;
    for (int s = 0; s < n_seg; ++s) {
        const int c = count[s];
        count[s] = o;
        o += c;
    }
    next[1] = N;
}
static __global__ void regime_scatter_kernel(int N, const int* __restrict__ seg, int* count, int* order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) order[atomicAdd(&count[seg[i]], 1)] = i;
}

template <int NT, int S>
__host__ __device__ constexpr int multi_min_blocks() {
    return NT == 256 ? (S <= 2 ? 3 : 2) : 1;
}

constexpr int MULTI_PLAIN = 0, MULTI_FULL = 1, MULTI_SLOTS = 2, MULTI_CLEAN = 3, MULTI_NE64 = 4;

template <int NT, int D, int S, int MODE>
__global__ void __launch_bounds__(NT, multi_min_blocks<NT, S>()) fit_multi_kernel(const FitParams P,
                                                                                  const MultiWs Wk) {
    using Gm = Gram<D>;
    constexpr int NB = D + 1;
    constexpr int NV = Gm::NV;
    static_assert(S >= 1 && S <= NT / 32, "one warp per lane runs the lane's Adam step");
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = P.M;
    const int p = M.n_pix, H = M.pad, nm = M.n_model;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr bool FULL = MODE == MULTI_FULL;
    constexpr bool CLEAN = FULL || MODE == MULTI_CLEAN;      // the Clean update compiled in
    constexpr bool NE64 = FULL || MODE == MULTI_NE64;        // the FP64 normal equations compiled in
    const MultiSmem L(p, H, nm, NT, D, M.K, S, NE64);
    float* red = sm + L.red;
    float* out = sm + L.out;
    __shared__ float s_x[S][5], s_b[S][NB], s_w[S];
    __shared__ int s_h[S], s_k[S][2], s_i[S], s_need[S], s_next, s_cln[S];
    __shared__ double s_redd[3 * (NT / 32)], s_tot[3];

    // Adam and stop-rule state of lane s: registers of warp s (parameter k on
    // its lane k < 5; step count, ring slot and rule state on every lane).
    float xk = 0.0f, mk = 0.0f, vk = 0.0f, prev = 0.0f;
    int rise = 0, ri = 0, t = 0, t0 = 0;
    double b1t = 1.0, b2t = 1.0;
    // resumable slots (P.S.x set): a lane takes running slots, resumes each from
    // its saved state and suspends it after P.S.budget steps
    const bool slots = (MODE == MULTI_FULL || MODE == MULTI_SLOTS) && P.S.x != nullptr;

    if (tid < S) {
        s_i[tid] = -1;
        s_need[tid] = 1;
        s_cln[tid] = -1;
    }
    for (int q = tid; q < S * L.lane; q += NT) sm[q] = 0.0f;
    __syncthreads();

    const float inv_p = 1.0f / (float)p;
    const int j0 = tid * PPT;
    const bool own_pix = j0 < p;
    const bool own_mod = j0 < nm;
    const float xstep = 2.0f / (float)p;

    for (;;) {
        // ---- take the next spectrum into every lane whose fit stopped
#pragma unroll 1
        for (int s = 0; s < S; ++s) {
            if (!s_need[s]) continue;
            float* base = sm + s * L.lane;
            for (;;) {
                if (tid == 0) {
                    const int q = atomicAdd(Wk.next, 1);
                    s_next = Wk.list ? (q < Wk.next[1] ? Wk.list[q] : P.N) : q;
                }
                __syncthreads();
                const int i = s_next;
                if (i >= P.N) {
                    if (tid == 0) {
                        s_i[s] = -1;
                        s_need[s] = 0;
                    }
                    __syncthreads();
                    break;
                }
                const bool take = slots ? P.status[i] == 128u : !isnan(Wk.wq[i]);
                if (!take) {              // slot not running, or result written by the preprocessing
                    __syncthreads();
                    continue;
                }
                const float w = slots ? P.S.w[i] : Wk.wq[i];
                if (warp == s) {
                    if (slots) {
                        t0 = t = P.S.t[i];
                        ri = t0 % P.O.window;
                        prev = P.S.prev[i];
                        rise = P.S.rise[i];
                        b1t = t0 > 0 ? P.S.b12[2 * i] : 1.0;        // saved with the slot, exactly
                        b2t = t0 > 0 ? P.S.b12[2 * i + 1] : 1.0;
                        if (lane < 5) {
                            xk = P.S.x[5 * i + lane];
                            mk = P.S.m[5 * i + lane];
                            vk = P.S.v[5 * i + lane];
                        }
                        for (int q = lane; q < WINMAX; q += 32) base[L.ring + q] = P.S.ring[(size_t)i * WINMAX + q];
                    } else {
                        mk = vk = prev = 0.0f;
                        rise = ri = t = t0 = 0;
                        b1t = b2t = 1.0;
                        if (lane < 5) {
                            const float xx = (P.theta0[5 * i + lane] - M.plo[lane]) / M.phalf[lane] - 1.0f;
                            xk = fminf(1.0f, fmaxf(-1.0f, xx));
                        }
                    }
                    if (lane < 5) s_x[s][lane] = xk;
                    __syncwarp();
                    const int hn = warp_prepare_step(M, s_x[s], base + L.phi, base + L.dphi, base + L.g,
                                                     base + L.gmu, base + L.gsg, s_k[s]);
                    if (lane == 0) {
                        s_h[s] = hn;
                        s_i[s] = i;
                        s_need[s] = 0;
                        s_w[s] = w;
                    }
                }
                __syncthreads();
                break;
            }
        }
        bool any = false;
        int kb = M.K, ke = 0;
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (s_i[s] >= 0) {
                any = true;
                kb = min(kb, s_k[s][0]);
                ke = max(ke, s_k[s][1]);
            }
        if (!any) break;

        // ---- a3 for every lane: F'_s = phi_s C (Eq. 1), each table value loaded once.
        // Adjacent model pixels go through one packed FMA (__ffma2_rn: two IEEE
        // fmas, the same results as fmaf), halving the FMA instructions.
        if (own_mod) {
            float2 acc[S][PPT / 2];
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int r = 0; r < PPT / 2; ++r) acc[s][r] = make_float2(0.0f, 0.0f);
            const float* crow = M.Cp + j0;
#pragma unroll 4
            for (int k = kb; k < ke; ++k) {
                float2 pk[S];
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const float v = sm[s * L.lane + L.phi + k];
                    pk[s] = make_float2(v, v);
                }
                const float* ck = crow + (size_t)k * M.ldc;
#pragma unroll
                for (int q = 0; q < PPT / 8; ++q) {
                    float c[8];
                    ldg8(ck + 8 * q, c);
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            acc[s][4 * q + e] = __ffma2_rn(pk[s], make_float2(c[2 * e], c[2 * e + 1]), acc[s][4 * q + e]);
                }
            }
#pragma unroll
            for (int s = 0; s < S; ++s) {
                float* Fp = sm + s * L.lane + L.Fp;
#pragma unroll
                for (int r = 0; r < PPT; ++r)
                    if (j0 + r < nm) Fp[skew(j0 + r + 16)] = (r & 1) ? acc[s][r >> 1].y : acc[s][r >> 1].x;
            }
        }
        // F' pads (model pixels [-16, 0) and [n_model, n_model + 16)) over the last delta
        if (tid < 32) {
            const int m = tid < 16 ? tid - 16 : nm + tid - 16;
#pragma unroll
            for (int s = 0; s < S; ++s) sm[s * L.lane + L.Fp + skew(m + 16)] = 0.0f;
        }
        __syncthreads();

        // ---- per lane: a4 broadening, a5 normal equations and solve, a6 residual,
        // a7 (i) tap sums; the code of fit_kernel with the lane's buffers
        // one copy of the per-lane code (lane loop not unrolled: the unrolled form
        // missed in the instruction cache); each thread's four sums of a lane
        // wait in shared memory for the end-of-step reduction
#pragma unroll 1
        for (int s = 0; s < S; ++s) {
            if (s_i[s] < 0) continue;
            float* Fp = sm + s * L.lane + L.Fp;
            float* Db = sm + s * L.lane + L.Db;      // the same buffer, delta layout
            const float* g = sm + s * L.lane + L.g;
            const float* gmu = sm + s * L.lane + L.gmu;
            const float* gsg = sm + s * L.lane + L.gsg;
            const float* yr = Wk.yw + (size_t)s_i[s] * 2 * Wk.ldw;
            const float* wr = yr + Wk.ldw;
            const int h = s_h[s];
            const int nblk = (2 * h + 1 + TB - 1) / TB;

            float fpp[PPT];
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

            // the lane's y and W, read from its workspace row (L2) here and again
            // for the residual: with four lanes there is no room to keep them
            float gacc[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) gacc[q] = 0.0f;
            if (own_pix) {
#pragma unroll
                for (int r4 = 0; r4 < PPT; r4 += 4) {
                    const float4 y4 = *reinterpret_cast<const float4*>(yr + j0 + r4);
                    const float4 w4 = *reinterpret_cast<const float4*>(wr + j0 + r4);
                    const float yv[4] = {y4.x, y4.y, y4.z, y4.w}, wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int r = r4 + u, j = j0 + r;
                        const float Wj = j < p ? wv[u] : 0.0f;
                        if (Wj != 0.0f) {
                            float Pl[NB];
                            legendre<D>(fmaf((float)j, xstep, -1.0f), Pl);
                            const float f = fpp[r];
                            const float vv = Wj * f * f, uu = Wj * f * yv[u];
#pragma unroll
                            for (int a = 0; a < NB; ++a) {
                                const float va = vv * Pl[a];
#pragma unroll
                                for (int b2 = a; b2 < NB; ++b2)
                                    gacc[Gm::idx(a, b2)] = fmaf(va, Pl[b2], gacc[Gm::idx(a, b2)]);
                                gacc[Gm::NG + a] = fmaf(uu, Pl[a], gacc[Gm::NG + a]);
                            }
                        }
                    }
                }
            }
            solve_continuum<D, NT, NE64>(gacc, P.O.fp64_ne, red, out, s_b[s]);

            // a6: residual (Eq. 7), loss (Eq. 9); delta = W eps c (unscaled)
            float racc[2] = {0.0f, 0.0f};
            {
                float bl[NB];
#pragma unroll
                for (int a = 0; a < NB; ++a) bl[a] = s_b[s][a];
                const bool solved = isfinite(bl[0]);
                if (own_pix && solved) {
#pragma unroll
                    for (int r4 = 0; r4 < PPT; r4 += 4) {
                        const float4 y4 = *reinterpret_cast<const float4*>(yr + j0 + r4);
                        const float4 w4 = *reinterpret_cast<const float4*>(wr + j0 + r4);
                        const float yv[4] = {y4.x, y4.y, y4.z, y4.w}, wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int r = r4 + u, j = j0 + r;
                            float dlt = 0.0f;
                            const float Wj = j < p ? wv[u] : 0.0f;
                            if (Wj != 0.0f) {
                                float Pl[NB];
                                legendre<D>(fmaf((float)j, xstep, -1.0f), Pl);
                                float c = 0.0f;
#pragma unroll
                                for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
                                const float e = yv[u] - c * fpp[r];
                                racc[0] = fmaf(Wj * e, e, racc[0]);
                                if (c <= 0.0f) racc[1] = 1.0f;
                                dlt = Wj * e * c;
                            }
                            fpp[r] = dlt;
                        }
                    }
                }
                if (!solved) racc[0] = NAN;
            }
            float bmu = 0.0f, bsg = 0.0f;
            // a7 (i): a_s = sum_j delta_j F'_{j+H-s}, into d/dmu and d/dsigma
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
                        bmu = fmaf(gmu[s0 + e + H], a[e], bmu);
                        bsg = fmaf(gsg[s0 + e + H], a[e], bsg);
                    }
                }
            }
            float* part = sm + L.part + 4 * s * NT + tid;
            part[0] = racc[0];
            part[NT] = racc[1];
            part[2 * NT] = bmu;
            part[3 * NT] = bsg;
            __syncthreads();      // the lane's last F' window is read: the buffer takes delta
            if (own_pix)
#pragma unroll
                for (int r = 0; r < PPT; ++r)
                    if (j0 + r < p) Db[skew(j0 + r + L.dofs)] = fpp[r];
            // delta pads: pixels [-dofs, 0) and [p, p + 2H + 32)
            if (tid < 4 * H + 40) {
                const int q = tid < L.dofs ? tid : p + tid;
                Db[skew(q)] = 0.0f;
            }
        }
        __syncthreads();     // every lane's delta buffer complete

        // ---- a7 (ii): dF'_s = g_s (x) delta_s per lane, then one table pass for all
        // lanes: d l / d phi_k = sum_m dF'_m C_km folded into the basis derivatives
        // basis sums d l / d(Teff, logg, FeH) of each lane; the lane's other four
        // sums join them from shared memory after the table pass
        float bph[S][3];
#pragma unroll
        for (int s = 0; s < S; ++s) bph[s][0] = bph[s][1] = bph[s][2] = 0.0f;
        if (own_mod) {
            float dfp[S][PPT];
#pragma unroll
            for (int s = 0; s < S; ++s) {
#pragma unroll
                for (int r = 0; r < PPT; ++r) dfp[s][r] = 0.0f;
                if (s_i[s] < 0) continue;
                const float* Db = sm + s * L.lane + L.Db;
                const float* g = sm + s * L.lane + L.g;
                const int h = s_h[s];
                const int nblk = (2 * h + 1 + TB - 1) / TB;
                for (int bk = 0; bk < nblk; ++bk) {
                    const int s0 = -h + bk * TB;
                    float gg[TB], win[PPT + TB - 1];
#pragma unroll
                    for (int e = 0; e < TB; ++e) gg[e] = g[s0 + e + H];
                    const int base = j0 - H + s0 + L.dofs;
#pragma unroll
                    for (int q = 0; q < PPT + TB - 1; ++q) win[q] = Db[skew(base + q)];
#pragma unroll
                    for (int e = 0; e < TB; ++e)
#pragma unroll
                        for (int r = 0; r < PPT; ++r) dfp[s][r] = fmaf(gg[e], win[r + e], dfp[s][r]);
                }
            }
            // lanes in pairs: one packed FMA carries the dot products of lanes
            // 2u and 2u + 1 (each the same sequence of fmas as alone)
            constexpr int SP = (S + 1) / 2;
            float2 dpair[SP][PPT];
#pragma unroll
            for (int u = 0; u < SP; ++u)
#pragma unroll
                for (int r = 0; r < PPT; ++r)
                    dpair[u][r] = make_float2(dfp[2 * u][r], 2 * u + 1 < S ? dfp[2 * u + 1][r] : 0.0f);
            const float* crow = M.Cp + j0;
#pragma unroll 4
            for (int k = kb; k < ke; ++k) {
                const float* ck = crow + (size_t)k * M.ldc;
                float c[PPT];
#pragma unroll
                for (int q = 0; q < PPT / 8; ++q) {
                    float c8[8];
                    ldg8(ck + 8 * q, c8);
#pragma unroll
                    for (int e = 0; e < 8; ++e) c[8 * q + e] = c8[e];
                }
#pragma unroll
                for (int u = 0; u < SP; ++u) {
                    float2 a2 = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int r = 0; r < PPT; ++r) a2 = __ffma2_rn(dpair[u][r], make_float2(c[r], c[r]), a2);
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int s = 2 * u + h2;
                        if (s >= S) continue;
                        const float a = h2 ? a2.y : a2.x;
                        const float4 dk = reinterpret_cast<const float4*>(sm + s * L.lane + L.dphi)[k];
                        bph[s][0] = fmaf(dk.x, a, bph[s][0]);
                        bph[s][1] = fmaf(dk.y, a, bph[s][1]);
                        bph[s][2] = fmaf(dk.z, a, bph[s][2]);
                    }
                }
            }
        }
        float bacc[S * NADJ];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const bool act = s_i[s] >= 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) bacc[NADJ * s + q] = act ? sm[L.part + (4 * s + q) * NT + tid] : 0.0f;
#pragma unroll
            for (int q = 0; q < 3; ++q) bacc[NADJ * s + 4 + q] = bph[s][q];
        }
        reduce_to_warp0<S * NADJ, NT>(bacc, red, out);
        __syncthreads();

        // ---- a8 per lane on warp s: chain rule to x, stop rules, Adam, next basis + taps
        if (warp < S && s_i[warp] >= 0) {
            const int s = warp;
            const int i = s_i[s];
            const float* o = out + NADJ * s;
            float* base = sm + s * L.lane;
            float* ring = base + L.ring;
            const float l = sqrtf(o[0] * inv_p);
            const bool nonpos = o[1] > 0.0f;
            const float kappa = l > 0.0f ? -1.0f / ((float)p * l) : 0.0f;
            float gk = 0.0f;
            if (lane < 5) {
                const float src = lane < 3 ? o[4 + lane] : o[lane - 1] / M.kms_px;
                gk = kappa * src * M.phalf[lane];
            }
            const bool fin = __all_sync(0xffffffffu, lane >= 5 || isfinite(gk));
            uint32_t st = 0;
            if (lane == 0) {
                if (!isfinite(s_b[s][0])) st = 32u;
                else if (!(fin && isfinite(l))) st = 16u;
                if (!st) {
                    const int Wn = P.O.window;
                    if (t >= Wn && fabsf(l - ring[ri]) < P.O.tol) st = 1u;
                    rise = (t >= 1 && l > prev) ? rise + 1 : 0;
                    if (!st && rise >= Wn) st = 2u;
                    if (!st && t >= P.O.max_steps) st = 4u;
                    ring[ri] = l;
                    ri = ri + 1 == Wn ? 0 : ri + 1;
                    prev = l;
                }
                if (st && st <= 4u && nonpos) st |= 8u;
            }
            st = __shfl_sync(0xffffffffu, st, 0);
            if (st) {
                if (lane < 5) P.theta[5 * i + lane] = phys_of(M, lane, xk);
                if (lane == 0) {
                    P.loss[i] = l;
                    P.steps[i] = t;
                    P.status[i] = st;
                    if (P.weight) P.weight[i] = s_w[s];
                    s_need[s] = 1;
                }
                if (P.cont && lane < NB) P.cont[(size_t)i * NB + lane] = s_b[s][lane];
            } else {
                b1t *= (double)P.O.beta1;
                b2t *= (double)P.O.beta2;
                const float step = P.O.lr / (float)(1.0 - b1t);
                const float bc2s = sqrtf((float)(1.0 - b2t));
                if (lane < 5) {
                    mk = P.O.beta1 * mk + (1.0f - P.O.beta1) * gk;
                    vk = P.O.beta2 * vk + (1.0f - P.O.beta2) * gk * gk;
                    const float denom = sqrtf(vk) / bc2s + P.O.eps;
                    xk = fminf(1.0f, fmaxf(-1.0f, xk - step * mk / denom));
                    s_x[s][lane] = xk;
                }
                __syncwarp();
                if (slots && t + 1 - t0 >= P.S.budget) {
                    // suspend: save the slot state; the slot stays running (a Clean
                    // update of this step still follows below)
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
                        s_need[s] = 1;
                    }
                    for (int q = lane; q < WINMAX; q += 32) P.S.ring[(size_t)i * WINMAX + q] = ring[q];
                }
                if (CLEAN && clean_step(P.O, t)) {
                    // the Clean update below needs the basis and taps of x_t
                    if (lane == 0) s_cln[s] = t;
                } else {
                    const int hn = warp_prepare_step(M, s_x[s], base + L.phi, base + L.dphi, base + L.g,
                                                     base + L.gmu, base + L.gsg, s_k[s]);
                    if (lane == 0) s_h[s] = hn;
                }
                ++t;
            }
        }
        __syncthreads();

        // ---- stage 6 Clean update of every lane that evaluated a Clean step,
        // from the residual at x_t (the code of fit_kernel's update).  The lane's
        // F' of x_t was overwritten by its delta, so one table pass recomputes
        // it; two other lanes' buffers, free between steps, hold r and m.
        if constexpr (CLEAN && S >= 3) {
            if (P.O.clean) {
#pragma unroll 1
                for (int s = 0; s < S; ++s) {
                    const int tc = s_cln[s];
                    if (tc < 0) continue;
                    const int i = s_i[s];
                    float* base = sm + s * L.lane;
                    float* Fp = base + L.Fp;
                    float* Rb = sm + ((s + 1) % S) * L.lane + L.Fp;
                    float* Mb = sm + ((s + 2) % S) * L.lane + L.Fp;
                    if (own_mod) {
                        float acc[PPT];
#pragma unroll
                        for (int r = 0; r < PPT; ++r) acc[r] = 0.0f;
                        const float* crow = M.Cp + j0;
#pragma unroll 2
                        for (int k = s_k[s][0]; k < s_k[s][1]; ++k) {
                            const float pk = base[L.phi + k];
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
                    if (tid < 32) Fp[skew((tid < 16 ? tid - 16 : nm + tid - 16) + 16)] = 0.0f;
                    __syncthreads();
                    const int h = s_h[s];
                    const int nblk = (2 * h + 1 + TB - 1) / TB;
                    const float* g = base + L.g;
                    float fpp[PPT];
#pragma unroll
                    for (int r = 0; r < PPT; ++r) fpp[r] = 0.0f;
                    if (own_pix) {
                        for (int bk = 0; bk < nblk; ++bk) {
                            const int s0 = -h + bk * TB;
                            float gg[TB], win[PPT + TB - 1];
#pragma unroll
                            for (int e = 0; e < TB; ++e) gg[e] = g[s0 + e + H];
                            const int wb0 = j0 + H - s0 - (TB - 1) + 16;
#pragma unroll
                            for (int q = 0; q < PPT + TB - 1; ++q) win[q] = Fp[skew(wb0 + q)];
#pragma unroll
                            for (int e = 0; e < TB; ++e)
#pragma unroll
                                for (int r = 0; r < PPT; ++r) fpp[r] = fmaf(gg[e], win[r - e + TB - 1], fpp[r]);
                        }
                    }
                    const float* yr = Wk.yw + (size_t)i * 2 * Wk.ldw;
                    float* wr = Wk.yw + (size_t)i * 2 * Wk.ldw + Wk.ldw;
                    const float imean = slots ? P.S.imean[i] : Wk.im[i], wgt = s_w[s];
                    const size_t row = (size_t)i * p;
                    float bl[NB];
#pragma unroll
                    for (int a = 0; a < NB; ++a) bl[a] = s_b[s][a];
                    float wbv[PPT];
                    uint32_t used = 0;
#pragma unroll
                    for (int r = 0; r < PPT; ++r) {
                        const int j = j0 + r;
                        wbv[r] = 0.0f;
                        if (j < p) {
                            const float f = P.flux[row + j], iv = P.ivar[row + j];
                            const bool use = P.good[row + j] && iv > 0.0f && isfinite(f) && isfinite(iv);
                            const bool edge = j < P.O.edge_px || j >= p - P.O.edge_px;
                            const float wb = (use && !edge && wgt > 0.0f) ? iv / imean : 0.0f;
                            float Pl[NB];
                            legendre<D>(fmaf((float)j, xstep, -1.0f), Pl);
                            float c = 0.0f;
#pragma unroll
                            for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
                            const float model = c * fpp[r];
                            const float sw = sqrtf(wb);
                            Rb[skew(j + L.dofs)] = sw * (yr[j] - model);
                            Mb[skew(j + 16)] = sw * model;
                            wbv[r] = wb;
                            if (wr[j] > 0.0f) used |= 1u << r;
                        }
                    }
                    __syncthreads();
                    const int upd = tc / P.O.clean_every;
                    const uint32_t keep = cta_clean_mask<NT, PPT>(p, j0, Rb, L.dofs, Mb, 16, used,
                                                                  upd == 1 ? 0.5f : 0.2f,
                                                                  reinterpret_cast<uint8_t*>(Mb), s_redd,
                                                                  s_tot, nullptr);
#pragma unroll
                    for (int r = 0; r < PPT; ++r)
                        if (j0 + r < p) wr[j0 + r] = ((keep >> r) & 1u) ? wbv[r] : 0.0f;
                    if (warp == s) {
                        const int hn = warp_prepare_step(M, s_x[s], base + L.phi, base + L.dphi, base + L.g,
                                                         base + L.gmu, base + L.gsg, s_k[s]);
                        if (lane == 0) {
                            s_h[s] = hn;
                            s_cln[s] = -1;
                        }
                    }
                    __syncthreads();
                }
            }
        }
    }
}

}  // namespace lasp
