// Grouped tensor-core fit (mixed precision): every Adam step (stage 8) runs
// over the whole active group of spectra as four kernels --
//   K1  F' = phi(theta) C            tcgen05, M = 128 model pixels x N = 128 spectra
//   K2  broadening, continuum WLS (FP32 or FP64 normal equations), residual,
//       loss and the adjoint down to dF' (CUDA cores, one CTA per spectrum);
//       dF' is written straight into the swizzled K-major operand image of K3
//   K3  dphi = dF' C^T               tcgen05, M = 128 spectra x N = 32 terms,
//       K = n_model pixels streamed through a 4-stage bulk-copy pipeline
//   K4  chain rule, Adam, stop rules, next active list (one warp per spectrum)
// -- so both contractions of Eq. 1 (forward and adjoint) run on the tensor
// cores with the table shared by 128 spectra, and converged spectra leave the
// active list at once.  Steps are replayed from CUDA graphs of 8 steps.
// This header holds the kernels and the host driver of one fit; the entry
// points are in lasp_grouped.cu.
#pragma once

#include <cuda_bf16.h>
#include <cmath>
#include <vector>

#include "lasp_clean.cuh"
#include "lasp_fit.cuh"
#include "lasp_prof.cuh"
#include "lasp_tc.cuh"
#include "lasp_tc_ptx.cuh"

namespace lasp {

int cuda_rc(cudaError_t e);

// Group state of the joint loss (LASP_LOSS_JOINT): the group RMS L of the
// current step, its member count, the group stop status and the stop-rule
// history, updated once per step by K3j.
struct GroupState {
    float L;
    int n_act;
    uint32_t status;
    int step;
    float prev;
    int rise;
    float ring[WINMAX];
};

struct Grp {
    ModelDev M;
    FitOpts O;
    int N, ldf, nch, nblk;        // spectra, F' row stride, K3 chunks, 128-spectrum blocks
    int n_kb, kp;                 // K blocks of 32 basis terms; kp = 32 n_kb (dphi row stride)
    int NB;                       // Legendre coefficients D + 1
    // per spectrum state
    float *x, *m, *v, *ring, *prev, *w, *imean, *loss, *gmu, *gsg, *b;
    int *rise, *t, *flags;
    // active lists (double buffered) and their counts
    int* list[2];
    int* count;                   // count[0], count[1]: active list lengths; count[2]: err
    float* Fp;                    // N x ldf
    float* taps;                  // N x 3 x TAPBUF: g, dg/dmu, dg/dsigma of the spectrum's next step
    int* hh;                      // N: kernel half width of those taps
    const float2* bct;            // per step t: (lr / (1 - beta1^t), sqrt(1 - beta2^t)), from FP64
    // joint loss: S_i of the step (K2), the step it belongs to, the group state (K3j)
    float* Sstep;
    int* act;
    GroupState* gs;
    float *Y, *Wt;                // N x ldp: y = flux / w and W of section 3.3 step 2 (0 beyond p)
    int ldp;                      // row stride of Y and Wt: n_pix rounded up to 16
    uint8_t *A_hi, *A_lo;         // K3 A images: nblk x nch x 16 KB
    float* dphi;                  // KSPLIT x list position x kp (partial sums)
    int* err;                     // count[2]: set when a bounded wait gives up (K1, K3); K4 then
                                  // ends every fit it steps with LASP_ST_TIMEOUT
    uint32_t wait0;               // poll limit of each K1 CTA's first table-copy wait
    // inputs / outputs
    const float *flux, *ivar, *theta0;
    const uint8_t* good;
    float *theta, *loss_out, *cont, *weight;
    int32_t* steps;
    uint32_t* status;
};


namespace {

constexpr uint32_t kWait = 1u << 22;
constexpr int K3_STAGES = 4;
constexpr int CHUNK_STEPS = 8;     // steps per captured graph (even)
constexpr int KSPLIT = 4;          // K3: pixel ranges per 128-spectrum block

// K3 pipeline depth for n_kb K blocks: four stages where they fit in shared memory.
__host__ __device__ inline int k3_stages(int n_kb) {
    const int stage = 2 * TC_TILE_BYTES + 2 * n_kb * TC_BK_CHUNK_BYTES;
    return 4 * stage + 1024 <= 227 * 1024 ? 4 : 3;
}
__host__ inline size_t k3_smem_bytes(int n_kb) {
    return (size_t)k3_stages(n_kb) * (2 * TC_TILE_BYTES + 2 * n_kb * TC_BK_CHUNK_BYTES) + 1024;
}

// ---------------------------------------------------------------- K0 prep
// One CTA per spectrum: blockIdx.x, or idx[blockIdx.x] for spectra admitted
// into a persistent pool; spectra with data join the active list of parity 0.
template <int NT>
__global__ void __launch_bounds__(NT) k0_prep(const Grp G, const int32_t* __restrict__ idx) {
    extern __shared__ __align__(16) float sm[];
    const int i = idx ? idx[blockIdx.x] : blockIdx.x;
    const int p = G.M.n_pix;
    const int pa = (p + 3) & ~3;
    float* y = sm;
    float* W = sm + pa;
    float* sortbuf = sm + 2 * pa;
    float* red = sortbuf + pa;
    const size_t row = (size_t)i * p;
    float w, imean;
    const int n_obj = prep_spectrum<NT>(G.flux + row, G.ivar + row, G.good + row, p, G.O.edge_px,
                                        G.O.quantile, y, W, sortbuf, red, &w, &imean);
    __syncthreads();
    // y and W for every step of K2, zero-padded to the row stride
    for (int j = threadIdx.x; j < G.ldp; j += NT) {
        G.Y[(size_t)i * G.ldp + j] = j < p ? y[j] : 0.0f;
        G.Wt[(size_t)i * G.ldp + j] = j < p ? W[j] : 0.0f;
    }
    if (threadIdx.x < 32) {
        // kernel taps of the first step (x0), for K2
        float th[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float xx = (G.theta0[5 * i + k] - G.M.plo[k]) / G.M.phalf[k] - 1.0f;
            th[k] = phys_of(G.M, k, fminf(1.0f, fmaxf(-1.0f, xx)));
        }
        float* tp = G.taps + (size_t)i * 3 * TAPBUF;
        const int h = kernel_taps_warp(th[3] / G.M.kms_px, th[4] / G.M.kms_px, G.M.pad, tp, tp + TAPBUF,
                                       tp + 2 * TAPBUF);
        if (threadIdx.x == 0) G.hh[i] = h;
    }
    if (threadIdx.x == 0) {
        G.w[i] = w;
        G.imean[i] = imean;
        float x[5];
        for (int k = 0; k < 5; ++k) {
            float xx = (G.theta0[5 * i + k] - G.M.plo[k]) / G.M.phalf[k] - 1.0f;
            x[k] = fminf(1.0f, fmaxf(-1.0f, xx));
            G.x[5 * i + k] = x[k];
            G.m[5 * i + k] = 0.0f;
            G.v[5 * i + k] = 0.0f;
        }
        G.prev[i] = 0.0f;
        G.rise[i] = 0;
        G.t[i] = 0;
        if (n_obj < G.NB + 5 || !(w > 0.0f) || !isfinite(w)) {
            for (int k = 0; k < 5; ++k) G.theta[5 * i + k] = phys_of(G.M, k, x[k]);
            G.loss_out[i] = NAN;
            G.steps[i] = 0;
            G.status[i] = LASP_ST_NODATA;
            if (G.weight) G.weight[i] = w;
            if (G.cont)
                for (int a = 0; a < G.NB; ++a) G.cont[(size_t)i * G.NB + a] = NAN;
            G.flags[i] = -1;
        } else {
            G.flags[i] = n_obj;
            const int pos = atomicAdd(&G.count[0], 1);
            G.list[0][pos] = i;
        }
    }
}

// ---------------------------------------------------------------- K1 forward
template <int PREC>
__global__ void __launch_bounds__(128) k1_interp(const Grp G, int par, const uint8_t* __restrict__ img,
                                                  const uint8_t* __restrict__ img_lo, int n_tiles) {
    const int count = G.count[par];
    const int s0 = blockIdx.x * 128;
    if (s0 >= count) return;
    extern __shared__ uint8_t smraw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int n_kb = G.n_kb;
    const uint32_t blk_bytes = (uint32_t)n_kb * TC_TILE_BYTES;
    uint8_t* Ahi = base;
    uint8_t* Alo = base + blk_bytes;
    uint8_t* Bhi = base + 2 * blk_bytes;
    uint8_t* Blo = base + 3 * blk_bytes;
    __shared__ __align__(8) uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok, s_id[128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const ModelDev& M = G.M;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 128);
        tc::tmem_relinquish();
    }
    {
        // B operand row tid: the basis of the spectrum at list position s0 + tid,
        // n_kb blocks of 32 terms (zero beyond K; for a piecewise interpolator the
        // rows of regimes inactive at its Teff are zero)
        float phi[KROWS];
        for (int k = 0; k < 32 * n_kb; ++k) phi[k] = 0.0f;
        const int pos = s0 + tid;
        int id = -1;
        if (pos < count) {
            id = G.list[par][pos];
            float th[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) th[q] = phys_of(M, q, G.x[5 * id + q]);
            for (int k = 0; k < M.K; ++k) basis_term(M, k, th, phi, nullptr);
        }
        s_id[tid] = id;
        for (int b = 0; b < n_kb; ++b) {
            uint8_t* bh = Bhi + b * TC_TILE_BYTES;
            uint8_t* bl = Blo + b * TC_TILE_BYTES;
            if (PREC == 2) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    __nv_bfloat16 bb[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) bb[q] = __float2bfloat16_rn(c < 4 ? phi[32 * b + 8 * c + q] : 0.0f);
                    *reinterpret_cast<uint4*>(bh + tc::sw128_off(tid, c)) = *reinterpret_cast<uint4*>(bb);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float h[4], l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        h[q] = tc::to_tf32(phi[32 * b + 4 * c + q]);
                        l[q] = tc::to_tf32(phi[32 * b + 4 * c + q] - h[q]);
                    }
                    *reinterpret_cast<float4*>(bh + tc::sw128_off(tid, c)) = make_float4(h[0], h[1], h[2], h[3]);
                    if (PREC == 3)
                        *reinterpret_cast<float4*>(bl + tc::sw128_off(tid, c)) = make_float4(l[0], l[1], l[2], l[3]);
                }
            }
        }
    }
    if (tid == 0) {
        tc::mbar_init(&bar_tma, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
        s_ok = 1;
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = tc::idesc_f32acc(PREC == 2 ? 1u : 2u, 128, 128);
    bool pending = false, mma_pending = false;
    uint32_t phase = 0;
    for (int t = blockIdx.y; t < n_tiles; t += gridDim.y) {
    if (tid == 0) {
        const uint32_t bytes = (PREC == 3 ? 2u : 1u) * blk_bytes;
        tc::mbar_arrive_expect_tx(&bar_tma, bytes);
        tc::bulk_g2s(Ahi, img + (size_t)t * blk_bytes, blk_bytes, &bar_tma);
        if (PREC == 3) tc::bulk_g2s(Alo, img_lo + (size_t)t * blk_bytes, blk_bytes, &bar_tma);
        pending = true;
        // the CTA's first wait comes before any MMA: its limit may be shortened for tests
        if (!tc::mbar_wait_bounded(&bar_tma, phase, t == (int)blockIdx.y ? G.wait0 : kWait)) {
            atomicExch(G.err, 1);
            s_ok = 0;
        } else {
            pending = false;
            tc::tc_fence_after();
            for (int b = 0; b < n_kb; ++b) {
                const uint64_t ah = tc::desc_kmajor_sw128(tc::smem_u32(Ahi + b * TC_TILE_BYTES));
                const uint64_t bh = tc::desc_kmajor_sw128(tc::smem_u32(Bhi + b * TC_TILE_BYTES));
                constexpr int NK = PREC == 2 ? 2 : 4;
#pragma unroll
                for (int ks = 0; ks < NK; ++ks) {
                    const uint64_t adv = (uint64_t)(ks * 32) >> 4;
                    const uint32_t acc = (b > 0 || ks > 0) ? 1u : 0u;
                    if (PREC == 2) tc::mma_bf16(tmem, ah + adv, bh + adv, idesc, acc);
                    else tc::mma_tf32(tmem, ah + adv, bh + adv, idesc, acc);
                }
                if (PREC == 3) {
                    const uint64_t al = tc::desc_kmajor_sw128(tc::smem_u32(Alo + b * TC_TILE_BYTES));
                    const uint64_t bl = tc::desc_kmajor_sw128(tc::smem_u32(Blo + b * TC_TILE_BYTES));
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t adv = (uint64_t)(ks * 32) >> 4;
                        tc::mma_tf32(tmem, ah + adv, bl + adv, idesc, 1);
                        tc::mma_tf32(tmem, al + adv, bh + adv, idesc, 1);
                    }
                }
            }
            tc::mma_commit(&bar_mma);
            mma_pending = true;
        }
    }
    __syncthreads();
    if (!s_ok) break;
    {
        if (!tc::mbar_wait_bounded(&bar_mma, phase, kWait)) {
            atomicExch(G.err, 1);
            s_ok = 0;
        } else {
            tc::tc_fence_after();
            const int mpix = t * TC_TILE + warp * 32 + lane;
#pragma unroll 1
            for (int c = 0; c < 8; ++c) {
                if (s0 + c * 16 >= count) break;
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
                if (mpix < M.n_model) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int id = s_id[c * 16 + q];
                        if (id >= 0) G.Fp[(size_t)id * G.ldf + mpix] = v[q];
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (!s_ok) break;
    if (tid == 0) mma_pending = false;
    phase ^= 1u;
    }
    // after a timeout: the copy and the MMAs still in flight complete (bounded) before exit
    if (tid == 0 && pending) tc::mbar_wait_bounded(&bar_tma, phase, kWait);
    if (tid == 0 && mma_pending) tc::mbar_wait_bounded(&bar_mma, phase, kWait);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------- K2 step body
struct RestSmem {
    int y, W, Fp, Db, g, gmu, gsg, red, out, total, dofs;
    __host__ __device__ RestSmem(int p, int H, int n_model, int NT, int D) {
        const int NB = D + 1, NV = NB * (NB + 1) / 2 + NB;
        const int nv_max = round32(NV > 4 ? NV : 4);
        dofs = 2 * H + 8;
        int o = 0;
        y = o;    o += skew_size(p);
        W = o;    o += skew_size(p);
        Fp = o;   o += skew_size(n_model + 32);
        Db = o;   o += skew_size(p + 4 * H + 40);
        g = o;    o += TAPBUF;
        gmu = o;  o += TAPBUF;
        gsg = o;  o += TAPBUF;
        red = o;  o += (NT / 32) * (nv_max > 2 * round32(NV) ? nv_max : 2 * round32(NV));
        out = o;  o += 2 * nv_max + 16;
        total = o;
    }
};

// Stage 6 Clean update in the grouped pipeline, between K3 and K4 of a step:
// for every active spectrum whose evaluated step t is a Clean step, the mask
// update from the residual at x_t (K1's F', K2's continuum b, and the taps of
// x_t, which K4 has not replaced yet), written into its W row for the steps
// that follow.  The same rules as the fused kernels' update; other spectra
// return at once.  Shared memory: RestSmem.
template <int NT, int D>
__global__ void __launch_bounds__(NT) kc_clean(const Grp G, int par) {
    constexpr int NB = D + 1;
    const int pos = blockIdx.x;
    if (pos >= G.count[par]) return;
    const int id = G.list[par][pos];
    const int t = G.t[id];
    if (!clean_step(G.O, t)) return;
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = G.M;
    const int p = M.n_pix, H = M.pad, nm = M.n_model;
    const int tid = threadIdx.x;
    const RestSmem L(p, H, nm, NT, D);
    float* Fp = sm + L.Fp;
    float* Rb = sm + L.Db;
    float* Mb = sm + L.W;
    float* g = sm + L.g;
    __shared__ double s_redd[3 * (NT / 32)], s_tot[3];
    const int j0 = tid * PPT;
    const bool own_pix = j0 < p;
    for (int q = tid; q < skew_size(nm + 32); q += NT) Fp[q] = 0.0f;
    __syncthreads();
    for (int m = tid; m < nm; m += NT) Fp[skew(m + 16)] = G.Fp[(size_t)id * G.ldf + m];
    const float* tp = G.taps + (size_t)id * 3 * TAPBUF;
    for (int q = tid; q < TAPBUF; q += NT) g[q] = tp[q];
    __syncthreads();
    const int h = G.hh[id];
    const int nblk = (2 * h + 1 + TB - 1) / TB;
    constexpr int HP = PPT / 2;
    float fpp[PPT];
    {
        float2 f2[HP];
#pragma unroll
        for (int r = 0; r < HP; ++r) f2[r] = make_float2(0.0f, 0.0f);
        if (own_pix) {
            for (int bk = 0; bk < nblk; ++bk) {
                const int s0 = -h + bk * TB;
                float gg[TB];
                float2 w2[HP + TB - 1];
#pragma unroll
                for (int e = 0; e < TB; ++e) gg[e] = g[s0 + e + H];
                const int base = j0 + H - s0 - (TB - 1) + 16;
#pragma unroll
                for (int q = 0; q < HP + TB - 1; ++q) w2[q] = make_float2(Fp[skew(base + q)], Fp[skew(base + q + HP)]);
#pragma unroll
                for (int e = 0; e < TB; ++e) {
                    const float2 g2 = make_float2(gg[e], gg[e]);
#pragma unroll
                    for (int r = 0; r < HP; ++r) f2[r] = __ffma2_rn(g2, w2[r - e + TB - 1], f2[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < HP; ++r) {
            fpp[r] = f2[r].x;
            fpp[r + HP] = f2[r].y;
        }
    }
    float bl[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) bl[a] = G.b[(size_t)id * NB + a];
    const float imean = G.imean[id], wgt = G.w[id];
    const size_t row = (size_t)id * p;
    const float* yr = G.Y + (size_t)id * G.ldp;
    float* wr = G.Wt + (size_t)id * G.ldp;
    const float xstep = 2.0f / (float)p;
    float wbv[PPT];
    uint32_t used = 0;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int j = j0 + r;
        wbv[r] = 0.0f;
        if (j < p) {
            const float f = G.flux[row + j], iv = G.ivar[row + j];
            const bool use = G.good[row + j] && iv > 0.0f && isfinite(f) && isfinite(iv);
            const bool edge = j < G.O.edge_px || j >= p - G.O.edge_px;
            const float wb = (use && !edge && wgt > 0.0f) ? iv / imean : 0.0f;
            float Pl[NB];
            legendre<D>(fmaf((float)j, xstep, -1.0f), Pl);
            float c = 0.0f;
#pragma unroll
            for (int a = 0; a < NB; ++a) c = fmaf(bl[a], Pl[a], c);
            const float model = c * fpp[r];
            const float sw = sqrtf(wb);
            Rb[skew(j + L.dofs)] = sw * (yr[j] - model);
            Mb[skew(j)] = sw * model;
            wbv[r] = wb;
            if (wr[j] > 0.0f) used |= 1u << r;
        }
    }
    __syncthreads();
    const int upd = t / G.O.clean_every;
    const uint32_t keep = cta_clean_mask<NT, PPT>(p, j0, Rb, L.dofs, Mb, 0, used, upd == 1 ? 0.5f : 0.2f,
                                                  reinterpret_cast<uint8_t*>(Mb), s_redd, s_tot, nullptr);
#pragma unroll
    for (int r = 0; r < PPT; ++r)
        if (j0 + r < p) wr[j0 + r] = ((keep >> r) & 1u) ? wbv[r] : 0.0f;
}

template <int PREC>
__device__ __forceinline__ void store_dfp(const Grp& G, int pos, int m0, const float (&d)[PPT]) {
    // K3 A image of block pos/128: chunk of 32 (TF32) or 64 (BF16) model pixels,
    // row pos%128, K-major with the 128-byte swizzle.
    const int blk = pos >> 7, r = pos & 127;
    if (PREC == 2) {
        const int c = m0 >> 6;
        uint8_t* tile = G.A_hi + ((size_t)blk * G.nch + c) * TC_TILE_BYTES;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = ((m0 & 63) >> 3) + h;
            __nv_bfloat16 bb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) bb[e] = __float2bfloat16_rn(d[8 * h + e]);
            *reinterpret_cast<uint4*>(tile + tc::sw128_off(r, q)) = *reinterpret_cast<uint4*>(bb);
        }
    } else {
        const int c = m0 >> 5;
        const size_t toff = ((size_t)blk * G.nch + c) * TC_TILE_BYTES;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int q = ((m0 & 31) >> 2) + h;
            float hh[4], ll[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                hh[e] = tc::to_tf32(d[4 * h + e]);
                ll[e] = tc::to_tf32(d[4 * h + e] - hh[e]);
            }
            *reinterpret_cast<float4*>(G.A_hi + toff + tc::sw128_off(r, q)) = make_float4(hh[0], hh[1], hh[2], hh[3]);
            if (PREC == 3)
                *reinterpret_cast<float4*>(G.A_lo + toff + tc::sw128_off(r, q)) =
                    make_float4(ll[0], ll[1], ll[2], ll[3]);
        }
    }
}

// NE64: the FP64 normal equations (LASP_NE_FP64) compiled in; without it the
// step body keeps the register budget of three CTAs per SM.
template <int NT, int D, int PREC, bool NE64 = false>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 1) k2_rest(const Grp G, int par) {
    using Gm = Gram<D>;
    constexpr int NB = D + 1;
    constexpr int NV = Gm::NV;
    const int pos = blockIdx.x;
    if (pos >= G.count[par]) return;
    const int id = G.list[par][pos];
    extern __shared__ __align__(16) float sm[];
    const ModelDev& M = G.M;
    const int p = M.n_pix, H = M.pad, nm = M.n_model;
    const int tid = threadIdx.x;
    const RestSmem L(p, H, nm, NT, D);
    float* y = sm + L.y;
    float* W = sm + L.W;
    float* Fp = sm + L.Fp;
    float* Db = sm + L.Db;
    float* g = sm + L.g;
    float* gmu = sm + L.gmu;
    float* gsg = sm + L.gsg;
    float* red = sm + L.red;
    float* out = sm + L.out;
    double* outd = reinterpret_cast<double*>(sm + ((L.out + 1) & ~1));
    __shared__ float s_b[NB];
    __shared__ int s_h;

    const int j0 = tid * PPT;
    const bool own_pix = j0 < p;
    const bool own_mod = j0 < nm;
    // F' of this spectrum (K1 output) and its y, W rows (K0 output): 256-bit
    // loads issued first (rows are padded to 16 floats), stored after the taps
    float fa[8], fb[8], ya[8], yb[8], wa[8], wb[8];
    if (own_mod) {
        const float* src = G.Fp + (size_t)id * G.ldf + j0;
        ldg8(src, fa);
        ldg8(src + 8, fb);
    }
    if (own_pix) {
        const float* ys = G.Y + (size_t)id * G.ldp + j0;
        const float* ws = G.Wt + (size_t)id * G.ldp + j0;
        ldg8(ys, ya);
        ldg8(ys + 8, yb);
        ldg8(ws, wa);
        ldg8(ws + 8, wb);
    }
    // kernel taps of this step (written by K0 or the previous K4), zero past 2H
    {
        const float* tp = G.taps + (size_t)id * 3 * TAPBUF;
        for (int q = tid; q < 3 * TAPBUF; q += NT) {
            const int c = q / TAPBUF, s0 = q - c * TAPBUF;
            g[c * TAPBUF + s0] = s0 <= 2 * H ? tp[q] : 0.0f;
        }
        if (tid == 0) s_h = G.hh[id];
    }
    // zero only the pads of F' (model pixels [-16, 0) and [nm, nm + 16)) and of
    // the delta buffer (j outside [0, p)); the interiors are overwritten
    for (int q = tid; q < 32; q += NT) {
        const int mm = q < 16 ? q - 16 : nm + q - 16;
        Fp[skew(mm + 16)] = 0.0f;
    }
    for (int q = tid; q < L.dofs + 2 * H + 32; q += NT) {
        const int j = q < L.dofs ? q - L.dofs : p + q - L.dofs;
        Db[skew(j + L.dofs)] = 0.0f;
    }
    if (own_pix) {
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int j = j0 + r;
            if (j < p) {
                y[skew(j)] = r < 8 ? ya[r & 7] : yb[r & 7];
                W[skew(j)] = r < 8 ? wa[r & 7] : wb[r & 7];
            }
        }
    }
    if (own_mod) {
#pragma unroll
        for (int r = 0; r < PPT; ++r)
            if (j0 + r < nm) Fp[skew(j0 + r + 16)] = r < 8 ? fa[r & 7] : fb[r & 7];
    }
    __syncthreads();
    const int h = s_h;
    const int nblk = (2 * h + 1 + TB - 1) / TB;
    const float xstep = 2.0f / (float)p;

    // F'' (Eq. 5) and the normal equations (Eq. 6).  The correlations pair
    // pixels r and r + PPT/2, the tap sums taps e and e + TB/2, the normal
    // equations the entries along a diagonal of G, each pair in one packed FMA
    // (__ffma2_rn: two IEEE fmas), so every sum takes the same fmas in the same
    // order as the scalar form and the step body issues fewer instructions
    // (K2 runs three CTAs per SM and is issue-bound: 147.5 -> 142.8 us a step
    // on 4096 LAMOST-like spectra).
    constexpr int HP = PPT / 2;
    float fpp[PPT];
    {
        float2 f2[HP];
#pragma unroll
        for (int r = 0; r < HP; ++r) f2[r] = make_float2(0.0f, 0.0f);
        if (own_pix) {
            for (int bk = 0; bk < nblk; ++bk) {
                const int s0 = -h + bk * TB;
                float gg[TB];
                float2 w2[HP + TB - 1];
#pragma unroll
                for (int e = 0; e < TB; ++e) gg[e] = g[s0 + e + H];
                const int base = j0 + H - s0 - (TB - 1) + 16;
#pragma unroll
                for (int q = 0; q < HP + TB - 1; ++q) w2[q] = make_float2(Fp[skew(base + q)], Fp[skew(base + q + HP)]);
#pragma unroll
                for (int e = 0; e < TB; ++e) {
                    const float2 g2 = make_float2(gg[e], gg[e]);
#pragma unroll
                    for (int r = 0; r < HP; ++r) f2[r] = __ffma2_rn(g2, w2[r - e + TB - 1], f2[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < HP; ++r) {
            fpp[r] = f2[r].x;
            fpp[r + HP] = f2[r].y;
        }
    }
    float gacc[NV];
    {
        GramPairs<D> gp;
        gp.zero();
        if (own_pix) {
#pragma unroll
            for (int r = 0; r < PPT; ++r) {
                const int j = j0 + r;
                const float Wj = j < p ? W[skew(j)] : 0.0f;
                if (Wj != 0.0f) {
                    float Pl[NB];
                    legendre<D>(fmaf((float)j, xstep, -1.0f), Pl);
                    const float f = fpp[r];
                    gp.add(Wj * f * f, Wj * f * y[skew(j)], Pl);
                }
            }
        }
        gp.unpack(gacc);
    }
    solve_continuum<D, NT, NE64>(gacc, G.O.fp64_ne, red, reinterpret_cast<float*>(outd), s_b);
    // residual (Eq. 7), loss (Eq. 9), delta = W eps c
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
                fpp[r] = dlt;
                if (j < p) Db[skew(j + L.dofs)] = dlt;
            }
        }
        if (!solved) racc[0] = NAN;
    }
    __syncthreads();     // delta buffer complete
    // adjoint of the kernel parameters through a_s = sum_j delta_j F'_{j+H-s};
    // bacc = [S, nonpos, mu, sigma] reduced together at the end
    float bacc[4] = {racc[0], racc[1], 0.0f, 0.0f};
    if (own_pix) {
        for (int bk = 0; bk < nblk; ++bk) {
            const int s0 = -h + bk * TB;
            float win[PPT + TB - 1];
            const int base = j0 + H - s0 - (TB - 1) + 16;
#pragma unroll
            for (int q = 0; q < PPT + TB - 1; ++q) win[q] = Fp[skew(base + q)];
            constexpr int TH = TB / 2;
            float2 a2[TH];
#pragma unroll
            for (int e = 0; e < TH; ++e) a2[e] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int r = 0; r < PPT; ++r) {
                const float2 d2 = make_float2(fpp[r], fpp[r]);
#pragma unroll
                for (int e = 0; e < TH; ++e)
                    a2[e] = __ffma2_rn(d2, make_float2(win[r - e + TB - 1], win[r - e - TH + TB - 1]), a2[e]);
            }
#pragma unroll
            for (int e = 0; e < TB; ++e) {
                const float ae = e < TH ? a2[e].x : a2[e - TH].y;
                bacc[2] = fmaf(gmu[s0 + e + H], ae, bacc[2]);
                bacc[3] = fmaf(gsg[s0 + e + H], ae, bacc[3]);
            }
        }
    }
    // dF'_m = sum_s g_s delta_{m-H+s}, written as the K3 operand (zero beyond n_model)
    const int kpix = PREC == 2 ? 64 * ((nm + 63) / 64) : 32 * ((nm + 31) / 32);
    if (j0 < kpix) {
        float dfp[PPT];
#pragma unroll
        for (int r = 0; r < PPT; ++r) dfp[r] = 0.0f;
        if (own_mod) {
            float2 f2[HP];
#pragma unroll
            for (int r = 0; r < HP; ++r) f2[r] = make_float2(0.0f, 0.0f);
            for (int bk = 0; bk < nblk; ++bk) {
                const int s0 = -h + bk * TB;
                float gg[TB];
                float2 w2[HP + TB - 1];
#pragma unroll
                for (int e = 0; e < TB; ++e) gg[e] = g[s0 + e + H];
                const int base = j0 - H + s0 + L.dofs;
#pragma unroll
                for (int q = 0; q < HP + TB - 1; ++q) w2[q] = make_float2(Db[skew(base + q)], Db[skew(base + q + HP)]);
#pragma unroll
                for (int e = 0; e < TB; ++e) {
                    const float2 g2 = make_float2(gg[e], gg[e]);
#pragma unroll
                    for (int r = 0; r < HP; ++r) f2[r] = __ffma2_rn(g2, w2[r + e], f2[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < HP; ++r) {
                dfp[r] = f2[r].x;
                dfp[r + HP] = f2[r].y;
            }
#pragma unroll
            for (int r = 0; r < PPT; ++r)
                if (j0 + r >= nm) dfp[r] = 0.0f;
        }
        store_dfp<PREC>(G, pos, j0, dfp);
    }
    reduce_to_warp0<4, NT>(bacc, red, out);
    if (tid == 0) {
        G.loss[id] = sqrtf(out[0] / (float)p);
        G.flags[id] = (out[1] > 0.0f ? 1 : 0) | (isfinite(s_b[0]) ? 0 : 2);
#pragma unroll
        for (int a = 0; a < NB; ++a) G.b[(size_t)id * NB + a] = s_b[a];
        G.gmu[id] = out[2];
        G.gsg[id] = out[3];
        if (G.O.joint) {
            G.Sstep[id] = out[0];
            G.act[id] = G.t[id];
        }
    }
}

// ---------------------------------------------------------------- K3j group loss
// Joint loss: L = sqrt(sum_i S_i / (N p)) over the spectra stepped this step
// with a finite S_i, summed in float-float in a fixed order (deterministic),
// and the stop rules on L.  One CTA.
template <int NTJ>
__global__ void __launch_bounds__(NTJ) k3j_group(const Grp G) {
    __shared__ float2 s_acc[NTJ];
    __shared__ int s_cnt[NTJ];
    GroupState* gs = G.gs;
    const int step = gs->step;
    const int tid = threadIdx.x;
    float2 acc = make_float2(0.0f, 0.0f);
    int cnt = 0;
    for (int id = tid; id < G.N; id += NTJ) {
        if (G.act[id] != step) continue;
        const float S = G.Sstep[id];
        if (isfinite(S)) {
            acc = ff_add(acc, S);
            ++cnt;
        }
    }
    s_acc[tid] = acc;
    s_cnt[tid] = cnt;
    __syncthreads();
    for (int off = NTJ / 2; off > 0; off >>= 1) {
        if (tid < off) {
            s_acc[tid] = ff_add2(s_acc[tid], s_acc[tid + off]);
            s_cnt[tid] += s_cnt[tid + off];
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int n = s_cnt[0];
        const float L = n > 0 ? sqrtf((s_acc[0].x + s_acc[0].y) / ((float)n * (float)G.M.n_pix)) : NAN;
        uint32_t st = 0;
        if (n > 0) {
            const int Wn = G.O.window;
            const int ri = step % Wn;
            if (step >= Wn && fabsf(L - gs->ring[ri]) < G.O.tol) st = LASP_ST_CONV_TOL;
            const int rise = (step >= 1 && L > gs->prev) ? gs->rise + 1 : 0;
            if (!st && rise >= Wn) st = LASP_ST_CONV_RISE;
            if (!st && step >= G.O.max_steps) st = LASP_ST_MAXSTEPS;
            gs->ring[ri] = L;
            gs->prev = L;
            gs->rise = rise;
        }
        gs->L = L;
        gs->n_act = n;
        gs->status = st;
        gs->step = step + 1;
    }
}

// ---------------------------------------------------------------- K3 backward contraction
template <int PREC>
__global__ void __launch_bounds__(128) k3_back(const Grp G, int par, const uint8_t* __restrict__ bk,
                                               const uint8_t* __restrict__ bk_lo) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) G.count[par ^ 1] = 0;  // list K4 fills next
    const int count = G.count[par];
    const int s0 = blockIdx.x * 128;
    if (s0 >= count) return;
    // this CTA's range of pixel chunks (split K; partial sums added in K4)
    const int per = (G.nch + KSPLIT - 1) / KSPLIT;
    const int c_beg = blockIdx.y * per;
    const int c_end = min(G.nch, c_beg + per);
    extern __shared__ uint8_t smraw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    // stage s: A hi (16 KB), A lo (16 KB), B hi (4 KB a K block), B lo (4 KB a K block);
    // the B operand of a chunk holds kp = 32 n_kb basis-term rows, the MMA's N
    const int kp = G.kp;
    const uint32_t bkb = (uint32_t)G.n_kb * TC_BK_CHUNK_BYTES;
    const int STAGE = 2 * TC_TILE_BYTES + 2 * (int)bkb;
    const int NS = k3_stages(G.n_kb);
    __shared__ __align__(8) uint64_t full[K3_STAGES], empty[K3_STAGES], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tcols = kp <= 32 ? 32u : (kp <= 64 ? 64u : 128u);
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, tcols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&done, 1);
        tc::fence_mbar_init();
        s_ok = 1;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::idesc_f32acc(PREC == 2 ? 1u : 2u, 128, (uint32_t)kp);
    const int nch = c_end - c_beg;
    const uint8_t* Ablk = G.A_hi + ((size_t)blockIdx.x * G.nch + c_beg) * TC_TILE_BYTES;
    const uint8_t* Ablk_lo =
        PREC == 3 ? G.A_lo + ((size_t)blockIdx.x * G.nch + c_beg) * TC_TILE_BYTES : nullptr;
    bk += (size_t)c_beg * bkb;
    if (PREC == 3) bk_lo += (size_t)c_beg * bkb;
    if (nch <= 0) {
        const int pos = s0 + tid;
        if (pos < count) {
            float* dst = G.dphi + ((size_t)blockIdx.y * G.nblk * 128 + pos) * kp;
            for (int k = 0; k < kp; ++k) dst[k] = 0.0f;
        }
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(tmem, tcols);
        return;
    }
    if (tid == 0) {
        const uint32_t bytes = (PREC == 3 ? 2u : 1u) * (uint32_t)(TC_TILE_BYTES + bkb);
        auto issue = [&](int c) {
            uint8_t* st = base + (c % NS) * STAGE;
            tc::mbar_arrive_expect_tx(&full[c % NS], bytes);
            tc::bulk_g2s(st, Ablk + (size_t)c * TC_TILE_BYTES, TC_TILE_BYTES, &full[c % NS]);
            tc::bulk_g2s(st + 2 * TC_TILE_BYTES, bk + (size_t)c * bkb, bkb, &full[c % NS]);
            if (PREC == 3) {
                tc::bulk_g2s(st + TC_TILE_BYTES, Ablk_lo + (size_t)c * TC_TILE_BYTES, TC_TILE_BYTES, &full[c % NS]);
                tc::bulk_g2s(st + 2 * TC_TILE_BYTES + bkb, bk_lo + (size_t)c * bkb, bkb, &full[c % NS]);
            }
        };
        const int pre = nch < NS ? nch : NS;
        for (int c = 0; c < pre; ++c) issue(c);
        int issued = pre;
        bool ok = true;
        for (int c = 0; c < nch && ok; ++c) {
            const int s = c % NS;
            if (!tc::mbar_wait_bounded(&full[s], (uint32_t)((c / NS) & 1), kWait)) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            uint8_t* st = base + s * STAGE;
            const uint64_t ah = tc::desc_kmajor_sw128(tc::smem_u32(st));
            const uint64_t bh = tc::desc_kmajor_sw128(tc::smem_u32(st + 2 * TC_TILE_BYTES));
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t adv = (uint64_t)(ks * 32) >> 4;
                const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                if (PREC == 2) tc::mma_bf16(tmem, ah + adv, bh + adv, idesc, acc);
                else tc::mma_tf32(tmem, ah + adv, bh + adv, idesc, acc);
            }
            if (PREC == 3) {
                const uint64_t al = tc::desc_kmajor_sw128(tc::smem_u32(st + TC_TILE_BYTES));
                const uint64_t bl = tc::desc_kmajor_sw128(tc::smem_u32(st + 2 * TC_TILE_BYTES + bkb));
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t adv = (uint64_t)(ks * 32) >> 4;
                    tc::mma_tf32(tmem, ah + adv, bl + adv, idesc, 1);
                    tc::mma_tf32(tmem, al + adv, bh + adv, idesc, 1);
                }
            }
            tc::mma_commit(&empty[s]);
            // refill the stage of the previous chunk once its MMAs are done
            if (c >= 1 && issued < nch) {
                const int sp = (c - 1) % NS;
                if (!tc::mbar_wait_bounded(&empty[sp], (uint32_t)(((c - 1) / NS) & 1), kWait)) {
                    ok = false;
                    break;
                }
                issue(issued++);
            }
        }
        tc::mma_commit(&done);        // arrives once every MMA issued so far has completed
        if (!ok) {
            atomicExch(G.err, 1);
            s_ok = 0;
            // let copies already issued and the MMAs in flight finish before the CTA exits
            for (int c = 0; c < issued; ++c)
                tc::mbar_wait_bounded(&full[c % NS], (uint32_t)((c / NS) & 1), kWait);
            tc::mbar_wait_bounded(&done, 0, kWait);
        }
    }
    __syncthreads();
    if (s_ok) {
        if (!tc::mbar_wait_bounded(&done, 0, kWait)) {
            atomicExch(G.err, 1);
            if (tid == 0) tc::mbar_wait_bounded(&done, 0, kWait);   // MMAs in flight: once more
        } else {
            tc::tc_fence_after();
            const int pos = s0 + warp * 32 + lane;
            float4* dst = reinterpret_cast<float4*>(G.dphi + ((size_t)blockIdx.y * G.nblk * 128 + pos) * kp);
            for (int c16 = 0; c16 < kp / 16; ++c16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * c16), v);
                if (pos < count)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[4 * c16 + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tcols);
}

// ---------------------------------------------------------------- K4 Adam + stop rules
template <int D>
__global__ void __launch_bounds__(256) k4_adam(const Grp G, int par) {
    constexpr int NB = D + 1;
    const int lane = threadIdx.x & 31;
    const int pos = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (pos >= G.count[par]) return;
    const int id = G.list[par][pos];
    const ModelDev& M = G.M;
    if (*(volatile int*)G.err) {
        // a bounded wait of this step gave up: the step's values are not valid,
        // so the fit ends here with LASP_ST_TIMEOUT (never reported converged)
        if (lane < 5) G.theta[5 * id + lane] = phys_of(M, lane, G.x[5 * id + lane]);
        if (lane == 0) {
            G.loss_out[id] = NAN;
            G.steps[id] = G.t[id];
            G.status[id] = LASP_ST_TIMEOUT;
            if (G.weight) G.weight[id] = G.w[id];
        }
        if (G.cont && lane < NB) G.cont[(size_t)id * NB + lane] = NAN;
        return;
    }
    // loads first: parameter k's Adam state on lane k, the basis adjoint sums on lane k < K
    float xk = 0.0f, mk = 0.0f, vk = 0.0f, gp = 0.0f;
    if (lane < 5) {
        xk = G.x[5 * id + lane];
        mk = G.m[5 * id + lane];
        vk = G.v[5 * id + lane];
    }
    // d l / d phi_k of rows k = lane, lane + 32, ... (split-K partials added in a fixed order)
    float gpk[NREG];
#pragma unroll
    for (int r = 0; r < NREG; ++r) {
        gpk[r] = 0.0f;
        const int k = lane + 32 * r;
        if (k < M.K)
#pragma unroll
            for (int q = 0; q < KSPLIT; ++q) gpk[r] += G.dphi[((size_t)q * G.nblk * 128 + pos) * G.kp + k];
    }
    gp = gpk[0];
    const float l = G.loss[id];
    const int flags = G.flags[id];
    const int t = G.t[id];
    float th[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) th[k] = phys_of(M, k, __shfl_sync(0xffffffffu, xk, k));
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
#pragma unroll
    for (int r = 0; r < NREG; ++r) {
        const int k = lane + 32 * r;
        if (k < M.K) {
            float d[3];
            basis_term_one(M, k, th, d);
            c0 = fmaf(gpk[r], d[0], c0);
            c1 = fmaf(gpk[r], d[1], c1);
            c2 = fmaf(gpk[r], d[2], c2);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    const int p = M.n_pix;
    const float kappa = l > 0.0f ? -1.0f / ((float)p * l) : 0.0f;
    float gk = 0.0f;
    if (lane < 5) {
        const float src = lane == 0 ? c0 : lane == 1 ? c1 : lane == 2 ? c2
                        : (lane == 3 ? G.gmu[id] : G.gsg[id]) / M.kms_px;
        gk = kappa * src * M.phalf[lane];
    }
    const bool fin = __all_sync(0xffffffffu, lane >= 5 || isfinite(gk));
    uint32_t st = 0;
    if (lane == 0) {
        if (flags & 2) st = LASP_ST_SINGULAR;
        else if (!(fin && isfinite(l))) st = LASP_ST_NONFINITE;
        if (!st && G.O.joint) {
            st = G.gs->status;                   // the group's stop rules (K3j)
        } else if (!st) {
            const int Wn = G.O.window;
            float* ring = G.ring + (size_t)id * WINMAX;
            const int ri = t % Wn;
            if (t >= Wn && fabsf(l - ring[ri]) < G.O.tol) st = LASP_ST_CONV_TOL;
            const int rise = (t >= 1 && l > G.prev[id]) ? G.rise[id] + 1 : 0;
            if (!st && rise >= Wn) st = LASP_ST_CONV_RISE;
            if (!st && t >= G.O.max_steps) st = LASP_ST_MAXSTEPS;
            ring[ri] = l;
            G.prev[id] = l;
            G.rise[id] = rise;
        }
        if (st && st <= LASP_ST_MAXSTEPS && (flags & 1)) st |= LASP_ST_NONPOS;
    }
    st = __shfl_sync(0xffffffffu, st, 0);
    if (st) {
        if (lane < 5) G.theta[5 * id + lane] = phys_of(M, lane, xk);
        if (lane == 0) {
            G.loss_out[id] = l;
            G.steps[id] = t;
            G.status[id] = st;
            if (G.weight) G.weight[id] = G.w[id];
        }
        if (G.cont && lane < NB) G.cont[(size_t)id * NB + lane] = G.b[(size_t)id * NB + lane];
        return;
    }
    // Adam (bias corrections from the FP64 table), parameter k on lane k; the
    // joint loss scales the gradient by l_i / (N L)
    const float2 bc = G.bct[t + 1];
    if (G.O.joint) gk *= l / ((float)G.gs->n_act * G.gs->L);
    if (lane < 5) {
        mk = G.O.beta1 * mk + (1.0f - G.O.beta1) * gk;
        vk = G.O.beta2 * vk + (1.0f - G.O.beta2) * gk * gk;
        const float denom = sqrtf(vk) / bc.y + G.O.eps;
        xk = fminf(1.0f, fmaxf(-1.0f, xk - bc.x * mk / denom));
        G.x[5 * id + lane] = xk;
        G.m[5 * id + lane] = mk;
        G.v[5 * id + lane] = vk;
    }
    if (lane == 0) {
        G.t[id] = t + 1;
        const int slot = atomicAdd(&G.count[par ^ 1], 1);
        G.list[par ^ 1][slot] = id;
    }
    // kernel taps of the next step, for K2
    const float mu = phys_of(M, 3, __shfl_sync(0xffffffffu, xk, 3)) / M.kms_px;
    const float sg = phys_of(M, 4, __shfl_sync(0xffffffffu, xk, 4)) / M.kms_px;
    float* tp = G.taps + (size_t)id * 3 * TAPBUF;
    const int h = kernel_taps_warp(mu, sg, M.pad, tp, tp + TAPBUF, tp + 2 * TAPBUF);
    if (lane == 0) G.hh[id] = h;
}

template <typename T>
int amalloc(T** p, size_t bytes, cudaStream_t st) {
    return cuda_rc(cudaMallocAsync((void**)p, bytes, st));
}

template <int D, int PREC, int NT, bool NE64 = false>
int run_grouped(Grp& G, const TcImages& tc, cudaStream_t st, int* launches) {
    const int N = G.N;
    const ModelDev& M = G.M;
    // K0
    {
        const int pa = (M.n_pix + 3) & ~3;
        const size_t smem = 4 * ((size_t)3 * pa + PREP_RED);
        int e = cuda_rc(cudaFuncSetAttribute(k0_prep<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        e = prof_time("k0_prep", st, [&]() {
            k0_prep<NT><<<N, NT, smem, st>>>(G, nullptr);
            return cuda_rc(cudaGetLastError());
        });
        if (e) return e;
    }
    const size_t smem1 = 4 * (size_t)G.n_kb * TC_TILE_BYTES + 1024;
    const size_t smem3 = k3_smem_bytes(G.n_kb);
    const RestSmem RS(M.n_pix, M.pad, M.n_model, NT, D);
    const size_t smem2 = 4 * (size_t)RS.total;
    int e = cuda_rc(cudaFuncSetAttribute(k1_interp<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
    if (!e) e = cuda_rc(cudaFuncSetAttribute(k2_rest<NT, D, PREC, NE64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    if (!e) e = cuda_rc(cudaFuncSetAttribute(k3_back<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3));
    if (!e && G.O.clean)
        e = cuda_rc(cudaFuncSetAttribute(kc_clean<NT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    if (e) return e;
    const uint8_t* img = (const uint8_t*)(PREC == 2 ? tc.bf16 : tc.tf32_hi);
    const uint8_t* img_lo = (const uint8_t*)tc.tf32_lo;
    const uint8_t* bk = (const uint8_t*)(PREC == 2 ? tc.bk_bf : tc.bk_hi);
    const uint8_t* bk_lo = (const uint8_t*)tc.bk_lo;
    const dim3 g1((N + 127) / 128, (tc.n_tiles + 3) / 4);
    const dim3 g3((N + 127) / 128, KSPLIT);
    const int g4 = (N + 7) / 8;
    auto one_step = [&](int par) {
        k1_interp<PREC><<<g1, 128, smem1, st>>>(G, par, img, img_lo, tc.n_tiles);
        k2_rest<NT, D, PREC, NE64><<<N, NT, smem2, st>>>(G, par);
        k3_back<PREC><<<g3, 128, smem3, st>>>(G, par, bk, bk_lo);
        if (G.O.joint) k3j_group<1024><<<1, 1024, 0, st>>>(G);
        if (G.O.clean) kc_clean<NT, D><<<N, NT, smem2, st>>>(G, par);
        k4_adam<D><<<g4, 256, 0, st>>>(G, par);
    };
    // every spectrum stops after at most max_steps + 1 evaluations
    const int max_chunks = (G.O.max_steps + 1 + CHUNK_STEPS - 1) / CHUNK_STEPS + 1;
    if (prof_on()) {
        // measurement mode: the same steps launched one by one without the
        // graph, each kernel timed on its own (lasp_profile)
        auto T = [&](const char* name, auto launch) {
            return prof_time(name, st, [&]() {
                launch();
                return cuda_rc(cudaGetLastError());
            });
        };
        int h_cnt[3] = {0, 0, 0};
        int nl = 1;
        for (int c = 0; !e && c < max_chunks; ++c) {
            for (int k = 0; !e && k < CHUNK_STEPS; ++k) {
                const int par = k & 1;
                e = T("k1_interp", [&] { k1_interp<PREC><<<g1, 128, smem1, st>>>(G, par, img, img_lo, tc.n_tiles); });
                if (!e) e = T("k2_rest", [&] { k2_rest<NT, D, PREC, NE64><<<N, NT, smem2, st>>>(G, par); });
                if (!e) e = T("k3_back", [&] { k3_back<PREC><<<g3, 128, smem3, st>>>(G, par, bk, bk_lo); });
                if (!e && G.O.joint) e = T("k3j_group", [&] { k3j_group<1024><<<1, 1024, 0, st>>>(G); });
                if (!e && G.O.clean) e = T("kc_clean", [&] { kc_clean<NT, D><<<N, NT, smem2, st>>>(G, par); });
                if (!e) e = T("k4_adam", [&] { k4_adam<D><<<g4, 256, 0, st>>>(G, par); });
                nl += (G.O.joint || G.O.clean ? 5 : 4);
            }
            if (!e) e = cuda_rc(cudaMemcpyAsync(h_cnt, G.count, sizeof(h_cnt), cudaMemcpyDeviceToHost, st));
            if (!e) e = cuda_rc(cudaStreamSynchronize(st));
            if (!e && h_cnt[0] == 0) break;
        }
        if (!e && h_cnt[2]) e = LASP_ETIMEOUT;
        *launches = nl;
        return e;
    }
    // capture CHUNK_STEPS steps (parities 0,1,0,1,...) into one graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap;
    if ((e = cuda_rc(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)))) return e;
    e = cuda_rc(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    if (!e) {
        cudaStream_t keep = st;
        st = cap;
        for (int k = 0; k < CHUNK_STEPS; ++k) one_step(k & 1);
        st = keep;
        e = cuda_rc(cudaStreamEndCapture(cap, &graph));
    }
    if (!e) e = cuda_rc(cudaGraphInstantiate(&exec, graph, 0));
    int h_cnt[3] = {0, 0, 0};       // active count, (other parity), timeout flag
    int nlaunch = 1;
    for (int c = 0; !e && c < max_chunks; ++c) {
        e = cuda_rc(cudaGraphLaunch(exec, st));
        nlaunch += (G.O.joint || G.O.clean ? 5 : 4) * CHUNK_STEPS;
        if (!e) e = cuda_rc(cudaMemcpyAsync(h_cnt, G.count, sizeof(h_cnt), cudaMemcpyDeviceToHost, st));
        if (!e) e = cuda_rc(cudaStreamSynchronize(st));
        if (!e && h_cnt[0] == 0) break;
    }
    // a timeout ended every fit it touched (K4): report it
    if (!e && h_cnt[2]) e = LASP_ETIMEOUT;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    *launches = nlaunch;
    return e;
}

}  // namespace

// The grouped fit at Legendre degree D for the handle's precision and
// normal-equation level: each degree is instantiated in its own translation
// unit (lasp_grouped.cu for D = 6, lasp_grp_d<D>.cu for the others).
template <int D>
int grp_run_deg(Grp& G, const TcImages& tc, const lasp_fit_opts* o, cudaStream_t st, int* launches) {
    const int NT = fit_threads(G.M.n_model);
    if (NT == 256) {
        if (o->precision == LASP_PREC_TF32) return run_grouped<D, 1, 256>(G, tc, st, launches);
        if (o->precision == LASP_PREC_BF16) return run_grouped<D, 2, 256>(G, tc, st, launches);
        if (o->fp64_normal_eq == LASP_NE_FP64) return run_grouped<D, 3, 256, true>(G, tc, st, launches);
        return run_grouped<D, 3, 256>(G, tc, st, launches);
    }
    if (o->precision == LASP_PREC_TF32) return run_grouped<D, 1, 512>(G, tc, st, launches);
    if (o->precision == LASP_PREC_BF16) return run_grouped<D, 2, 512>(G, tc, st, launches);
    if (o->fp64_normal_eq == LASP_NE_FP64) return run_grouped<D, 3, 512, true>(G, tc, st, launches);
    return run_grouped<D, 3, 512>(G, tc, st, launches);
}

}  // namespace lasp
