// Clean outlier masking (stage 6, Eq. 8) by one CTA -- sm_103a.
//
// From the weighted residual r_j = sqrt(W_j) eps_j and the weighted model
// m_j = sqrt(W_j) c_j F''_j of one spectrum: sigma = std of r over the used
// pixels; G_j = max(|m_j - m_{j-1}|, |m_j - m_{j+1}|); B: |r| - f G > k sigma
// with k = 3 relaxed to 4, 5, 7 while more than 3% of the used pixels are
// flagged; C: neighbours of B outliers with |r| - f G > 2 sigma; D:
// neighbours of flagged pixels with the same sign, no larger |r| and
// |r| - f G > sigma' (std over used pixels not in B or C), repeated until
// unchanged (at most 20 passes).  Thread t owns pixels 16 t .. 16 t + 15.
#pragma once

#include "lasp_common.cuh"

namespace lasp {

// Sum of three doubles over the CTA; the sums end in tot[0..2] for all threads.
template <int NT>
__device__ __forceinline__ void cta_sum3_f64(double a, double b, double c, double* redd, double* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        redd[3 * warp + 0] = a;
        redd[3 * warp + 1] = b;
        redd[3 * warp + 2] = c;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += redd[3 * w + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ float std_from_sums(const double* tot) {
    if (tot[2] <= 0.0) return 0.0f;
    const double mean = tot[0] / tot[2], var = tot[1] / tot[2] - mean * mean;
    return (float)sqrt(var > 0.0 ? var : 0.0);
}

// Rs, Ms: r and m of pixel j at skew(j + roff), skew(j + moff) (shared).  used: bit r of
// the thread's own pixel j0 + r.  fl: 2 (p + 2) bytes of shared scratch that
// may alias Ms.  redd: 3 (NT/32) doubles, tot: 3 doubles (shared).  Returns
// the thread's keep bits (used and not flagged); *k_used gets the k of B.
template <int NT, int PPTC>
__device__ uint32_t cta_clean_mask(int p, int j0, const float* Rs, int roff, float* Ms, int moff,
                                   uint32_t used, float fshift, uint8_t* fl, double* redd, double* tot,
                                   int* k_used) {
    constexpr int kPPT = PPTC;
    float lhs[kPPT];
    // sigma over used pixels; G and lhs from the model neighbours
    double s1 = 0.0, s2 = 0.0, n = 0.0;
#pragma unroll
    for (int r = 0; r < kPPT; ++r) {
        const int j = j0 + r;
        lhs[r] = 0.0f;
        if (j < p) {
            const float rj = Rs[skew(j + roff)], mj = Ms[skew(j + moff)];
            float gj = 0.0f;
            if (j > 0) gj = fabsf(mj - Ms[skew(j - 1 + moff)]);
            if (j < p - 1) {
                const float g2 = fabsf(mj - Ms[skew(j + 1 + moff)]);
                if (g2 > gj) gj = g2;
            }
            lhs[r] = __fsub_rn(fabsf(rj), __fmul_rn(fshift, gj));
            if ((used >> r) & 1u) {
                s1 += rj;
                s2 += (double)rj * rj;
                n += 1.0;
            }
        }
    }
    cta_sum3_f64<NT>(s1, s2, n, redd, tot);     // also: every thread is done with Ms
    const float sigma = std_from_sums(tot);
    const double n_used = tot[2];
    // B: counts for k = 3, 4, 5 (and 7 needs no count)
    const float ks[4] = {3.0f, 4.0f, 5.0f, 7.0f};
    double c3 = 0.0, c4 = 0.0, c5 = 0.0;
#pragma unroll
    for (int r = 0; r < kPPT; ++r)
        if ((used >> r) & 1u) {
            c3 += lhs[r] > ks[0] * sigma ? 1.0 : 0.0;
            c4 += lhs[r] > ks[1] * sigma ? 1.0 : 0.0;
            c5 += lhs[r] > ks[2] * sigma ? 1.0 : 0.0;
        }
    cta_sum3_f64<NT>(c3, c4, c5, redd, tot);
    int kk = 3;
    if (!(tot[0] > 0.03 * n_used)) kk = 0;
    else if (!(tot[1] > 0.03 * n_used)) kk = 1;
    else if (!(tot[2] > 0.03 * n_used)) kk = 2;
    const float kb = ks[kk];
    if (k_used) *k_used = (int)kb;
    uint8_t* A = fl;                 // flags, pixel j at A[j + 1] (A[0], A[p+1] = 0)
    uint8_t* Bf = fl + (p + 2);
    if (threadIdx.x == 0) {
        A[0] = A[p + 1] = 0;
        Bf[0] = Bf[p + 1] = 0;
    }
#pragma unroll
    for (int r = 0; r < kPPT; ++r) {
        const int j = j0 + r;
        if (j < p) A[j + 1] = (((used >> r) & 1u) && lhs[r] > kb * sigma) ? 1 : 0;
    }
    __syncthreads();
    // C: neighbours of B outliers; sigma' over used pixels not in B or C
    s1 = s2 = n = 0.0;
#pragma unroll
    for (int r = 0; r < kPPT; ++r) {
        const int j = j0 + r;
        if (j < p) {
            uint8_t f = A[j + 1];
            if (!f && ((used >> r) & 1u) && (A[j] || A[j + 2]) && lhs[r] > 2.0f * sigma) f = 1;
            Bf[j + 1] = f;
            if (((used >> r) & 1u) && !f) {
                const float rj = Rs[skew(j + roff)];
                s1 += rj;
                s2 += (double)rj * rj;
                n += 1.0;
            }
        }
    }
    cta_sum3_f64<NT>(s1, s2, n, redd, tot);
    const float sigp = std_from_sums(tot);
    // D: grow along same-sign, non-increasing residuals above sigma'
    uint8_t* cur = Bf;
    uint8_t* nxt = A;
    for (int it = 0; it < 20; ++it) {
        double ch = 0.0;
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            const int j = j0 + r;
            if (j < p) {
                uint8_t f = cur[j + 1];
                if (!f && ((used >> r) & 1u) && lhs[r] > sigp) {
                    const float rj = Rs[skew(j + roff)];
                    if (cur[j] && j > 0) {
                        const float ri = Rs[skew(j - 1 + roff)];
                        if (ri * rj > 0.0f && fabsf(rj) <= fabsf(ri)) f = 1;
                    }
                    if (cur[j + 2] && j < p - 1) {
                        const float ri = Rs[skew(j + 1 + roff)];
                        if (ri * rj > 0.0f && fabsf(rj) <= fabsf(ri)) f = 1;
                    }
                    if (f) ch += 1.0;
                }
                nxt[j + 1] = f;
            }
        }
        if (threadIdx.x == 0) nxt[0] = nxt[p + 1] = 0;
        cta_sum3_f64<NT>(ch, 0.0, 0.0, redd, tot);
        uint8_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
        if (!(tot[0] > 0.0)) break;
    }
    uint32_t keep = 0;
#pragma unroll
    for (int r = 0; r < kPPT; ++r) {
        const int j = j0 + r;
        if (j < p && ((used >> r) & 1u) && !cur[j + 1]) keep |= 1u << r;
    }
    return keep;
}

}  // namespace lasp
