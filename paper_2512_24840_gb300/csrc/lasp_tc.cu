// Tensor-core (tcgen05) interpolator contraction, Eq. 1: Fp = phi(theta) C.
//
// One CTA (4 warps) takes 128 spectra (the MMA N dimension) and loops over
// 128-pixel tiles of the model grid (the MMA M dimension), K = 32 basis
// terms.  The basis rows phi are written once into shared memory in the
// swizzled K-major layout; each table tile arrives by one bulk copy; one
// thread issues the MMAs into a 128 x 128 FP32 accumulator in TMEM; each warp
// then reads its 32 TMEM lanes (pixels) and writes 128-byte coalesced runs of
// F' per spectrum.
#include <cuda_bf16.h>

#include "lasp_tc.cuh"
#include "lasp_tc_ptx.cuh"

namespace lasp {

int cuda_rc(cudaError_t e);

namespace {

constexpr uint32_t kWaitLimit = 1u << 22;

// Forward images: tile t, K block b, row r (model pixel), 16-byte piece c.
__global__ void build_images_kernel(const float* __restrict__ C, int K, int n_model, int n_tiles, int n_kb,
                                    uint8_t* hi, uint8_t* lo, uint8_t* bf) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = n_tiles * n_kb * TC_TILE * 8;
    if (idx >= total) return;
    const int c = idx & 7, r = (idx >> 3) & (TC_TILE - 1), tb = idx >> 10;
    const int t = tb / n_kb, b = tb - t * n_kb;
    const int m = t * TC_TILE + r;
    const uint32_t off = (uint32_t)tb * TC_TILE_BYTES + tc::sw128_off(r, c);
    float v[4], h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 32 * b + 4 * c + q;
        v[q] = (m < n_model && k < K) ? C[(size_t)k * n_model + m] : 0.0f;
        h[q] = tc::to_tf32(v[q]);
        l[q] = tc::to_tf32(v[q] - h[q]);
    }
    *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    // BF16: piece c < 4 holds basis terms 32 b + 8c .. 32 b + 8c + 7, pieces 4..7 are zero
    __nv_bfloat16 bv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k = 32 * b + 8 * c + q;
        const float x = (c < 4 && m < n_model && k < K) ? C[(size_t)k * n_model + m] : 0.0f;
        bv[q] = __float2bfloat16_rn(x);
    }
    *reinterpret_cast<uint4*>(bf + off) = *reinterpret_cast<uint4*>(bv);
}

// Backward table images: chunk c, row k (basis term, 32 n_kb rows), 16-byte piece q.
__global__ void build_back_images_kernel(const float* __restrict__ C, int K, int n_model, int n_ch32,
                                         int n_ch64, int n_kb, uint8_t* hi, uint8_t* lo, uint8_t* bf) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int rows = 32 * n_kb;
    const int total = n_ch32 * rows * 8;
    if (idx >= total) return;
    const int q = idx & 7, k = (idx >> 3) % rows, c = (idx >> 3) / rows;
    const uint32_t off = (uint32_t)c * n_kb * TC_BK_CHUNK_BYTES + tc::sw128_off(k, q);
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int m = 32 * c + 4 * q + e;
        const float v = (k < K && m < n_model) ? C[(size_t)k * n_model + m] : 0.0f;
        h[e] = tc::to_tf32(v);
        l[e] = tc::to_tf32(v - h[e]);
    }
    *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    if (c < n_ch64) {
        __nv_bfloat16 b[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int m = 64 * c + 8 * q + e;
            b[e] = __float2bfloat16_rn((k < K && m < n_model) ? C[(size_t)k * n_model + m] : 0.0f);
        }
        *reinterpret_cast<uint4*>(bf + off) = *reinterpret_cast<uint4*>(b);
    }
}

// PREC: 1 TF32, 2 BF16, 3 split TF32 (hi*hi + hi*lo + lo*hi).  n_kb K
// blocks of 32 basis terms accumulate into one 128 x 128 accumulator.  Every
// wait is bounded; when one gives up the CTA sets *err, writes NaN into every
// output of the tiles it has not finished, lets its own copies and MMAs in
// flight complete (bounded again), frees its TMEM and returns.  wait0 bounds
// the first table-copy wait of the CTA (no MMA issued yet).
template <int PREC>
__global__ void __launch_bounds__(128) interp_tc_kernel(const ModelDev M, const float* __restrict__ theta,
                                                        float* __restrict__ Fp, int N,
                                                        const uint8_t* __restrict__ img_a,
                                                        const uint8_t* __restrict__ img_a_lo,
                                                        int n_tiles, int n_kb, int* err, uint32_t wait0) {
    extern __shared__ uint8_t smraw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const uint32_t blk_bytes = (uint32_t)n_kb * TC_TILE_BYTES;
    uint8_t* Ahi = base;
    uint8_t* Alo = base + blk_bytes;
    uint8_t* Bhi = base + 2 * blk_bytes;
    uint8_t* Blo = base + 3 * blk_bytes;
    __shared__ __align__(8) uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s0 = blockIdx.x * 128;

    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 128);
        tc::tmem_relinquish();
    }
    // B operand row tid: phi of spectrum s0 + tid, zero beyond N or K
    {
        float phi[KROWS];
        for (int k = 0; k < 32 * n_kb; ++k) phi[k] = 0.0f;
        if (s0 + tid < N) {
            float th[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) th[q] = theta[5 * (size_t)(s0 + tid) + q];
            for (int k = 0; k < M.K; ++k) basis_term(M, k, th, phi, nullptr);
        }
        for (int b = 0; b < n_kb; ++b) {
            uint8_t* bh = Bhi + b * TC_TILE_BYTES;
            uint8_t* bl = Blo + b * TC_TILE_BYTES;
            if (PREC == 2) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    __nv_bfloat16 bv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) bv[q] = __float2bfloat16_rn(c < 4 ? phi[32 * b + 8 * c + q] : 0.0f);
                    *reinterpret_cast<uint4*>(bh + tc::sw128_off(tid, c)) = *reinterpret_cast<uint4*>(bv);
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
    uint32_t phase = 0;
    bool copy_pending = false, mma_pending = false;
    int t = blockIdx.y;

    for (; t < n_tiles; t += gridDim.y) {
        if (tid == 0) {
            const uint32_t bytes = (PREC == 3 ? 2u : 1u) * blk_bytes;
            tc::mbar_arrive_expect_tx(&bar_tma, bytes);
            tc::bulk_g2s(Ahi, img_a + (size_t)t * blk_bytes, blk_bytes, &bar_tma);
            if (PREC == 3) tc::bulk_g2s(Alo, img_a_lo + (size_t)t * blk_bytes, blk_bytes, &bar_tma);
            copy_pending = true;
            if (!tc::mbar_wait_bounded(&bar_tma, phase, t == (int)blockIdx.y ? wait0 : kWaitLimit)) {
                atomicExch(err, 1);
                s_ok = 0;
            } else {
                copy_pending = false;
                tc::tc_fence_after();
                for (int b = 0; b < n_kb; ++b) {
                    const uint64_t ah = tc::desc_kmajor_sw128(tc::smem_u32(Ahi + b * TC_TILE_BYTES));
                    const uint64_t bh = tc::desc_kmajor_sw128(tc::smem_u32(Bhi + b * TC_TILE_BYTES));
                    // K = 32 basis terms = 128 bytes per row: 4 TF32 MMAs (K=8) or 2 BF16 MMAs (K=16)
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
        if (!tc::mbar_wait_bounded(&bar_mma, phase, kWaitLimit)) {
            atomicExch(err, 1);
            s_ok = 0;
        }
        tc::tc_fence_after();
        if (s_ok) {
            const int mpix = t * TC_TILE + warp * 32 + lane;
#pragma unroll 1
            for (int c = 0; c < 8; ++c) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
                if (mpix < M.n_model) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int s = s0 + c * 16 + q;
                        if (s < N) Fp[(size_t)s * M.n_model + mpix] = v[q];
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
    if (!s_ok) {
        // the tiles from t on are not computed: NaN marks them in the output
        for (int tt = t; tt < n_tiles; tt += gridDim.y) {
            const int mpix = tt * TC_TILE + tid;
            if (mpix < M.n_model)
                for (int s = s0; s < N && s < s0 + 128; ++s) Fp[(size_t)s * M.n_model + mpix] = NAN;
        }
        // copies and MMAs still in flight complete before the CTA's memory goes
        if (tid == 0 && copy_pending) tc::mbar_wait_bounded(&bar_tma, phase, kWaitLimit);
        if (tid == 0 && mma_pending) tc::mbar_wait_bounded(&bar_mma, phase, kWaitLimit);
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

}  // namespace

int tc_build_images(TcImages& t, const float* C, int K, int n_model) {
    t = TcImages{};
    t.n_tiles = (n_model + TC_TILE - 1) / TC_TILE;
    t.n_kb = (K + 31) / 32;
    const size_t bytes = (size_t)t.n_tiles * t.n_kb * TC_TILE_BYTES;
    int rc = cuda_rc(cudaMalloc(&t.tf32_hi, bytes));
    if (!rc) rc = cuda_rc(cudaMalloc(&t.tf32_lo, bytes));
    if (!rc) rc = cuda_rc(cudaMalloc(&t.bf16, bytes));
    if (rc) return rc;
    const int total = t.n_tiles * t.n_kb * TC_TILE * 8;
    build_images_kernel<<<(total + 255) / 256, 256>>>(C, K, n_model, t.n_tiles, t.n_kb, (uint8_t*)t.tf32_hi,
                                                       (uint8_t*)t.tf32_lo, (uint8_t*)t.bf16);
    rc = cuda_rc(cudaGetLastError());
    if (rc) return rc;
    t.n_chunks_tf32 = (n_model + 31) / 32;
    t.n_chunks_bf16 = (n_model + 63) / 64;
    const size_t bk = (size_t)t.n_chunks_tf32 * t.n_kb * TC_BK_CHUNK_BYTES;
    rc = cuda_rc(cudaMalloc(&t.bk_hi, bk));
    if (!rc) rc = cuda_rc(cudaMalloc(&t.bk_lo, bk));
    if (!rc) rc = cuda_rc(cudaMalloc(&t.bk_bf, bk));
    if (rc) return rc;
    const int tb = t.n_chunks_tf32 * 32 * t.n_kb * 8;
    build_back_images_kernel<<<(tb + 255) / 256, 256>>>(C, K, n_model, t.n_chunks_tf32, t.n_chunks_bf16, t.n_kb,
                                                         (uint8_t*)t.bk_hi, (uint8_t*)t.bk_lo,
                                                         (uint8_t*)t.bk_bf);
    rc = cuda_rc(cudaGetLastError());
    if (!rc) rc = cuda_rc(cudaDeviceSynchronize());
    return rc;
}

void tc_free_images(TcImages& t) {
    if (t.bk_hi) cudaFree(t.bk_hi);
    if (t.bk_lo) cudaFree(t.bk_lo);
    if (t.bk_bf) cudaFree(t.bk_bf);
    if (t.tf32_hi) cudaFree(t.tf32_hi);
    if (t.tf32_lo) cudaFree(t.tf32_lo);
    if (t.bf16) cudaFree(t.bf16);
    t = TcImages{};
}

// Synchronous: the call waits for its kernel and reads back the kernel's
// timeout flag (a stream-ordered allocation of this call).
int lasp_tc_interp_eval(const ModelDev& M, const TcImages& t, int N, const float* theta, float* Fp,
                        int precision, cudaStream_t st, int* launches) {
    if (!t.tf32_hi) return LASP_EINVAL;
    const size_t smem = 4 * (size_t)t.n_kb * TC_TILE_BYTES + 1024;
    dim3 grid((N + 127) / 128, t.n_tiles < 65535 ? t.n_tiles : 65535);
    int* err = nullptr;
    int rc = cuda_rc(cudaMallocAsync((void**)&err, sizeof(int), st));
    if (rc) return rc;
    rc = cuda_rc(cudaMemsetAsync(err, 0, sizeof(int), st));
    const uint32_t wait0 = first_wait_limit(kWaitLimit);
    auto go = [&](auto kern, const void* a, const void* alo) {
        int e = cuda_rc(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        kern<<<grid, 128, smem, st>>>(M, theta, Fp, N, (const uint8_t*)a, (const uint8_t*)alo, t.n_tiles, t.n_kb,
                                      err, wait0);
        return cuda_rc(cudaGetLastError());
    };
    if (!rc) {
        if (precision == LASP_PREC_TF32) rc = go(interp_tc_kernel<1>, t.tf32_hi, nullptr);
        else if (precision == LASP_PREC_BF16) rc = go(interp_tc_kernel<2>, t.bf16, nullptr);
        else if (precision == LASP_PREC_TF32X3) rc = go(interp_tc_kernel<3>, t.tf32_hi, t.tf32_lo);
        else rc = LASP_EINVAL;
    }
    int h_err = 0;
    if (!rc) {
        *launches = 1;
        rc = cuda_rc(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    const int rf = cuda_rc(cudaFreeAsync(err, st));
    if (!rc) rc = rf;
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
    if (!rc && h_err) rc = LASP_ETIMEOUT;
    return rc;
}

}  // namespace lasp

// ---------------------------------------------------------------------------
// Allocation-free form of the tensor-core contraction.
//
// The handle-based path keeps the swizzled table images and its wait-timeout
// flag in memory that lasp_init_interp allocates.  Here the same kernel gets
// that scratch from one file-scope __device__ array instead, so a call makes
// no device allocation at all.  Every GPU that loads the library holds the
// array (3 MiB + 256 B) until the process exits.

#include <mutex>

namespace lasp {
namespace {

constexpr int kStaticMaxTiles = LASP_STATIC_MAX_MODEL_PIX / TC_TILE;
constexpr size_t kStaticImageBytes = (size_t)kStaticMaxTiles * TC_TILE_BYTES;
constexpr size_t kStaticBytes = 3 * kStaticImageBytes + 256;

// [TF32 hi image | TF32 lo image | BF16 image | timeout flag]; the flag is
// zero at load (static storage) and cleared when a call reports it
static __device__ __align__(256) uint8_t g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
uint8_t* g_static_addr[kMaxDevices] = {};
bool g_static_sm103[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once
// per device (with that device current), together with the check that the
// device is an sm_103 part.  Host code never touches the array through its
// name: on the host the name is only a stand-in for the symbol.
int static_scratch(uint8_t** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LASP_ENODEV;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return LASP_ENODEV;
        g_static_sm103[dev] = major == 10 && minor == 3;
        if (!g_static_sm103[dev]) return LASP_ENODEV;
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return LASP_ECUDA;
        // the timeout flag starts at zero: set once, finished before the first call goes on
        uint8_t* flag = static_cast<uint8_t*>(p) + 3 * kStaticImageBytes;
        if (cudaMemset(flag, 0, 256) != cudaSuccess || cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess)
            return LASP_ECUDA;
        g_static_addr[dev] = static_cast<uint8_t*>(p);
    }
    if (!g_static_sm103[dev]) return LASP_ENODEV;
    *out = g_static_addr[dev];
    return LASP_OK;
}

int static_model(const lasp_interp_desc* d, const float* coeff, ModelDev* M) {
    if (d->K < 1 || d->K > KMAX || d->n_pix < 16 || d->pad < 0 || d->pad > HMAX || !(d->dln > 0.0) ||
        !d->exps)
        return LASP_EINVAL;
    for (int k = 0; k < 3 * d->K; ++k)
        if (d->exps[k] < 0 || d->exps[k] > 8) return LASP_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!(d->basis_hi[k] > d->basis_lo[k])) return LASP_EINVAL;
    for (int k = 0; k < 5; ++k)
        if (!(d->box_hi[k] > d->box_lo[k])) return LASP_EINVAL;
    if (!(d->box_lo[0] > 0.0) || !(d->box_lo[4] > 0.0)) return LASP_EINVAL;
    const double kms = 299792.458 * d->dln;
    const double mumax = fmax(fabs(d->box_lo[3]), fabs(d->box_hi[3])) / kms;
    if ((int)ceil(mumax + 5.0 * d->box_hi[4] / kms) > d->pad) return LASP_EGRID;
    *M = ModelDev{};
    M->C = coeff;
    M->K = d->K;
    M->n_pix = d->n_pix;
    M->pad = d->pad;
    M->n_model = d->n_pix + 2 * d->pad;
    M->kms_px = (float)kms;
    M->n_reg = 1;
    M->reg_row[0] = 0;
    M->reg_row[1] = d->K;
    for (int k = 0; k < 3; ++k) {
        M->rblo[0][k] = (float)d->basis_lo[k];
        M->rbscale[0][k] = (float)(2.0 / (d->basis_hi[k] - d->basis_lo[k]));
    }
    for (int k = 0; k < 5; ++k) {
        M->plo[k] = (float)d->box_lo[k];
        M->phalf[k] = (float)(0.5 * (d->box_hi[k] - d->box_lo[k]));
    }
    for (int k = 0; k < 3 * d->K; ++k) M->exps[k] = d->exps[k];
    return LASP_OK;
}

}  // namespace
}  // namespace lasp

extern "C" int lasp_interp_eval_static(const lasp_interp_desc* desc, const float* coeff, int N,
                                       const float* theta, float* Fp, int precision, void* stream) {
    using namespace lasp;
    set_last_launches(0);
    if (!desc || N < 0) return LASP_EINVAL;
    if (precision != LASP_PREC_TF32 && precision != LASP_PREC_BF16 && precision != LASP_PREC_TF32X3)
        return LASP_EINVAL;
    ModelDev M;
    int rc = static_model(desc, coeff, &M);
    if (rc) return rc;
    if (M.n_model > LASP_STATIC_MAX_MODEL_PIX) return LASP_EINVAL;
    if (N == 0) return LASP_OK;
    if (!coeff || !theta || !Fp) return LASP_EINVAL;
    uint8_t* base = nullptr;
    rc = static_scratch(&base);
    if (rc) return rc;
    uint8_t* hi = base;
    uint8_t* lo = base + kStaticImageBytes;
    uint8_t* bf = base + 2 * kStaticImageBytes;
    int* err = reinterpret_cast<int*>(base + 3 * kStaticImageBytes);
    cudaStream_t st = (cudaStream_t)stream;
    // A wait that gave up in an earlier call left its flag set (and NaN in the
    // rows it did not compute).  Outside stream capture the flag is read after
    // the stream's earlier work, cleared, and reported here; during capture it
    // stays set for the next call made outside capture.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    rc = cuda_rc(cudaStreamIsCapturing(st, &cs));
    if (rc) return rc;
    if (cs == cudaStreamCaptureStatusNone) {
        int prev = 0;
        rc = cuda_rc(cudaMemcpyAsync(&prev, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
        if (!rc && prev) {
            rc = cuda_rc(cudaMemsetAsync(err, 0, sizeof(int), st));
            return rc ? rc : LASP_ETIMEOUT;
        }
        if (rc) return rc;
    }
    const int n_tiles = (M.n_model + TC_TILE - 1) / TC_TILE;
    const int total = n_tiles * TC_TILE * 8;
    build_images_kernel<<<(total + 255) / 256, 256, 0, st>>>(coeff, M.K, M.n_model, n_tiles, 1, hi, lo, bf);
    rc = cuda_rc(cudaGetLastError());
    if (rc) return rc;
    const size_t smem = 4 * TC_TILE_BYTES + 1024;
    dim3 grid((N + 127) / 128, n_tiles);
    const uint32_t wait0 = first_wait_limit(kWaitLimit);
    auto go = [&](auto kern, const uint8_t* a, const uint8_t* alo) {
        int e = cuda_rc(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        kern<<<grid, 128, smem, st>>>(M, theta, Fp, N, a, alo, n_tiles, 1, err, wait0);
        return cuda_rc(cudaGetLastError());
    };
    if (precision == LASP_PREC_TF32) rc = go(interp_tc_kernel<1>, hi, nullptr);
    else if (precision == LASP_PREC_BF16) rc = go(interp_tc_kernel<2>, bf, nullptr);
    else rc = go(interp_tc_kernel<3>, hi, lo);
    if (!rc) set_last_launches(2);
    return rc;
}
