// Launchers of the FP32 CUDA-core kernels, one translation unit per Legendre
// degree D (explicitly instantiated in lasp_k_d<D>.cu).
#pragma once

#include "lasp_fit.cuh"
#include "lasp_fit_multi.cuh"
#include "lasp_lm.cuh"
#include "lasp_model.cuh"
#include "lasp_prof.cuh"

namespace lasp {

int cuda_rc(cudaError_t e);

template <int D> int launch_fit(const FitParams& P, cudaStream_t st);
template <int D> int launch_fit_multi(const FitParams& P, cudaStream_t st, int* n_launch = nullptr);
template <int D> int launch_fit_multi_slots(const FitParams& P, const MultiWs& W, int n_running, cudaStream_t st);
template <int D> int launch_fit_prep_slots(const FitParams& P, const MultiWs& W, const int32_t* idx, int count,
                                           cudaStream_t st);
template <int D> int launch_errors(const ErrParams& P, cudaStream_t st);
template <int D> int launch_forward(const ModelParams& P, cudaStream_t st);
template <int D> int launch_backward(const ModelParams& P, cudaStream_t st);
template <int D> int launch_lm(const LmParams& P, cudaStream_t st);

// Spectra per CTA of the batch fit (fit_multi_kernel).
constexpr int FIT_LANES = 4;

// Whether resumable slots of this table and degree run on fit_multi_kernel
// (its shared memory fits), with y, W rows of 2 ldw floats per slot.
inline bool fit_multi_slots_ok(int p, int H, int nm, int K, int D) {
    const int NT = fit_threads(nm);
    return fit_multi_smem_bytes(p, H, nm, NT, D, K, FIT_LANES, true) <= 227 * 1024 &&
           4 * (size_t)fit_prep_smem_floats(p) <= 227 * 1024;
}

#ifdef LASP_DEFINE_LAUNCHERS
template <typename Kern>
static int set_smem_attr(Kern k, size_t bytes) {
    if (bytes > 227 * 1024) return -1;
    return cuda_rc(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <int D>
int launch_fit(const FitParams& P, cudaStream_t st) {
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    return prof_time("fit_kernel", st, [&]() {
        if (fit_threads(nm) == 256) {
            size_t smem = fit_smem_bytes(p, H, nm, 256, D, P.M.K);
            int e = set_smem_attr(fit_kernel<256, D>, smem);
            if (e) return e;
            fit_kernel<256, D><<<P.N, 256, smem, st>>>(P);
        } else {
            size_t smem = fit_smem_bytes(p, H, nm, 512, D, P.M.K);
            int e = set_smem_attr(fit_kernel<512, D>, smem);
            if (e) return e;
            fit_kernel<512, D><<<P.N, 512, smem, st>>>(P);
        }
        return cuda_rc(cudaGetLastError());
    });
}


// One-shot batch fit: fit_prep_kernel (one CTA per spectrum), then FIT_LANES
// spectra per CTA on a persistent grid of as many CTAs as the SMs hold.  The
// workspace (spectrum counter, w, mean ivar and the y, W rows of every
// spectrum: about 8 p bytes a spectrum) is taken from the stream-ordered pool
// for the launch.
// Falls back to fit_kernel where the lanes' buffers or the workspace do not fit.
template <int D>
int launch_fit_multi(const FitParams& P, cudaStream_t st, int* n_launch) {
    constexpr int S = FIT_LANES;
    if (n_launch) *n_launch = 1;             // fit_kernel alone where it falls back
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    const int NT = fit_threads(nm);
    const bool full = P.O.clean || P.O.fp64_ne == LASP_NE_FP64;
    const size_t smem = fit_multi_smem_bytes(p, H, nm, NT, D, P.M.K, S, full);
    const size_t smem_prep = 4 * (size_t)fit_prep_smem_floats(p);
    // resumable slots, and Clean with too few lanes for its scratch, stay on fit_kernel
    if (P.S.x || (P.O.clean && S < 3) || smem > 227 * 1024 || smem_prep > 227 * 1024) return launch_fit<D>(P, st);
    // Clean and the FP64 normal equations each on their own variant, both on the full one
    const bool ne64 = P.O.fp64_ne == LASP_NE_FP64;
    const int mode = ne64 ? (P.O.clean ? MULTI_FULL : MULTI_NE64) : P.O.clean ? MULTI_CLEAN : MULTI_PLAIN;
    void (*kern)(const FitParams, const MultiWs) =
        mode == MULTI_FULL    ? (NT == 256 ? fit_multi_kernel<256, D, S, MULTI_FULL> : fit_multi_kernel<512, D, S, MULTI_FULL>)
        : mode == MULTI_NE64  ? (NT == 256 ? fit_multi_kernel<256, D, S, MULTI_NE64> : fit_multi_kernel<512, D, S, MULTI_NE64>)
        : mode == MULTI_CLEAN ? (NT == 256 ? fit_multi_kernel<256, D, S, MULTI_CLEAN> : fit_multi_kernel<512, D, S, MULTI_CLEAN>)
                              : (NT == 256 ? fit_multi_kernel<256, D, S, MULTI_PLAIN> : fit_multi_kernel<512, D, S, MULTI_PLAIN>);
    void (*prep)(const FitParams, const MultiWs) =
        NT == 256 ? fit_prep_kernel<256, D> : fit_prep_kernel<512, D>;
    int e = set_smem_attr(kern, smem);
    if (!e) e = set_smem_attr(prep, smem_prep);
    if (e) return e;
    int nb = 0, dev = 0, nsm = 0;
    e = cuda_rc(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem));
    if (!e) e = cuda_rc(cudaGetDevice(&dev));
    if (!e) e = cuda_rc(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (e) return e;
    if (nb < 1) return launch_fit<D>(P, st);
    const int grid = (int)std::min<long long>(((long long)P.N + S - 1) / S, (long long)nb * nsm);
    MultiWs W{};
    W.ldw = (p + 15) & ~15;
    const size_t rows = (size_t)P.N * 2 * W.ldw * sizeof(float);
    const size_t wq = ((size_t)P.N * sizeof(float) + 255) & ~(size_t)255;   // w, then the mean ivar
    const bool order = P.M.n_reg > 1;                  // piecewise: spectra taken grouped by regime
    const size_t ob = order ? 2 * wq : 0;              // segment and order, N ints each
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, 256 + 2 * wq + ob + rows, st) != cudaSuccess) {
        cudaGetLastError();
        return launch_fit<D>(P, st);          // no room for the workspace: one spectrum per CTA
    }
    W.next = static_cast<int*>(ws);
    W.wq = reinterpret_cast<float*>(static_cast<char*>(ws) + 256);
    W.im = reinterpret_cast<float*>(static_cast<char*>(ws) + 256 + wq);
    W.yw = reinterpret_cast<float*>(static_cast<char*>(ws) + 256 + 2 * wq + ob);
    e = cuda_rc(cudaMemsetAsync(ws, 0, 256, st));
    if (!e && order) {
        int* seg = reinterpret_cast<int*>(static_cast<char*>(ws) + 256 + 2 * wq);
        int* ord = reinterpret_cast<int*>(static_cast<char*>(ws) + 256 + 3 * wq);
        int* count = W.next + 16;                      // 2 NREG - 1 counters in the zeroed header
        const int nb256 = (P.N + 255) / 256;
        e = prof_time("regime_order_kernels", st, [&]() {
            regime_count_kernel<<<nb256, 256, 0, st>>>(P.M, P.N, P.theta0, seg, count);
            regime_offsets_kernel<<<1, 32, 0, st>>>(P.N, 2 * P.M.n_reg - 1, count, W.next);
            regime_scatter_kernel<<<nb256, 256, 0, st>>>(P.N, seg, count, ord);
            return cuda_rc(cudaGetLastError());
        });
        W.list = ord;
    }
    if (!e) e = prof_time("fit_prep_kernel", st, [&]() {
            prep<<<P.N, NT, smem_prep, st>>>(P, W);
            return cuda_rc(cudaGetLastError());
        });
    const char* name = mode == MULTI_FULL    ? "fit_multi_kernel<full>"
                       : mode == MULTI_NE64  ? "fit_multi_kernel<ne64>"
                       : mode == MULTI_CLEAN ? "fit_multi_kernel<clean>" : "fit_multi_kernel";
    if (!e) e = prof_time(name, st, [&]() {
            kern<<<grid, NT, smem, st>>>(P, W);
            return cuda_rc(cudaGetLastError());
        });
    const int ef = cuda_rc(cudaFreeAsync(ws, st));
    if (n_launch) *n_launch = order ? 5 : 2;  // (the regime order,) fit_prep_kernel, fit_multi_kernel
    return e ? e : ef;
}

// One step launch of a slot pool on fit_multi_kernel: a persistent grid whose
// lanes take the running slots through W.next (cleared here), at most one
// CTA per FIT_LANES of the caller's running count.
template <int D>
int launch_fit_multi_slots(const FitParams& P, const MultiWs& W, int n_running, cudaStream_t st) {
    constexpr int S = FIT_LANES;
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    const int NT = fit_threads(nm);
    // the Clean update and the FP64 normal equations only where the options ask for them
    const bool full = P.O.clean || P.O.fp64_ne == LASP_NE_FP64;
    const size_t smem = fit_multi_smem_bytes(p, H, nm, NT, D, P.M.K, S, full);
    void (*kern)(const FitParams, const MultiWs) =
        full ? (NT == 256 ? fit_multi_kernel<256, D, S, MULTI_FULL> : fit_multi_kernel<512, D, S, MULTI_FULL>)
             : (NT == 256 ? fit_multi_kernel<256, D, S, MULTI_SLOTS> : fit_multi_kernel<512, D, S, MULTI_SLOTS>);
    int e = set_smem_attr(kern, smem);
    if (e) return e;
    int nb = 0, dev = 0, nsm = 0;
    e = cuda_rc(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem));
    if (!e) e = cuda_rc(cudaGetDevice(&dev));
    if (!e) e = cuda_rc(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (e) return e;
    if (nb < 1) return cuda_rc(cudaErrorLaunchOutOfResources);
    const long long nr = std::min(P.N, std::max(1, n_running));
    const int grid = (int)std::min<long long>((nr + S - 1) / S, (long long)nb * nsm);
    // the running slots first, so that lanes take work without scanning idle
    // slots and CTAs left without work end at once (freeing their SMs)
    e = cuda_rc(cudaMemsetAsync(W.next, 0, 2 * sizeof(int), st));
    if (e) return e;
    e = prof_time("slots_running_list", st, [&]() {
        slots_running_list<<<(P.N + 255) / 256, 256, 0, st>>>(P.N, P.status, const_cast<int*>(W.list), W.next);
        return cuda_rc(cudaGetLastError());
    });
    if (e) return e;
    return prof_time("fit_multi_kernel<slots>", st, [&]() {
        kern<<<grid, NT, smem, st>>>(P, W);
        return cuda_rc(cudaGetLastError());
    });
}

// Preprocessing of `count` freshly admitted slots (idx: device slot indices).
template <int D>
int launch_fit_prep_slots(const FitParams& P, const MultiWs& W, const int32_t* idx, int count,
                          cudaStream_t st) {
    const int p = P.M.n_pix;
    const int NT = fit_threads(P.M.n_model);      // as the batch fit's preprocessing: the same sums
    const size_t smem = 4 * (size_t)fit_prep_smem_floats(p);
    void (*prep)(const FitParams, const MultiWs, const int32_t*) =
        NT == 256 ? fit_prep_slots_kernel<256, D> : fit_prep_slots_kernel<512, D>;
    int e = set_smem_attr(prep, smem);
    if (e) return e;
    return prof_time("fit_prep_slots_kernel", st, [&]() {
        prep<<<count, NT, smem, st>>>(P, W, idx);
        return cuda_rc(cudaGetLastError());
    });
}

template <int D>
int launch_errors(const ErrParams& P, cudaStream_t st) {
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    const bool f64 = P.O.fp64_ne == LASP_NE_FP64;
    auto go = [&](auto kern, int NT) {
        const size_t smem = err_smem_bytes(p, H, nm, NT);
        int e = set_smem_attr(kern, smem);
        if (!e) kern<<<P.N, NT, smem, st>>>(P);
        return e;
    };
    return prof_time(f64 ? "errors_kernel<fp64>" : "errors_kernel", st, [&]() {
        int e;
        if (fit_threads(nm) == 256) e = f64 ? go(errors_kernel<256, D, true>, 256) : go(errors_kernel<256, D, false>, 256);
        else e = f64 ? go(errors_kernel<512, D, true>, 512) : go(errors_kernel<512, D, false>, 512);
        return e ? e : cuda_rc(cudaGetLastError());
    });
}

template <int D>
int launch_forward(const ModelParams& P, cudaStream_t st) {
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    size_t smem = model_smem_bytes(p, H, nm);
    if (fit_threads(nm) == 256) {
        int e = set_smem_attr(forward_kernel<256, D>, smem);
        if (e) return e;
        forward_kernel<256, D><<<P.N, 256, smem, st>>>(P);
    } else {
        int e = set_smem_attr(forward_kernel<512, D>, smem);
        if (e) return e;
        forward_kernel<512, D><<<P.N, 512, smem, st>>>(P);
    }
    return cuda_rc(cudaGetLastError());
}

template <int D>
int launch_backward(const ModelParams& P, cudaStream_t st) {
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    size_t smem = model_smem_bytes(p, H, nm);
    if (fit_threads(nm) == 256) {
        int e = set_smem_attr(backward_kernel<256, D>, smem);
        if (e) return e;
        backward_kernel<256, D><<<P.N, 256, smem, st>>>(P);
    } else {
        int e = set_smem_attr(backward_kernel<512, D>, smem);
        if (e) return e;
        backward_kernel<512, D><<<P.N, 512, smem, st>>>(P);
    }
    return cuda_rc(cudaGetLastError());
}

template <int D>
int launch_lm(const LmParams& P, cudaStream_t st) {
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    return prof_time("lm_kernel", st, [&]() {
        if (fit_threads(nm) == 256) {
            size_t smem = lm_smem_bytes(p, H, nm, 256);
            int e = set_smem_attr(lm_kernel<256, D>, smem);
            if (e) return e;
            lm_kernel<256, D><<<P.N, 256, smem, st>>>(P);
        } else {
            size_t smem = lm_smem_bytes(p, H, nm, 512);
            int e = set_smem_attr(lm_kernel<512, D>, smem);
            if (e) return e;
            lm_kernel<512, D><<<P.N, 512, smem, st>>>(P);
        }
        return cuda_rc(cudaGetLastError());
    });
}

#define LASP_INSTANTIATE(D)                                                  \
    template int launch_fit<D>(const FitParams&, cudaStream_t);             \
    template int launch_fit_multi<D>(const FitParams&, cudaStream_t, int*); \
    template int launch_fit_multi_slots<D>(const FitParams&, const MultiWs&, int, cudaStream_t); \
    template int launch_fit_prep_slots<D>(const FitParams&, const MultiWs&, const int32_t*, int, cudaStream_t); \
    template int launch_errors<D>(const ErrParams&, cudaStream_t);          \
    template int launch_forward<D>(const ModelParams&, cudaStream_t);       \
    template int launch_backward<D>(const ModelParams&, cudaStream_t);      \
    template int launch_lm<D>(const LmParams&, cudaStream_t);
#endif

}  // namespace lasp
