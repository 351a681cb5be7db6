// Launchers of the FP32 CUDA-core kernels, one translation unit per Legendre
// degree D (explicitly instantiated in lasp_k_d<D>.cu).
#pragma once

#include "lasp_fit.cuh"
#include "lasp_lm.cuh"
#include "lasp_model.cuh"

namespace lasp {

int cuda_rc(cudaError_t e);

template <int D> int launch_fit(const FitParams& P, cudaStream_t st);
template <int D> int launch_errors(const ErrParams& P, cudaStream_t st);
template <int D> int launch_forward(const ModelParams& P, cudaStream_t st);
template <int D> int launch_backward(const ModelParams& P, cudaStream_t st);
template <int D> int launch_lm(const LmParams& P, cudaStream_t st);

#ifdef LASP_DEFINE_LAUNCHERS
template <typename Kern>
static int set_smem_attr(Kern k, size_t bytes) {
    if (bytes > 227 * 1024) return -1;
    return cuda_rc(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <int D>
int launch_fit(const FitParams& P, cudaStream_t st) {
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    if (p <= 16 * 256) {
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
}

template <int D>
int launch_errors(const ErrParams& P, cudaStream_t st) {
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    if (p <= 16 * 256) {
        size_t smem = err_smem_bytes(p, H, nm, 256);
        int e = set_smem_attr(errors_kernel<256, D>, smem);
        if (e) return e;
        errors_kernel<256, D><<<P.N, 256, smem, st>>>(P);
    } else {
        size_t smem = err_smem_bytes(p, H, nm, 512);
        int e = set_smem_attr(errors_kernel<512, D>, smem);
        if (e) return e;
        errors_kernel<512, D><<<P.N, 512, smem, st>>>(P);
    }
    return cuda_rc(cudaGetLastError());
}

template <int D>
int launch_forward(const ModelParams& P, cudaStream_t st) {
    const int p = P.M.n_pix, H = P.M.pad, nm = P.M.n_model;
    size_t smem = model_smem_bytes(p, H, nm);
    if (p <= 16 * 256) {
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
    if (p <= 16 * 256) {
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
    if (p <= 16 * 256) {
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
}

#define LASP_INSTANTIATE(D)                                                  \
    template int launch_fit<D>(const FitParams&, cudaStream_t);             \
    template int launch_errors<D>(const ErrParams&, cudaStream_t);          \
    template int launch_forward<D>(const ModelParams&, cudaStream_t);       \
    template int launch_backward<D>(const ModelParams&, cudaStream_t);      \
    template int launch_lm<D>(const LmParams&, cudaStream_t);
#endif

}  // namespace lasp
