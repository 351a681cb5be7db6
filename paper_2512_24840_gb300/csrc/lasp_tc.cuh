// Tensor-core (tcgen05) forms of the interpolator contraction -- sm_103a.
#pragma once

#include "lasp.h"
#include "lasp_common.cuh"

namespace lasp {

struct TcImages {
    void* tf32_hi = nullptr;   // per 128-pixel tile: 128 rows x 32 k, TF32, 128B-swizzled
    void* tf32_lo = nullptr;
    void* bf16 = nullptr;
    int n_tiles = 0;
};

inline int tc_build_images(TcImages& t, const float* C, int K, int n_model) {
    (void)C; (void)K; (void)n_model;
    t = TcImages{};
    return LASP_OK;
}

inline void tc_free_images(TcImages& t) {
    if (t.tf32_hi) cudaFree(t.tf32_hi);
    if (t.tf32_lo) cudaFree(t.tf32_lo);
    if (t.bf16) cudaFree(t.bf16);
    t = TcImages{};
}

inline int lasp_tc_fit_batch(const ModelDev&, const TcImages&, const lasp_batch*, const lasp_fit_opts*,
                             lasp_result*, void*, int*) {
    return LASP_EINVAL;
}

inline int lasp_tc_interp_eval(const ModelDev&, const TcImages&, int, const float*, float*, int,
                               cudaStream_t, int*) {
    return LASP_EINVAL;
}

}  // namespace lasp
