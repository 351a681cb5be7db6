// Tensor-core (tcgen05) forms of the interpolator contraction (Eq. 1), sm_103a.
//
// The table is kept as per-tile images ready for the MMA: tile t holds model
// pixels 128 t .. 128 t + 127 as 128 rows of 32 basis terms per K block
// (n_kb blocks of 32 terms: one for a single regime, up to three for the
// stacked rows of a piecewise interpolator), K-major with the 128-byte
// swizzle, so one 1D bulk copy brings a tile into shared memory in MMA layout.
// TF32 is stored as a hi/lo split (hi = tf32(C), lo = tf32(C - hi)); BF16
// occupies the first 64 bytes of each 128-byte row.
#pragma once

#include "lasp.h"
#include "lasp_common.cuh"

namespace lasp {

constexpr int TC_TILE = 128;            // model pixels per tile (MMA M)
constexpr int TC_TILE_BYTES = 128 * 128; // 16 KB per image tile

struct TcImages {
    void* tf32_hi = nullptr;          // tile t, block b at (t n_kb + b) 16 KB
    void* tf32_lo = nullptr;
    void* bf16 = nullptr;
    int n_tiles = 0;
    int n_kb = 1;                     // K blocks of 32 basis terms
    // Backward images (dphi = dF' C^T): per chunk of model pixels (32 for TF32,
    // 64 for BF16) a (32 n_kb)-row (basis term) x 128-byte tile, K-major in
    // pixels, 128-byte swizzle (4 KB per K block, the blocks contiguous).
    void* bk_hi = nullptr;
    void* bk_lo = nullptr;
    void* bk_bf = nullptr;
    int n_chunks_tf32 = 0;
    int n_chunks_bf16 = 0;
};
constexpr int TC_BK_CHUNK_BYTES = 32 * 128;

int tc_build_images(TcImages& t, const float* C, int K, int n_model);

// Poll limit of the first bounded wait of each CTA of a tensor-core kernel
// (a table-copy wait, issued before any MMA): `normal`, unless the testing hook
// lasp_test_wait_limit has set a shorter one.
uint32_t first_wait_limit(uint32_t normal);
// Kernel count reported by lasp_last_launches for the calling thread.
void set_last_launches(int n);
void tc_free_images(TcImages& t);

int lasp_tc_interp_eval(const ModelDev& M, const TcImages& t, int N, const float* theta, float* Fp,
                        int precision, cudaStream_t st, int* launches);

// Persistent grouped pipeline over the slot arrays of a lasp_slots pool
// (served fits at tensor-core precision); see lasp_grouped.cu.
struct GrpPool;
int grp_pool_create(const ModelDev& M, const TcImages& tc, int n, const lasp_fit_opts* o, float* flux,
                    float* ivar, uint8_t* good, float* theta0, float* theta, float* loss, int32_t* steps,
                    uint32_t* status, float* cont, float* weight, GrpPool** out);
int grp_pool_admit(GrpPool* P, int count, const int32_t* idx_dev, cudaStream_t st);
int grp_pool_step(GrpPool* P, int budget, cudaStream_t st, int* launches);
void grp_pool_free(GrpPool* P);

int lasp_tc_fit_batch(const ModelDev& M, const TcImages& t, const lasp_batch* b, const lasp_fit_opts* o,
                      lasp_result* r, void* stream, int* launches);

}  // namespace lasp
