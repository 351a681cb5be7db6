// Host-only check that every grid lasp_init_interp accepts can be launched:
// for each margin H <= HMAX and each n_pix >= 16 with n_pix + 2 H <= 8192, the
// block chosen by fit_threads covers the model grid (16 model pixels a
// thread), and the dynamic shared memory of every per-spectrum kernel, at
// every Legendre degree and with the largest table (96 rows), together with
// the kernel's static shared arrays stays within the 227 KB a CTA may opt
// into.  The static arrays are allowed for as ptxas -v reports them for
// sm_103a: under 1 KB in every kernel but kc_clean (12 KB, with the step
// body's dynamic layout).  The multi-lane fit may exceed the limit (the
// launcher then falls back to the one-spectrum fit), so it is reported but
// not required.  Built as host code (no kernel is launched, no device is
// touched); exits non-zero on a failure.
#include <cstdio>

#include "lasp_grouped.cuh"
#include "lasp_launch.cuh"

using namespace lasp;

namespace {

struct Worst {
    const char* name;
    bool required;
    size_t static_bytes;      // allowance for the kernel's static shared arrays
    size_t bytes = 0;
    int p = 0, H = 0, D = 0;
    void see(size_t b, int p_, int H_, int D_) {
        if (b > bytes) bytes = b, p = p_, H = H_, D = D_;
    }
};

}  // namespace

int main() {
    const size_t limit = 227 * 1024, small = 2048;
    Worst fit{"fit_kernel", true, small}, multi{"fit_multi_kernel (full)", false, small},
        lm{"lm_kernel", true, small}, model{"forward/backward_kernel", true, small},
        err{"errors_kernel", true, small}, rest{"k2_rest/kc_clean", true, 13 * 1024},
        k0{"k0_prep", true, small}, prep{"fit_prep_kernel", true, small};
    long uncovered = 0;
    for (int H = 0; H <= HMAX; ++H)
        for (int p = 16; p + 2 * H <= MODEL_PIX_MAX; ++p) {
            const int nm = p + 2 * H, NT = fit_threads(nm);
            if (NT * PPT < nm) ++uncovered;
            for (int D = 2; D <= 8; D += 2) {
                fit.see(fit_smem_bytes(p, H, nm, NT, D, KROWS), p, H, D);
                multi.see(fit_multi_smem_bytes(p, H, nm, NT, D, KROWS, FIT_LANES, true), p, H, D);
                rest.see(4 * (size_t)RestSmem(p, H, nm, NT, D).total, p, H, D);
            }
            lm.see(lm_smem_bytes(p, H, nm, NT), p, H, 0);
            model.see(model_smem_bytes(p, H, nm), p, H, 0);
            err.see(err_smem_bytes(p, H, nm, NT), p, H, 0);
            k0.see(4 * ((size_t)3 * ((p + 3) & ~3) + PREP_RED), p, H, 0);
            prep.see(4 * (size_t)fit_prep_smem_floats(p), p, H, 0);
        }
    int fail = uncovered != 0;
    printf("grids whose block does not cover the model grid: %ld\n", uncovered);
    for (const Worst* w : {&fit, &multi, &lm, &model, &err, &rest, &k0, &prep}) {
        const bool over = w->bytes + w->static_bytes > limit;
        printf("%-26s largest %7zu B at n_pix=%d H=%d D=%d%s\n", w->name, w->bytes, w->p, w->H, w->D,
               over ? (w->required ? "  OVER THE LIMIT" : "  (falls back)") : "");
        if (over && w->required) fail = 1;
    }
    // tensor-core contractions: up to three K blocks of 32 terms
    for (int n_kb = 1; n_kb <= 3; ++n_kb) {
        const size_t k1 = 4 * (size_t)n_kb * TC_TILE_BYTES + 1024, k3 = k3_smem_bytes(n_kb);
        printf("k1_interp / k3_back, %d K block(s): %zu / %zu B\n", n_kb, k1, k3);
        if (k1 + small > limit || k3 + small > limit) fail = 1;
    }
    return fail;
}
