// C-ABI of liblasp.so: validation, interpolator handle, launches.
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lasp.h"
#include "lasp_clean.cuh"
#include "lasp_launch.cuh"
#include "lasp_prof.cuh"
#include "lasp_tc.cuh"

using namespace lasp;

struct lasp_interp_s {
    ModelDev M;              // device table pointer + constants
    int device;
    float* C;                // K x n_model FP32
    float* Cp;               // K x ldc FP32, rows padded to 16 floats
    TcImages tc;             // tensor-core tile images of the table
};

namespace {

thread_local int g_last_launches = 0;
std::atomic<int> g_test_wait0{-1};      // lasp_test_wait_limit: -1 = normal limits

// lasp_profile: per-kernel launch counts and device milliseconds since the last read
std::atomic<int> g_prof{0};
std::mutex g_prof_mu;
std::vector<lasp_kernel_time> g_prof_tab;

}  // namespace

namespace lasp {
bool prof_on() { return g_prof.load(std::memory_order_relaxed) != 0; }

void prof_add(const char* name, float ms) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (lasp_kernel_time& k : g_prof_tab)
        if (std::strncmp(k.name, name, sizeof(k.name)) == 0) {
            k.launches += 1;
            k.ms += ms;
            return;
        }
    lasp_kernel_time k{};
    std::strncpy(k.name, name, sizeof(k.name) - 1);
    k.launches = 1;
    k.ms = ms;
    g_prof_tab.push_back(k);
}
}  // namespace lasp

namespace lasp {
int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return LASP_OK;
    // The runtime also keeps a failed call as this thread's last error, which
    // the launch checks read with cudaGetLastError: reset it here, so that an
    // error already returned (a failed allocation, say) is not reported again
    // by a later, unrelated launch.  An error that corrupts the context is
    // returned by every later call regardless.
    (void)cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return LASP_ENOMEM;
    return LASP_ECUDA;
}

uint32_t first_wait_limit(uint32_t normal) {
    const int w = g_test_wait0.load(std::memory_order_relaxed);
    return w >= 0 ? (uint32_t)w : normal;
}

void set_last_launches(int n) { g_last_launches = n; }
}  // namespace lasp

namespace {

constexpr double kCkms = 299792.458;

int cuda_err(cudaError_t e) { return lasp::cuda_rc(e); }

bool valid_deg(int D) { return D == 2 || D == 4 || D == 6 || D == 8; }

int check_device(int* dev) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return LASP_ENODEV;
    }
    if (cudaGetDevice(dev) != cudaSuccess) return LASP_ENODEV;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, *dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, *dev) != cudaSuccess)
        return LASP_ENODEV;
    if (major != 10 || minor != 3) return LASP_ENODEV;   // built for sm_103a only
    return LASP_OK;
}

template <typename F>
int dispatch_deg(int D, F&& f) {
    switch (D) {
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 6: return f(std::integral_constant<int, 6>{});
        case 8: return f(std::integral_constant<int, 8>{});
        default: return LASP_EINVAL;
    }
}

int check_opts(const lasp_fit_opts* o, int n_pix) {
    if (!o) return LASP_EINVAL;
    if (!(o->lr > 0.0f) || !(o->beta1 >= 0.0f && o->beta1 < 1.0f) ||
        !(o->beta2 >= 0.0f && o->beta2 < 1.0f) || !(o->eps >= 0.0f) || !(o->tol >= 0.0f))
        return LASP_EINVAL;
    if (o->window < 1 || o->window > WINMAX || o->max_steps < 0 || o->max_steps > 1000000)
        return LASP_EINVAL;
    if (!valid_deg(o->legendre_deg)) return LASP_EINVAL;
    if (o->edge_px < 0 || 2 * o->edge_px >= n_pix) return LASP_EINVAL;
    if (!(o->quantile >= 0.0f && o->quantile <= 1.0f)) return LASP_EINVAL;
    if (o->precision < LASP_PREC_FP32 || o->precision > LASP_PREC_TF32X3) return LASP_EINVAL;
    if (o->fp64_normal_eq < LASP_NE_FP32 || o->fp64_normal_eq > LASP_NE_FP64) return LASP_EINVAL;
    if (o->clean && (o->clean_every < 1 || o->clean_max < 0)) return LASP_EINVAL;
    if (o->optimizer != LASP_OPT_ADAM && o->optimizer != LASP_OPT_LM) return LASP_EINVAL;
    if (o->optimizer == LASP_OPT_LM && (o->precision != LASP_PREC_FP32 || o->clean)) return LASP_EINVAL;
    if (o->loss_mode != LASP_LOSS_SEPARABLE && o->loss_mode != LASP_LOSS_JOINT) return LASP_EINVAL;
    if (o->loss_mode == LASP_LOSS_JOINT &&
        (o->precision == LASP_PREC_FP32 || o->optimizer != LASP_OPT_ADAM || o->clean))
        return LASP_EINVAL;
    return LASP_OK;
}

FitOpts to_dev(const lasp_fit_opts* o) {
    FitOpts d;
    d.lr = o->lr;
    d.beta1 = o->beta1;
    d.beta2 = o->beta2;
    d.eps = o->eps;
    d.tol = o->tol;
    d.window = o->window;
    d.max_steps = o->max_steps;
    d.edge_px = o->edge_px;
    d.quantile = o->quantile;
    d.fp64_ne = o->fp64_normal_eq;
    d.clean = o->clean ? 1 : 0;
    d.clean_every = o->clean_every;
    d.clean_max = o->clean_max;
    d.joint = o->loss_mode == LASP_LOSS_JOINT ? 1 : 0;
    return d;
}

int check_batch(const lasp_interp_s* h, const lasp_batch* b) {
    if (!h || !b || b->N < 0 || b->n_pix != h->M.n_pix) return LASP_EINVAL;
    if (b->N > 0 && (!b->flux || !b->ivar || !b->good || !b->theta0)) return LASP_EINVAL;
    return LASP_OK;
}

}  // namespace

extern "C" {

int lasp_version(void) { return 1; }

int lasp_last_launches(void) { return g_last_launches; }

int lasp_profile(int on) {
    g_prof.store(on ? 1 : 0, std::memory_order_relaxed);
    return LASP_OK;
}

int lasp_profile_read(lasp_kernel_time* out, int max, int* n) {
    if (!n || max < 0 || (max > 0 && !out)) return LASP_EINVAL;
    std::lock_guard<std::mutex> g(g_prof_mu);
    int k = 0;
    for (; k < max && k < (int)g_prof_tab.size(); ++k) out[k] = g_prof_tab[k];
    *n = k;
    g_prof_tab.clear();
    return LASP_OK;
}

int lasp_test_wait_limit(int polls) {
    g_test_wait0.store(polls < 0 ? -1 : polls, std::memory_order_relaxed);
    return LASP_OK;
}

const char* lasp_strerror(int code) {
    switch (code) {
        case LASP_OK: return "ok";
        case LASP_EINVAL: return "invalid argument";
        case LASP_ENOMEM: return "device allocation failed";
        case LASP_ECUDA: return "CUDA runtime error";
        case LASP_ETIMEOUT: return "bounded device wait timed out";
        case LASP_EGRID: return "table padding too small for the parameter box";
        case LASP_ENODEV: return "no sm_103 CUDA device";
        default: return "unknown error";
    }
}

void lasp_default_opts(lasp_fit_opts* o) {
    if (!o) return;
    o->lr = 0.1f;
    o->beta1 = 0.9f;
    o->beta2 = 0.999f;
    o->eps = 1e-8f;
    o->tol = 1e-5f;
    o->window = 50;
    o->max_steps = 5000;
    o->legendre_deg = 6;
    o->edge_px = 0;
    o->quantile = 0.5f;
    o->precision = LASP_PREC_FP32;
    o->fp64_normal_eq = 0;
    o->clean = 0;
    o->clean_every = 30;
    o->clean_max = 11;
    o->optimizer = LASP_OPT_ADAM;
    o->loss_mode = LASP_LOSS_SEPARABLE;
}

int lasp_init_interp_piecewise(const lasp_piecewise_desc* d, const float* coeff, lasp_interp* out) {
    if (!d || !coeff || !out) return LASP_EINVAL;
    *out = nullptr;
    if (d->n_reg < 1 || d->n_reg > NREG || d->n_pix < 16 || d->pad < 0 || d->pad > HMAX ||
        d->n_pix + 2 * d->pad > MODEL_PIX_MAX || !(d->dln > 0.0) || !d->exps)
        return LASP_EINVAL;
    int K = 0;
    for (int r = 0; r < d->n_reg; ++r) {
        if (d->K[r] < 1) return LASP_EINVAL;
        K += d->K[r];
        for (int k = 0; k < 3; ++k)
            if (!(d->basis_hi[r][k] > d->basis_lo[r][k])) return LASP_EINVAL;
    }
    if (K > KROWS || (d->n_reg == 1 && K > KMAX)) return LASP_EINVAL;
    for (int q = 0; q + 1 < 2 * (d->n_reg - 1); ++q)
        if (!(d->teff_blend[q + 1] > d->teff_blend[q])) return LASP_EINVAL;
    for (int k = 0; k < 3 * K; ++k)
        if (d->exps[k] < 0 || d->exps[k] > 8) return LASP_EINVAL;
    for (int k = 0; k < 5; ++k)
        if (!(d->box_hi[k] > d->box_lo[k])) return LASP_EINVAL;
    if (!(d->box_lo[0] > 0.0) || !(d->box_lo[4] > 0.0)) return LASP_EINVAL;
    // the widest kernel reachable in the box must fit in the table margin (Eq. 5)
    const double kms = kCkms * d->dln;
    const double mumax = std::fmax(std::fabs(d->box_lo[3]), std::fabs(d->box_hi[3])) / kms;
    const int hmax = (int)std::ceil(mumax + 5.0 * d->box_hi[4] / kms);
    if (hmax > d->pad) return LASP_EGRID;
    int dev;
    int rc = check_device(&dev);
    if (rc) return rc;

    lasp_interp_s* h = new (std::nothrow) lasp_interp_s();
    if (!h) return LASP_ENOMEM;
    h->device = dev;
    ModelDev& M = h->M;
    M.K = K;
    M.n_pix = d->n_pix;
    M.pad = d->pad;
    M.n_model = d->n_pix + 2 * d->pad;
    M.kms_px = (float)kms;
    M.n_reg = d->n_reg;
    M.reg_row[0] = 0;
    for (int r = 0; r < d->n_reg; ++r) {
        M.reg_row[r + 1] = M.reg_row[r] + d->K[r];
        for (int k = 0; k < 3; ++k) {
            M.rblo[r][k] = (float)d->basis_lo[r][k];
            M.rbscale[r][k] = (float)(2.0 / (d->basis_hi[r][k] - d->basis_lo[r][k]));
        }
    }
    for (int q = 0; q < 2 * (d->n_reg - 1); ++q) M.tb[q] = (float)d->teff_blend[q];
    for (int k = 0; k < 5; ++k) {
        M.plo[k] = (float)d->box_lo[k];
        M.phalf[k] = (float)(0.5 * (d->box_hi[k] - d->box_lo[k]));
    }
    std::memset(M.exps, 0, sizeof(M.exps));
    for (int k = 0; k < 3 * K; ++k) M.exps[k] = d->exps[k];
    const size_t nC = (size_t)K * M.n_model;
    rc = cuda_err(cudaMalloc(&h->C, nC * sizeof(float)));
    if (rc) {
        delete h;
        return rc;
    }
    M.ldc = (M.n_model + 15) & ~15;
    rc = cuda_err(cudaMemcpy(h->C, coeff, nC * sizeof(float), cudaMemcpyHostToDevice));
    if (!rc) rc = cuda_err(cudaMalloc(&h->Cp, (size_t)K * M.ldc * sizeof(float)));
    if (!rc) rc = cuda_err(cudaMemset(h->Cp, 0, (size_t)K * M.ldc * sizeof(float)));
    if (!rc)
        rc = cuda_err(cudaMemcpy2D(h->Cp, (size_t)M.ldc * sizeof(float), coeff,
                                   (size_t)M.n_model * sizeof(float), (size_t)M.n_model * sizeof(float),
                                   (size_t)K, cudaMemcpyHostToDevice));
    // tensor-core tile images: the rows in K blocks of 32 terms (three at most)
    if (!rc) rc = tc_build_images(h->tc, h->C, K, M.n_model);
    // the copies above run on the legacy default stream; finish them before a fit on another stream
    if (!rc) rc = cuda_err(cudaStreamSynchronize(cudaStreamLegacy));
    if (rc) {
        tc_free_images(h->tc);
        cudaFree(h->C);
        cudaFree(h->Cp);
        delete h;
        return rc;
    }
    M.C = h->C;
    M.Cp = h->Cp;
    *out = h;
    return LASP_OK;
}

int lasp_init_interp(const lasp_interp_desc* d, const float* coeff, lasp_interp* out) {
    if (!d || !coeff || !out) return LASP_EINVAL;
    *out = nullptr;
    if (d->K < 1 || d->K > KMAX) return LASP_EINVAL;
    lasp_piecewise_desc pd{};
    pd.n_reg = 1;
    pd.K[0] = d->K;
    pd.n_pix = d->n_pix;
    pd.pad = d->pad;
    pd.dln = d->dln;
    pd.exps = d->exps;
    for (int k = 0; k < 3; ++k) {
        pd.basis_lo[0][k] = d->basis_lo[k];
        pd.basis_hi[0][k] = d->basis_hi[k];
    }
    for (int k = 0; k < 5; ++k) {
        pd.box_lo[k] = d->box_lo[k];
        pd.box_hi[k] = d->box_hi[k];
    }
    return lasp_init_interp_piecewise(&pd, coeff, out);
}

void lasp_free_interp(lasp_interp h) {
    if (!h) return;
    tc_free_images(h->tc);
    cudaFree(h->C);
    cudaFree(h->Cp);
    delete h;
}

int lasp_fit_batch(lasp_interp h, const lasp_batch* b, const lasp_fit_opts* o, lasp_result* r,
                   void* stream) {
    g_last_launches = 0;
    int rc = check_batch(h, b);
    if (rc) return rc;
    rc = check_opts(o, b->n_pix);
    if (rc) return rc;
    if (!r || (b->N > 0 && (!r->theta || !r->loss || !r->steps || !r->status))) return LASP_EINVAL;
    if (b->N == 0) return LASP_OK;
    if (o->precision != LASP_PREC_FP32) {
        return lasp_tc_fit_batch(h->M, h->tc, b, o, r, stream, &g_last_launches);
    }
    if (o->optimizer == LASP_OPT_LM) {
        LmParams L{};
        L.M = h->M;
        L.O = to_dev(o);
        L.N = b->N;
        L.max_iter = o->max_steps;
        L.rtol = o->tol;
        L.flux = b->flux;
        L.ivar = b->ivar;
        L.good = b->good;
        L.theta0 = b->theta0;
        L.theta = r->theta;
        L.loss = r->loss;
        L.steps = r->steps;
        L.status = r->status;
        L.weight = r->weight;
        L.cont = r->cont_coeff;
        cudaStream_t st = (cudaStream_t)stream;
        int e = dispatch_deg(o->legendre_deg, [&](auto dd) {
            constexpr int D = decltype(dd)::value;
            return launch_lm<D>(L, st);
        });
        g_last_launches = e ? 0 : 1;
        return e;
    }
    FitParams P{};
    P.M = h->M;
    P.O = to_dev(o);
    P.N = b->N;
    P.flux = b->flux;
    P.ivar = b->ivar;
    P.good = b->good;
    P.theta0 = b->theta0;
    P.theta = r->theta;
    P.loss = r->loss;
    P.steps = r->steps;
    P.status = r->status;
    P.cont = r->cont_coeff;
    P.weight = r->weight;
    cudaStream_t st = (cudaStream_t)stream;
    // several spectra per CTA (the same result as fit_kernel, bit for bit)
    int nl = 0;
    int e = dispatch_deg(o->legendre_deg, [&](auto dd) {
        constexpr int D = decltype(dd)::value;
        return launch_fit_multi<D>(P, st, &nl);
    });
    g_last_launches = e ? 0 : nl;
    return e;
}

int lasp_errors(lasp_interp h, const lasp_batch* b, const lasp_fit_opts* o, const float* theta,
                float* sigma, double* cov, uint32_t* status, void* stream) {
    g_last_launches = 0;
    int rc = check_batch(h, b);
    if (rc) return rc;
    rc = check_opts(o, b->n_pix);
    if (rc) return rc;
    if (b->N > 0 && (!theta || !sigma)) return LASP_EINVAL;
    if (b->N == 0) return LASP_OK;
    ErrParams P;
    P.M = h->M;
    P.O = to_dev(o);
    P.N = b->N;
    P.flux = b->flux;
    P.ivar = b->ivar;
    P.good = b->good;
    P.theta = theta;
    P.sigma = sigma;
    P.cov = cov;
    P.status = status;
    cudaStream_t st = (cudaStream_t)stream;
    int e = dispatch_deg(o->legendre_deg, [&](auto dd) {
        constexpr int D = decltype(dd)::value;
        return launch_errors<D>(P, st);
    });
    g_last_launches = e ? 0 : 1;
    return e;
}

int lasp_forward(lasp_interp h, int N, const float* theta, const float* b, int deg, float* model,
                 void* stream) {
    g_last_launches = 0;
    if (!h || N < 0 || !valid_deg(deg)) return LASP_EINVAL;
    if (N == 0) return LASP_OK;
    if (!theta || !b || !model) return LASP_EINVAL;
    ModelParams P{};
    P.M = h->M;
    P.N = N;
    P.D = deg;
    P.theta = theta;
    P.b = b;
    P.model = model;
    cudaStream_t st = (cudaStream_t)stream;
    int e = dispatch_deg(deg, [&](auto dd) {
        constexpr int D = decltype(dd)::value;
        return launch_forward<D>(P, st);
    });
    g_last_launches = e ? 0 : 1;
    return e;
}

int lasp_backward(lasp_interp h, int N, const float* theta, const float* b, int deg,
                  const float* gmodel, float* gtheta, float* gb, void* stream) {
    g_last_launches = 0;
    if (!h || N < 0 || !valid_deg(deg)) return LASP_EINVAL;
    if (N == 0) return LASP_OK;
    if (!theta || !b || !gmodel || !gtheta || !gb) return LASP_EINVAL;
    ModelParams P{};
    P.M = h->M;
    P.N = N;
    P.D = deg;
    P.theta = theta;
    P.b = b;
    P.gmodel = gmodel;
    P.gtheta = gtheta;
    P.gb = gb;
    cudaStream_t st = (cudaStream_t)stream;
    int e = dispatch_deg(deg, [&](auto dd) {
        constexpr int D = decltype(dd)::value;
        return launch_backward<D>(P, st);
    });
    g_last_launches = e ? 0 : 1;
    return e;
}

int lasp_interp_eval(lasp_interp h, int N, const float* theta, float* Fp, int precision,
                     void* stream) {
    g_last_launches = 0;
    if (!h || N < 0 || precision < LASP_PREC_FP32 || precision > LASP_PREC_TF32X3) return LASP_EINVAL;
    if (N == 0) return LASP_OK;
    if (!theta || !Fp) return LASP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision != LASP_PREC_FP32)
        return lasp_tc_interp_eval(h->M, h->tc, N, theta, Fp, precision, st, &g_last_launches);
    dim3 grid(N, (h->M.n_model + 255) / 256);
    interp_fp32_kernel<256><<<grid, 256, 0, st>>>(h->M, theta, Fp);
    g_last_launches = 1;
    return cuda_err(cudaGetLastError());
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Resumable fit slots (continuous batching).

namespace {

__global__ void slots_scatter_kernel(int count, int n_pix, const int32_t* __restrict__ idx,
                                     const float* __restrict__ f_st, const float* __restrict__ iv_st,
                                     const uint8_t* __restrict__ g_st, const float* __restrict__ th_st,
                                     float* flux, float* ivar, uint8_t* good, float* theta0, int* t,
                                     uint32_t* status) {
    const int r = blockIdx.x;
    if (r >= count) return;
    const int slot = idx[r];
    const size_t src = (size_t)r * n_pix, dst = (size_t)slot * n_pix;
    for (int j = threadIdx.x; j < n_pix; j += blockDim.x) {
        flux[dst + j] = f_st[src + j];
        ivar[dst + j] = iv_st[src + j];
        good[dst + j] = g_st[src + j];
    }
    if (threadIdx.x < 5) theta0[5 * slot + threadIdx.x] = th_st[5 * r + threadIdx.x];
    if (threadIdx.x == 0) {
        t[slot] = -1;
        status[slot] = LASP_ST_RUNNING;
    }
}

}  // namespace

struct lasp_slots_s {
    lasp_interp h;
    int n;
    lasp_fit_opts opts;
    float *flux, *ivar, *theta0;
    uint8_t* good;
    float *f_st, *iv_st, *th_st;
    uint8_t* g_st;
    int32_t* idx_st;
    lasp::SlotState S;
    float *theta, *loss, *cont, *weight;
    int32_t* steps;
    uint32_t* status;
    lasp::GrpPool* grp = nullptr;   // tensor-core precisions: the grouped pipeline over the slots
    // FP32 pools on fit_multi_kernel: y, W rows of 2 ldw floats per slot (Clean
    // masks included) and the lanes' slot counter; otherwise fit_kernel
    bool multi = false;
    int ldw = 0;
    float* yw = nullptr;
    int* ctr = nullptr;
    int* list = nullptr;             // the running slots of a step
};

namespace {

lasp::FitParams slot_params(const lasp_slots_s* s) {
    lasp::FitParams P{};
    P.M = s->h->M;
    P.O = to_dev(&s->opts);
    P.N = s->n;
    P.S = s->S;
    P.flux = s->flux;
    P.ivar = s->ivar;
    P.good = s->good;
    P.theta0 = s->theta0;
    P.theta = s->theta;
    P.loss = s->loss;
    P.steps = s->steps;
    P.status = s->status;
    P.cont = s->cont;
    P.weight = s->weight;
    return P;
}

lasp::MultiWs slot_ws(const lasp_slots_s* s) {
    lasp::MultiWs W{};
    W.yw = s->yw;
    W.ldw = s->ldw;
    W.next = s->ctr;
    W.list = s->list;
    return W;
}

}  // namespace

namespace lasp {
int slots_n_pix(lasp_slots s) { return s ? s->h->M.n_pix : 0; }
}  // namespace lasp


extern "C" {

void lasp_slots_free(lasp_slots s) {
    if (!s) return;
    if (s->grp) grp_pool_free(s->grp);
    void* ptrs[] = {s->flux, s->ivar, s->theta0, s->good, s->f_st, s->iv_st, s->th_st, s->g_st,
                    s->idx_st, s->S.x, s->S.m, s->S.v, s->S.ring, s->S.prev, s->S.rise, s->S.t, s->S.b12,
                    s->S.w, s->S.imean, s->S.cmask, s->theta, s->loss, s->cont, s->weight, s->steps,
                    s->status, s->yw, s->ctr, s->list};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete s;
}

int lasp_slots_create(lasp_interp h, int n_slots, const lasp_fit_opts* o, lasp_slots* out) {
    if (!h || !out || n_slots < 1) return LASP_EINVAL;
    *out = nullptr;
    int rc = check_opts(o, h->M.n_pix);
    if (rc) return rc;
    if (o->loss_mode != LASP_LOSS_SEPARABLE) return LASP_EINVAL;
    if (o->precision != LASP_PREC_FP32 && o->legendre_deg != 6)
        return LASP_EINVAL;
    lasp_slots_s* s = new (std::nothrow) lasp_slots_s();
    if (!s) return LASP_ENOMEM;
    s->h = h;
    s->n = n_slots;
    s->opts = *o;
    const size_t n = (size_t)n_slots, p = (size_t)h->M.n_pix, NB = (size_t)o->legendre_deg + 1;
    auto alloc = [&](auto** ptr, size_t bytes) {
        if (rc) return;
        rc = cuda_err(cudaMalloc((void**)ptr, bytes));
        if (!rc) rc = cuda_err(cudaMemset(*ptr, 0, bytes));
    };
    alloc(&s->flux, n * p * 4);
    alloc(&s->ivar, n * p * 4);
    alloc(&s->good, n * p);
    alloc(&s->theta0, n * 5 * 4);
    alloc(&s->f_st, n * p * 4);
    alloc(&s->iv_st, n * p * 4);
    alloc(&s->g_st, n * p);
    alloc(&s->th_st, n * 5 * 4);
    alloc(&s->idx_st, n * 4);
    alloc(&s->S.x, n * 5 * 4);
    alloc(&s->S.m, n * 5 * 4);
    alloc(&s->S.v, n * 5 * 4);
    alloc(&s->S.ring, n * WINMAX * 4);
    alloc(&s->S.prev, n * 4);
    alloc(&s->S.rise, n * 4);
    alloc(&s->S.t, n * 4);
    alloc(&s->S.b12, n * 2 * 8);
    alloc(&s->S.w, n * 4);
    alloc(&s->S.imean, n * 4);
    const lasp::ModelDev& M = h->M;
    s->multi = o->precision == LASP_PREC_FP32 &&
               fit_multi_slots_ok(M.n_pix, M.pad, M.n_model, M.K, o->legendre_deg);
    if (s->multi) {
        s->ldw = (int)((p + 15) & ~(size_t)15);
        alloc(&s->yw, n * 2 * (size_t)s->ldw * 4);
        alloc(&s->ctr, 256);
        alloc(&s->list, n * 4);
    } else if (o->clean) {
        alloc(&s->S.cmask, n * (size_t)((p + 15) / 16) * 2);
    }
    alloc(&s->theta, n * 5 * 4);
    alloc(&s->loss, n * 4);
    alloc(&s->cont, n * NB * 4);
    alloc(&s->weight, n * 4);
    alloc(&s->steps, n * 4);
    alloc(&s->status, n * 4);
    if (!rc && o->precision != LASP_PREC_FP32)
        rc = grp_pool_create(h->M, h->tc, n_slots, o, s->flux, s->ivar, s->good, s->theta0, s->theta, s->loss,
                             s->steps, s->status, s->cont, s->weight, &s->grp);
    // the zero fills above are queued on the legacy default stream, which a caller's non-blocking
    // stream does not wait for: finish them before the pool can be admitted into
    if (!rc) rc = cuda_err(cudaStreamSynchronize(cudaStreamLegacy));
    if (rc) {
        lasp_slots_free(s);
        return rc;
    }
    *out = s;
    return LASP_OK;
}

int lasp_slots_admit(lasp_slots s, int count, const int32_t* slot_idx, const float* flux,
                     const float* ivar, const uint8_t* good, const float* theta0, void* stream) {
    g_last_launches = 0;
    if (!s || count < 0 || count > s->n) return LASP_EINVAL;
    if (count == 0) return LASP_OK;
    if (!slot_idx || !flux || !ivar || !good || !theta0) return LASP_EINVAL;
    for (int r = 0; r < count; ++r)
        if (slot_idx[r] < 0 || slot_idx[r] >= s->n) return LASP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t p = (size_t)s->h->M.n_pix, c = (size_t)count;
    int rc = prof_time("slots_admit_h2d", st, [&] {
        int r = cuda_err(cudaMemcpyAsync(s->f_st, flux, c * p * 4, cudaMemcpyHostToDevice, st));
        if (!r) r = cuda_err(cudaMemcpyAsync(s->iv_st, ivar, c * p * 4, cudaMemcpyHostToDevice, st));
        if (!r) r = cuda_err(cudaMemcpyAsync(s->g_st, good, c * p, cudaMemcpyHostToDevice, st));
        if (!r) r = cuda_err(cudaMemcpyAsync(s->th_st, theta0, c * 5 * 4, cudaMemcpyHostToDevice, st));
        if (!r) r = cuda_err(cudaMemcpyAsync(s->idx_st, slot_idx, c * 4, cudaMemcpyHostToDevice, st));
        return r;
    });
    if (rc) return rc;
    rc = prof_time("slots_scatter_kernel", st, [&] {
        slots_scatter_kernel<<<count, 256, 0, st>>>(count, (int)p, s->idx_st, s->f_st, s->iv_st, s->g_st,
                                                     s->th_st, s->flux, s->ivar, s->good, s->theta0, s->S.t,
                                                     s->status);
        return cuda_err(cudaGetLastError());
    });
    g_last_launches = 1;
    if (!rc && s->grp) {
        rc = grp_pool_admit(s->grp, count, s->idx_st, st);     // prep + join the active list
        g_last_launches = 2;
    }
    if (!rc && s->multi) {
        const FitParams P = slot_params(s);
        const MultiWs W = slot_ws(s);
        rc = dispatch_deg(s->opts.legendre_deg, [&](auto dd) {
            constexpr int D = decltype(dd)::value;
            return launch_fit_prep_slots<D>(P, W, s->idx_st, count, st);
        });
        g_last_launches = 2;
    }
    return rc;
}

int lasp_slots_step(lasp_slots s, int budget, void* stream) {
    return lasp_slots_step_running(s, budget, s ? s->n : 1, stream);
}

int lasp_slots_step_running(lasp_slots s, int budget, int n_running, void* stream) {
    g_last_launches = 0;
    if (!s || budget < 1 || n_running < 1) return LASP_EINVAL;
    if (s->grp) return grp_pool_step(s->grp, budget, (cudaStream_t)stream, &g_last_launches);
    FitParams P = slot_params(s);
    P.S.budget = budget;
    const MultiWs W = slot_ws(s);
    cudaStream_t st = (cudaStream_t)stream;
    int e = dispatch_deg(s->opts.legendre_deg, [&](auto dd) {
        constexpr int D = decltype(dd)::value;
        return s->multi ? launch_fit_multi_slots<D>(P, W, n_running, st) : launch_fit<D>(P, st);
    });
    g_last_launches = e ? 0 : 1;
    return e;
}

int lasp_slots_fetch(lasp_slots s, float* theta, float* loss, int32_t* steps, uint32_t* status,
                     float* weight, void* stream) {
    if (!s) return LASP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)s->n;
    return prof_time("slots_fetch_d2h", st, [&] {
        int rc = LASP_OK;
        if (!rc && theta) rc = cuda_err(cudaMemcpyAsync(theta, s->theta, n * 5 * 4, cudaMemcpyDeviceToHost, st));
        if (!rc && loss) rc = cuda_err(cudaMemcpyAsync(loss, s->loss, n * 4, cudaMemcpyDeviceToHost, st));
        if (!rc && steps) rc = cuda_err(cudaMemcpyAsync(steps, s->steps, n * 4, cudaMemcpyDeviceToHost, st));
        if (!rc && status) rc = cuda_err(cudaMemcpyAsync(status, s->status, n * 4, cudaMemcpyDeviceToHost, st));
        if (!rc && weight) rc = cuda_err(cudaMemcpyAsync(weight, s->weight, n * 4, cudaMemcpyDeviceToHost, st));
        return rc;
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Flux-conserving resampling (stage 3, Eqs. 2-4) as exact overlap integrals.

namespace {

__global__ void resample_kernel(int K, int q, double lam1, double dlam, const float* __restrict__ in,
                                int n_out, double ln0, double dln, float* __restrict__ out) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)K * n_out) return;
    const int k = (int)(idx / n_out), i = (int)(idx % n_out);
    const double a = exp(ln0 + (i - 0.5) * dln), b = exp(ln0 + (i + 0.5) * dln);
    const double e0 = lam1 - 0.5 * dlam;
    long ka = (long)floor((a - e0) / dlam), kb = (long)floor((b - e0) / dlam);
    if (ka < 0) ka = 0;
    if (kb > q - 1) kb = q - 1;
    double acc = 0.0;
    const float* row = in + (size_t)k * q;
    for (long m = ka; m <= kb; ++m) {
        const double lo = fmax(a, e0 + m * dlam), hi = fmin(b, e0 + (m + 1) * dlam);
        if (hi > lo) acc += (double)row[m] * (hi - lo);
    }
    out[(size_t)k * n_out + i] = (float)(acc / (b - a));
}

}  // namespace

extern "C" int lasp_resample_linear(int K, int q, double lam1, double dlam, const float* coeff_lin,
                                    int n_out, double ln_lam0, double dln, float* coeff_out,
                                    void* stream) {
    g_last_launches = 0;
    if (K < 1 || q < 1 || n_out < 0 || !(dlam > 0.0) || !(dln > 0.0) || !(lam1 > 0.0)) return LASP_EINVAL;
    if (n_out == 0) return LASP_OK;
    if (!coeff_lin || !coeff_out) return LASP_EINVAL;
    const long total = (long)K * n_out;
    resample_kernel<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        K, q, lam1, dlam, coeff_lin, n_out, ln_lam0, dln, coeff_out);
    g_last_launches = 1;
    return cuda_err(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Clean mask of N spectra (stage 6, Eq. 8), one CTA per spectrum.

namespace {

template <int NT>
__global__ void __launch_bounds__(NT) clean_mask_kernel(int p, const float* __restrict__ r,
                                                        const float* __restrict__ m,
                                                        const uint8_t* __restrict__ used, float fshift,
                                                        uint8_t* keep, int32_t* k_used) {
    extern __shared__ __align__(16) float sm[];
    const int i = blockIdx.x, tid = threadIdx.x;
    float* Rs = sm;
    float* Ms = sm + skew_size(p + 32);
    double* redd = reinterpret_cast<double*>(Ms + skew_size(p + 32));
    double* tot = redd + 3 * (NT / 32);
    __shared__ int s_k;
    const size_t row = (size_t)i * p;
    const int j0 = tid * PPT;
    uint32_t ub = 0;
    for (int q = 0; q < PPT; ++q) {
        const int j = j0 + q;
        if (j < p) {
            Rs[skew(j + 16)] = r[row + j];
            Ms[skew(j + 16)] = m[row + j];
            if (used[row + j]) ub |= 1u << q;
        }
    }
    __syncthreads();
    const uint32_t kb = cta_clean_mask<NT, PPT>(p, j0, Rs, 16, Ms, 16, ub, fshift,
                                                reinterpret_cast<uint8_t*>(Ms), redd, tot, &s_k);
    for (int q = 0; q < PPT; ++q) {
        const int j = j0 + q;
        if (j < p) keep[row + j] = (kb >> q) & 1u;
    }
    if (tid == 0 && k_used) k_used[i] = s_k;
}

}  // namespace

extern "C" int lasp_clean_mask(int N, int p, const float* r, const float* m, const uint8_t* used,
                               float fshift, uint8_t* keep, int32_t* k_used, void* stream) {
    g_last_launches = 0;
    if (N < 0 || p < 1 || p > 16 * 512) return LASP_EINVAL;
    if (N == 0) return LASP_OK;
    if (!r || !m || !used || !keep) return LASP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t smem = 4 * (2 * (size_t)skew_size(p + 32)) + 8 * (3 * 16 + 4);
    int e;
    if (p <= 16 * 256) {
        e = cuda_err(cudaFuncSetAttribute(clean_mask_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        clean_mask_kernel<256><<<N, 256, smem, st>>>(p, r, m, used, fshift, keep, k_used);
    } else {
        e = cuda_err(cudaFuncSetAttribute(clean_mask_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        clean_mask_kernel<512><<<N, 512, smem, st>>>(p, r, m, used, fshift, keep, k_used);
    }
    g_last_launches = 1;
    return cuda_err(cudaGetLastError());
}
