// C-ABI of liblasp.so: validation, interpolator handle, launches.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lasp.h"
#include "lasp_launch.cuh"
#include "lasp_tc.cuh"

using namespace lasp;

struct lasp_interp_s {
    ModelDev M;              // device table pointer + constants
    int device;
    float* C;                // K x n_model FP32
    float* Cp;               // K x ldc FP32, rows padded to 16 floats
    TcImages tc;             // tensor-core tile images of the table
};

namespace lasp {
int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return LASP_OK;
    if (e == cudaErrorMemoryAllocation) return LASP_ENOMEM;
    return LASP_ECUDA;
}
}  // namespace lasp

namespace {

thread_local int g_last_launches = 0;

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
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, *dev) != cudaSuccess) return LASP_ENODEV;
    if (prop.major != 10 || prop.minor != 3) return LASP_ENODEV;   // built for sm_103a only
    return LASP_OK;
}

int threads_for(int n_pix) { return n_pix <= 16 * 256 ? 256 : 512; }

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
    d.fp64_ne = o->fp64_normal_eq ? 1 : 0;
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
}

int lasp_init_interp(const lasp_interp_desc* d, const float* coeff, lasp_interp* out) {
    if (!d || !coeff || !out) return LASP_EINVAL;
    *out = nullptr;
    if (d->K < 1 || d->K > KMAX || d->n_pix < 16 || d->n_pix > 16 * 512 || d->pad < 0 ||
        d->pad > HMAX || !(d->dln > 0.0) || !d->exps)
        return LASP_EINVAL;
    for (int k = 0; k < 3 * d->K; ++k)
        if (d->exps[k] < 0 || d->exps[k] > 8) return LASP_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!(d->basis_hi[k] > d->basis_lo[k])) return LASP_EINVAL;
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
    M.K = d->K;
    M.n_pix = d->n_pix;
    M.pad = d->pad;
    M.n_model = d->n_pix + 2 * d->pad;
    M.kms_px = (float)kms;
    for (int k = 0; k < 3; ++k) {
        M.blo[k] = (float)d->basis_lo[k];
        M.bscale[k] = (float)(2.0 / (d->basis_hi[k] - d->basis_lo[k]));
    }
    for (int k = 0; k < 5; ++k) {
        M.plo[k] = (float)d->box_lo[k];
        M.phalf[k] = (float)(0.5 * (d->box_hi[k] - d->box_lo[k]));
    }
    std::memset(M.exps, 0, sizeof(M.exps));
    for (int k = 0; k < 3 * d->K; ++k) M.exps[k] = d->exps[k];
    const size_t nC = (size_t)d->K * M.n_model;
    rc = cuda_err(cudaMalloc(&h->C, nC * sizeof(float)));
    if (rc) {
        delete h;
        return rc;
    }
    M.ldc = (M.n_model + 15) & ~15;
    rc = cuda_err(cudaMemcpy(h->C, coeff, nC * sizeof(float), cudaMemcpyHostToDevice));
    if (!rc) rc = cuda_err(cudaMalloc(&h->Cp, (size_t)d->K * M.ldc * sizeof(float)));
    if (!rc) rc = cuda_err(cudaMemset(h->Cp, 0, (size_t)d->K * M.ldc * sizeof(float)));
    if (!rc)
        rc = cuda_err(cudaMemcpy2D(h->Cp, (size_t)M.ldc * sizeof(float), coeff,
                                   (size_t)M.n_model * sizeof(float), (size_t)M.n_model * sizeof(float),
                                   (size_t)d->K, cudaMemcpyHostToDevice));
    if (!rc) rc = tc_build_images(h->tc, h->C, d->K, M.n_model);
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
    if (o->precision != LASP_PREC_FP32) return lasp_tc_fit_batch(h->M, h->tc, b, o, r, stream, &g_last_launches);
    FitParams P;
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
    int e = dispatch_deg(o->legendre_deg, [&](auto dd) {
        constexpr int D = decltype(dd)::value;
        return launch_fit<D>(P, st);
    });
    g_last_launches = e ? 0 : 1;
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
