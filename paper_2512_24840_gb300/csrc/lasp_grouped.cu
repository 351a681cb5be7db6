// Entry points of the grouped tensor-core fit (lasp_grouped.cuh): the
// one-shot batch fit (lasp_tc_fit_batch), which dispatches on the Legendre
// degree, and the persistent pools of served fits (degree 6).
#include "lasp_grouped.cuh"

namespace lasp {

extern template int grp_run_deg<2>(Grp&, const TcImages&, const lasp_fit_opts*, cudaStream_t, int*);
extern template int grp_run_deg<4>(Grp&, const TcImages&, const lasp_fit_opts*, cudaStream_t, int*);
extern template int grp_run_deg<8>(Grp&, const TcImages&, const lasp_fit_opts*, cudaStream_t, int*);

int lasp_tc_fit_batch(const ModelDev& M, const TcImages& tc, const lasp_batch* b, const lasp_fit_opts* o,
                      lasp_result* r, void* stream, int* launches) {
    *launches = 0;
    if (!tc.tf32_hi || !tc.bk_hi) return LASP_EINVAL;
    // FP64 normal equations are compiled into the split-TF32 step body only
    if (o->fp64_normal_eq == LASP_NE_FP64 && o->precision != LASP_PREC_TF32X3) return LASP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Grp G{};
    G.M = M;
    G.O.lr = o->lr;
    G.O.beta1 = o->beta1;
    G.O.beta2 = o->beta2;
    G.O.eps = o->eps;
    G.O.tol = o->tol;
    G.O.window = o->window;
    G.O.max_steps = o->max_steps;
    G.O.edge_px = o->edge_px;
    G.O.quantile = o->quantile;
    G.O.fp64_ne = o->fp64_normal_eq;
    G.O.joint = o->loss_mode == LASP_LOSS_JOINT ? 1 : 0;
    G.O.clean = o->clean ? 1 : 0;
    G.O.clean_every = o->clean_every;
    G.O.clean_max = o->clean_max;
    const int N = b->N;
    const int NB = o->legendre_deg + 1;
    G.N = N;
    G.NB = NB;
    G.ldf = (M.n_model + 15) & ~15;
    G.ldp = (M.n_pix + 15) & ~15;
    G.nch = o->precision == LASP_PREC_BF16 ? tc.n_chunks_bf16 : tc.n_chunks_tf32;
    G.nblk = (N + 127) / 128;
    G.n_kb = tc.n_kb;
    G.kp = 32 * tc.n_kb;
    G.flux = b->flux;
    G.ivar = b->ivar;
    G.good = b->good;
    G.theta0 = b->theta0;
    G.theta = r->theta;
    G.loss_out = r->loss;
    G.steps = r->steps;
    G.status = r->status;
    G.cont = r->cont_coeff;
    G.weight = r->weight;
    G.wait0 = first_wait_limit(kWait);
    const size_t n = (size_t)N;
    int e = LASP_OK;
    auto A = [&](auto** ptr, size_t bytes) {
        if (!e) e = amalloc(ptr, bytes, st);
    };
    A(&G.x, n * 20); A(&G.m, n * 20); A(&G.v, n * 20); A(&G.ring, n * WINMAX * 4);
    A(&G.prev, n * 4); A(&G.w, n * 4); A(&G.imean, n * 4); A(&G.loss, n * 4); A(&G.gmu, n * 4);
    A(&G.gsg, n * 4); A(&G.b, n * NB * 4); A(&G.rise, n * 4); A(&G.t, n * 4); A(&G.flags, n * 4);
    A(&G.list[0], n * 4); A(&G.list[1], n * 4); A(&G.count, 16);
    A(&G.Fp, n * G.ldf * 4);
    A(&G.taps, n * 3 * TAPBUF * 4);
    A(&G.hh, n * 4);
    if (o->loss_mode == LASP_LOSS_JOINT) {
        A(&G.Sstep, n * 4);
        A(&G.act, n * 4);
        A(&G.gs, sizeof(GroupState));
        if (!e) e = cuda_rc(cudaMemsetAsync(G.act, 0xff, n * 4, st));
        if (!e) e = cuda_rc(cudaMemsetAsync(G.gs, 0, sizeof(GroupState), st));
    }
    float2* bct = nullptr;
    A(&bct, ((size_t)o->max_steps + 2) * sizeof(float2));
    if (!e) {
        // bias corrections per step, in double as PyTorch's Adam takes them
        std::vector<float2> hb((size_t)o->max_steps + 2);
        for (size_t t = 0; t < hb.size(); ++t) {
            const double b1t = std::pow((double)o->beta1, (double)t), b2t = std::pow((double)o->beta2, (double)t);
            hb[t] = make_float2(t ? (float)((double)o->lr / (1.0 - b1t)) : 0.0f, t ? (float)std::sqrt(1.0 - b2t) : 1.0f);
        }
        e = cuda_rc(cudaMemcpyAsync(bct, hb.data(), hb.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
        if (!e) e = cuda_rc(cudaStreamSynchronize(st));
    }
    G.bct = bct;
    A(&G.Y, n * G.ldp * 4);
    A(&G.Wt, n * G.ldp * 4);
    A(&G.A_hi, (size_t)G.nblk * G.nch * TC_TILE_BYTES);
    if (o->precision == LASP_PREC_TF32X3) A(&G.A_lo, (size_t)G.nblk * G.nch * TC_TILE_BYTES);
    A(&G.dphi, (size_t)KSPLIT * G.nblk * 128 * G.kp * 4);
    if (!e) e = cuda_rc(cudaMemsetAsync(G.count, 0, 16, st));
    G.err = G.count + 2;
    if (!e) {
        switch (o->legendre_deg) {
            case 2: e = grp_run_deg<2>(G, tc, o, st, launches); break;
            case 4: e = grp_run_deg<4>(G, tc, o, st, launches); break;
            case 6: e = grp_run_deg<6>(G, tc, o, st, launches); break;
            case 8: e = grp_run_deg<8>(G, tc, o, st, launches); break;
            default: e = LASP_EINVAL;
        }
    }
    void* ptrs[] = {G.x, G.m, G.v, G.ring, G.prev, G.w, G.imean, G.loss, G.gmu, G.gsg, G.b, G.rise,
                    G.t, G.flags, G.list[0], G.list[1], G.count, G.Fp, G.Y, G.Wt, G.A_hi, G.A_lo, G.dphi,
                    G.taps, G.hh, bct, G.Sstep, G.act, G.gs};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, st);
    return e;
}

// ---------------------------------------------------------------------------
// Persistent grouped pipeline over slots (served mixed precision).  The state
// of every slot lives in the Grp arrays; admission preps the admitted slots
// and appends them to the active list of parity 0; a step replays the captured
// graph of CHUNK_STEPS steps (so a chunk is rounded up to a multiple of it),
// after which the parity is 0 again.  K4 writes each finished fit's results
// into the slot outputs.

struct GrpPool {
    Grp G{};
    TcImages tc{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float2* bct = nullptr;
    int (*admit)(GrpPool*, int, const int32_t*, cudaStream_t) = nullptr;
};

namespace {

template <int D, int PREC, int NT>
int pool_setup(GrpPool* P) {
    Grp& G = P->G;
    const ModelDev& M = G.M;
    const TcImages& tc = P->tc;
    const int N = G.N;
    const int pa = (M.n_pix + 3) & ~3;
    const size_t smem0 = 4 * ((size_t)3 * pa + PREP_RED);
    const size_t smem1 = 4 * (size_t)G.n_kb * TC_TILE_BYTES + 1024;
    const size_t smem3 = k3_smem_bytes(G.n_kb);
    const RestSmem RS(M.n_pix, M.pad, M.n_model, NT, D);
    const size_t smem2 = 4 * (size_t)RS.total;
    int e = cuda_rc(cudaFuncSetAttribute(k0_prep<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0));
    if (!e) e = cuda_rc(cudaFuncSetAttribute(k1_interp<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
    if (!e) e = cuda_rc(cudaFuncSetAttribute(k2_rest<NT, D, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    if (!e) e = cuda_rc(cudaFuncSetAttribute(k3_back<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3));
    if (!e && G.O.clean)
        e = cuda_rc(cudaFuncSetAttribute(kc_clean<NT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    if (e) return e;
    P->admit = [](GrpPool* Q, int count, const int32_t* idx, cudaStream_t st) -> int {
        const int pq = (Q->G.M.n_pix + 3) & ~3;
        const size_t sm0 = 4 * ((size_t)3 * pq + PREP_RED);
        k0_prep<NT><<<count, NT, sm0, st>>>(Q->G, idx);
        return cuda_rc(cudaGetLastError());
    };
    const uint8_t* img = (const uint8_t*)(PREC == 2 ? tc.bf16 : tc.tf32_hi);
    const uint8_t* img_lo = (const uint8_t*)tc.tf32_lo;
    const uint8_t* bk = (const uint8_t*)(PREC == 2 ? tc.bk_bf : tc.bk_hi);
    const uint8_t* bk_lo = (const uint8_t*)tc.bk_lo;
    const dim3 g1((N + 127) / 128, (tc.n_tiles + 3) / 4);
    const dim3 g3((N + 127) / 128, KSPLIT);
    const int g4 = (N + 7) / 8;
    cudaStream_t cap;
    if ((e = cuda_rc(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)))) return e;
    e = cuda_rc(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    if (!e) {
        for (int k = 0; k < CHUNK_STEPS; ++k) {
            const int par = k & 1;
            k1_interp<PREC><<<g1, 128, smem1, cap>>>(G, par, img, img_lo, tc.n_tiles);
            k2_rest<NT, D, PREC><<<N, NT, smem2, cap>>>(G, par);
            k3_back<PREC><<<g3, 128, smem3, cap>>>(G, par, bk, bk_lo);
            if (G.O.clean) kc_clean<NT, D><<<N, NT, smem2, cap>>>(G, par);
            k4_adam<D><<<g4, 256, 0, cap>>>(G, par);
        }
        e = cuda_rc(cudaStreamEndCapture(cap, &P->graph));
    }
    if (!e) e = cuda_rc(cudaGraphInstantiate(&P->exec, P->graph, 0));
    cudaStreamDestroy(cap);
    return e;
}

}  // namespace

void grp_pool_free(GrpPool* P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    Grp& G = P->G;
    void* ptrs[] = {G.x, G.m, G.v, G.ring, G.prev, G.w, G.imean, G.loss, G.gmu, G.gsg, G.b, G.rise,
                    G.t, G.flags, G.list[0], G.list[1], G.count, G.Fp, G.Y, G.Wt, G.A_hi, G.A_lo, G.dphi,
                    G.taps, G.hh, P->bct};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete P;
}

int grp_pool_create(const ModelDev& M, const TcImages& tc, int n, const lasp_fit_opts* o, float* flux,
                    float* ivar, uint8_t* good, float* theta0, float* theta, float* loss, int32_t* steps,
                    uint32_t* status, float* cont, float* weight, GrpPool** out) {
    *out = nullptr;
    // served tensor-core pools: float-float or FP32 normal equations
    if (!tc.tf32_hi || !tc.bk_hi || o->legendre_deg != 6 || o->fp64_normal_eq == LASP_NE_FP64) return LASP_EINVAL;
    GrpPool* P = new (std::nothrow) GrpPool();
    if (!P) return LASP_ENOMEM;
    P->tc = tc;
    Grp& G = P->G;
    G.M = M;
    G.O.lr = o->lr;
    G.O.beta1 = o->beta1;
    G.O.beta2 = o->beta2;
    G.O.eps = o->eps;
    G.O.tol = o->tol;
    G.O.window = o->window;
    G.O.max_steps = o->max_steps;
    G.O.edge_px = o->edge_px;
    G.O.quantile = o->quantile;
    G.O.fp64_ne = o->fp64_normal_eq;
    G.O.clean = o->clean ? 1 : 0;
    G.O.clean_every = o->clean_every;
    G.O.clean_max = o->clean_max;
    G.N = n;
    G.NB = o->legendre_deg + 1;
    G.ldf = (M.n_model + 15) & ~15;
    G.ldp = (M.n_pix + 15) & ~15;
    G.nch = o->precision == LASP_PREC_BF16 ? tc.n_chunks_bf16 : tc.n_chunks_tf32;
    G.nblk = (n + 127) / 128;
    G.n_kb = tc.n_kb;
    G.kp = 32 * tc.n_kb;
    G.flux = flux;
    G.ivar = ivar;
    G.good = good;
    G.theta0 = theta0;
    G.theta = theta;
    G.loss_out = loss;
    G.steps = steps;
    G.status = status;
    G.cont = cont;
    G.weight = weight;
    G.wait0 = first_wait_limit(kWait);
    const size_t N = (size_t)n;
    int e = LASP_OK;
    auto A = [&](auto** ptr, size_t bytes) {
        if (!e) e = cuda_rc(cudaMalloc((void**)ptr, bytes));
        if (!e) e = cuda_rc(cudaMemset(*ptr, 0, bytes));
    };
    A(&G.x, N * 20); A(&G.m, N * 20); A(&G.v, N * 20); A(&G.ring, N * WINMAX * 4);
    A(&G.prev, N * 4); A(&G.w, N * 4); A(&G.imean, N * 4); A(&G.loss, N * 4); A(&G.gmu, N * 4);
    A(&G.gsg, N * 4); A(&G.b, N * G.NB * 4); A(&G.rise, N * 4); A(&G.t, N * 4); A(&G.flags, N * 4);
    A(&G.list[0], N * 4); A(&G.list[1], N * 4); A(&G.count, 16);
    G.err = G.count + 2;
    A(&G.Fp, N * G.ldf * 4);
    A(&G.Y, N * G.ldp * 4);
    A(&G.Wt, N * G.ldp * 4);
    A(&G.taps, N * 3 * TAPBUF * 4);
    A(&G.hh, N * 4);
    A(&G.A_hi, (size_t)G.nblk * G.nch * TC_TILE_BYTES);
    if (o->precision == LASP_PREC_TF32X3) A(&G.A_lo, (size_t)G.nblk * G.nch * TC_TILE_BYTES);
    A(&G.dphi, (size_t)KSPLIT * G.nblk * 128 * G.kp * 4);
    A(&P->bct, ((size_t)o->max_steps + 2) * sizeof(float2));
    if (!e) {
        std::vector<float2> hb((size_t)o->max_steps + 2);
        for (size_t t = 0; t < hb.size(); ++t) {
            const double b1t = std::pow((double)o->beta1, (double)t), b2t = std::pow((double)o->beta2, (double)t);
            hb[t] = make_float2(t ? (float)((double)o->lr / (1.0 - b1t)) : 0.0f, t ? (float)std::sqrt(1.0 - b2t) : 1.0f);
        }
        e = cuda_rc(cudaMemcpy(P->bct, hb.data(), hb.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
    G.bct = P->bct;
    if (!e) {
        const int NT = fit_threads(M.n_model);
        if (NT == 256) {
            e = o->precision == LASP_PREC_TF32   ? pool_setup<6, 1, 256>(P)
                : o->precision == LASP_PREC_BF16 ? pool_setup<6, 2, 256>(P)
                                                 : pool_setup<6, 3, 256>(P);
        } else {
            e = o->precision == LASP_PREC_TF32   ? pool_setup<6, 1, 512>(P)
                : o->precision == LASP_PREC_BF16 ? pool_setup<6, 2, 512>(P)
                                                 : pool_setup<6, 3, 512>(P);
        }
    }
    if (e) {
        grp_pool_free(P);
        return e;
    }
    *out = P;
    return LASP_OK;
}

int grp_pool_admit(GrpPool* P, int count, const int32_t* idx_dev, cudaStream_t st) {
    return count > 0 ? P->admit(P, count, idx_dev, st) : LASP_OK;
}

int grp_pool_step(GrpPool* P, int budget, cudaStream_t st, int* launches) {
    const int replays = (budget + CHUNK_STEPS - 1) / CHUNK_STEPS;
    // a timeout ends only the fits stepped while it was set (LASP_ST_TIMEOUT)
    int e0 = cuda_rc(cudaMemsetAsync(P->G.err, 0, sizeof(int), st));
    if (e0) return e0;
    for (int r = 0; r < replays; ++r) {
        const int e = cuda_rc(cudaGraphLaunch(P->exec, st));
        if (e) return e;
    }
    *launches = replays * (P->G.O.clean ? 5 : 4) * CHUNK_STEPS;
    return LASP_OK;
}

}  // namespace lasp
