// Native continuous-batching scheduler over slot pools (lasp_server_*).
//
// One lane per interpolator: a lasp_slots pool, its own CUDA stream, a pinned
// submission ring and pinned result buffers.  Submissions copy into the ring
// under the lane's mutex; a tick admits ring entries into free slots (one or
// two host-to-device copies of contiguous ring ranges), runs one chunk of Adam
// steps on every lane, fetches the slots' status and results, waits for the
// lanes, and retires finished fits into a result queue.  Ring entries are
// released for reuse only after the tick that copied them has completed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "lasp.h"

namespace lasp {
int slots_n_pix(lasp_slots s);   // pixel count of a slot pool's grid (lasp_capi.cu)
}

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

int cuda_e(cudaError_t e) {
    if (e == cudaSuccess) return LASP_OK;
    (void)cudaGetLastError();    // returned here: not to be reported again by a later launch check
    return e == cudaErrorMemoryAllocation ? LASP_ENOMEM : LASP_ECUDA;
}

struct Lane {
    lasp_slots pool = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int n = 0, n_pix = 0, ring = 0;
    // pinned submission ring, entries [released, staged) in use, [admitted, staged) waiting
    float *r_flux = nullptr, *r_ivar = nullptr, *r_th0 = nullptr;
    uint8_t* r_good = nullptr;
    std::vector<int64_t> r_id, r_tsub;        // caller tag and submit time per entry
    int64_t staged = 0, admitted = 0, released = 0;
    std::mutex mu;                        // guards the ring counters and entries
    // slots
    int32_t* h_idx = nullptr;             // pinned admission slot indices
    float *o_theta = nullptr, *o_loss = nullptr;
    int32_t* o_steps = nullptr;
    uint32_t* o_status = nullptr;
    std::vector<int> free_slots;
    std::vector<int64_t> slot_id, slot_tsub;   // tag and submit time per slot
    std::vector<uint8_t> slot_busy;
    std::atomic<int> busy{0};                  // slots running (written by the ticking thread)
    int64_t admitted_this_tick = 0;
};

}  // namespace

struct lasp_server_s {
    std::vector<Lane*> lanes;
    int chunk = 1;
    std::mutex out_mu;
    std::deque<lasp_served> out;
};

namespace {

void free_lane(Lane* L) {
    if (!L) return;
    if (L->pool) lasp_slots_free(L->pool);
    if (L->done) cudaEventDestroy(L->done);
    if (L->stream) cudaStreamDestroy(L->stream);
    void* pinned[] = {L->r_flux, L->r_ivar, L->r_th0, L->r_good, L->h_idx,
                      L->o_theta, L->o_loss, L->o_steps, L->o_status};
    for (void* p : pinned)
        if (p) cudaFreeHost(p);
    delete L;
}

// Admit waiting ring entries into free slots and launch one chunk (lane stream).
// The slot bookkeeping is committed only once every admission call has been
// accepted; a failed admission leaves the slots free and the entries waiting.
int launch_lane(Lane* L, int chunk) {
    int64_t first, count;
    {
        std::lock_guard<std::mutex> g(L->mu);
        first = L->admitted;
        count = L->staged - L->admitted;
    }
    if (count > (int64_t)L->free_slots.size()) count = (int64_t)L->free_slots.size();
    // the slots taken, from the back of the free list
    for (int64_t r = 0; r < count; ++r) L->h_idx[r] = L->free_slots[L->free_slots.size() - 1 - (size_t)r];
    int64_t done = 0;
    while (done < count) {
        const int64_t e = (first + done) % L->ring;
        const int64_t m = std::min(count - done, (int64_t)L->ring - e);
        const size_t p = (size_t)L->n_pix;
        int rc = lasp_slots_admit(L->pool, (int)m, L->h_idx + done, L->r_flux + e * p, L->r_ivar + e * p,
                                  L->r_good + e * p, L->r_th0 + e * 5, L->stream);
        if (rc) {
            // nothing is committed: the slots stay free and the entries wait for the next tick
            // (slots whose admission was already enqueued are overwritten when reused)
            L->admitted_this_tick = first;
            return rc;
        }
        done += m;
    }
    {
        std::lock_guard<std::mutex> g(L->mu);
        for (int64_t r = 0; r < count; ++r) {
            const int s = L->free_slots.back();
            L->free_slots.pop_back();
            const int64_t e = (first + r) % L->ring;
            L->slot_id[s] = L->r_id[e];
            L->slot_tsub[s] = L->r_tsub[e];
            L->slot_busy[s] = 1;
        }
        L->admitted = first + count;
    }
    L->admitted_this_tick = first + count;
    L->busy.fetch_add((int)count);
    if (L->busy == 0) return LASP_OK;
    int rc = lasp_slots_step_running(L->pool, chunk, L->busy, L->stream);
    if (!rc)
        rc = lasp_slots_fetch(L->pool, L->o_theta, L->o_loss, L->o_steps, L->o_status, nullptr, L->stream);
    if (!rc) rc = cuda_e(cudaEventRecord(L->done, L->stream));
    return rc;
}

}  // namespace

extern "C" {

int lasp_server_create(int n_lanes, const lasp_interp* interps, const int* n_slots, const int* ring,
                       const lasp_fit_opts* opts, int chunk, lasp_server* out) {
    if (!out) return LASP_EINVAL;
    *out = nullptr;
    if (n_lanes < 1 || n_lanes > 8 || !interps || !n_slots || !ring || !opts || chunk < 1)
        return LASP_EINVAL;
    lasp_server_s* S = new (std::nothrow) lasp_server_s();
    if (!S) return LASP_ENOMEM;
    S->chunk = chunk;
    int rc = LASP_OK;
    for (int l = 0; l < n_lanes && !rc; ++l) {
        if (!interps[l] || n_slots[l] < 1 || ring[l] < 1) {
            rc = LASP_EINVAL;
            break;
        }
        Lane* L = new (std::nothrow) Lane();
        if (!L) {
            rc = LASP_ENOMEM;
            break;
        }
        S->lanes.push_back(L);
        rc = lasp_slots_create(interps[l], n_slots[l], opts, &L->pool);
        if (rc) break;
        L->n = n_slots[l];
        L->ring = ring[l];
        L->n_pix = lasp::slots_n_pix(L->pool);
        const size_t p = (size_t)L->n_pix, R = (size_t)L->ring, n = (size_t)L->n;
        rc = cuda_e(cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking));
        if (!rc) rc = cuda_e(cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->r_flux, R * p * 4, cudaHostAllocDefault));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->r_ivar, R * p * 4, cudaHostAllocDefault));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->r_good, R * p, cudaHostAllocDefault));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->r_th0, R * 5 * 4, cudaHostAllocDefault));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->h_idx, n * 4, cudaHostAllocDefault));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->o_theta, n * 5 * 4, cudaHostAllocDefault));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->o_loss, n * 4, cudaHostAllocDefault));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->o_steps, n * 4, cudaHostAllocDefault));
        if (!rc) rc = cuda_e(cudaHostAlloc((void**)&L->o_status, n * 4, cudaHostAllocDefault));
        if (rc) break;
        L->r_id.assign(R, -1);
        L->r_tsub.assign(R, 0);
        L->slot_id.assign(n, 0);
        L->slot_tsub.assign(n, 0);
        L->slot_busy.assign(n, 0);
        L->free_slots.reserve(n);
        for (int s = L->n - 1; s >= 0; --s) L->free_slots.push_back(s);
    }
    if (rc) {
        for (Lane* L : S->lanes) free_lane(L);
        delete S;
        return rc;
    }
    *out = S;
    return LASP_OK;
}

void lasp_server_destroy(lasp_server S) {
    if (!S) return;
    for (Lane* L : S->lanes) {
        if (L->stream) cudaStreamSynchronize(L->stream);
        free_lane(L);
    }
    delete S;
}

int lasp_server_submit(lasp_server S, int lane, const float* flux, const float* ivar, const uint8_t* good,
                       const float* theta0, int64_t tag) {
    if (!S || lane < 0 || lane >= (int)S->lanes.size() || !flux || !ivar || !good || !theta0)
        return LASP_EINVAL;
    Lane* L = S->lanes[lane];
    const size_t p = (size_t)L->n_pix;
    std::lock_guard<std::mutex> g(L->mu);
    if (L->staged - L->released >= L->ring) return LASP_EBUSY;
    const int64_t e = L->staged % L->ring;
    std::memcpy(L->r_flux + e * p, flux, p * 4);
    std::memcpy(L->r_ivar + e * p, ivar, p * 4);
    std::memcpy(L->r_good + e * p, good, p);
    std::memcpy(L->r_th0 + e * 5, theta0, 5 * 4);
    L->r_id[e] = tag;
    L->r_tsub[e] = now_ns();
    L->staged += 1;
    return LASP_OK;
}

int lasp_server_submit_n(lasp_server S, int lane, int n, const float* flux, const float* ivar,
                         const uint8_t* good, const float* theta0, const int64_t* tags, int* n_taken) {
    if (n_taken) *n_taken = 0;
    if (!S || lane < 0 || lane >= (int)S->lanes.size() || n < 0 || !n_taken) return LASP_EINVAL;
    if (n == 0) return LASP_OK;
    if (!flux || !ivar || !good || !theta0 || !tags) return LASP_EINVAL;
    Lane* L = S->lanes[lane];
    const size_t p = (size_t)L->n_pix;
    std::lock_guard<std::mutex> g(L->mu);
    const int64_t room = L->ring - (L->staged - L->released);
    const int k = (int)std::min<int64_t>(n, room > 0 ? room : 0);
    const int64_t t = now_ns();
    // at most two contiguous ranges of ring entries (the second after the wrap)
    for (int i = 0; i < k;) {
        const int64_t e = (L->staged + i) % L->ring;
        const int run = (int)std::min<int64_t>(k - i, L->ring - e);
        std::memcpy(L->r_flux + e * p, flux + (size_t)i * p, (size_t)run * p * 4);
        std::memcpy(L->r_ivar + e * p, ivar + (size_t)i * p, (size_t)run * p * 4);
        std::memcpy(L->r_good + e * p, good + (size_t)i * p, (size_t)run * p);
        std::memcpy(L->r_th0 + e * 5, theta0 + (size_t)i * 5, (size_t)run * 5 * 4);
        for (int j = 0; j < run; ++j) {
            L->r_id[e + j] = tags[i + j];
            L->r_tsub[e + j] = t;
        }
        i += run;
    }
    L->staged += k;
    *n_taken = k;
    return k == n ? LASP_OK : LASP_EBUSY;
}

int lasp_server_tick(lasp_server S, int* n_finished) {
    if (n_finished) *n_finished = 0;
    if (!S) return LASP_EINVAL;
    int rc = LASP_OK;
    for (Lane* L : S->lanes)
        if (!rc) rc = launch_lane(L, S->chunk);
    int fin = 0;
    bool timed_out = false;
    for (size_t l = 0; l < S->lanes.size(); ++l) {
        Lane* L = S->lanes[l];
        if (L->busy == 0) {
            std::lock_guard<std::mutex> g(L->mu);
            L->released = L->admitted_this_tick > L->released ? L->admitted_this_tick : L->released;
            continue;
        }
        const int e = cuda_e(cudaEventSynchronize(L->done));
        if (!rc) rc = e;
        if (e) continue;
        {
            std::lock_guard<std::mutex> g(L->mu);
            L->released = L->admitted_this_tick;   // the copies of this tick's entries are done
        }
        const int64_t t = now_ns();
        std::vector<lasp_served> done;
        for (int s = 0; s < L->n; ++s) {
            if (!L->slot_busy[s] || L->o_status[s] == LASP_ST_RUNNING) continue;
            lasp_served r;
            r.tag = L->slot_id[s];
            r.lane = (int)l;
            std::memcpy(r.theta, L->o_theta + 5 * (size_t)s, sizeof(r.theta));
            r.loss = L->o_loss[s];
            r.steps = L->o_steps[s];
            r.status = L->o_status[s];
            r.t_submit_ns = L->slot_tsub[s];
            r.t_done_ns = t;
            if (r.status & LASP_ST_TIMEOUT) timed_out = true;
            done.push_back(r);
            L->slot_busy[s] = 0;
            L->free_slots.push_back(s);
            L->busy.fetch_sub(1);
        }
        fin += (int)done.size();
        std::lock_guard<std::mutex> g(S->out_mu);
        for (const lasp_served& r : done) S->out.push_back(r);
    }
    if (n_finished) *n_finished = fin;
    // a bounded device wait gave up in this tick: its fits are retired with
    // LASP_ST_TIMEOUT, and the tick reports it
    if (!rc && timed_out) rc = LASP_ETIMEOUT;
    return rc;
}

int lasp_server_poll(lasp_server S, lasp_served* out, int max, int* n) {
    if (!S || !n || max < 0 || (max > 0 && !out)) return LASP_EINVAL;
    std::lock_guard<std::mutex> g(S->out_mu);
    int k = 0;
    while (k < max && !S->out.empty()) {
        out[k++] = S->out.front();
        S->out.pop_front();
    }
    *n = k;
    return LASP_OK;
}

int lasp_server_pending(lasp_server S, int64_t* n) {
    if (!S || !n) return LASP_EINVAL;
    int64_t c = 0;
    for (Lane* L : S->lanes) {
        std::lock_guard<std::mutex> g(L->mu);
        c += (L->staged - L->admitted) + L->busy;
    }
    *n = c;
    return LASP_OK;
}

}  // extern "C"
