// Per-kernel timing for measurement (lasp_profile / lasp_profile_read).
//
// While profiling is on, the launchers bracket each kernel launch with CUDA
// events on the launching stream and wait for the closing event, so each
// kernel's device time is known on its own; the sums are kept per kernel name
// until read.  Off by default: the launch paths then pay one relaxed load.
#pragma once

#include <cuda_runtime.h>

namespace lasp {

bool prof_on();
void prof_add(const char* name, float ms);

// Runs f() (which launches on st and returns a LASP_* code); when profiling
// is on, times it with events on st and adds the time under `name`.
template <typename F>
int prof_time(const char* name, cudaStream_t st, F&& f) {
    if (!prof_on()) return f();
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        cudaGetLastError();
        return f();
    }
    cudaEventRecord(a, st);
    const int e = f();
    cudaEventRecord(b, st);
    float ms = 0.0f;
    if (!e && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
        prof_add(name, ms);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

}  // namespace lasp
