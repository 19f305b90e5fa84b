// Per-kernel-class launch counts and CUDA-event spans (the library's tracing hook).
#include "internal.h"

namespace gbxc {

void Profiler::begin(int kind, cudaStream_t s) {
    if (!on) return;
    cudaEvent_t e;
    if (pool.empty()) {
        if (cudaEventCreate(&e) != cudaSuccess) return;
    } else {
        e = pool.back();
        pool.pop_back();
    }
    cudaEventRecord(e, s);
    open_kind = kind;
    open_ev = e;
}

void Profiler::end(int kind, cudaStream_t s, int nlaunch) {
    launches[kind] += nlaunch;
    if (!on || open_kind != kind || !open_ev) return;
    cudaEvent_t e;
    if (pool.empty()) {
        if (cudaEventCreate(&e) != cudaSuccess) return;
    } else {
        e = pool.back();
        pool.pop_back();
    }
    cudaEventRecord(e, s);
    pending.push_back({kind, open_ev, e});
    open_kind = -1;
    open_ev = nullptr;
}

void Profiler::collect() {
    for (auto &r : pending) {
        cudaEventSynchronize(r.b);
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.kind] += t;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
}

void Profiler::reset() {
    collect();
    for (int k = 0; k < GBXC_NKERNEL; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
}

void Profiler::release() {
    collect();
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    if (open_ev) cudaEventDestroy(open_ev);
    open_ev = nullptr;
}

}  // namespace gbxc
