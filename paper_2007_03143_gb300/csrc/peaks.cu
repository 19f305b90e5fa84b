// Arithmetic-pipe peaks of the device, measured (no counterpart in the paper; the rooflines of
// the collocation and of the float64 contractions are stated against them).
//
// Each thread runs 8 independent multiply-add chains of `iters` steps (16 flops per step and
// thread), so the FMA pipe, not the dependency latency, sets the rate; 8 blocks of 256 threads
// per SM.  The chains' sum is stored so nothing is eliminated.  Time: CUDA events around one
// launch after a warm-up launch.
#include <cuda_runtime.h>

#include "gbxc.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int time_chains(int sms, int iters, double *tflops) {
    const int blocks = sms * 8, threads = 256;
    T *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) return GBXC_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a contraction towards b / (1 - a): values stay bounded, no denormals or overflow
    const T a = (T)0.999, b = (T)1e-3;
    fma_chains<T><<<blocks, threads>>>(out, iters / 8, a, b);
    cudaEventRecord(e0);
    fma_chains<T><<<blocks, threads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.f) return GBXC_ECUDA;
    *tflops = 16.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
    return GBXC_OK;
}

}  // namespace

extern "C" int gbxc_measure_alu_peaks(int device, double *fp32_tflops, double *fp64_tflops) {
    if (!fp32_tflops || !fp64_tflops) return GBXC_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return GBXC_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
        return GBXC_ECUDA;
    int rc = time_chains<float>(sms, 1 << 16, fp32_tflops);
    if (rc != GBXC_OK) return rc;
    return time_chains<double>(sms, 1 << 12, fp64_tflops);
}
