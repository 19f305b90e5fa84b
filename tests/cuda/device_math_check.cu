// Checks of the library's own device math against CUDA's float64 results and the stated
// error bounds (built and run by tests/test_gpu_device_math.py):
//   dfl::exp_neg (double-float exp(-t), table-driven) against exp() in float64 over t in [0, 90];
//   slc::slice5 (Ozaki slices) against the float64 value it cuts: reconstruction error,
//   integrality and magnitude of every slice, exactness in bf16.
// Prints one JSON line; exit status 0 when every bound holds.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdint>
#include <vector>

#include "dfloat.cuh"
#include "slicing.cuh"

using namespace gbxc;

__global__ void exp_kernel(int n, double *rel, double *absd, const float2 *tab) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // t from 0 to 90 with an irregular low part
    double t = 90.0 * (double)i / (double)n + 1e-9 * (double)(i % 13);
    dfl::df td = dfl::from_double(t);
    double ref = exp(-dfl::to_double(td));
    double got = dfl::to_double(dfl::exp_neg(td, tab));
    absd[i] = fabs(got - ref);
    rel[i] = ref > 0 ? fabs(got - ref) / ref : 0.0;
}

// splitmix64 for the test values
__device__ uint64_t mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void slice_kernel(int n, double *err, float *qmax, int *bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t r = mix((uint64_t)i * 7919u + 17u);
    // a double-float value with a random sign, mantissa and exponent in [-60, 20]
    double mant = 1.0 + (double)(r >> 11) * (1.0 / 9007199254740992.0);
    int ex = (int)((r >> 3) % 81) - 60;
    double v = ((r & 1) ? -1.0 : 1.0) * ldexp(mant, ex);
    float h = (float)v;
    float l = (float)(v - (double)h);
    // the row exponent: the value's own, or up to 30 above it (a smaller element of a row)
    int e = slc::exp_of(fabsf(h)) + (int)((r >> 40) % 31) * ((r >> 2) & 1);
    float q[slc::NSL];
    slc::slice5(h, l, e, q);
    double sum = 0.0;
    int b = 0;
    for (int s = 0; s < slc::NSL; ++s) {
        double units = ldexp((double)q[s], 6 + 7 * s);   // q_s as an integer
        if (units != rint(units)) b |= 1;
        double lim = s == 3 ? 72.0 : 64.0;
        if (fabs(units) > lim) b |= 2;
        if (__bfloat162float(__float2bfloat16_rn(q[s])) != q[s]) b |= 4;
        qmax[(size_t)i * slc::NSL + s] = (float)fabs(units);
        sum += (double)q[s];
    }
    double target = ldexp((double)h + (double)l, -e);
    if (fabs(target) > 1.0) b |= 8;
    err[i] = fabs(sum - target);
    bad[i] = b;
}

int main() {
    const int n = 1 << 22;
    double *rel, *absd, *serr;
    float *qmax;
    int *bad;
    cudaMalloc(&rel, n * sizeof(double));
    cudaMalloc(&absd, n * sizeof(double));
    cudaMalloc(&serr, n * sizeof(double));
    cudaMalloc(&qmax, (size_t)n * slc::NSL * sizeof(float));
    cudaMalloc(&bad, n * sizeof(int));
    float2 htab[64], *tab;
    dfl::make_exp2_table(htab);
    cudaMalloc(&tab, sizeof(htab));
    cudaMemcpy(tab, htab, sizeof(htab), cudaMemcpyHostToDevice);
    exp_kernel<<<(n + 255) / 256, 256>>>(n, rel, absd, tab);
    slice_kernel<<<(n + 255) / 256, 256>>>(n, serr, qmax, bad);
    cudaError_t e = cudaDeviceSynchronize();
    std::vector<double> hr(n), ha(n), hs(n);
    std::vector<float> hq((size_t)n * slc::NSL);
    std::vector<int> hb(n);
    cudaMemcpy(hr.data(), rel, n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaMemcpy(ha.data(), absd, n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaMemcpy(hs.data(), serr, n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaMemcpy(hq.data(), qmax, hq.size() * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(hb.data(), bad, n * sizeof(int), cudaMemcpyDeviceToHost);
    double rel70 = 0, abs_tail = 0, serr_max = 0;
    float qm[slc::NSL] = {0, 0, 0, 0, 0};
    int nbad = 0, flags = 0;
    for (int i = 0; i < n; ++i) {
        double t = 90.0 * (double)i / (double)n;
        if (t <= 70.0) rel70 = fmax(rel70, hr[i]);
        else abs_tail = fmax(abs_tail, ha[i]);
        serr_max = fmax(serr_max, hs[i]);
        for (int s = 0; s < slc::NSL; ++s) qm[s] = fmaxf(qm[s], hq[(size_t)i * slc::NSL + s]);
        if (hb[i]) ++nbad;
        flags |= hb[i];
    }
    bool ok = e == cudaSuccess && rel70 < 1e-12 && abs_tail < 1e-36 && serr_max <= ldexp(1.0, -34) && nbad == 0;
    printf("{\"cuda\": \"%s\", \"exp_max_rel_t_le_70\": %.3e, \"exp_max_abs_t_gt_70\": %.3e, "
           "\"slice_max_err\": %.3e, \"slice_max_units\": [%g, %g, %g, %g, %g], \"slice_bad\": %d, "
           "\"slice_flags\": %d, \"ok\": %s}\n",
           cudaGetErrorString(e), rel70, abs_tail, serr_max, qm[0], qm[1], qm[2], qm[3], qm[4], nbad, flags,
           ok ? "true" : "false");
    return ok ? 0 : 1;
}
