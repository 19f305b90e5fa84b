// The bounded mbarrier wait the tensor-core kernels use (umma::mbar_wait_for): a wait on a
// barrier that nothing arrives at gives up after its limit and reports it, a completed phase
// is seen at once, and the context stays usable afterwards (built and run by
// tests/test_gpu_bounded_wait.py).  No fault, trap or endless loop is involved: the expiring
// wait is limited to 2e7 clock cycles (about 10 ms).
// Prints one JSON line; exit status 0 when every check holds.
#include <cuda_runtime.h>

#include <cstdio>

#include "umma.cuh"

using namespace gbxc;

__global__ void wait_kernel(int *status) {
    __shared__ uint64_t bar[2];
    if (threadIdx.x == 0) {
        umma::mbar_init(&bar[0], 1);
        umma::mbar_init(&bar[1], 1);
        umma::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // bar[0]: nobody arrives, so phase 0 never completes within the limit
        status[0] = umma::mbar_wait_for(&bar[0], 0, 20000000LL) ? 0 : 1;
        // bar[1]: one arrival completes phase 0
        umma::mbar_arrive(&bar[1]);
        status[1] = umma::mbar_wait_for(&bar[1], 0, 20000000LL) ? 1 : 0;
    }
}

__global__ void add_one(int *v) { v[threadIdx.x] += 1; }

int main() {
    int *d = nullptr;
    if (cudaMalloc(&d, 64 * sizeof(int)) != cudaSuccess) return 2;
    cudaMemset(d, 0, 64 * sizeof(int));
    wait_kernel<<<1, 32>>>(d);
    cudaError_t e1 = cudaDeviceSynchronize();
    int st[2] = {-1, -1};
    cudaMemcpy(st, d, sizeof(st), cudaMemcpyDeviceToHost);
    cudaMemset(d, 0, 64 * sizeof(int));
    add_one<<<1, 64>>>(d);                       // the context still runs work
    cudaError_t e2 = cudaDeviceSynchronize();
    int v[64];
    cudaMemcpy(v, d, sizeof(v), cudaMemcpyDeviceToHost);
    int sum = 0;
    for (int k = 0; k < 64; ++k) sum += v[k];
    cudaFree(d);
    const bool ok = e1 == cudaSuccess && e2 == cudaSuccess && st[0] == 1 && st[1] == 1 && sum == 64;
    printf("{\"timed_out\": %d, \"completed_seen\": %d, \"after\": %d, \"err1\": %d, \"err2\": %d}\n", st[0], st[1],
           sum, (int)e1, (int)e2);
    return ok ? 0 : 1;
}
