// Atomic partition weights w_i = p_A(r_i) w^q_i (Sec. 2.2, Eqs. atomic_partition and num_int;
// Algorithm 4's partition-weight update), in float64 on the GPU, one thread per grid point.
//
// Becke (1988) cell function: s(mu) = (1 - p(p(p(mu))))/2, p(x) = 1.5x - 0.5x^3.
// SSF (1996): s(mu) = (1 - g(mu))/2 with g the degree-7 polynomial in mu/a on
// |mu| < a (a = 0.64) and g = +-1 outside; plus SSF's own-atom shortcut.
// P_B(r) = prod_{C != B} s(mu_BC), mu_BC = (|r-R_B| - |r-R_C|)/R_BC,
// p_A = P_A / sum_B P_B.
//
// The natoms^2 loop is screened in the SSF case by two exact rules (the skipped factors are
// exactly 0 or 1; only the order of the products changes).  (1) P_B = 0 when mu_Bn >= a for
// the atom n nearest to the point.  (2) By the triangle inequality |r-R_C| >= R_BC - |r-R_B|,
// so mu_BC <= 2|r-R_B|/R_BC - 1, which is <= -a (s = 1 exactly) once R_BC >= 2|r-R_B|/(1-a):
// the factors of P_B are taken over B's neighbours in order of distance (lists built on the
// host per molecule) and stop there.  The outer loop over B stays in atom order, so the
// threads of a warp take the same B together (a candidate list per point, from the nearest
// atom's neighbours, was measured slower: divergent).
#include <cstdint>

#include "internal.h"

namespace gbxc {
namespace {

constexpr double kSsfA = 0.64;
constexpr int kMaxAtomsSmem = 1024;

__device__ __forceinline__ double becke_s(double mu) {
    double f = mu;
    f = 1.5 * f - 0.5 * f * f * f;
    f = 1.5 * f - 0.5 * f * f * f;
    f = 1.5 * f - 0.5 * f * f * f;
    return 0.5 * (1.0 - f);
}

__device__ __forceinline__ double ssf_s(double mu) {
    if (mu <= -kSsfA) return 1.0;
    if (mu >= kSsfA) return 0.0;
    double z = mu / kSsfA;
    double z2 = z * z;
    double g = z * (35.0 + z2 * (-35.0 + z2 * (21.0 - 5.0 * z2))) / 16.0;
    return 0.5 * (1.0 - g);
}

// CACHE: the point's distances to every atom are computed once into shared memory
// ([atom][thread], so the threads of a warp read one row) and the SSF pair loops read them.
template <bool CACHE>
__global__ void partition_weights_kernel(WeightsArgs a) {
    extern __shared__ double sm[];
    double *ax = sm, *ay = sm + a.natoms, *az = sm + 2 * a.natoms;
    double *dc = sm + 3 * a.natoms;   // CACHE: natoms x blockDim.x
    for (int k = threadIdx.x; k < a.natoms; k += blockDim.x) {
        ax[k] = a.atoms[3 * k];
        ay[k] = a.atoms[3 * k + 1];
        az[k] = a.atoms[3 * k + 2];
    }
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.npts) return;
    double px = a.x[i], py = a.y[i], pz = a.z[i];
    int A = a.parent[i];
    auto dist0 = [&](int k) {
        double dx = px - ax[k], dy = py - ay[k], dz = pz - az[k];
        return sqrt(dx * dx + dy * dy + dz * dz);
    };
    auto dist = [&](int k) {
        if constexpr (CACHE) return dc[(size_t)k * blockDim.x + threadIdx.x];
        else return dist0(k);
    };
    auto rab = [&](int k, int l) {
        double dx = ax[k] - ax[l], dy = ay[k] - ay[l], dz = az[k] - az[l];
        return sqrt(dx * dx + dy * dy + dz * dz);
    };
    double p;
    if (a.natoms == 1) {
        p = 1.0;
    } else if (a.scheme == GBXC_SSF && dist0(A) < 0.5 * (1.0 - kSsfA) * a.rnn[A]) {
        p = 1.0;
    } else if (a.scheme == GBXC_SSF) {
        int nearest = 0;
        double dn = dist0(0);
        if constexpr (CACHE) dc[threadIdx.x] = dn;
        for (int k = 1; k < a.natoms; ++k) {
            double d = dist0(k);
            if constexpr (CACHE) dc[(size_t)k * blockDim.x + threadIdx.x] = d;
            if (d < dn) { dn = d; nearest = k; }
        }
        double sum = 0.0, pa = 0.0;
        for (int B = 0; B < a.natoms; ++B) {   // every thread of a warp visits the same B
            const double dB = dist(B);
            double PB = 1.0;
            if (B != nearest && (dB - dn) / rab(B, nearest) >= kSsfA) {
                PB = 0.0;
            } else {
                const int *nb = a.nbr + (size_t)B * (a.natoms - 1);
                const double *nr = a.nbr_r + (size_t)B * (a.natoms - 1);
                const double lim = 2.0 * dB / (1.0 - kSsfA);
                for (int k = 0; k < a.natoms - 1 && PB != 0.0; ++k) {
                    const double R = nr[k];
                    if (R >= lim) break;          // every further factor is exactly 1
                    PB *= ssf_s((dB - dist(nb[k])) / R);
                }
            }
            sum += PB;
            if (B == A) pa = PB;
        }
        p = pa / sum;
    } else {   // Becke: every pair
        double sum = 0.0, pa = 0.0;
        for (int B = 0; B < a.natoms; ++B) {
            double dB = dist0(B);
            double PB = 1.0;
            for (int C = 0; C < a.natoms; ++C) {
                if (C == B) continue;
                PB *= becke_s((dB - dist0(C)) / rab(B, C));
            }
            sum += PB;
            if (B == A) pa = PB;
        }
        p = pa / sum;
    }
    a.w[i] = a.wq[i] * p;
}

}  // namespace

cudaError_t launch_partition_weights(const WeightsArgs &a, cudaStream_t s) {
    if (a.npts == 0) return cudaSuccess;
    if (a.natoms > kMaxAtomsSmem) return cudaErrorInvalidValue;
    // SSF with the distance cache when 128 threads' distances fit in 200 KB (up to 195 atoms)
    const size_t cache = sizeof(double) * (size_t)a.natoms * 128;
    const bool use_cache = a.scheme == GBXC_SSF && cache <= (size_t)200 * 1024;
    int threads = 128;
    int64_t blocks = (a.npts + threads - 1) / threads;
    size_t smem = sizeof(double) * 3 * a.natoms + (use_cache ? cache : 0);
    if (a.prof) a.prof->begin(GBXC_K_WEIGHTS, s);
    if (use_cache) {
        cudaError_t e = cudaFuncSetAttribute(partition_weights_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        partition_weights_kernel<true><<<(unsigned)blocks, threads, smem, s>>>(a);
    } else {
        partition_weights_kernel<false><<<(unsigned)blocks, threads, smem, s>>>(a);
    }
    if (a.prof) a.prof->end(GBXC_K_WEIGHTS, s);
    return cudaGetLastError();
}

}  // namespace gbxc
