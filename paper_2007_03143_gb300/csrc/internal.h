// Internal data structures shared by the host code and the CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gbxc.h"

namespace gbxc {

constexpr int TILE = 128;        // grid points per tile (the M extent of the tensor-core tiles)
constexpr int FBLK = 32;         // function padding granule (one 64-byte K block of bf16 operands)

// One contracted Cartesian shell (Eq. gau_cart), as the kernels read it.
struct DevShell {
    double c[3];
    int L, nprim, fofs;
    int pure;   // 1: the 2L+1 real solid harmonics (L >= 2) instead of the Cartesian functions
    double alpha[GBXC_MAX_PRIM];
    double coeff[GBXC_MAX_PRIM];
};

// Host-side batch plan (Sec. 2.2, Algorithm 1, Algorithm 3).
struct HostPlan {
    // points in batch order
    std::vector<double> x, y, z, wq;
    std::vector<int> parent;
    std::vector<int64_t> point_index;
    // merged batches
    std::vector<int64_t> batch_ptr;   // nbatch+1 into the point arrays
    std::vector<int64_t> shell_ptr;   // nbatch+1
    std::vector<int> shell_idx;
    std::vector<int64_t> func_ptr;    // nbatch+1
    std::vector<int> func_idx;
    std::vector<double> work;
    int nleaf = 0;
    // 128-point tiles
    std::vector<int> tile_batch;
    std::vector<int64_t> tile_first;  // first point (batch order) of the tile
    std::vector<int> tile_count;
    std::vector<int64_t> tile_row;    // prefix sum of padded N_b^j over tiles (slab row offset)
    std::vector<int64_t> batch_tile;  // nbatch+1 into the tile arrays
    int64_t npts = 0;                 // points (the arrays above may live on the device only)
    int nbatch() const { return (int)batch_ptr.size() - 1; }
    int64_t ntiles() const { return (int64_t)tile_batch.size(); }
};

// Device views of the resident plan of one molecule.
struct DevPlan {
    double *x = nullptr, *y = nullptr, *z = nullptr, *wq = nullptr, *w = nullptr;
    int *parent = nullptr;
    int64_t *shell_ptr = nullptr;
    int *shell_idx = nullptr;
    int64_t *func_ptr = nullptr;
    int *func_idx = nullptr;
    int *tile_batch = nullptr;
    int64_t *tile_first = nullptr;
    int *tile_count = nullptr;
    int64_t *tile_row = nullptr;
    int64_t *batch_tile = nullptr;
    int64_t *batch_ptr = nullptr;
};

// Grid generation and planning on the host (host_plan.cpp).  Bitwise contract:
// the same coordinates and the same batches as the reference CPU planner in the
// same process (plain IEEE double arithmetic, no contraction; logarithms, sines and cosines
// written out with basic operations instead of libm, so the plan is the same on every host).
// 1-D factors of the atomic grid: Mura-Knowles radii and weights (r^2 included), and the
// angular product rule's unit vectors and weights.
struct GridTables {
    std::vector<double> r, wr, ux, uy, uz, wa;
};
void grid_tables(const gbxc_grid_spec &spec, GridTables &T);
// True when a Lebedev-Laikov rule of n points is tabulated (lebedev_rules.inc).
bool lebedev_supported(int n);
void build_molecular_grid(const std::vector<double> &xyz, const gbxc_grid_spec &spec,
                          std::vector<double> &x, std::vector<double> &y, std::vector<double> &z,
                          std::vector<double> &wq, std::vector<int> &parent);
double shell_cutoff(const double *alpha, int nprim, double eta);
void build_plan(const std::vector<double> &xyz, const std::vector<DevShell> &shells,
                const std::vector<double> &rcut, int nbf, const gbxc_grid_spec &spec,
                const std::vector<double> &x, const std::vector<double> &y,
                const std::vector<double> &z, const std::vector<double> &wq,
                const std::vector<int> &parent, HostPlan &plan);

inline int64_t pad_funcs(int64_t n) { return (n + FBLK - 1) / FBLK * FBLK; }
// Functions of a shell: (L+1)(L+2)/2 Cartesian, or 2L+1 real solid harmonics when pure.
inline int shell_nfunc(const DevShell &s) { return s.pure ? 2 * s.L + 1 : (s.L + 1) * (s.L + 2) / 2; }
// The planner as device kernels (device_plan.cu): the same grid and plan as
// build_molecular_grid + build_plan, bit for bit.  *status: 0 done, 1 grid too large,
// 2 internal stack overflow (cannot happen for depth <= 16).
// The point arrays in batch order stay on the device: x, y, z, wq, parent and point_index
// are allocated here (cudaMalloc; the caller frees them) and the host plan's copies stay
// empty (plan.npts holds the count).
struct DevPoints {
    double *x = nullptr, *y = nullptr, *z = nullptr, *wq = nullptr;
    int *parent = nullptr;
    int64_t *point_index = nullptr;
};
cudaError_t device_plan(const std::vector<double> &xyz, const std::vector<DevShell> &shells,
                        const std::vector<double> &rcut, const gbxc_grid_spec &spec, HostPlan &plan,
                        DevPoints &out, cudaStream_t s, int *status);
// The planner's last steps, shared by the host and the device planner: merge leaves with
// equal shell lists (first occurrence first), lay out points, functions, work and tiles.
void merge_leaves(const std::vector<std::vector<int>> &keeps, std::vector<std::vector<int>> &bshells,
                  std::vector<std::vector<int>> &bleaves);
void batch_metadata(size_t natoms, const std::vector<DevShell> &shells, const std::vector<std::vector<int>> &bshells,
                    const std::vector<int64_t> &batch_size, HostPlan &plan);
void plan_from_leaves(size_t natoms, const std::vector<DevShell> &shells,
                      const std::vector<std::vector<int64_t>> &leaves, const std::vector<std::vector<int>> &keeps,
                      const std::vector<double> &x, const std::vector<double> &y, const std::vector<double> &z,
                      const std::vector<double> &wq, const std::vector<int> &parent, HostPlan &plan);

// Per-kernel-class launch counter and optional CUDA-event timer (profiler.cpp).
// Kernel classes are the GBXC_K_* constants of gbxc.h.
struct Profiler {
    bool on = false;
    long long launches[GBXC_NKERNEL] = {};
    double ms[GBXC_NKERNEL] = {};
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    int open_kind = -1;
    cudaEvent_t open_ev = nullptr;
    void begin(int kind, cudaStream_t s);
    void end(int kind, cudaStream_t s, int nlaunch = 1);
    void collect();
    void reset();
    void release();
};

// ---------------------------------------------------------------------------
// kernel launchers (one translation unit each)
// ---------------------------------------------------------------------------
struct WeightsArgs {
    const double *x, *y, *z, *wq;
    const int *parent;
    const double *atoms;      // natoms x 3
    const double *rnn;        // natoms nearest-neighbour distances
    const int *nbr;           // natoms x (natoms - 1): the other atoms of each atom by distance
    const double *nbr_r;      // their distances
    double *w;
    int64_t npts;
    int natoms;
    int scheme;
    Profiler *prof;
};
cudaError_t launch_partition_weights(const WeightsArgs &a, cudaStream_t s);

// One molecule of a grouped launch over several molecules (gbxc_integrate_many): its P, its
// V accumulator, its P as double-float planes (tensor-core form), function count and functional.
struct MolRef {
    const double *P;
    double *Vacc;
    const float2 *pdf;                // P region of the tensor-core form (mixed.h: pdf_slices)
    int nbf;
    int functional;
};

// Tiles of one chunk are [t0, t1); slab rows are tile_row[t] - row0.  A grouped chunk spans the
// batches of several molecules in one combined plan: batch_mol[j] names batch j's molecule in
// mols[], whose P, V_acc, nbf and functional then replace the fields below.
struct ChunkArgs {
    DevPlan plan;
    const DevShell *shells;
    int nbf;
    int64_t t0, t1, row0, rows;
    int max_nfunc;            // largest N_b^j of the chunk's batches
    int functional;
    const double *P;          // nbf x nbf
    double *Vacc;             // nbf x nbf accumulator (W = Z^T Phi scattered, not yet symmetrised)
    double *tileE, *tileN;    // per-tile partial sums (indexed by global tile id)
    void *scratch;            // chunk slabs
    const int *vtasks;        // 5 ints per task: batch, mb, nb, t0, t1
    int nvtasks;
    Profiler *prof;
    const int *batch_mol = nullptr;   // grouped chunks only (device)
    const MolRef *mols = nullptr;     // grouped chunks only (device)
};
cudaError_t launch_fp64_chunk(const ChunkArgs &a, cudaStream_t s);
// Spin-unrestricted chunk: a.P / a.Vacc carry spin a, Pb / Vacc_b spin b.
cudaError_t launch_fp64_chunk_uks(const ChunkArgs &a, const double *Pb, double *Vacc_b, cudaStream_t s);
// Meta-GGA chunk (a.functional is a meta-GGA): X and the three Y^k = (d_k Phi) P^j, rho, tau,
// the functional, Z and W^k, and four V contractions into a.Vacc.
cudaError_t launch_fp64_chunk_mgga(const ChunkArgs &a, cudaStream_t s);

struct FinishArgs {
    const double *Vacc;
    double *V;                // nbf x nbf symmetric result
    int nbf;
    const double *tileE, *tileN;
    const int64_t *batch_tile;
    int b0, b1;
    double *Eb, *Nb;          // per batch (nbatch), device
    double *tot;              // [E, N] device
    Profiler *prof;
};
cudaError_t launch_finish(const FinishArgs &a, cudaStream_t s);

// Allocation-free float64 variant: the static device scratch (slab address and size, and the
// address of its non-finite-P flag), one chunk of the float64 pipeline with per-tile V tasks,
// the in-place V + V^T, and {E, N} <- NaN if the flag is set.
cudaError_t noalloc_scratch(void **ptr, size_t *bytes, double **flag);
cudaError_t launch_poison_if_flagged(const double *flag, double *EN, cudaStream_t s);
cudaError_t launch_fp64_chunk_noalloc(const ChunkArgs &a, cudaStream_t s);
cudaError_t launch_symmetrize_inplace(double *V, int nbf, cudaStream_t s);
// V = V_acc + V_acc^T
cudaError_t launch_symmetrize(const double *Vacc, double *V, int nbf, cudaStream_t s);
// *flag <- 1.0 if P[0 .. n) holds a NaN or an infinity (zeroed first when reset).
cudaError_t launch_check_finite(const double *P, int64_t n, double *flag, bool reset, cudaStream_t s);

}  // namespace gbxc
