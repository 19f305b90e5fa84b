// Batching and screening plan on the GPU (Sec. 2.2 micro-batching and the grid-partition
// figure, Eq. rcut, Algorithm 1): the atomic grids, the recursive cuboid subdivision of each
// atom's points and Algorithm 1 on every leaf, as device kernels whose results are identical
// to the host planner's (host_plan.cpp).  Identity holds because every step is the same IEEE
// float64 operation in the same order (explicitly rounded intrinsics, no contraction) or an
// exact one (comparisons, minima and maxima, stable partitions):
//
//   expand_grid      x = c + r_k u_q, w^q = w_k w_q from the host-built 1-D tables
//   subdivide_atoms  one block per atom walks the atom's cell tree depth first (a stack in
//                    shared memory), so leaves come out in the host recursion's order; a
//                    cell's points are split into its 27 or 8 children by a stable counting
//                    scatter, which keeps every child's points in ascending order
//   screen_leaves    tight box of each leaf, Algorithm 1 for every shell -> bit masks
//   layout_points    the points of the merged batches in batch order, left on the device
//
// Merging leaves with equal shell lists and the batch metadata (function lists, work, tiles)
// run on the host, shared with the host planner (merge_leaves, batch_metadata); only leaf
// ranges and shell masks cross to the host.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace gbxc {
namespace {

constexpr int PT = 256;                       // threads per block
constexpr int NW = PT / 32;
constexpr int kMaxDepth = 16;
constexpr int STACK = kMaxDepth * 26 + 2;     // depth-first: at most 26 pending siblings per level

struct Tables {
    const double *r, *wr, *ux, *uy, *uz, *wa;
    int nang;
};

__global__ void expand_grid(const double *__restrict__ atoms, Tables T, int64_t npa, int64_t npts,
                            double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                            double *__restrict__ wq, int *__restrict__ parent) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t A = i / npa, rem = i % npa;
        const int k = (int)(rem / T.nang), q = (int)(rem % T.nang);
        const double rk = T.r[k];
        x[i] = __dadd_rn(atoms[3 * A], __dmul_rn(rk, T.ux[q]));
        y[i] = __dadd_rn(atoms[3 * A + 1], __dmul_rn(rk, T.uy[q]));
        z[i] = __dadd_rn(atoms[3 * A + 2], __dmul_rn(rk, T.uz[q]));
        wq[i] = __dmul_rn(T.wr[k], T.wa[q]);
        parent[i] = (int)A;
    }
}

struct CellRec {
    int b, e, depth, pad;
    double lo[3], hi[3];
};

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Tight box of points idx[b, e) (or of b .. e - 1 themselves when idx is null), by the whole
// block; the result is in lo/hi (shared).  Minima and maxima are exact in any order.
__device__ void block_box(const double *x, const double *y, const double *z, const int *idx, int64_t b, int64_t e,
                          double *lo, double *hi, double (*red)[NW]) {
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
        const int64_t q = idx ? idx[p] : p;
        const double v[3] = {x[q], y[q], z[q]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], v[d]);
            mx[d] = fmax(mx[d], v[d]);
        }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        mn[d] = warp_min(mn[d]);
        mx[d] = warp_max(mx[d]);
        if (lane == 0) {
            red[d][w] = mn[d];
            red[3 + d][w] = mx[d];
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        double a = red[d][0], c = red[3 + d][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            a = fmin(a, red[d][k]);
            c = fmax(c, red[3 + d][k]);
        }
        lo[d] = a;
        hi[d] = c;
    }
    __syncthreads();
}

// One block per atom; leaves (ranges of idx) go to leaf_b/leaf_e at the atom's offset.
__global__ void __launch_bounds__(PT) subdivide_atoms(const double *__restrict__ x, const double *__restrict__ y,
                                                      const double *__restrict__ z, const double *__restrict__ atoms,
                                                      int natoms, int64_t npa, int max_batch, int *__restrict__ idx,
                                                      int *__restrict__ tmp, int *__restrict__ leaf_b,
                                                      int *__restrict__ leaf_e, int *__restrict__ leaf_n,
                                                      int *__restrict__ err) {
    __shared__ CellRec stack[STACK];
    __shared__ CellRec cur;
    __shared__ int sp, nleaf;
    __shared__ double cuts[3][4];
    __shared__ double red[6][NW];
    __shared__ double box_lo[3], box_hi[3];
    __shared__ int cnt[27], offs[27], run[27], tot[27];
    __shared__ int wcnt[NW][27];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * npa;
    for (int64_t p = tid; p < npa; p += PT) idx[base + p] = (int)(base + p);
    block_box(x, y, z, nullptr, base, base + npa, box_lo, box_hi, red);
    if (tid == 0) {
        sp = 0;
        nleaf = 0;
        CellRec r;
        r.b = (int)base;
        r.e = (int)(base + npa);
        r.depth = 0;
        r.pad = 0;
        for (int d = 0; d < 3; ++d) {
            r.lo[d] = box_lo[d];
            r.hi[d] = box_hi[d];
        }
        stack[sp++] = r;
    }
    __syncthreads();
    while (true) {
        if (tid == 0) {
            if (sp > 0) cur = stack[--sp];
            else cur.b = -1;
        }
        __syncthreads();
        if (cur.b < 0) break;
        const int b = cur.b, e = cur.e;
        if (e - b <= max_batch || cur.depth >= kMaxDepth) {   // a leaf
            if (tid == 0) {
                leaf_b[base + nleaf] = b;
                leaf_e[base + nleaf] = e;
                ++nleaf;
            }
            __syncthreads();
            continue;
        }
        // a cell holding any atomic centre (inclusive bounds) is cut in thirds, any other in halves
        int inside = 0;
        for (int a = tid; a < natoms; a += PT) {
            const double *R = atoms + 3 * a;
            if (cur.lo[0] <= R[0] && R[0] <= cur.hi[0] && cur.lo[1] <= R[1] && R[1] <= cur.hi[1] &&
                cur.lo[2] <= R[2] && R[2] <= cur.hi[2])
                inside = 1;
        }
        const int thirds = __syncthreads_or(inside);
        const int nc = thirds ? 3 : 2, nch = nc * nc * nc;
        if (tid < 3) {
            const double lo = cur.lo[tid], hi = cur.hi[tid];
            cuts[tid][0] = lo;
            if (thirds) {
                cuts[tid][1] = __dadd_rn(lo, __ddiv_rn(__dsub_rn(hi, lo), 3.0));
                cuts[tid][2] = __dadd_rn(lo, __ddiv_rn(__dmul_rn(2.0, __dsub_rn(hi, lo)), 3.0));
                cuts[tid][3] = hi;
            } else {
                cuts[tid][1] = __dmul_rn(0.5, __dadd_rn(lo, hi));
                cuts[tid][2] = hi;
            }
        }
        if (tid < 27) {
            cnt[tid] = 0;
            run[tid] = 0;
        }
        __syncthreads();
        auto child_of = [&](int q) {
            const double v[3] = {x[q], y[q], z[q]};
            int c[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int k = 0;
                for (int s = 1; s < nc; ++s) k += (v[d] >= cuts[d][s]) ? 1 : 0;
                c[d] = k;
            }
            return (c[2] * nc + c[1]) * nc + c[0];
        };
        for (int p = b + tid; p < e; p += PT) atomicAdd(&cnt[child_of(idx[p])], 1);
        __syncthreads();
        if (tid == 0) {
            int o = 0;
            for (int c = 0; c < nch; ++c) {
                offs[c] = o;
                o += cnt[c];
            }
        }
        __syncthreads();
        // stable scatter, PT points at a time in order: rank = earlier points of the same
        // child in this chunk (lower lanes of the warp, then earlier warps)
        for (int c0 = b; c0 < e; c0 += PT) {
            const int p = c0 + tid;
            const bool act = p < e;
            const int val = act ? idx[p] : 0;
            const int cid = act ? child_of(val) : 31;
            const unsigned same = __match_any_sync(0xffffffffu, cid);
            const int lower = __popc(same & ((1u << lane) - 1u));
            for (int k = tid; k < NW * 27; k += PT) (&wcnt[0][0])[k] = 0;
            __syncthreads();
            if (act && lower == 0) wcnt[w][cid] = __popc(same);
            __syncthreads();
            if (tid < nch) {
                int acc = 0;
                for (int ww = 0; ww < NW; ++ww) {
                    const int v = wcnt[ww][tid];
                    wcnt[ww][tid] = acc;
                    acc += v;
                }
                tot[tid] = acc;
            }
            __syncthreads();
            if (act) tmp[b + offs[cid] + run[cid] + wcnt[w][cid] + lower] = val;
            __syncthreads();
            if (tid < nch) run[tid] += tot[tid];
            __syncthreads();
        }
        for (int p = b + tid; p < e; p += PT) idx[p] = tmp[p];
        __syncthreads();
        if (tid == 0) {   // children pushed last-first, so they are visited in z-, y-, x-order
            for (int c = nch - 1; c >= 0; --c) {
                if (cnt[c] == 0) continue;
                if (sp >= STACK) {
                    atomicOr(err, 1);
                    continue;
                }
                const int ix = c % nc, iy = (c / nc) % nc, iz = c / (nc * nc);
                CellRec r;
                r.b = b + offs[c];
                r.e = r.b + cnt[c];
                r.depth = cur.depth + 1;
                r.pad = 0;
                r.lo[0] = cuts[0][ix];
                r.lo[1] = cuts[1][iy];
                r.lo[2] = cuts[2][iz];
                r.hi[0] = cuts[0][ix + 1];
                r.hi[1] = cuts[1][iy + 1];
                r.hi[2] = cuts[2][iz + 1];
                stack[sp++] = r;
            }
        }
        __syncthreads();
    }
    if (tid == 0) leaf_n[blockIdx.x] = nleaf;
}

// Leaves of all atoms, atom by atom, into one list.
__global__ void gather_leaves(const int *__restrict__ leaf_b, const int *__restrict__ leaf_e,
                              const int *__restrict__ leaf_n, const int64_t *__restrict__ leaf_ofs, int64_t npa,
                              int *__restrict__ out_b, int *__restrict__ out_e) {
    const int A = blockIdx.x;
    for (int k = threadIdx.x; k < leaf_n[A]; k += blockDim.x) {
        out_b[leaf_ofs[A] + k] = leaf_b[(int64_t)A * npa + k];
        out_e[leaf_ofs[A] + k] = leaf_e[(int64_t)A * npa + k];
    }
}

// Algorithm 1 (typo and inverted return corrected): keep shell s iff r_cut^2 minus the
// squared distance from its centre to the leaf's tight box is >= 0; one block per leaf,
// one bit per shell.
__global__ void __launch_bounds__(PT) screen_leaves(const double *__restrict__ x, const double *__restrict__ y,
                                                    const double *__restrict__ z, const int *__restrict__ idx,
                                                    const int *__restrict__ lb, const int *__restrict__ le,
                                                    const double *__restrict__ centres, const double *__restrict__ rcut,
                                                    int nsh, int nwords, uint32_t *__restrict__ mask) {
    __shared__ double red[6][NW];
    __shared__ double V[3], W[3];
    const int l = blockIdx.x;
    block_box(x, y, z, idx, lb[l], le[l], V, W, red);
    const int lane = threadIdx.x & 31;
    for (int wi = threadIdx.x >> 5; wi < nwords; wi += NW) {
        const int s = wi * 32 + lane;
        bool keep = false;
        if (s < nsh) {
            const double rc = rcut[s];
            double d = __dmul_rn(rc, rc);
            for (int p = 0; p < 3; ++p) {
                const double R = centres[3 * s + p];
                if (R < V[p]) {
                    const double t = __dsub_rn(R, V[p]);
                    d = __dsub_rn(d, __dmul_rn(t, t));
                } else if (R > W[p]) {
                    const double t = __dsub_rn(R, W[p]);
                    d = __dsub_rn(d, __dmul_rn(t, t));
                }
            }
            keep = d >= 0.0;
        }
        const unsigned bits = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) mask[(int64_t)l * nwords + wi] = bits;
    }
}

// Points of the merged batches in batch order: leaf order[k] goes to out_ofs[k].
__global__ void layout_points(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                              const double *__restrict__ wq, const int *__restrict__ parent, const int *__restrict__ idx,
                              const int *__restrict__ lb, const int *__restrict__ le, const int *__restrict__ order,
                              const int64_t *__restrict__ out_ofs, DevPoints out) {
    const int l = order[blockIdx.x];
    const int b = lb[l], n = le[l] - b;
    const int64_t o = out_ofs[blockIdx.x];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int p = idx[b + t];
        out.x[o + t] = x[p];
        out.y[o + t] = y[p];
        out.z[o + t] = z[p];
        out.wq[o + t] = wq[p];
        out.parent[o + t] = parent[p];
        out.point_index[o + t] = p;
    }
}

template <typename T>
struct DevBuf {
    T *p = nullptr;
    ~DevBuf() { cudaFree(p); }
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)); }
};

template <typename T>
cudaError_t upload(DevBuf<T> &b, const std::vector<T> &v, cudaStream_t s) {
    cudaError_t e = b.alloc(v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

template <typename T>
cudaError_t download(std::vector<T> &v, const T *p, size_t n, cudaStream_t s) {
    v.resize(n);
    if (!n) return cudaSuccess;
    return cudaMemcpyAsync(v.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s);
}

#define DP_CHECK(expr)                         \
    do {                                       \
        cudaError_t e_ = (expr);               \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

}  // namespace

cudaError_t device_plan(const std::vector<double> &xyz, const std::vector<DevShell> &shells,
                        const std::vector<double> &rcut, const gbxc_grid_spec &spec, HostPlan &plan,
                        DevPoints &out, cudaStream_t s, int *status) {
    *status = 0;
    out = DevPoints{};
    const int natoms = (int)(xyz.size() / 3);
    GridTables T;
    grid_tables(spec, T);
    const int64_t nang = (int64_t)T.ux.size(), npa = (int64_t)spec.nrad * nang, npts = natoms * npa;
    if (npts >= (int64_t)1 << 31 || natoms == 0 || npa == 0) {
        *status = 1;
        return cudaSuccess;
    }
    DevBuf<double> d_atoms, d_r, d_wr, d_ux, d_uy, d_uz, d_wa, dx, dy, dz, dwq, d_cent, d_rcut;
    DevBuf<int> d_parent, d_idx, d_tmp, d_lb, d_le, d_ln, d_err, d_fb, d_fe, d_order;
    DevBuf<int64_t> d_lofs, d_oofs;
    DevBuf<uint32_t> d_mask;
    DP_CHECK(upload(d_atoms, xyz, s));
    DP_CHECK(upload(d_r, T.r, s));
    DP_CHECK(upload(d_wr, T.wr, s));
    DP_CHECK(upload(d_ux, T.ux, s));
    DP_CHECK(upload(d_uy, T.uy, s));
    DP_CHECK(upload(d_uz, T.uz, s));
    DP_CHECK(upload(d_wa, T.wa, s));
    DP_CHECK(dx.alloc(npts));
    DP_CHECK(dy.alloc(npts));
    DP_CHECK(dz.alloc(npts));
    DP_CHECK(dwq.alloc(npts));
    DP_CHECK(d_parent.alloc(npts));
    DP_CHECK(d_idx.alloc(npts));
    DP_CHECK(d_tmp.alloc(npts));
    DP_CHECK(d_lb.alloc(npts));
    DP_CHECK(d_le.alloc(npts));
    DP_CHECK(d_ln.alloc(natoms));
    DP_CHECK(d_err.alloc(1));
    DP_CHECK(cudaMemsetAsync(d_err.p, 0, sizeof(int), s));
    Tables tb{d_r.p, d_wr.p, d_ux.p, d_uy.p, d_uz.p, d_wa.p, (int)nang};
    expand_grid<<<(unsigned)std::min<int64_t>((npts + PT - 1) / PT, 4096), PT, 0, s>>>(d_atoms.p, tb, npa, npts, dx.p,
                                                                                       dy.p, dz.p, dwq.p, d_parent.p);
    DP_CHECK(cudaGetLastError());
    subdivide_atoms<<<natoms, PT, 0, s>>>(dx.p, dy.p, dz.p, d_atoms.p, natoms, npa, spec.max_batch, d_idx.p, d_tmp.p,
                                          d_lb.p, d_le.p, d_ln.p, d_err.p);
    DP_CHECK(cudaGetLastError());
    std::vector<int> ln;
    int herr = 0;
    DP_CHECK(download(ln, d_ln.p, natoms, s));
    DP_CHECK(cudaMemcpyAsync(&herr, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DP_CHECK(cudaStreamSynchronize(s));
    if (herr) {
        *status = 2;
        return cudaSuccess;
    }
    std::vector<int64_t> lofs(natoms + 1, 0);
    for (int A = 0; A < natoms; ++A) lofs[A + 1] = lofs[A] + ln[A];
    const int64_t nleaf = lofs[natoms];
    DP_CHECK(upload(d_lofs, lofs, s));
    DP_CHECK(d_fb.alloc(nleaf));
    DP_CHECK(d_fe.alloc(nleaf));
    gather_leaves<<<natoms, PT, 0, s>>>(d_lb.p, d_le.p, d_ln.p, d_lofs.p, npa, d_fb.p, d_fe.p);
    DP_CHECK(cudaGetLastError());
    const int nsh = (int)shells.size(), nwords = (nsh + 31) / 32;
    std::vector<double> cent(3 * (size_t)nsh);
    for (int k = 0; k < nsh; ++k)
        for (int d = 0; d < 3; ++d) cent[3 * k + d] = shells[k].c[d];
    DP_CHECK(upload(d_cent, cent, s));
    DP_CHECK(upload(d_rcut, rcut, s));
    DP_CHECK(d_mask.alloc((size_t)nleaf * nwords));
    if (nleaf > 0 && nwords > 0)
        screen_leaves<<<(unsigned)nleaf, PT, 0, s>>>(dx.p, dy.p, dz.p, d_idx.p, d_fb.p, d_fe.p, d_cent.p, d_rcut.p,
                                                     nsh, nwords, d_mask.p);
    DP_CHECK(cudaGetLastError());
    std::vector<int> fb, fe;
    std::vector<uint32_t> mask;
    DP_CHECK(download(fb, d_fb.p, nleaf, s));
    DP_CHECK(download(fe, d_fe.p, nleaf, s));
    DP_CHECK(download(mask, d_mask.p, (size_t)nleaf * nwords, s));
    DP_CHECK(cudaStreamSynchronize(s));
    // merge on the host (small: one shell list per leaf), then the points in batch order on
    // the device
    std::vector<std::vector<int>> keeps(nleaf), bshells, bleaves;
    for (int64_t l = 0; l < nleaf; ++l)
        for (int k = 0; k < nsh; ++k)
            if (mask[l * nwords + (k >> 5)] >> (k & 31) & 1u) keeps[l].push_back(k);
    merge_leaves(keeps, bshells, bleaves);
    std::vector<int> order;
    std::vector<int64_t> oofs, bsize;
    int64_t pos = 0;
    for (const auto &bl : bleaves) {
        const int64_t p0 = pos;
        for (int l : bl) {
            order.push_back(l);
            oofs.push_back(pos);
            pos += fe[l] - fb[l];
        }
        bsize.push_back(pos - p0);
    }
    DP_CHECK(upload(d_order, order, s));
    DP_CHECK(upload(d_oofs, oofs, s));
    DevPoints pts;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&pts.x, npts * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&pts.y, npts * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&pts.z, npts * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&pts.wq, npts * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&pts.parent, npts * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&pts.point_index, npts * sizeof(int64_t));
    if (e == cudaSuccess && nleaf > 0)
        layout_points<<<(unsigned)nleaf, PT, 0, s>>>(dx.p, dy.p, dz.p, dwq.p, d_parent.p, d_idx.p, d_fb.p, d_fe.p,
                                                    d_order.p, d_oofs.p, pts);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(pts.x);
        cudaFree(pts.y);
        cudaFree(pts.z);
        cudaFree(pts.wq);
        cudaFree(pts.parent);
        cudaFree(pts.point_index);
        return e;
    }
    plan.x.clear(); plan.y.clear(); plan.z.clear(); plan.wq.clear();
    plan.parent.clear(); plan.point_index.clear();
    plan.nleaf = (int)nleaf;
    batch_metadata((size_t)natoms, shells, bshells, bsize, plan);
    out = pts;
    return cudaSuccess;
}

}  // namespace gbxc
