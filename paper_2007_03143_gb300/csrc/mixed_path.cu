// Tensor-core form of the batched integration (Algorithm 4) on sm_103a.
//
// The two contractions run on the 5th-generation tensor cores (tcgen05.mma, bf16 inputs,
// fp32 accumulators in tensor memory, operands staged by TMA with the 32-byte swizzle):
//
//   X^j = P^j Phi^j (Eq. x_mat)      Ozaki-style exact slicing.  Every row of Phi (a grid
//        point) and of P^j (a function) is scaled by a power of two to |v| <= 1 and cut
//        into 5 integer slices v = sum_s q_s 2^-(6+7s) (34 bits, |q_s| <= 64 for s <= 2).  The 15 slice products
//        with s + t <= 4 are issued per K step into four accumulators: level d = s + t for
//        d = 0, 1, 2, whose partial sums are integer multiples of 2^-(12+7d) below 2^24
//        units so the fp32 sums are exact, and levels 3-4 together (rounded, 2^-21 below
//        level 0).  X = (acc0 + acc1 + acc2 + acc3) 2^(e_i + f_mu), summed in double-float.
//        The exactness needs K <= 1184 functions per accumulation; a batch with more
//        functions runs its K in segments of 1184, each exact, added in double-float.
//   W^j = Z^jT Phi^j (Eq. vxc_batch) the same slicing over K = grid points (at most 8 tiles =
//        1024 points per V task, so levels 0-2 stay exact).  Phi is taken from the X
//        contraction's slices (Phi_i,nu 2^-e_i, one exponent per point), read MN-major, and
//        Z_i,mu 2^e_i is sliced per function over the task's points, so the product needs
//        only Z's exponents; the meta-GGA terms slice both operands per function.
//
// Everything that decides E_xc to 1e-9 stays above fp32 precision: collocation in
// float64 written as double-float pairs, rho and grad rho summed in double-float, the
// partition weights, the functional and all E/N/V accumulation in float64.
//
// Kernels per chunk of tiles: pslice (P^j row slices), colloc (Phi, grad Phi, Phi slices),
// xgemm (tcgen05), rho (rho, grad rho, functional, E/N partials, per-point Z coefficients),
// z_slice (Z 2^e_i in double-float, group exponent maxima, Z slices per V task), vgemm
// (tcgen05, scatter into V_acc with float64 atomics).  The spin-unrestricted form runs z_slice
// once per spin; the meta-GGA form forms Z and W^k in its rho kernel (two passes over Phi) and
// slices them with slice_v.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <utility>

#include "mixed.h"
#include "dfloat.cuh"
#include "group.cuh"
#include "slicing.cuh"
#include "solid_harmonics.cuh"
#include "umma.cuh"
#include "xc_functional.cuh"

namespace gbxc {
namespace {

using slc::NSL;
using slc::pow2f;
using slc::scale2;
using slc::slice5;
using slc::exp_of;
constexpr int XSEG = 74;        // 16-wide K steps per X segment: K <= 1184 functions keeps the
                                // exact accumulator levels exact; longer K runs in segments
constexpr int MGGA_FB = 1184;   // functions per block of the meta-GGA kernel's shared maxima
constexpr int VKS = 8;          // tiles per V task: K <= 1024 points keeps levels 0-2 exact
// The functional runs in float64 at every point: float32 PBE above rho = 1e-8 was measured
// at |dE_xc| = 6e-6 Eh on the 16-water workload, above the 1e-6 Eh bound of this form.

// ---------------------------------------------------------------- scratch layout
struct MixedSlabs {
    float2 *phi;            // [rows][128]: Phi as (hi, lo) pairs
    float *ghi;             // 3 planes [rows][128]: hi words of dPhi/dx, /dy, /dz
    __nv_bfloat16 *glo;     // 3 planes [rows][128]: their lo words rounded to bf16 (hi + lo
                            // then carries about 32 bits, enough for grad rho; the Z pass
                            // reads the hi words alone)
    float2 *x;              // 1 plane [rows][128]: X (later Z) as (hi, lo)
    __nv_bfloat16 *ax;      // 5 planes [4 rows][32]: Phi slices, K-blocked per tile
    __nv_bfloat16 *vz;      // 5 planes [4 rows][32]: Z slices, point-blocked per tile
    __nv_bfloat16 *vphi;    // 5 planes [4 rows][32]: Phi slices, point-blocked per tile (the
                            // meta-GGA form; the others read Phi from ax)
    int *zexp, *fexp;       // [rows]: per tile and function, exponent of max |Z|, |Phi| over
                            // the tile's points (group maxima on the group's first tile; fexp
                            // in the meta-GGA form only)
    int *pexp;              // [tiles][128] point exponents e_i
};

__host__ __device__ inline MixedSlabs mixed_slabs(void *base, int64_t rows) {
    char *p = static_cast<char *>(base);
    MixedSlabs s;
    s.phi = reinterpret_cast<float2 *>(p);
    p += (size_t)2 * rows * TILE * 4;
    s.ghi = reinterpret_cast<float *>(p);
    p += (size_t)3 * rows * TILE * 4;
    s.glo = reinterpret_cast<__nv_bfloat16 *>(p);
    p += (size_t)3 * rows * TILE * 2;
    s.x = reinterpret_cast<float2 *>(p);
    p += (size_t)2 * rows * TILE * 4;
    s.ax = reinterpret_cast<__nv_bfloat16 *>(p);
    p += (size_t)NSL * rows * TILE * 2;
    s.vz = reinterpret_cast<__nv_bfloat16 *>(p);
    p += (size_t)NSL * rows * TILE * 2;
    s.vphi = reinterpret_cast<__nv_bfloat16 *>(p);
    p += (size_t)NSL * rows * TILE * 2;
    s.zexp = reinterpret_cast<int *>(p);
    p += (size_t)rows * 4;
    s.fexp = reinterpret_cast<int *>(p);
    p += (size_t)rows * 4;
    s.pexp = reinterpret_cast<int *>(p);
    return s;
}

struct MixedArgs {
    MixedSlabs s;
    int64_t rows;
    int j0;                      // first batch of the chunk
    const int64_t *pofs;         // per batch of the chunk: first row of its P slices
    __nv_bfloat16 *pslices;      // 5 planes, plane pitch pplane rows of 32
    int64_t pplane;
    const float2 *pdf;           // the P region (pairs, slices, row exponents)
    int *err;
    int keep_z;                  // z_slice also writes Z over X (per-batch debugging copy)
    int pad_all;                 // the collocation writes zeros for every padding point of a tile
                                 // (the meta-GGA kernels read all 128 points); otherwise only up
                                 // to the count rounded up to 8 (z_slice reads 8-point groups),
                                 // and the X epilogue stores live rows only
};

__device__ __forceinline__ int pad32(int n) { return (n + 31) & ~31; }

// ---------------------------------------------------------------- double-float helpers
using dfl::df;
using dfl::two_sum;
__device__ __forceinline__ df df_mul(df a, df b) { return dfl::mul(a, b); }
__device__ __forceinline__ df df_add(df a, df b) { return dfl::add(a, b); }
__device__ __forceinline__ double df_to_d(df a) { return dfl::to_double(a); }
__device__ __forceinline__ df d_to_df(double d) { return dfl::from_double(d); }

// ---------------------------------------------------------------- pslice
// The P region once per integration (the only float64 pass over P), one block per row mu:
// the double-float pairs (hi, lo) of the row, the exponent of its largest |P_mu,nu| over all
// nu, and the 5 slices of every element in that scale.  The X contraction gathers its P^j
// operand from these planes: P^j's row maximum over a batch's functions is at most the row's
// maximum over all functions, so a batch's slices lose only the bits of that ratio (none when
// the row peaks inside the batch, as a density matrix's rows do near the diagonal).
constexpr int PP_THREADS = 256;
__global__ void __launch_bounds__(PP_THREADS) p_prepare(const double *__restrict__ P, float2 *__restrict__ pdf,
                                                       int nbf) {
    const int mu = blockIdx.x;
    const double *row = P + (size_t)mu * nbf;
    float2 *drow = pdf + (size_t)mu * nbf;
    float mx = 0.f;
    for (int nu = threadIdx.x; nu < nbf; nu += PP_THREADS) {
        const df d = d_to_df(row[nu]);
        drow[nu] = make_float2(d.h, d.l);
        mx = fmaxf(mx, fabsf(d.h));
    }
    __shared__ float red[PP_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
#pragma unroll
    for (int w = 0; w < PP_THREADS / 32; ++w) mx = fmaxf(mx, red[w]);
    const int e = exp_of(mx);
    char *base = reinterpret_cast<char *>(pdf);
    if (threadIdx.x == 0) reinterpret_cast<int *>(base + pdf_exps_offset(nbf))[mu] = e;
    uint4 *sl = reinterpret_cast<uint4 *>(base + pdf_slices_offset(nbf)) + (size_t)mu * nbf;
    for (int nu = threadIdx.x; nu < nbf; nu += PP_THREADS) {
        const float2 v = drow[nu];
        float q[NSL];
        slice5(v.x, v.y, e, q);
        __nv_bfloat162 b01 = __floats2bfloat162_rn(q[0], q[1]), b23 = __floats2bfloat162_rn(q[2], q[3]);
        __nv_bfloat162 b4 = __floats2bfloat162_rn(q[4], 0.f);
        sl[nu] = make_uint4(*reinterpret_cast<uint32_t *>(&b01), *reinterpret_cast<uint32_t *>(&b23),
                            *reinterpret_cast<uint32_t *>(&b4), 0u);
    }
}

// P^j's slices for the X contraction's B operand, gathered from the P region (p_prepare): two
// rows mu of P^j per warp (lanes 0-15 the first, 16-31 the second), eight rows per block
// (tasks: batch, first row of eight), two consecutive nu per lane, so that each slice plane of
// the two rows (two consecutive 64-byte rows of the K-blocked layout) is one 128-byte store
// per warp.  The slices are P's own, cut with the row's exponent over all functions, so no
// pass over the batch's row is needed first.  Rows and columns past N_b^j are zeros.
constexpr int PS_WARPS = 4;
constexpr int PS_ROWS = 2 * PS_WARPS;
__global__ void __launch_bounds__(32 * PS_WARPS) pslice_kernel(ChunkArgs a, MixedArgs m, const int *tasks) {
    const int jl = tasks[2 * blockIdx.x], mu0 = tasks[2 * blockIdx.x + 1];
    const int j = m.j0 + jl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hl = lane & 15;
    const int64_t f0 = a.plan.func_ptr[j];
    const int n = (int)(a.plan.func_ptr[j + 1] - f0);
    const int np = pad32(n);
    const int mu = mu0 + 2 * warp + (lane >> 4);   // < np: np is a multiple of 32, mu0 of 8
    const int *F = a.plan.func_idx + f0;
    const float2 *pdf = m.pdf;
    int nbf = a.nbf;
    if (a.batch_mol) {   // grouped chunk: the batch's own molecule
        const MolRef r = mol_of(a, j);
        pdf = r.pdf;
        nbf = r.nbf;
    }
    const uint4 *tab = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(pdf) + pdf_slices_offset(nbf));
    const uint4 *row = tab + ((mu < n) ? (size_t)F[mu] * nbf : 0);
    const int64_t pofs = m.pofs[jl];
    for (int kb = 0; kb < np / 32; ++kb) {
        const int nu = kb * 32 + 2 * hl;
        const bool in0 = mu < n && nu < n, in1 = mu < n && nu + 1 < n;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        const uint4 p0 = in0 ? __ldg(row + F[nu]) : z;
        const uint4 p1 = in1 ? __ldg(row + F[nu + 1]) : z;
        // slice s of an element: half s of (x, y, z); the pair (nu, nu + 1) of each plane
        const uint32_t w[NSL] = {__byte_perm(p0.x, p1.x, 0x5410), __byte_perm(p0.x, p1.x, 0x7632),
                                 __byte_perm(p0.y, p1.y, 0x5410), __byte_perm(p0.y, p1.y, 0x7632),
                                 __byte_perm(p0.z, p1.z, 0x5410)};
        const size_t o = (size_t)(pofs + (int64_t)kb * np + mu) * 32 + 2 * hl;
#pragma unroll
        for (int s = 0; s < NSL; ++s) *reinterpret_cast<uint32_t *>(m.pslices + (size_t)s * m.pplane * 32 + o) = w[s];
    }
}

// ---------------------------------------------------------------- collocation
// x^a y^b z^c from the power tables (index >= 1; the zeroth powers are never read); `one`
// tells that all exponents are 0, i.e. the value is exactly 1 and need not multiply anything.
__device__ __forceinline__ df pow3(const df *xp, const df *yp, const df *zp, int a, int b, int c, bool &one) {
    one = (a == 0 && b == 0 && c == 0);
    df r{1.f, 0.f};
    bool have = false;
    if (a > 0) {
        r = xp[a];
        have = true;
    }
    if (b > 0) {
        r = have ? df_mul(r, yp[b]) : yp[b];
        have = true;
    }
    if (c > 0) r = have ? df_mul(r, zp[c]) : zp[c];
    return r;
}

// The (L+1)(L+2)/2 Cartesian functions of one shell at one point (Eq. gau_cart) and their
// gradients, from X, Y, Z = r - A and the radial sums g = sum_k d_k e_k and
// h = sum_k (-2 alpha_k d_k) e_k (e_k = exp(-alpha_k r^2)):
//   phi = x^l y^m z^n g,  d/dx phi = l x^(l-1) y^m z^n g + x^(l+1) y^m z^n h  (y, z alike).
// L is a template parameter so every monomial index is a compile-time constant.
template <int L>
__device__ __forceinline__ void colloc_shell(df X, df Y, df Z, df g, df h, const MixedSlabs &sl, size_t plane,
                                             size_t o, bool live, float &mx) {
    df xp[L + 1], yp[L + 1], zp[L + 1];
    xp[0] = yp[0] = zp[0] = {1.f, 0.f};
#pragma unroll
    for (int k = 1; k <= L; ++k) {
        xp[k] = df_mul(xp[k - 1], X);
        yp[k] = df_mul(yp[k - 1], Y);
        zp[k] = df_mul(zp[k - 1], Z);
    }
    const df Xh = df_mul(X, h), Yh = df_mul(Y, h), Zh = df_mul(Z, h);
    int f = 0;
#pragma unroll
    for (int l = L; l >= 0; --l)
#pragma unroll
        for (int mm = L - l; mm >= 0; --mm) {
            const int nn = L - l - mm;
            // after unrolling every exponent is a constant: factors equal to 1 are skipped
            bool one;
            const df mono = pow3(xp, yp, zp, l, mm, nn, one);
            df v[4];
            v[0] = one ? g : df_mul(mono, g);
            v[1] = one ? Xh : df_mul(mono, Xh);
            v[2] = one ? Yh : df_mul(mono, Yh);
            v[3] = one ? Zh : df_mul(mono, Zh);
            if (l > 0) {
                const df b = pow3(xp, yp, zp, l - 1, mm, nn, one);
                df t = one ? g : df_mul(b, g);
                if (l > 1) t = dfl::mul_f(t, (float)l);
                v[1] = df_add(v[1], t);
            }
            if (mm > 0) {
                const df b = pow3(xp, yp, zp, l, mm - 1, nn, one);
                df t = one ? g : df_mul(b, g);
                if (mm > 1) t = dfl::mul_f(t, (float)mm);
                v[2] = df_add(v[2], t);
            }
            if (nn > 0) {
                const df b = pow3(xp, yp, zp, l, mm, nn - 1, one);
                df t = one ? g : df_mul(b, g);
                if (nn > 1) t = dfl::mul_f(t, (float)nn);
                v[3] = df_add(v[3], t);
            }
            const size_t of = o + (size_t)f * TILE;
            sl.phi[of] = live ? make_float2(v[0].h, v[0].l) : make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sl.ghi[c * plane + of] = live ? v[c + 1].h : 0.f;
                sl.glo[c * plane + of] = __float2bfloat16_rn(live ? v[c + 1].l : 0.f);
            }
            if (live) mx = fmaxf(mx, fabsf(v[0].h));
            ++f;
        }
}

// Double-float arithmetic for the pure-shell combinations (solid_harmonics.cuh).
struct DfOps {
    __device__ static df add(df a, df b) { return dfl::add(a, b); }
    __device__ static df sub(df a, df b) { return dfl::sub(a, b); }
    __device__ static df scale(df a, double k) {
        const float kh = (float)k;
        return dfl::mul(a, {kh, (float)(k - (double)kh)});
    }
};

// A pure shell (L = 2 or 3), one component at a time (value, d/dx, d/dy, d/dz): the
// Cartesian values of that component, then its 2L+1 real solid harmonics, written as rows
// o, o + TILE, ... (the same formulas as colloc_shell for each component).
template <int L>
__device__ __forceinline__ void colloc_pure_shell(df X, df Y, df Z, df g, df h, const MixedSlabs &sl, size_t plane,
                                                  size_t o, bool live, float &mx) {
    constexpr int NC = (L + 1) * (L + 2) / 2, NO = 2 * L + 1;
    df xp[L + 1], yp[L + 1], zp[L + 1];
    xp[0] = yp[0] = zp[0] = {1.f, 0.f};
#pragma unroll
    for (int k = 1; k <= L; ++k) {
        xp[k] = df_mul(xp[k - 1], X);
        yp[k] = df_mul(yp[k - 1], Y);
        zp[k] = df_mul(zp[k - 1], Z);
    }
    const df R[4] = {g, df_mul(X, h), df_mul(Y, h), df_mul(Z, h)};
#pragma unroll
    for (int comp = 0; comp < 4; ++comp) {
        df cv[NC], out[NO];
        int f = 0;
#pragma unroll
        for (int l = L; l >= 0; --l)
#pragma unroll
            for (int mm = L - l; mm >= 0; --mm) {
                const int nn = L - l - mm;
                const df ym_zn = df_mul(yp[mm], zp[nn]);
                df v = df_mul(df_mul(xp[l], ym_zn), R[comp]);
                if (comp == 1 && l > 0)
                    v = df_add(v, df_mul(dfl::mul_f(df_mul(xp[l > 0 ? l - 1 : 0], ym_zn), (float)l), g));
                if (comp == 2 && mm > 0)
                    v = df_add(v, df_mul(dfl::mul_f(df_mul(df_mul(xp[l], yp[mm > 0 ? mm - 1 : 0]), zp[nn]), (float)mm), g));
                if (comp == 3 && nn > 0)
                    v = df_add(v, df_mul(dfl::mul_f(df_mul(df_mul(xp[l], yp[mm]), zp[nn > 0 ? nn - 1 : 0]), (float)nn), g));
                cv[f++] = v;
            }
        sph::pure<L, DfOps>(cv, out);
#pragma unroll
        for (int k = 0; k < NO; ++k) {
            const size_t of = o + (size_t)k * TILE;
            if (comp == 0) {
                sl.phi[of] = live ? make_float2(out[k].h, out[k].l) : make_float2(0.f, 0.f);
                if (live) mx = fmaxf(mx, fabsf(out[k].h));
            } else {
                sl.ghi[(comp - 1) * plane + of] = live ? out[k].h : 0.f;
                sl.glo[(comp - 1) * plane + of] = __float2bfloat16_rn(live ? out[k].l : 0.f);
            }
        }
    }
}

// Thread per point; Eq. gau_cart and its gradient in double-float arithmetic on the
// float32 pipe (exp(-alpha r^2) by dfl::exp_neg), stored as (hi, lo) pairs; then the
// point's Ozaki slices of Phi, K-blocked by 32 functions.  Consecutive shells on one centre
// share X, Y, Z and r^2.
struct Exp2Table {
    float2 v[64];   // 2^(-j/64) as (hi, lo): the table of dfl::exp_neg
};

template <bool HAS_PURE>   // instantiated without the pure-shell path for Cartesian bases
__global__ void __launch_bounds__(TILE, 7) colloc_mixed(ChunkArgs a, MixedArgs m, const DfShell *__restrict__ shells,
                                                     const __grid_constant__ Exp2Table e2t) {
    __shared__ float2 tab[64];
    if (threadIdx.x < 64) tab[threadIdx.x] = e2t.v[threadIdx.x];
    __syncthreads();
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int cnt = a.plan.tile_count[t];
    int64_t r0 = a.plan.tile_row[t] - a.row0;
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int np = pad32(n);
    bool live = i < cnt;
    // padding points past the count rounded up to 8 are read by no kernel of the spin-restricted
    // and spin-unrestricted forms except the W contraction, whose 16-point K steps read their
    // Phi slices up to the count rounded up to 16: those get zero slices, nothing else is
    // computed or stored for them (no barrier follows)
    if (!m.pad_all && i >= ((cnt + 7) & ~7)) {
        m.s.pexp[(t - a.t0) * TILE + i] = 0;
        if (i < ((cnt + 15) & ~15)) {
            const size_t plane = (size_t)m.rows * TILE;
            for (int kb = 0; kb < np / 32; ++kb) {
                const size_t orow = (size_t)(4 * r0 + (int64_t)kb * TILE + i) * 32;
#pragma unroll
                for (int s = 0; s < NSL; ++s)
#pragma unroll
                    for (int c8 = 0; c8 < 32; c8 += 8)
                        *reinterpret_cast<uint4 *>(m.s.ax + (size_t)s * plane + orow + c8) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        return;
    }
    int64_t p = a.plan.tile_first[t] + i;
    df px = d_to_df(live ? a.plan.x[p] : 0.0), py = d_to_df(live ? a.plan.y[p] : 0.0),
       pz = d_to_df(live ? a.plan.z[p] : 0.0);
    const size_t plane = (size_t)m.rows * TILE;
    const float2 *phi = m.s.phi;
    int64_t s0 = a.plan.shell_ptr[j], s1 = a.plan.shell_ptr[j + 1];
    int row = 0;
    float mx = 0.f;
    float cx = __int_as_float(0x7fc00000), cy = 0.f, cz = 0.f;   // centre of X, Y, Z (NaN: none yet)
    df X{0.f, 0.f}, Y{0.f, 0.f}, Z{0.f, 0.f}, r2{0.f, 0.f};
    for (int64_t si = s0; si < s1; ++si) {
        const DfShell &sh = shells[a.plan.shell_idx[si]];
        if (!(sh.ch[0] == cx && sh.ch[1] == cy && sh.ch[2] == cz)) {   // uniform over the block
            cx = sh.ch[0];
            cy = sh.ch[1];
            cz = sh.ch[2];
            X = dfl::sub(px, {sh.ch[0], sh.cl[0]});
            Y = dfl::sub(py, {sh.ch[1], sh.cl[1]});
            Z = dfl::sub(pz, {sh.ch[2], sh.cl[2]});
            r2 = df_add(df_add(df_mul(X, X), df_mul(Y, Y)), df_mul(Z, Z));
        }
        df g = {0.f, 0.f}, h = {0.f, 0.f};
        for (int k = 0; k < sh.nprim; ++k) {
            df ex = dfl::exp_neg(df_mul({sh.ah[k], sh.al[k]}, r2), tab);
            g = df_add(g, df_mul({sh.dh[k], sh.dl[k]}, ex));
            h = df_add(h, df_mul({sh.gh[k], sh.gl[k]}, ex));
        }
        const size_t o = (size_t)(r0 + row) * TILE + i;
        if constexpr (HAS_PURE) {
            if (sh.pure) {   // L = 2 or 3
                if (sh.L == 2) colloc_pure_shell<2>(X, Y, Z, g, h, m.s, plane, o, live, mx);
                else colloc_pure_shell<3>(X, Y, Z, g, h, m.s, plane, o, live, mx);
                row += 2 * sh.L + 1;
                continue;
            }
        }
        switch (sh.L) {
            case 0: colloc_shell<0>(X, Y, Z, g, h, m.s, plane, o, live, mx); row += 1; break;
            case 1: colloc_shell<1>(X, Y, Z, g, h, m.s, plane, o, live, mx); row += 3; break;
            case 2: colloc_shell<2>(X, Y, Z, g, h, m.s, plane, o, live, mx); row += 6; break;
            default: colloc_shell<3>(X, Y, Z, g, h, m.s, plane, o, live, mx); row += 10; break;
        }
    }
    int e = exp_of(mx);
    m.s.pexp[(t - a.t0) * TILE + i] = e;
    for (; row < np; ++row) {
        size_t o = (size_t)(r0 + row) * TILE + i;
        m.s.phi[o] = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            m.s.ghi[c * plane + o] = 0.f;
            m.s.glo[c * plane + o] = __float2bfloat16_rn(0.f);
        }
    }
    // Ozaki slices of this point's row of Phi: K block kb -> row 4 r0 + 128 kb + i, 32 values,
    // eight functions per 16-byte store of each slice plane; the next eight values are loaded
    // while the current ones are cut
    const int ngr = np / 8;
    float2 nx[8];
    auto load8 = [&](int gi) {
        if (gi < ngr) {
#pragma unroll
            for (int k = 0; k < 8; ++k) nx[k] = phi[(size_t)(r0 + 8 * gi + k) * TILE + i];
        }
    };
    load8(0);
#pragma unroll 1
    for (int gi = 0; gi < ngr; ++gi) {
        float2 cur[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) cur[k] = nx[k];
        load8(gi + 1);
        uint32_t w[NSL][4];
#pragma unroll
        for (int pr = 0; pr < 4; ++pr) {
            float q0[NSL], q1[NSL];
            slice5(cur[2 * pr].x, cur[2 * pr].y, e, q0);
            slice5(cur[2 * pr + 1].x, cur[2 * pr + 1].y, e, q1);
#pragma unroll
            for (int s = 0; s < NSL; ++s) {
                __nv_bfloat162 b2 = __floats2bfloat162_rn(q0[s], q1[s]);
                w[s][pr] = *reinterpret_cast<uint32_t *>(&b2);
            }
        }
        const size_t orow = (size_t)(4 * r0 + (int64_t)(gi >> 2) * TILE + i) * 32 + (gi & 3) * 8;
#pragma unroll
        for (int s = 0; s < NSL; ++s)
            *reinterpret_cast<uint4 *>(m.s.ax + (size_t)s * plane + orow) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
}

// ---------------------------------------------------------------- tcgen05 GEMM core
// Slice products of one K step, by accumulator: level d = s + t for d = 0, 1, 2 in
// accumulators 0, 1, 2 (exact: integer multiples of 2^-(12+7d) below 2^24 units for
// K <= 1184 functions or 1024 points) and levels 3-4 in accumulator 3 (rounded, 2^-21 below
// level 0).  The issue order is listed in issue_op().
constexpr int XACC = 4;
constexpr int BM = 128;                        // M extent of one MMA (points or functions)
constexpr int EPI_WARPS = 16;
constexpr int TQ = 8;                          // slots of the task ring (producer -> MMA and epilogue)
constexpr int GEMM_THREADS = 32 * (4 + EPI_WARPS);   // 4 control warps + the epilogue warps

// Geometry of the persistent GEMM for an N tile of BN functions: one pipeline stage holds
// one 16-wide K step of every slice of both operands (the global rows of 32 values are
// fetched as two 32-byte halves with the 32-byte swizzle; the K step after it reads the
// other halves of the same 64-byte rows, mostly from L2); tensor memory holds NBUF
// accumulator sets of 4 x BN columns.
template <int BN_>
struct GemmCfg {
    static constexpr int BN = BN_;
    static constexpr int NBUF = 512 / (XACC * BN);
    static constexpr int TMEM_COLS = NBUF * XACC * BN;   // 512 columns
    static constexpr int STAGES = BN == 128 ? 5 : 7;
    static constexpr int EPI_COLS = BN / (EPI_WARPS / 4);  // columns per epilogue warp
    static constexpr int A_BYTES = NSL * BM * 32;
    static constexpr int B_BYTES = NSL * BN * 32;
    // MN-major B (the V contraction's Phi from the X-side slices): BN / 32 boxes of 32
    // functions x 16 points x NSL slices, rows of 64 B
    static constexpr int MN_BOX = NSL * 16 * 64;
    static_assert(B_BYTES == (BN / 32) * MN_BOX, "MN-major B fills the B stage");
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TOTAL = 1024 + STAGES * STAGE + 512;   // + barriers and the task ring
    static_assert(NBUF >= 1 && NBUF <= 2, "one or two accumulator sets");
    static_assert(TOTAL <= 227 * 1024, "shared memory");
};

// The 15 MMAs of one 16-wide K step with compile-time operand offsets.  `first` is 0 only
// for the first K step of a task: then the first product into each accumulator overwrites
// it (levels 0, 1, 2, 3 start at ops 0, 1, 3, 6).
template <int BN, int BPL, int Q>   // BPL: B slice-plane stride in 16-byte units
__device__ __forceinline__ void issue_op(uint32_t tmem, uint64_t a0, uint64_t b0, uint32_t idesc, uint32_t first) {
    constexpr int A[15] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4};
    constexpr int B[15] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0};
    constexpr int C[15] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3};
    constexpr bool LEAD[15] = {true, true, false, true, false, false, true, false, false, false,
                               false, false, false, false, false};
    const uint64_t ad = a0 + (uint64_t)(A[Q] * (BM * 32 / 16));
    const uint64_t bd = b0 + (uint64_t)(B[Q] * BPL);
    const uint32_t acc = LEAD[Q] ? first : 1u;
    umma::mma_bf16(tmem + C[Q] * BN, ad, bd, idesc, acc);
}

template <int BN, int BPL, int... Q>
__device__ __forceinline__ void issue_ops(uint32_t tmem, uint64_t a0, uint64_t b0, uint32_t idesc, uint32_t first,
                                          std::integer_sequence<int, Q...>) {
    (issue_op<BN, BPL, Q>(tmem, a0, b0, idesc, first), ...);
}

template <int BN, int BPL>
__device__ __forceinline__ void issue_slice_mmas(uint32_t tmem, uint64_t a0, uint64_t b0, uint32_t idesc,
                                                 uint32_t first) {
    issue_ops<BN, BPL>(tmem, a0, b0, idesc, first, std::make_integer_sequence<int, 15>{});
}

// ---------------------------------------------------------------- persistent GEMM
// One CTA per SM; its producer claims tasks from a global counter in list order and hands
// each to the MMA thread and the epilogue warps through a ring in shared memory.  Roles:
//   warp 0 lane 0  task claims and TMA producer; its stage ring runs across task boundaries
//   warp 1 lane 0  MMA issuer (15 slice products per 16-wide K step into 4 accumulators)
//   warp 2         owns the tensor-memory allocation (all 512 columns)
//   warps 4-19     epilogue; warp w reads TMEM lanes 32 (w % 4) .. +31 and one quarter of
//                  the columns of each accumulator
// Task tau uses accumulator set tau % NBUF (with two sets the epilogue of one task overlaps
// the MMAs of the next); tmem_full[b] (MMA -> epilogue) and tmem_empty[b] (epilogue -> MMA)
// hand set b over.  The epilogue is kept short: a 4-term combine, power-of-two scaling
// from exponent bits, one store or one float64 atomic per element.

struct XGeom {
    int64_t t, r0, pofs;
    int j, jl, n, np, nc;
};
__device__ __forceinline__ XGeom x_geom(const ChunkArgs &a, const MixedArgs &m, const int *tasks, int k) {
    XGeom g;
    g.t = tasks[2 * k];
    g.nc = tasks[2 * k + 1];
    g.j = a.plan.tile_batch[g.t];
    g.n = (int)(a.plan.func_ptr[g.j + 1] - a.plan.func_ptr[g.j]);
    g.np = pad32(g.n);
    g.r0 = a.plan.tile_row[g.t] - a.row0;
    g.jl = g.j - m.j0;
    g.pofs = m.pofs[g.jl];
    return g;
}

struct VGeom {
    int64_t tb, te;
    int j, mc, nc, n, np;
};
__device__ __forceinline__ VGeom v_geom(const ChunkArgs &a, const int *tasks, int k) {
    VGeom g;
    const int *q = tasks + 5 * k;
    g.j = q[0];
    g.mc = q[1];
    g.nc = q[2];
    g.tb = q[3];
    g.te = q[4];
    g.n = (int)(a.plan.func_ptr[g.j + 1] - a.plan.func_ptr[g.j]);
    g.np = pad32(g.n);
    return g;
}

// 16-wide K steps of a task.  Steps that cover only zero padding are skipped, their products
// being exact zeros: for X the functions past N_b^j (the P^j and Phi slices of the rows up to
// the 32-padded count are zero), for W the points past the count of the task's last tile (the
// only tile of a batch that can be partial; Z is zero there).
__device__ __forceinline__ int x_ksteps(const XGeom &g) { return (g.n + 15) >> 4; }
// X segments of a task: batches with more than 1,184 functions accumulate K in segments of
// XSEG steps, each exact in its own level accumulators; the epilogue adds segment s > 0 to
// the X already stored by segment s - 1 (same CTA, same thread, in order) in double-float.
__device__ __forceinline__ int x_nseg(const XGeom &g) { return (x_ksteps(g) + XSEG - 1) / XSEG; }
__device__ __forceinline__ int v_ksteps(const ChunkArgs &a, const VGeom &g) {
    return (int)(g.te - g.tb - 1) * 8 + ((a.plan.tile_count[g.te - 1] + 15) >> 4);
}

// The four level accumulators as an unnormalised pair: levels 0 + 1 by two-sum (exact), levels
// 2-4 added to the low word (|v2| + |v3| < 2^-13 of level 0, so the rounding stays below 2^-37)
__device__ __forceinline__ df combine4(uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
    df s = two_sum(__uint_as_float(v0), __uint_as_float(v1));
    return {s.h, __fadd_rn(s.l, __fadd_rn(__uint_as_float(v2), __uint_as_float(v3)))};
}

// (double)f * 2^k from the bit fields, for a zero or normal float and a result exponent that
// stays normal (k in [-296, 258] here); partial sums of the slice products are multiples of
// 2^-40 or zero, so subnormal inputs do not occur
__device__ __forceinline__ double f2d_scaled(float f, int k) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t ex = (b >> 23) & 0xFFu;
    if (ex == 0) return 0.0;
    const uint64_t d = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(ex + 896 + k) << 52) |
                       ((uint64_t)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}

// KIND 0: X^j = P^j Phi^j tiles (tasks: point tile, BN-function column chunk).
// KIND 1: W^j = Z^T Phi tiles (tasks: batch, 128-row block, BN-column block, tile range),
//         Phi from slices cut per function over the task's points (the meta-GGA terms).
// KIND 2: the same tiles with Z scaled by 2^e_i and Phi from the X contraction's slices (cut
//         per point, read MN-major): the spin-restricted and spin-unrestricted forms.
template <int KIND, int BN_>
__global__ void __launch_bounds__(GEMM_THREADS, 1) gemm_persistent(const __grid_constant__ CUtensorMap ta,
                                                                   const __grid_constant__ CUtensorMap tb,
                                                                   ChunkArgs a, MixedArgs m, const int *tasks,
                                                                   int ntasks, int *task_ctr) {
    using GL = GemmCfg<BN_>;
    constexpr int BN = GL::BN, NBUF = GL::NBUF, TMEM_COLS = GL::TMEM_COLS, GEMM_STAGES = GL::STAGES,
                  EPI_COLS = GL::EPI_COLS;
    extern __shared__ uint8_t smem_raw[];
    uint32_t base = umma::smem_u32(smem_raw);
    uint8_t *smem = smem_raw + (((base + 1023) & ~1023u) - base);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + GEMM_STAGES * GL::STAGE);
    uint64_t *empty = full + GEMM_STAGES;
    uint64_t *tfull = empty + GEMM_STAGES;   // [NBUF]
    uint64_t *tempty = tfull + NBUF;         // [NBUF]
    uint64_t *drain = tempty + NBUF;
    uint64_t *tqf = drain + 1;               // [TQ] producer -> consumers: the slot holds a task
    uint64_t *tqe = tqf + TQ;                // [TQ] consumers -> producer: the slot was read
    int *tq = reinterpret_cast<int *>(tqe + TQ);   // [TQ] task indices (-1: no more tasks)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tq + TQ);
    __shared__ volatile int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < GEMM_STAGES; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            umma::mbar_init(&tfull[b], 1);
            umma::mbar_init(&tempty[b], EPI_WARPS);
        }
        umma::mbar_init(drain, 1);
        for (int q = 0; q < TQ; ++q) {
            umma::mbar_init(&tqf[q], 1);
            umma::mbar_init(&tqe[q], 1 + EPI_WARPS);   // the MMA thread and one lane per epilogue warp
        }
        umma::fence_mbar_init();
        umma::prefetch_tmap(&ta);
        umma::prefetch_tmap(&tb);
    }
    if (warp == 2) umma::tmem_alloc(tmem_slot, TMEM_COLS);
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {   // ------------------------------------------------ producer
            // Tasks are claimed from a global counter (dynamic scheduling: tasks that share an
            // operand tile, e.g. the N chunks of one point tile, start at nearly the same time
            // on neighbouring CTAs and find it in L2) and published to the MMA and epilogue warps
            // through the ring; -1 ends the ring.
            uint32_t gk = 0;
            for (uint32_t pt = 0;; ++pt) {
                const uint32_t slot = pt % TQ;
                if (pt >= TQ && !umma::mbar_wait(&tqe[slot], ((pt / TQ) - 1) & 1)) {
                    atomicOr(m.err, 1);
                    abort_flag = 1;
                    break;   // the slot was not read: the consumers' waits on it expire
                }
                int k = abort_flag ? -1 : atomicAdd(task_ctr, 1);
                if (k >= ntasks) k = -1;
                tq[slot] = k;
                umma::mbar_arrive(&tqf[slot]);
                if (k < 0) break;
                XGeom xg;
                VGeom vg;
                int nks;   // 16-wide K steps: two per stored block of 32
                if (KIND == 0) {
                    xg = x_geom(a, m, tasks, k);
                    nks = x_ksteps(xg);
                } else {
                    vg = v_geom(a, tasks, k);
                    nks = v_ksteps(a, vg);
                }
                for (int ks = 0; ks < nks; ++ks, ++gk) {
                    const int kb = ks >> 1, kx = (ks & 1) * 16;
                    int s = gk % GEMM_STAGES;
                    if (gk >= GEMM_STAGES && !umma::mbar_wait(&empty[s], ((gk / GEMM_STAGES) - 1) & 1)) {
                        atomicOr(m.err, 1);
                        abort_flag = 1;
                        break;   // the next ring slot then carries -1
                    }
                    int ay, by;
                    int64_t rx = 0;   // KIND 2: the X-side Phi slice rows of this 16-point step
                    if (KIND == 0) {
                        ay = (int)(4 * xg.r0 + (int64_t)kb * TILE);
                        by = (int)(xg.pofs + (int64_t)kb * xg.np + xg.nc * BN);
                    } else {
                        int64_t t = vg.tb + kb / 4;
                        int64_t b0 = 4 * (a.plan.tile_row[t] - a.row0) + (int64_t)(kb % 4) * vg.np;
                        ay = (int)(b0 + vg.mc * BM);
                        by = (int)(b0 + vg.nc * BN);
                        rx = 4 * (a.plan.tile_row[t] - a.row0) + (int64_t)(ks & 7) * 16 +
                             (int64_t)vg.nc * (BN / 32) * TILE;
                    }
                    uint8_t *sa = smem + s * GL::STAGE;
                    if (KIND == 2) {
                        // Phi_i,nu 2^-e_i from the X-side slices (rows: K block of 32 functions x
                        // 128 points): one box of 32 functions x 16 points per 32 live columns,
                        // MN-major in shared memory; columns past them are not read by the MMA
                        const int nbox = (min(BN, vg.n - vg.nc * BN) + 31) / 32;
                        umma::mbar_arrive_expect_tx(&full[s], GL::A_BYTES + nbox * GL::MN_BOX);
                        umma::tma_load_3d(sa, &ta, &full[s], kx, ay, 0);
                        for (int bx = 0; bx < nbox; ++bx)
                            umma::tma_load_3d(sa + GL::A_BYTES + bx * GL::MN_BOX, &tb, &full[s], 0,
                                              (int)(rx + (int64_t)bx * TILE), 0);
                    } else {
                        umma::mbar_arrive_expect_tx(&full[s], GL::STAGE);
                        umma::tma_load_3d(sa, &ta, &full[s], kx, ay, 0);
                        umma::tma_load_3d(sa + GL::A_BYTES, &tb, &full[s], kx, by, 0);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ------------------------------------------------ MMA issuer
            uint32_t gk = 0, tau = 0;
            for (uint32_t ct = 0;; ++ct) {
                const uint32_t slot = ct % TQ;
                if (!umma::mbar_wait(&tqf[slot], (ct / TQ) & 1)) {
                    atomicOr(m.err, 2);
                    abort_flag = 1;
                    break;
                }
                const int k = tq[slot];
                umma::mbar_arrive(&tqe[slot]);
                if (k < 0) break;
                if (abort_flag) continue;   // keep reading the ring until it ends, issue nothing
                int nks, ncols, nseg = 1;
                if (KIND == 0) {
                    XGeom g = x_geom(a, m, tasks, k);
                    nks = x_ksteps(g);
                    nseg = x_nseg(g);
                    ncols = min(BN, ((g.n - g.nc * BN) + 15) & ~15);
                } else {
                    VGeom g = v_geom(a, tasks, k);
                    nks = v_ksteps(a, g);
                    ncols = min(BN, ((g.n - g.nc * BN) + 15) & ~15);
                }
                const uint32_t idesc = umma::idesc_bf16(BM, ncols, KIND == 2);
                for (int sg = 0; sg < nseg && !abort_flag; ++sg, ++tau) {   // one accumulator set each
                    const uint32_t b = tau % NBUF, use = tau / NBUF;
                    if (tau >= NBUF && !umma::mbar_wait(&tempty[b], (use - 1) & 1)) {
                        atomicOr(m.err, 2);
                        abort_flag = 1;
                        break;
                    }
                    umma::fence_after_sync();
                    const uint32_t tacc = tmem + b * (XACC * BN);
                    const int ks0 = KIND == 0 ? sg * XSEG : 0;
                    const int ks1 = KIND == 0 ? min(nks, ks0 + XSEG) : nks;
                    for (int ks = ks0; ks < ks1; ++ks, ++gk) {
                        int s = gk % GEMM_STAGES;
                        if (!umma::mbar_wait(&full[s], (gk / GEMM_STAGES) & 1)) {
                            atomicOr(m.err, 2);
                            abort_flag = 1;
                            break;
                        }
                        umma::fence_after_sync();
                        uint32_t sa = umma::smem_u32(smem + s * GL::STAGE), sb = sa + GL::A_BYTES;
                        // descriptors of slice 0; every other slice is a fixed offset in 16-byte
                        // units (slice tiles BM x 32 B and BN x 32 B apart; MN-major B: 1 KB
                        // apart inside each box, boxes MN_BOX apart along N)
                        const uint64_t a0 = umma::desc_sw32(sa);
                        if (KIND == 2) {
                            const uint64_t b0 = umma::desc_mn_sw64(sb, GL::MN_BOX, 512);
                            issue_slice_mmas<BN, 1024 / 16>(tacc, a0, b0, idesc, ks == ks0 ? 0u : 1u);
                        } else {
                            const uint64_t b0 = umma::desc_sw32(sb);
                            issue_slice_mmas<BN, BN * 32 / 16>(tacc, a0, b0, idesc, ks == ks0 ? 0u : 1u);
                        }
                        umma::mma_commit(&empty[s]);
                    }
                    if (abort_flag) break;
                    umma::mma_commit(&tfull[b]);
                }
            }
            // every MMA this thread issued has completed before the allocation is released
            umma::mma_commit(drain);
            if (!umma::mbar_wait(drain, 0)) atomicOr(m.err, 4);
        }
    } else if (warp >= 4) {   // ---------------------------------------------- epilogue
        // Per accumulator hand-over, each epilogue warp first stages the column data of its own
        // EPI_COLS columns (X: the row exponents of P; V: global function indices and Phi group
        // exponents) in its own shared-memory slots, one column per lane, then reads them back
        // after a __syncwarp: no barrier spans the epilogue warps.
        __shared__ int wcol_a[EPI_WARPS][EPI_COLS], wcol_b[EPI_WARPS][EPI_COLS];
        const int q = warp & 3, cpart = (warp - 4) >> 2, ew = warp - 4;
        const int i = q * 32 + lane;
        int *col_a = wcol_a[ew], *col_b = wcol_b[ew];
        uint32_t tau = 0, ct = 0;
        // the next task of the ring (-1: no more tasks; -2: the wait expired)
        auto ring_next = [&]() -> int {
            const uint32_t slot = ct % TQ;
            if (!umma::mbar_wait(&tqf[slot], (ct / TQ) & 1)) {
                atomicOr(m.err, 4);
                abort_flag = 1;
                return -2;
            }
            ++ct;
            const int k = tq[slot];
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&tqe[slot]);
            return k;
        };
        // one accumulator hand-over: segment sg of X task k, or V task k
        auto epilogue = [&](int k, int sg) {
            const uint32_t b = tau % NBUF, use = tau / NBUF;
            ++tau;
            if (lane < EPI_COLS) {
                const int cc = cpart * EPI_COLS + lane;
                if (KIND == 0) {
                    XGeom g = x_geom(a, m, tasks, k);
                    const int mu = g.nc * BN + cc;
                    const float2 *pdf = m.pdf;
                    int nbf = a.nbf;
                    if (a.batch_mol) {
                        const MolRef r = mol_of(a, g.j);
                        pdf = r.pdf;
                        nbf = r.nbf;
                    }
                    const int *pe = reinterpret_cast<const int *>(reinterpret_cast<const char *>(pdf) +
                                                                  pdf_exps_offset(nbf));
                    col_a[lane] = mu < g.n ? pe[a.plan.func_idx[a.plan.func_ptr[g.j] + mu]] : 0;
                } else {
                    VGeom g = v_geom(a, tasks, k);
                    const int nu = g.nc * BN + cc;
                    const int64_t rg = a.plan.tile_row[g.tb] - a.row0;
                    col_a[lane] = nu < g.n ? a.plan.func_idx[a.plan.func_ptr[g.j] + nu] : 0;
                    col_b[lane] = (KIND == 1 && nu < g.n) ? m.s.fexp[rg + nu] : 0;
                }
            }
            __syncwarp();
            if (abort_flag) return;
            if (!umma::mbar_wait(&tfull[b], use & 1)) {
                atomicOr(m.err, 4);
                abort_flag = 1;
                return;
            }
            umma::fence_after_sync();
            __syncwarp();
            const uint32_t lane_base = tmem + b * (XACC * BN) + ((uint32_t)(q * 32) << 16);
            if (KIND == 0) {
                XGeom g = x_geom(a, m, tasks, k);
                const int ei = m.s.pexp[(g.t - a.t0) * TILE + i];
                const bool row_used = m.pad_all || i < a.plan.tile_count[g.t];
#pragma unroll 1
                for (int c = cpart * EPI_COLS; c < (cpart + 1) * EPI_COLS; c += 16) {
                    if (g.nc * BN + c >= g.n) break;   // warp-uniform
                    uint32_t v0[16], v1[16], v2[16], v3[16];
                    umma::tmem_ld16_nw(lane_base + c, v0);
                    umma::tmem_ld16_nw(lane_base + BN + c, v1);
                    umma::tmem_ld16_nw(lane_base + 2 * BN + c, v2);
                    umma::tmem_ld16_nw(lane_base + 3 * BN + c, v3);
                    umma::tmem_wait_ld();
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk) {
                        const int mu = g.nc * BN + c + kk;
                        if (mu < g.n && row_used) {
                            df x = combine4(v0[kk], v1[kk], v2[kk], v3[kk]);
                            const int sc = min(max(ei + col_a[c - cpart * EPI_COLS + kk], -252), 252);
                            const float s1 = pow2f(sc >> 1), s2 = pow2f(sc - (sc >> 1));
                            float2 *xo = m.s.x + (size_t)(g.r0 + mu) * TILE + i;
                            df xs{__fmul_rn(__fmul_rn(x.h, s1), s2), __fmul_rn(__fmul_rn(x.l, s1), s2)};
                            if (sg > 0) {   // a later K segment: add to the segments before it
                                const float2 o = *xo;
                                xs = df_add({o.x, o.y}, xs);
                            }
                            *xo = make_float2(xs.h, xs.l);
                        }
                    }
                }
            } else {
                // W^j is added transposed (V_acc[nu][mu] += W[mu][nu]); the final
                // V = V_acc + V_acc^T is unchanged, and the 32 lanes of a warp (consecutive
                // mu) then update neighbouring words of one row of V_acc
                VGeom g = v_geom(a, tasks, k);
                const MolRef mr = mol_of(a, g.j);   // V_acc and nbf of the batch's molecule
                const int mu = g.mc * BM + i;
                const size_t colg = (mu < g.n) ? (size_t)a.plan.func_idx[a.plan.func_ptr[g.j] + mu] : 0;
                const int64_t rg = a.plan.tile_row[g.tb] - a.row0;   // group exponents on the first tile
                const int ez = (mu < g.n) ? m.s.zexp[rg + mu] : 0;
#pragma unroll 1
                for (int c = cpart * EPI_COLS; c < (cpart + 1) * EPI_COLS; c += 16) {
                    if (g.nc * BN + c >= g.n) break;   // warp-uniform
                    uint32_t v0[16], v1[16], v2[16], v3[16];
                    umma::tmem_ld16_nw(lane_base + c, v0);
                    umma::tmem_ld16_nw(lane_base + BN + c, v1);
                    umma::tmem_ld16_nw(lane_base + 2 * BN + c, v2);
                    umma::tmem_ld16_nw(lane_base + 3 * BN + c, v3);
                    umma::tmem_wait_ld();
                    if (mu < g.n) {
#pragma unroll
                        for (int kk = 0; kk < 16; ++kk) {
                            const int nu = g.nc * BN + c + kk;
                            if (nu < g.n) {
                                df w = combine4(v0[kk], v1[kk], v2[kk], v3[kk]);
                                const int lc = c - cpart * EPI_COLS + kk;
                                const int sc = ez + col_b[lc];
                                atomicAdd(&mr.Vacc[(size_t)col_a[lc] * mr.nbf + colg],
                                          f2d_scaled(w.h, sc) + f2d_scaled(w.l, sc));
                            }
                        }
                    }
                }
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&tempty[b]);
        };
        for (;;) {
            const int k = ring_next();
            if (k < 0) break;
            // one pass per accumulator hand-over: the K segments of an X task, one pass for V
            const int nseg = KIND == 0 ? x_nseg(x_geom(a, m, tasks, k)) : 1;
            for (int sg = 0; sg < nseg; ++sg) epilogue(k, sg);
        }
    }
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 2) umma::tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------- rho, functional (spin-restricted)
// rho and grad rho (Eqs. eval_local_den, eval_local_den_grad) in double-float over the batch's
// functions, the functional and the tile's E/N partials (Eq. exc_batch) in float64.  Z (Eq.
// z_mat) is not formed here: the per-point coefficients a_i = 1/2 w vrho and
// b_i = 2 w vsigma grad rho go, as float64, to the first four rows of the tile's X plane (X is
// dead once rho is formed; a tile has at least FBLK = 32 rows), and z_slice forms Z from them
// while slicing it, so Z never travels through memory.  Thread i reads and writes column i
// only, so the overwrite needs no barrier.
__global__ void __launch_bounds__(TILE) rho_mixed(ChunkArgs a, MixedArgs m) {
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int cnt = a.plan.tile_count[t];
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int64_t r0 = a.plan.tile_row[t] - a.row0;
    const size_t plane = (size_t)m.rows * TILE;
    const float2 *phi = m.s.phi;
    df rho{0.f, 0.f}, gx{0.f, 0.f}, gy{0.f, 0.f}, gz{0.f, 0.f};
    if (i < cnt) {   // padding points contribute nothing (their coefficients stay zero)
#pragma unroll 2
        for (int mu = 0; mu < n; ++mu) {
            size_t o = (size_t)(r0 + mu) * TILE + i;
            const float2 xv = m.s.x[o], f0 = phi[o];
            const float h1 = m.s.ghi[o], h2 = m.s.ghi[plane + o], h3 = m.s.ghi[2 * plane + o];
            const float l1 = __bfloat162float(m.s.glo[o]), l2 = __bfloat162float(m.s.glo[plane + o]),
                        l3 = __bfloat162float(m.s.glo[2 * plane + o]);
            df x{xv.x, xv.y};
            rho = df_add(rho, df_mul({f0.x, f0.y}, x));
            gx = df_add(gx, df_mul({h1, l1}, x));
            gy = df_add(gy, df_mul({h2, l2}, x));
            gz = df_add(gz, df_mul({h3, l3}, x));
        }
    }
    double r = df_to_d(rho);
    double dx = 2.0 * df_to_d(gx), dy = 2.0 * df_to_d(gy), dz = 2.0 * df_to_d(gz);
    double e = 0.0, nn = 0.0;
    double coef[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < cnt) {
        double w = a.plan.w[a.plan.tile_first[t] + i];
        double sigma = dx * dx + dy * dy + dz * dz;
        double f, vr, vs;
        xc::evaluate<double>(mol_of(a, j).functional, r, sigma, f, vr, vs);
        e = w * f;
        nn = w * r;
        coef[0] = 0.5 * w * vr;
        double b = 2.0 * w * vs;
        coef[1] = b * dx;
        coef[2] = b * dy;
        coef[3] = b * dz;
    }
    double *cz = reinterpret_cast<double *>(m.s.x);
#pragma unroll
    for (int q = 0; q < 4; ++q) cz[(size_t)(r0 + q) * TILE + i] = coef[q];
    __shared__ double re[TILE], rn[TILE];
    re[i] = e;
    rn[i] = nn;
    __syncthreads();
    for (int s = TILE / 2; s > 0; s >>= 1) {
        if (i < s) {
            re[i] += re[i + s];
            rn[i] += rn[i + s];
        }
        __syncthreads();
    }
    if (i == 0) {
        a.tileE[t] = re[0];
        a.tileN[t] = rn[0];
    }
}

// ---------------------------------------------------------------- Z and its slices (spin-restricted)
// Per K group (the up to VKS tiles of one batch that form one V task) and function row mu:
// Z_i,mu = a_i Phi_i,mu + b_i . grad Phi_i,mu (Eq. z_mat, double-float, gradient hi words),
// times 2^e_i, the exponent of point i's Phi slices: the W contraction takes Phi from the
// slices the X contraction uses (Phi_i,nu 2^-e_i, cut per point), so
// W_mu,nu = sum_i (Z_i,mu 2^e_i)(Phi_i,nu 2^-e_i) and only the scaled Z is sliced here, per
// function over the group's points (the exponent of max |Z 2^e| per tile, their maximum over
// the group, to the group's first tile for the V epilogue).  The block's eight 16-thread slots
// cover G2 tiles (the group size rounded up to a power of two) for 8 / G2 rows at a time, 8
// points per thread, so Z stays in registers while the slots exchange their tile exponents
// through shared memory (one barrier per step, double-buffered): every element is read once.  The blocks of a group's
// tiles share its rows (row step k to block k mod group size), so the grid keeps one block per
// tile.  With keep_z the values of Z are also written over X for the per-batch debugging copy;
// the group's first block then does every row, because those writes cover the coefficient rows
// the other blocks read.
// Shared-memory slot of point p's coefficient: an XOR of p's octet bits (p >> 4) into its low
// three bits, so the 16 threads of a slot (points 8 pg + k, one k) read 16 distinct bank pairs
// instead of two.
__device__ __forceinline__ int cf_slot(int p) { return p ^ ((p >> 4) & 7); }

// Dynamic shared memory: the coefficients of the chunk's largest group (4 KB per tile), so that
// eight blocks fit an SM when the groups are short (batches of at most 512 points)
__host__ __device__ constexpr size_t z_slice_smem(int max_group) {
    return (size_t)max_group * 4 * TILE * sizeof(float2);
}

__global__ void __launch_bounds__(TILE, 4) z_slice(ChunkArgs a, MixedArgs m) {
    const int64_t t = a.t0 + blockIdx.x;
    const int j = a.plan.tile_batch[t];
    const int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    const int np = pad32(n);
    const int64_t s0 = a.plan.batch_tile[j] > a.t0 ? a.plan.batch_tile[j] : a.t0;
    const int64_t s1 = a.plan.batch_tile[j + 1] < a.t1 ? a.plan.batch_tile[j + 1] : a.t1;
    const int64_t g0 = s0 + (t - s0) / VKS * VKS;
    const int ng = (int)((g0 + VKS < s1 ? g0 + VKS : s1) - g0);
    const int ub = (int)(t - g0), nblk = m.keep_z ? 1 : ng;
    if (ub >= nblk) return;   // block-uniform
    const int64_t rg = a.plan.tile_row[g0] - a.row0;
    const size_t plane = (size_t)m.rows * TILE;
    // the group's per-point coefficients (a, b_x, b_y, b_z) times 2^e_i as double-float pairs,
    // [tile][4][TILE], so that the products form Z 2^e_i
    extern __shared__ float2 cf[];
    __shared__ int64_t trow[VKS];
    __shared__ int tcnt[VKS];
    __shared__ int red[2][8];   // per step parity and slot: tile exponents of |Z 2^e|
    const double *cz = reinterpret_cast<const double *>(m.s.x);
    for (int u = 0; u < ng; ++u) {
        const int64_t ru = a.plan.tile_row[g0 + u] - a.row0;
        const int cu = a.plan.tile_count[g0 + u];
        if (threadIdx.x == 0) {
            trow[u] = ru;
            tcnt[u] = cu;
        }
        const int ep = threadIdx.x < cu ? m.s.pexp[(g0 + u - a.t0) * TILE + threadIdx.x] : 0;
        const double pe = (double)pow2f(min(max(ep, -126), 127));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const df c = d_to_df(cz[(size_t)(ru + q) * TILE + threadIdx.x] * pe);
            cf[(u * 4 + q) * TILE + cf_slot(threadIdx.x)] = make_float2(c.h, c.l);
        }
    }
    __syncthreads();
    const int lg = ng > 4 ? 3 : ng > 2 ? 2 : ng > 1 ? 1 : 0;   // G2 = 2^lg tiles per row
    const int R = 8 >> lg;                                       // rows per step
    const int slot = threadIdx.x >> 4, pg = threadIdx.x & 15;
    const int u = slot & ((1 << lg) - 1), rr = slot >> lg;
    const int pk = pg >> 2, col = (pg & 3) * 8;
    const int64_t ru = u < ng ? trow[u] : 0;
    // padding points (past the tile's count) have Z = 0 and Phi = 0: a thread whose 8 points
    // are all padding loads nothing, and stores its (zero) slices only if the V contraction
    // reads them, i.e. below the count rounded up to its 16-point K steps
    const int cu = u < ng ? tcnt[u] : 0;
    const bool live8 = 8 * pg < cu, need8 = 8 * pg < ((cu + 15) & ~15);
    // the next step's Phi and grad Phi are loaded while this step's Z is formed and sliced
    float4 nf[4], nh[3][2];
    auto load = [&](int c2) {
        const int mu2 = c2 * R + rr;
        if (c2 * R < n && u < ng && mu2 < n && live8) {
            const size_t o2 = (size_t)(ru + mu2) * TILE + 8 * pg;
            const float4 *fs = reinterpret_cast<const float4 *>(m.s.phi + o2);
#pragma unroll
            for (int q = 0; q < 4; ++q) nf[q] = fs[q];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float4 *h = reinterpret_cast<const float4 *>(m.s.ghi + d * plane + o2);
                nh[d][0] = h[0];
                nh[d][1] = h[1];
            }
        }
    };
    load(ub);
    int par = 0;
    for (int c = ub; c * R < n; c += nblk, par ^= 1) {
        const int mu = c * R + rr;
        const bool act = u < ng && mu < n;
        float4 cfs[4], ch[3][2];
#pragma unroll
        for (int q = 0; q < 4; ++q) cfs[q] = nf[q];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ch[d][0] = nh[d][0];
            ch[d][1] = nh[d][1];
        }
        load(c + nblk);
        float zh[8], zl[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) zh[e] = zl[e] = 0.f;
        float az = 0.f;
        const size_t o = (size_t)(ru + mu) * TILE + 8 * pg;
        if (act && live8) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {   // points 2q, 2q + 1
                const float4 f4 = cfs[q];
                const float4 a1 = ch[0][q >> 1], a2 = ch[1][q >> 1], a3 = ch[2][q >> 1];
                const float gxs[2] = {(q & 1) ? a1.z : a1.x, (q & 1) ? a1.w : a1.y};
                const float gys[2] = {(q & 1) ? a2.z : a2.x, (q & 1) ? a2.w : a2.y};
                const float gzs[2] = {(q & 1) ? a3.z : a3.x, (q & 1) ? a3.w : a3.y};
                const float fh[2] = {f4.x, f4.z}, fl[2] = {f4.y, f4.w};
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int e = 2 * q + k, sp = cf_slot(8 * pg + e);
                    const float2 *cu4 = cf + u * 4 * TILE + sp;
                    const float2 c0 = cu4[0], c1 = cu4[TILE], c2 = cu4[2 * TILE], c3 = cu4[3 * TILE];
                    df z = df_mul({c0.x, c0.y}, {fh[k], fl[k]});
                    z = df_add(z, dfl::mul_f({c1.x, c1.y}, gxs[k]));
                    z = df_add(z, dfl::mul_f({c2.x, c2.y}, gys[k]));
                    z = df_add(z, dfl::mul_f({c3.x, c3.y}, gzs[k]));
                    zh[e] = z.h;
                    zl[e] = z.l;
                    az = fmaxf(az, fabsf(z.h));
                }
            }
        }
#pragma unroll
        for (int q = 8; q > 0; q >>= 1)   // over the 16 threads of the slot (one tile row)
            az = fmaxf(az, __shfl_xor_sync(0xffffffffu, az, q));
        if (pg == 0) red[par][slot] = act ? exp_of(az) : -1000;
        __syncthreads();
        int ez = -1000;
        for (int v = 0; v < (1 << lg); ++v) ez = max(ez, red[par][(rr << lg) + v]);
        if (!act) continue;
        if (m.keep_z && live8) {   // Z itself: the scaling by 2^e_i undone (exact)
            float4 *zo = reinterpret_cast<float4 *>(m.s.x + o);
            const int *pe = m.s.pexp + (g0 + u - a.t0) * TILE + 8 * pg;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e0 = -min(max(pe[2 * q], -126), 127), e1 = -min(max(pe[2 * q + 1], -126), 127);
                zo[q] = make_float4(scale2(zh[2 * q], e0), scale2(zl[2 * q], e0), scale2(zh[2 * q + 1], e1),
                                    scale2(zl[2 * q + 1], e1));
            }
        }
        uint32_t wz[NSL][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // points 2q, 2q + 1
            float a0[NSL], a1[NSL];
            slice5(zh[2 * q], zl[2 * q], ez, a0);
            slice5(zh[2 * q + 1], zl[2 * q + 1], ez, a1);
#pragma unroll
            for (int sl = 0; sl < NSL; ++sl) {
                __nv_bfloat162 bz = __floats2bfloat162_rn(a0[sl], a1[sl]);
                wz[sl][q] = *reinterpret_cast<uint32_t *>(&bz);
            }
        }
        const size_t orow = (size_t)(4 * ru + (int64_t)pk * np + mu) * 32 + col;
        if (need8) {
#pragma unroll
            for (int sl = 0; sl < NSL; ++sl)
                *reinterpret_cast<uint4 *>(m.s.vz + (size_t)sl * plane + orow) =
                    make_uint4(wz[sl][0], wz[sl][1], wz[sl][2], wz[sl][3]);
        }
        if (u == 0 && pg == 0) m.s.zexp[rg + mu] = ez;
    }
}

// ---------------------------------------------------------------- spin-unrestricted rho, functional
// Both spin densities and their gradients in double-float over X_a (in the slab) and X_b (in
// x2), the spin-polarised functional in float64, the tile's E/N partials, and per spin the
// coefficients of Z^s = 1/2 w v_s Phi + w (2 s_ss grad rho_s + s_ab grad rho_s') . grad Phi:
// spin a's in the first four rows of the tile's X_a plane, spin b's in those of x2, as in
// rho_mixed, so that z_slice forms and slices each Z^s in turn.  Padding points load nothing.
__global__ void __launch_bounds__(TILE) rho_mixed_uks(ChunkArgs a, MixedArgs m, float2 *__restrict__ x2) {
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int cnt = a.plan.tile_count[t];
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int64_t r0 = a.plan.tile_row[t] - a.row0;
    const size_t plane = (size_t)m.rows * TILE;
    const float2 *phi = m.s.phi;
    df rho[2] = {{0.f, 0.f}, {0.f, 0.f}};
    df g[2][3] = {{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}};
    if (i < cnt) {
#pragma unroll 2
        for (int mu = 0; mu < n; ++mu) {
            size_t o = (size_t)(r0 + mu) * TILE + i;
            const float2 xa = m.s.x[o], xb = x2[o], f0 = phi[o];
            const df gr[3] = {{m.s.ghi[o], __bfloat162float(m.s.glo[o])},
                              {m.s.ghi[plane + o], __bfloat162float(m.s.glo[plane + o])},
                              {m.s.ghi[2 * plane + o], __bfloat162float(m.s.glo[2 * plane + o])}};
            const df xs[2] = {{xa.x, xa.y}, {xb.x, xb.y}};
#pragma unroll
            for (int sp = 0; sp < 2; ++sp) {
                rho[sp] = df_add(rho[sp], df_mul({f0.x, f0.y}, xs[sp]));
#pragma unroll
                for (int d = 0; d < 3; ++d) g[sp][d] = df_add(g[sp][d], df_mul(gr[d], xs[sp]));
            }
        }
    }
    double r[2], gd[2][3];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
        r[sp] = df_to_d(rho[sp]);
#pragma unroll
        for (int d = 0; d < 3; ++d) gd[sp][d] = 2.0 * df_to_d(g[sp][d]);
    }
    double e = 0.0, nn = 0.0, coef[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
    if (i < cnt) {
        const double w = a.plan.w[a.plan.tile_first[t] + i];
        const double saa = gd[0][0] * gd[0][0] + gd[0][1] * gd[0][1] + gd[0][2] * gd[0][2];
        const double sab = gd[0][0] * gd[1][0] + gd[0][1] * gd[1][1] + gd[0][2] * gd[1][2];
        const double sbb = gd[1][0] * gd[1][0] + gd[1][1] * gd[1][1] + gd[1][2] * gd[1][2];
        double f, va, vb, s_aa, s_ab, s_bb;
        xc::evaluate_pol<double>(a.functional, r[0], r[1], saa, sab, sbb, f, va, vb, s_aa, s_ab, s_bb);
        e = w * f;
        nn = w * (r[0] + r[1]);
        coef[0][0] = 0.5 * w * va;
        coef[1][0] = 0.5 * w * vb;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            coef[0][d + 1] = w * (2.0 * s_aa * gd[0][d] + s_ab * gd[1][d]);
            coef[1][d + 1] = w * (2.0 * s_bb * gd[1][d] + s_ab * gd[0][d]);
        }
    }
    double *cza = reinterpret_cast<double *>(m.s.x), *czb = reinterpret_cast<double *>(x2);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        cza[(size_t)(r0 + q) * TILE + i] = coef[0][q];
        czb[(size_t)(r0 + q) * TILE + i] = coef[1][q];
    }
    __shared__ double re[TILE], rn[TILE];
    re[i] = e;
    rn[i] = nn;
    __syncthreads();
    for (int st = TILE / 2; st > 0; st >>= 1) {
        if (i < st) {
            re[i] += re[i + st];
            rn[i] += rn[i + st];
        }
        __syncthreads();
    }
    if (i == 0) {
        a.tileE[t] = re[0];
        a.tileN[t] = rn[0];
    }
}

// ---------------------------------------------------------------- meta-GGA (tensor-core form)
// The meta-GGA's kinetic energy density needs Y^k = (d_k Phi) P^j for k = x, y, z: the X
// contraction again with d_k Phi as its A operand.  grad_slices cuts d_k Phi (hi words and
// bf16 lo words) into the K-blocked Ozaki slices the collocation writes for Phi, with per
// point exponents of max_mu |d_k Phi|: component k's slices at ax_g + k NSL plane, its
// exponents at pexp_g + k 4 rows (the stride of the slab's own point exponents).
__global__ void __launch_bounds__(TILE) grad_slices(ChunkArgs a, MixedArgs m, __nv_bfloat16 *__restrict__ ax_g,
                                                    int *__restrict__ pexp_g) {
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int np = pad32(n);
    int64_t r0 = a.plan.tile_row[t] - a.row0;
    const size_t plane = (size_t)m.rows * TILE;
    for (int k = 0; k < 3; ++k) {
        const float *gh = m.s.ghi + (size_t)k * plane;
        const __nv_bfloat16 *gl = m.s.glo + (size_t)k * plane;
        float mx = 0.f;
        for (int mu = 0; mu < n; ++mu) mx = fmaxf(mx, fabsf(gh[(size_t)(r0 + mu) * TILE + i]));
        const int e = exp_of(mx);
        pexp_g[(size_t)k * 4 * m.rows + (t - a.t0) * TILE + i] = e;
        __nv_bfloat16 *ax = ax_g + (size_t)k * NSL * plane;
        for (int kb = 0; kb < np / 32; ++kb) {
            const size_t orow = (size_t)(4 * r0 + (int64_t)kb * TILE + i) * 32;
#pragma unroll 1
            for (int c8 = 0; c8 < 32; c8 += 8) {
                uint32_t w[NSL][4];
#pragma unroll
                for (int pr = 0; pr < 4; ++pr) {
                    size_t o = (size_t)(r0 + kb * 32 + c8 + 2 * pr) * TILE + i;
                    float q0[NSL], q1[NSL];
                    slice5(gh[o], __bfloat162float(gl[o]), e, q0);
                    slice5(gh[o + TILE], __bfloat162float(gl[o + TILE]), e, q1);
#pragma unroll
                    for (int s = 0; s < NSL; ++s) {
                        __nv_bfloat162 b2 = __floats2bfloat162_rn(q0[s], q1[s]);
                        w[s][pr] = *reinterpret_cast<uint32_t *>(&b2);
                    }
                }
#pragma unroll
                for (int s = 0; s < NSL; ++s)
                    *reinterpret_cast<uint4 *>(ax + (size_t)s * plane + orow + c8) =
                        make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
            }
        }
    }
}

// rho, grad rho and tau = 1/2 sum_k sum_mu d_k Phi Y^k in double-float (X in the slab, Y^k
// in y_g + k plane), the meta-GGA functional in float64, then Z over X and
// W^k = 1/4 w vtau d_k Phi over Y^k, with the per-tile maxima of |Z| (zexp), |Phi| (fexp),
// |W^k| (wexp_g + k rows) and |d_k Phi| (gexp_g + k rows) for the V-side slicing.
__global__ void __launch_bounds__(TILE) rho_z_mixed_mgga(ChunkArgs a, MixedArgs m, float2 *__restrict__ y_g,
                                                          int *__restrict__ wexp_g, int *__restrict__ gexp_g) {
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int cnt = a.plan.tile_count[t];
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int np = pad32(n);
    int64_t r0 = a.plan.tile_row[t] - a.row0;
    const size_t plane = (size_t)m.rows * TILE;
    const float2 *phi = m.s.phi;
    df rho{0.f, 0.f}, tau{0.f, 0.f}, gr[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 2
    for (int mu = 0; mu < n; ++mu) {
        size_t o = (size_t)(r0 + mu) * TILE + i;
        const float2 xv = m.s.x[o], f0 = phi[o];
        const df x{xv.x, xv.y};
        rho = df_add(rho, df_mul({f0.x, f0.y}, x));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const df gk{m.s.ghi[k * plane + o], __bfloat162float(m.s.glo[k * plane + o])};
            const float2 yv = y_g[k * plane + o];
            gr[k] = df_add(gr[k], df_mul(gk, x));
            tau = df_add(tau, df_mul(gk, {yv.x, yv.y}));
        }
    }
    const double r = df_to_d(rho), ta = 0.5 * df_to_d(tau);
    const double dx = 2.0 * df_to_d(gr[0]), dy = 2.0 * df_to_d(gr[1]), dz = 2.0 * df_to_d(gr[2]);
    double e = 0.0, nn = 0.0, ca_d = 0.0, bx_d = 0.0, by_d = 0.0, bz_d = 0.0, ct_d = 0.0;
    if (i < cnt) {
        const double w = a.plan.w[a.plan.tile_first[t] + i];
        double f, vr, vs, vt;
        xc::mvs_x(r, dx * dx + dy * dy + dz * dz, ta, f, vr, vs, vt);
        e = w * f;
        nn = w * r;
        ca_d = 0.5 * w * vr;
        const double b = 2.0 * w * vs;
        bx_d = b * dx;
        by_d = b * dy;
        bz_d = b * dz;
        ct_d = 0.25 * w * vt;
    }
    // the per-function maxima over the tile's points, in blocks of MGGA_FB functions
    __shared__ int zmax[MGGA_FB], fmx[MGGA_FB], wmax[3][MGGA_FB], gmax[3][MGGA_FB];
    const df cz = d_to_df(ca_d), cbx = d_to_df(bx_d), cby = d_to_df(by_d), cbz = d_to_df(bz_d), ct = d_to_df(ct_d);
    const int lane = i & 31;
    for (int fb = 0; fb < np; fb += MGGA_FB) {
        const int fe = min(np, fb + MGGA_FB), ne = min(n, fe);
        for (int mu = fb + i; mu < fe; mu += TILE) {
            zmax[mu - fb] = 0;
            fmx[mu - fb] = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                wmax[k][mu - fb] = 0;
                gmax[k][mu - fb] = 0;
            }
        }
        __syncthreads();
#pragma unroll 2
        for (int mu = fb; mu < ne; ++mu) {
            size_t o = (size_t)(r0 + mu) * TILE + i;
            const float2 f0 = phi[o];
            const float h1 = m.s.ghi[o], h2 = m.s.ghi[plane + o], h3 = m.s.ghi[2 * plane + o];
            df z = df_mul(cz, {f0.x, f0.y});
            z = df_add(z, dfl::mul_f(cbx, h1));
            z = df_add(z, dfl::mul_f(cby, h2));
            z = df_add(z, dfl::mul_f(cbz, h3));
            m.s.x[o] = make_float2(z.h, z.l);
            float az = fabsf(z.h), ap = fabsf(f0.x), aw[3], ag[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float hk = m.s.ghi[k * plane + o];
                const df wk = df_mul(ct, {hk, __bfloat162float(m.s.glo[k * plane + o])});
                y_g[k * plane + o] = make_float2(wk.h, wk.l);
                aw[k] = fabsf(wk.h);
                ag[k] = fabsf(hk);
            }
#pragma unroll
            for (int q = 16; q > 0; q >>= 1) {
                az = fmaxf(az, __shfl_xor_sync(0xffffffffu, az, q));
                ap = fmaxf(ap, __shfl_xor_sync(0xffffffffu, ap, q));
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    aw[k] = fmaxf(aw[k], __shfl_xor_sync(0xffffffffu, aw[k], q));
                    ag[k] = fmaxf(ag[k], __shfl_xor_sync(0xffffffffu, ag[k], q));
                }
            }
            if (lane == 0) {
                atomicMax(&zmax[mu - fb], __float_as_int(az));
                atomicMax(&fmx[mu - fb], __float_as_int(ap));
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    atomicMax(&wmax[k][mu - fb], __float_as_int(aw[k]));
                    atomicMax(&gmax[k][mu - fb], __float_as_int(ag[k]));
                }
            }
        }
        __syncthreads();
        for (int mu = fb + i; mu < ne; mu += TILE) {
            m.s.zexp[r0 + mu] = exp_of(__int_as_float(zmax[mu - fb]));
            m.s.fexp[r0 + mu] = exp_of(__int_as_float(fmx[mu - fb]));
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                wexp_g[(size_t)k * m.rows + r0 + mu] = exp_of(__int_as_float(wmax[k][mu - fb]));
                gexp_g[(size_t)k * m.rows + r0 + mu] = exp_of(__int_as_float(gmax[k][mu - fb]));
            }
        }
        __syncthreads();   // the next block's reset waits for these reads
    }
    __shared__ double re[TILE], rn[TILE];
    re[i] = e;
    rn[i] = nn;
    __syncthreads();
    for (int st = TILE / 2; st > 0; st >>= 1) {
        if (i < st) {
            re[i] += re[i + st];
            rn[i] += rn[i + st];
        }
        __syncthreads();
    }
    if (i == 0) {
        a.tileE[t] = re[0];
        a.tileN[t] = rn[0];
    }
}

// ---------------------------------------------------------------- V-side slicing
// Thread per point.  The K group of the tile (the V task it belongs to) shares one
// exponent per function for Z and one for Phi: the maximum of the per-tile exponents.
// The group's first tile stores those maxima for the V epilogue over its own per-tile
// entries; a reader in another block that sees the new value takes the same maximum, so
// no ordering between the blocks of a group is needed.
// GRAD: the meta-GGA's terms W^k^T d_k Phi, with W^k in the X/Z plane (m.s.x) and d_k Phi read
// from its hi words `gh` and bf16 lo words `gl` instead of Phi.
template <bool GRAD>
__global__ void __launch_bounds__(TILE) slice_v(ChunkArgs a, MixedArgs m, const float *__restrict__ gh,
                                                const __nv_bfloat16 *__restrict__ gl) {
    int64_t t = a.t0 + blockIdx.x;
    int j = a.plan.tile_batch[t];
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int np = pad32(n);
    int64_t s0 = a.plan.batch_tile[j] > a.t0 ? a.plan.batch_tile[j] : a.t0;
    int64_t s1 = a.plan.batch_tile[j + 1] < a.t1 ? a.plan.batch_tile[j + 1] : a.t1;
    int64_t g0 = s0 + (t - s0) / VKS * VKS;
    int64_t g1 = g0 + VKS < s1 ? g0 + VKS : s1;
    int64_t r0 = a.plan.tile_row[t] - a.row0;
    int64_t rg = a.plan.tile_row[g0] - a.row0;
    const size_t plane = (size_t)m.rows * TILE;
    // thread = (function row within 8, group of 8 points): 64-byte loads, 16-byte stores
    const int lr = threadIdx.x >> 4, pg = threadIdx.x & 15;
    const int pk = pg >> 2, col = (pg & 3) * 8;
    for (int mu = lr; mu < n; mu += 8) {
        int ez = -1000, ep = -1000;
        for (int64_t u = g0; u < g1; ++u) {
            int64_t ru = a.plan.tile_row[u] - a.row0;
            ez = max(ez, m.s.zexp[ru + mu]);
            ep = max(ep, m.s.fexp[ru + mu]);
        }
        const size_t o = (size_t)(r0 + mu) * TILE + 8 * pg;
        const float4 *zs = reinterpret_cast<const float4 *>(m.s.x + o);
        const float4 *fs = reinterpret_cast<const float4 *>(m.s.phi + o);
        float gfh[8], gfl[8];
        if constexpr (GRAD) {
            const float4 h0 = *reinterpret_cast<const float4 *>(gh + o), h1 = *reinterpret_cast<const float4 *>(gh + o + 4);
            const uint4 lw = *reinterpret_cast<const uint4 *>(gl + o);
            const uint32_t lu[4] = {lw.x, lw.y, lw.z, lw.w};
            gfh[0] = h0.x; gfh[1] = h0.y; gfh[2] = h0.z; gfh[3] = h0.w;
            gfh[4] = h1.x; gfh[5] = h1.y; gfh[6] = h1.z; gfh[7] = h1.w;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&lu[q]));
                gfl[2 * q] = f.x;
                gfl[2 * q + 1] = f.y;
            }
        }
        uint32_t wz[NSL][4], wp[NSL][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // points 2q, 2q + 1 as (hi, lo, hi, lo)
            const float4 z4 = zs[q];
            float4 f4;
            if constexpr (GRAD) f4 = make_float4(gfh[2 * q], gfl[2 * q], gfh[2 * q + 1], gfl[2 * q + 1]);
            else f4 = fs[q];
            float a0[NSL], a1[NSL], b0[NSL], b1[NSL];
            slice5(z4.x, z4.y, ez, a0);
            slice5(z4.z, z4.w, ez, a1);
            slice5(f4.x, f4.y, ep, b0);
            slice5(f4.z, f4.w, ep, b1);
#pragma unroll
            for (int s = 0; s < NSL; ++s) {
                __nv_bfloat162 bz = __floats2bfloat162_rn(a0[s], a1[s]);
                __nv_bfloat162 bp = __floats2bfloat162_rn(b0[s], b1[s]);
                wz[s][q] = *reinterpret_cast<uint32_t *>(&bz);
                wp[s][q] = *reinterpret_cast<uint32_t *>(&bp);
            }
        }
        const size_t orow = (size_t)(4 * r0 + (int64_t)pk * np + mu) * 32 + col;
#pragma unroll
        for (int s = 0; s < NSL; ++s) {
            *reinterpret_cast<uint4 *>(m.s.vz + (size_t)s * plane + orow) = make_uint4(wz[s][0], wz[s][1], wz[s][2], wz[s][3]);
            *reinterpret_cast<uint4 *>(m.s.vphi + (size_t)s * plane + orow) =
                make_uint4(wp[s][0], wp[s][1], wp[s][2], wp[s][3]);
        }
        if (t == g0 && pg == 0) {
            m.s.zexp[rg + mu] = ez;
            m.s.fexp[rg + mu] = ep;
        }
    }
}

// ---------------------------------------------------------------- host helpers
// Slabs of rows of 32 bf16 (64 B) in `planes` planes; K-major boxes of 16 values x box_rows
// rows with the 32-byte swizzle, or (mn) boxes of all 32 values x 16 rows with the 64-byte
// swizzle, the MN-major operand layout.
CUtensorMap make_map(MixedCtx &c, void *ptr, int64_t rows, int64_t plane_rows, int planes, int box_rows,
                     cudaError_t &err, bool mn = false) {
    CUtensorMap mp;
    std::memset(&mp, 0, sizeof(mp));
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(c.encode_fn);
    cuuint64_t dims[3] = {32, (cuuint64_t)std::max<int64_t>(rows, 1), (cuuint64_t)planes};
    cuuint64_t strides[2] = {64, (cuuint64_t)plane_rows * 64};
    cuuint32_t box[3] = {mn ? 32u : 16u, (cuuint32_t)box_rows, (cuuint32_t)planes};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = encode(&mp, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ptr, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, mn ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) err = cudaErrorInvalidValue;
    return mp;
}

template <typename T>
cudaError_t grow(T *&p, size_t &cap, size_t need) {
    if (need <= cap && p) return cudaSuccess;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(need, 1) * sizeof(T));
    if (e == cudaSuccess) cap = need;
    return e;
}

}  // namespace

MixedSlabOffsets mixed_slab_offsets(int64_t rows) {
    const size_t plane = (size_t)rows * TILE;
    MixedSlabOffsets o;
    o.phi = 0;
    o.ghi = o.phi + plane * 8;
    o.glo = o.ghi + 3 * plane * 4;
    o.x = o.glo + 3 * plane * 2;
    return o;
}

size_t mixed_row_bytes() { return (size_t)TILE * (8 + 12 + 6 + 8 + 3 * NSL * 2) + 8 + 16; }

bool mixed_tile_supported(int bn) { return bn == 128 || bn == 64; }

void append_mixed_vtasks(int j, int n, int64_t s0, int64_t s1, int bn, std::vector<int> &tasks) {
    int mblk = (n + BM - 1) / BM, nblk = (n + bn - 1) / bn;
    for (int64_t k = s0; k < s1; k += VKS) {
        int64_t k1 = std::min<int64_t>(k + VKS, s1);
        for (int mb = 0; mb < mblk; ++mb)
            for (int nb = 0; nb < nblk; ++nb) {
                tasks.push_back(j);
                tasks.push_back(mb);
                tasks.push_back(nb);
                tasks.push_back((int)k);
                tasks.push_back((int)k1);
            }
    }
}

void build_mixed_schedule(const HostPlan &plan, const std::vector<int64_t> &chunk_t0,
                          const std::vector<int64_t> &chunk_t1, int bn, MixedSchedule &s) {
    free_mixed_schedule(s);
    s.bn = bn;
    std::vector<int64_t> pofs;
    std::vector<int> xt, pt;
    for (size_t c = 0; c < chunk_t0.size(); ++c) {
        MixedSchedule::Chunk ch;
        ch.j0 = plan.tile_batch[chunk_t0[c]];
        ch.j1 = plan.tile_batch[chunk_t1[c] - 1];
        ch.prow0 = (int64_t)pofs.size();
        int64_t rows = 0;
        ch.max_np = 0;
        ch.xtask0 = (int64_t)xt.size() / 2;
        for (int64_t t = chunk_t0[c]; t < chunk_t1[c]; ++t) {
            int j = plan.tile_batch[t];
            int64_t n = plan.func_ptr[j + 1] - plan.func_ptr[j];
            for (int nc = 0; (int64_t)nc * bn < n; ++nc) {
                xt.push_back((int)t);
                xt.push_back(nc);
            }
        }
        ch.nxtask = (int64_t)xt.size() / 2 - ch.xtask0;
        ch.ptask0 = (int64_t)pt.size() / 2;
        for (int j = ch.j0; j <= ch.j1; ++j) {
            const int64_t np = pad_funcs(plan.func_ptr[j + 1] - plan.func_ptr[j]);
            for (int64_t mu0 = 0; mu0 < np; mu0 += PS_ROWS) {
                pt.push_back(j - ch.j0);
                pt.push_back((int)mu0);
            }
        }
        ch.nptask = (int64_t)pt.size() / 2 - ch.ptask0;
        for (int j = ch.j0; j <= ch.j1; ++j) {
            int64_t n = plan.func_ptr[j + 1] - plan.func_ptr[j];
            int64_t np = pad_funcs(n);
            pofs.push_back(rows);
            rows += (np / 32) * np;
            ch.max_np = std::max<int>(ch.max_np, (int)np);
        }
        ch.prows = rows;
        ch.max_group = 1;
        for (int j = ch.j0; j <= ch.j1; ++j) {
            const int64_t tb = std::max(plan.batch_tile[j], chunk_t0[c]);
            const int64_t te = std::min(plan.batch_tile[j + 1], chunk_t1[c]);
            ch.max_group = std::max<int>(ch.max_group, (int)std::min<int64_t>(VKS, te - tb));
        }
        s.max_prows = std::max(s.max_prows, rows);
        s.chunks.push_back(ch);
    }
    if (!xt.empty()) {
        cudaMalloc(&s.d_xtasks, xt.size() * sizeof(int));
        cudaMemcpy(s.d_xtasks, xt.data(), xt.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (!pt.empty()) {
        cudaMalloc(&s.d_ptasks, pt.size() * sizeof(int));
        cudaMemcpy(s.d_ptasks, pt.data(), pt.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (!pofs.empty()) {
        cudaMalloc(&s.d_pofs, pofs.size() * sizeof(int64_t));
        cudaMemcpy(s.d_pofs, pofs.data(), pofs.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    }
}

void free_mixed_schedule(MixedSchedule &s) {
    cudaFree(s.d_xtasks);
    cudaFree(s.d_ptasks);
    cudaFree(s.d_pofs);
    s = MixedSchedule{};
}

void free_mixed_resident(MixedResident &r) {
    cudaFree(r.d_shells);
    r = MixedResident{};
}

cudaError_t build_mixed_resident(const std::vector<DevShell> &shells, MixedResident &r) {
    std::vector<DfShell> h(shells.size());
    r.has_pure = false;
    auto split = [](double v, float &hi, float &lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    for (size_t s = 0; s < shells.size(); ++s) {
        const DevShell &d = shells[s];
        DfShell &o = h[s];
        std::memset(&o, 0, sizeof(o));
        for (int c = 0; c < 3; ++c) split(d.c[c], o.ch[c], o.cl[c]);
        for (int k = 0; k < d.nprim; ++k) {
            split(d.alpha[k], o.ah[k], o.al[k]);
            split(d.coeff[k], o.dh[k], o.dl[k]);
            split(-2.0 * d.alpha[k] * d.coeff[k], o.gh[k], o.gl[k]);
        }
        o.L = d.L;
        o.nprim = d.nprim;
        o.fofs = d.fofs;
        o.pure = d.pure;
        if (d.pure) r.has_pure = true;
    }
    cudaFree(r.d_shells);
    r.d_shells = nullptr;
    cudaError_t e = cudaMalloc(&r.d_shells, std::max<size_t>(h.size(), 1) * sizeof(DfShell));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(r.d_shells, h.data(), h.size() * sizeof(DfShell), cudaMemcpyHostToDevice);
}

void free_mixed_ctx(MixedCtx &c) {
    cudaFree(c.pdf);
    cudaFree(c.pdf2);
    cudaFree(c.x2);
    cudaFree(c.zexp2);
    cudaFree(c.ax_g);
    cudaFree(c.y_g);
    cudaFree(c.pexp_g);
    cudaFree(c.wexp_g);
    cudaFree(c.gexp_g);
    cudaFree(c.pslices);
    cudaFree(c.d_err);
    c = MixedCtx{};
}

cudaError_t mixed_init(MixedCtx &c) {
    if (!c.encode_fn) {
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &c.encode_fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || !c.encode_fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
    }
    static bool attr_set = false;
    if (!attr_set) {
        const cudaFuncAttribute smem = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(gemm_persistent<0, 128>, smem, GemmCfg<128>::TOTAL);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_persistent<1, 128>, smem, GemmCfg<128>::TOTAL);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_persistent<0, 64>, smem, GemmCfg<64>::TOTAL);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_persistent<1, 64>, smem, GemmCfg<64>::TOTAL);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_persistent<2, 128>, smem, GemmCfg<128>::TOTAL);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_persistent<2, 64>, smem, GemmCfg<64>::TOTAL);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (!c.num_sms) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        c.num_sms = sms > 0 ? sms : 1;
    }
    return cudaSuccess;
}

cudaError_t mixed_reserve(MixedCtx &c, const MixedSchedule &s, int nbf) {
    cudaError_t e0 = mixed_init(c);
    if (e0 != cudaSuccess) return e0;
    if (!c.d_err) {   // [0] error word of the bounded waits, [1] task counter of the GEMM launches
        cudaError_t e = cudaMalloc(&c.d_err, 4 * sizeof(int));
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = grow(c.pslices, c.pslice_rows, (size_t)std::max<int64_t>(s.max_prows, 1) * 32 * NSL);
    if (e != cudaSuccess) return e;
    return grow(c.pdf, c.pdf_cap, std::max<size_t>(mixed_pdf_floats(nbf), 1));
}

size_t mixed_reserve_bytes(const MixedSchedule &s, int nbf) {
    return (size_t)std::max<int64_t>(s.max_prows, 1) * 32 * NSL * 2 +
           mixed_pdf_floats(nbf) * 4;
}

cudaError_t mixed_begin(MixedCtx &c, const double *P, int nbf, cudaStream_t st) {
    int64_t nn = (int64_t)nbf * nbf;
    if (nn > 0) p_prepare<<<(unsigned)nbf, PP_THREADS, 0, st>>>(P, reinterpret_cast<float2 *>(c.pdf), nbf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(c.d_err, 0, sizeof(int), st);
}

cudaError_t mixed_prepare_p(const double *P, float *pdf, int nbf, cudaStream_t st) {
    int64_t nn = (int64_t)nbf * nbf;
    if (nn > 0) p_prepare<<<(unsigned)nbf, PP_THREADS, 0, st>>>(P, reinterpret_cast<float2 *>(pdf), nbf);
    return cudaGetLastError();
}

cudaError_t mixed_reset_error(MixedCtx &c, cudaStream_t st) { return cudaMemsetAsync(c.d_err, 0, sizeof(int), st); }

cudaError_t mixed_reserve_uks(MixedCtx &c, int64_t max_rows, int nbf) {
    const size_t rows = (size_t)std::max<int64_t>(max_rows, 1);
    cudaError_t e = grow(c.x2, c.x2_cap, rows * TILE);
    if (e != cudaSuccess) return e;
    e = grow(c.zexp2, c.zexp2_cap, rows);
    if (e != cudaSuccess) return e;
    return grow(c.pdf2, c.pdf2_cap, std::max<size_t>(mixed_pdf_floats(nbf), 1));
}

size_t mixed_reserve_uks_bytes(int64_t max_rows, int nbf) {
    const size_t rows = (size_t)std::max<int64_t>(max_rows, 1);
    return rows * TILE * 8 + rows * 4 + mixed_pdf_floats(nbf) * 4;
}

cudaError_t mixed_reserve_mgga(MixedCtx &c, int64_t max_rows) {
    const size_t rows = (size_t)std::max<int64_t>(max_rows, 1);
    cudaError_t e = grow(c.ax_g, c.ax_g_cap, (size_t)3 * NSL * rows * TILE);
    if (e == cudaSuccess) e = grow(c.y_g, c.y_g_cap, (size_t)3 * rows * TILE);
    if (e == cudaSuccess) e = grow(c.pexp_g, c.pexp_g_cap, (size_t)3 * 4 * rows);
    if (e == cudaSuccess) e = grow(c.wexp_g, c.wexp_g_cap, (size_t)3 * rows);
    if (e == cudaSuccess) e = grow(c.gexp_g, c.gexp_g_cap, (size_t)3 * rows);
    c.mgga_rows = e == cudaSuccess ? (int64_t)rows : 0;
    return e;
}

cudaError_t mixed_begin_uks(MixedCtx &c, const double *Pa, const double *Pb, int nbf, cudaStream_t st) {
    cudaError_t e = mixed_begin(c, Pa, nbf, st);
    if (e != cudaSuccess) return e;
    int64_t nn = (int64_t)nbf * nbf;
    if (nn > 0) p_prepare<<<(unsigned)nbf, PP_THREADS, 0, st>>>(Pb, reinterpret_cast<float2 *>(c.pdf2), nbf);
    return cudaGetLastError();
}

cudaError_t mixed_read_error(MixedCtx &c, int *err, cudaStream_t st) {
    *err = 0;
    if (!c.d_err) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(err, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

namespace {
MixedArgs chunk_mixed_args(const ChunkArgs &a, MixedCtx &c, const MixedSchedule &s,
                           const MixedSchedule::Chunk &ch, const float *pdf) {
    MixedArgs m;
    m.s = mixed_slabs(a.scratch, a.rows);
    m.rows = a.rows;
    m.j0 = ch.j0;
    m.pofs = s.d_pofs + ch.prow0;
    m.pslices = reinterpret_cast<__nv_bfloat16 *>(c.pslices);
    m.pplane = std::max<int64_t>(s.max_prows, 1);
    m.pdf = reinterpret_cast<const float2 *>(pdf);
    m.err = c.d_err;
    m.keep_z = c.keep_z;
    m.pad_all = 0;
    return m;
}

struct ChunkMaps {
    CUtensorMap tax, tp, tz, tph, tax_mn;
};

ChunkMaps chunk_maps(MixedCtx &c, const MixedArgs &m, const MixedSchedule &s, const MixedSchedule::Chunk &ch,
                     cudaError_t &err) {
    ChunkMaps q;
    q.tax = make_map(c, m.s.ax, 4 * m.rows, 4 * m.rows, NSL, BM, err);
    q.tp = make_map(c, m.pslices, ch.prows, m.pplane, NSL, s.bn, err);
    q.tz = make_map(c, m.s.vz, 4 * m.rows, 4 * m.rows, NSL, BM, err);
    q.tph = make_map(c, m.s.vphi, 4 * m.rows, 4 * m.rows, NSL, s.bn, err);
    q.tax_mn = make_map(c, m.s.ax, 4 * m.rows, 4 * m.rows, NSL, 16, err, true);
    return q;
}

void run_pslice(const ChunkArgs &a, const MixedArgs &m, const MixedSchedule &s, const MixedSchedule::Chunk &ch,
                cudaStream_t st) {
    Profiler &P = *a.prof;
    P.begin(GBXC_K_PGATHER, st);
    if (ch.nptask > 0)
        pslice_kernel<<<(unsigned)ch.nptask, 32 * PS_WARPS, 0, st>>>(a, m, s.d_ptasks + 2 * ch.ptask0);
    P.end(GBXC_K_PGATHER, st);
}

void run_colloc(const ChunkArgs &a, const MixedArgs &m, const MixedResident &r, int64_t nt, cudaStream_t st) {
    Profiler &P = *a.prof;
    P.begin(GBXC_K_COLLOC, st);
    static const Exp2Table e2t = [] {
        Exp2Table x;
        dfl::make_exp2_table(x.v);
        return x;
    }();
    if (r.has_pure)
        colloc_mixed<true><<<(unsigned)nt, TILE, 0, st>>>(a, m, r.d_shells, e2t);
    else
        colloc_mixed<false><<<(unsigned)nt, TILE, 0, st>>>(a, m, r.d_shells, e2t);
    P.end(GBXC_K_COLLOC, st);
}

void run_xgemm(const ChunkArgs &a, const MixedArgs &m, const ChunkMaps &q, MixedCtx &c, const MixedSchedule &s,
               const MixedSchedule::Chunk &ch, cudaStream_t st) {
    const int *xtasks = s.d_xtasks + 2 * ch.xtask0;
    int nx = (int)ch.nxtask;
    if (nx <= 0) return;
    Profiler &P = *a.prof;
    P.begin(GBXC_K_XGEMM, st);
    const unsigned g = (unsigned)std::min(nx, c.num_sms);
    int *ctr = c.d_err + 1;   // the launch's task counter, claimed by the CTAs' producers
    cudaMemsetAsync(ctr, 0, sizeof(int), st);
    if (s.bn == 64)
        gemm_persistent<0, 64><<<g, GEMM_THREADS, GemmCfg<64>::TOTAL, st>>>(q.tax, q.tp, a, m, xtasks, nx, ctr);
    else
        gemm_persistent<0, 128><<<g, GEMM_THREADS, GemmCfg<128>::TOTAL, st>>>(q.tax, q.tp, a, m, xtasks, nx, ctr);
    P.end(GBXC_K_XGEMM, st);
}

void run_vgemm(const ChunkArgs &a, const MixedArgs &m, const ChunkMaps &q, MixedCtx &c, const MixedSchedule &s,
               cudaStream_t st, bool phi_v_side = false);

void run_slice_vgemm(const ChunkArgs &a, const MixedArgs &m, const ChunkMaps &q, MixedCtx &c,
                     const MixedSchedule &s, int64_t nt, cudaStream_t st) {
    Profiler &P = *a.prof;
    P.begin(GBXC_K_SLICE, st);
    slice_v<false><<<(unsigned)nt, TILE, 0, st>>>(a, m, nullptr, nullptr);
    P.end(GBXC_K_SLICE, st);
    run_vgemm(a, m, q, c, s, st, true);
}

// W^j and its scatter into V_acc: Phi from the V-side slices (slice_v; meta-GGA) or from the
// X-side slices (z_slice's scaled Z; every other form)
void run_vgemm(const ChunkArgs &a, const MixedArgs &m, const ChunkMaps &q, MixedCtx &c, const MixedSchedule &s,
               cudaStream_t st, bool phi_v_side) {
    Profiler &P = *a.prof;
    if (a.nvtasks <= 0) return;
    P.begin(GBXC_K_VGEMM, st);
    const unsigned g = (unsigned)std::min(a.nvtasks, c.num_sms);
    int *ctr = c.d_err + 1;
    cudaMemsetAsync(ctr, 0, sizeof(int), st);
    if (phi_v_side && s.bn == 64)
        gemm_persistent<1, 64><<<g, GEMM_THREADS, GemmCfg<64>::TOTAL, st>>>(q.tz, q.tph, a, m, a.vtasks, a.nvtasks,
                                                                             ctr);
    else if (phi_v_side)
        gemm_persistent<1, 128><<<g, GEMM_THREADS, GemmCfg<128>::TOTAL, st>>>(q.tz, q.tph, a, m, a.vtasks,
                                                                               a.nvtasks, ctr);
    else if (s.bn == 64)
        gemm_persistent<2, 64><<<g, GEMM_THREADS, GemmCfg<64>::TOTAL, st>>>(q.tz, q.tax_mn, a, m, a.vtasks,
                                                                             a.nvtasks, ctr);
    else
        gemm_persistent<2, 128><<<g, GEMM_THREADS, GemmCfg<128>::TOTAL, st>>>(q.tz, q.tax_mn, a, m, a.vtasks,
                                                                               a.nvtasks, ctr);
    P.end(GBXC_K_VGEMM, st);
}
}  // namespace

cudaError_t launch_mixed_chunk(const ChunkArgs &a, MixedCtx &c, MixedResident &r, const MixedSchedule &s,
                               int chunk_index, cudaStream_t st) {
    if (!r.d_shells) return cudaErrorInvalidValue;
    int64_t nt = a.t1 - a.t0;
    if (nt <= 0) return cudaSuccess;
    const MixedSchedule::Chunk &ch = s.chunks[chunk_index];
    MixedArgs m = chunk_mixed_args(a, c, s, ch, c.pdf);
    cudaError_t err = cudaSuccess;
    const ChunkMaps q = chunk_maps(c, m, s, ch, err);
    if (err != cudaSuccess) return err;
    run_pslice(a, m, s, ch, st);
    run_colloc(a, m, r, nt, st);
    run_xgemm(a, m, q, c, s, ch, st);
    Profiler &P = *a.prof;
    P.begin(GBXC_K_RHO_Z, st);
    rho_mixed<<<(unsigned)nt, TILE, 0, st>>>(a, m);
    P.end(GBXC_K_RHO_Z, st);
    P.begin(GBXC_K_SLICE, st);
    z_slice<<<(unsigned)nt, TILE, z_slice_smem(ch.max_group), st>>>(a, m);
    P.end(GBXC_K_SLICE, st);
    run_vgemm(a, m, q, c, s, st);
    return cudaGetLastError();
}

// Meta-GGA chunk: the collocation, then the slices of d_k Phi; X and the three Y^k on the
// same P^j slices (Y^k through the X/Z plane of a per-component copy of the slab view); the
// rho/tau/functional/Z/W^k kernel; the V term Z^T Phi as in the spin-restricted form, then
// each W^k^T d_k Phi with its own slicing (W^k from its Y^k plane, d_k Phi from the gradient
// planes) into the same V_acc.
cudaError_t launch_mixed_chunk_mgga(const ChunkArgs &a, MixedCtx &c, MixedResident &r, const MixedSchedule &s,
                                    int chunk_index, cudaStream_t st) {
    if (!r.d_shells || !c.ax_g || !c.y_g || !c.pexp_g || !c.wexp_g || !c.gexp_g) return cudaErrorInvalidValue;
    if (a.rows > c.mgga_rows) return cudaErrorInvalidValue;
    int64_t nt = a.t1 - a.t0;
    if (nt <= 0) return cudaSuccess;
    const MixedSchedule::Chunk &ch = s.chunks[chunk_index];
    MixedArgs m = chunk_mixed_args(a, c, s, ch, c.pdf);
    m.pad_all = 1;   // rho_z_mixed_mgga and grad_slices read every point of a tile
    cudaError_t err = cudaSuccess;
    const ChunkMaps q = chunk_maps(c, m, s, ch, err);
    const size_t plane = (size_t)a.rows * TILE;
    __nv_bfloat16 *axg = reinterpret_cast<__nv_bfloat16 *>(c.ax_g);
    CUtensorMap tg[3];
    for (int k = 0; k < 3; ++k)
        tg[k] = make_map(c, axg + (size_t)k * NSL * plane, 4 * a.rows, 4 * a.rows, NSL, BM, err);
    if (err != cudaSuccess) return err;
    Profiler &P = *a.prof;
    run_pslice(a, m, s, ch, st);
    run_colloc(a, m, r, nt, st);
    P.begin(GBXC_K_COLLOC, st);
    grad_slices<<<(unsigned)nt, TILE, 0, st>>>(a, m, axg, c.pexp_g);
    P.end(GBXC_K_COLLOC, st);
    run_xgemm(a, m, q, c, s, ch, st);
    for (int k = 0; k < 3; ++k) {
        MixedArgs mk = m;
        mk.s.pexp = c.pexp_g + (size_t)k * 4 * a.rows;
        mk.s.x = c.y_g + (size_t)k * plane;
        ChunkMaps qk = q;
        qk.tax = tg[k];
        run_xgemm(a, mk, qk, c, s, ch, st);
    }
    P.begin(GBXC_K_RHO_Z, st);
    rho_z_mixed_mgga<<<(unsigned)nt, TILE, 0, st>>>(a, m, c.y_g, c.wexp_g, c.gexp_g);
    P.end(GBXC_K_RHO_Z, st);
    run_slice_vgemm(a, m, q, c, s, nt, st);
    for (int k = 0; k < 3; ++k) {
        MixedArgs mk = m;
        mk.s.x = c.y_g + (size_t)k * plane;
        mk.s.zexp = c.wexp_g + (size_t)k * a.rows;
        mk.s.fexp = c.gexp_g + (size_t)k * a.rows;
        P.begin(GBXC_K_SLICE, st);
        slice_v<true><<<(unsigned)nt, TILE, 0, st>>>(a, mk, m.s.ghi + (size_t)k * plane, m.s.glo + (size_t)k * plane);
        P.end(GBXC_K_SLICE, st);
        run_vgemm(a, mk, q, c, s, st, true);
    }
    return cudaGetLastError();
}

// Spin-unrestricted chunk: one collocation; P_a's slices and X_a (into the slab), then P_b's
// slices and X_b (into x2), both densities and the spin-polarised functional in one kernel
// (the Z^a coefficients over X_a, the Z^b coefficients over X_b), then z_slice and W^j per
// spin, spin b with x2 and zexp2 in place of the slab's X plane and Z exponents.  The Phi
// slices of the second slicing are the same values as the first's.
cudaError_t launch_mixed_chunk_uks(const ChunkArgs &a, MixedCtx &c, MixedResident &r, const MixedSchedule &s,
                                   int chunk_index, double *Vacc_b, cudaStream_t st) {
    if (!r.d_shells || !c.x2 || !c.zexp2 || !c.pdf2) return cudaErrorInvalidValue;
    if ((size_t)a.rows > c.zexp2_cap || (size_t)a.rows * TILE > c.x2_cap) return cudaErrorInvalidValue;
    int64_t nt = a.t1 - a.t0;
    if (nt <= 0) return cudaSuccess;
    const MixedSchedule::Chunk &ch = s.chunks[chunk_index];
    MixedArgs ma = chunk_mixed_args(a, c, s, ch, c.pdf);
    MixedArgs mb = chunk_mixed_args(a, c, s, ch, c.pdf2);
    mb.s.x = c.x2;
    mb.s.zexp = c.zexp2;
    cudaError_t err = cudaSuccess;
    const ChunkMaps q = chunk_maps(c, ma, s, ch, err);
    if (err != cudaSuccess) return err;
    run_pslice(a, ma, s, ch, st);
    run_colloc(a, ma, r, nt, st);
    run_xgemm(a, ma, q, c, s, ch, st);
    run_pslice(a, mb, s, ch, st);
    run_xgemm(a, mb, q, c, s, ch, st);
    Profiler &P = *a.prof;
    P.begin(GBXC_K_RHO_Z, st);
    rho_mixed_uks<<<(unsigned)nt, TILE, 0, st>>>(a, ma, c.x2);
    P.end(GBXC_K_RHO_Z, st);
    P.begin(GBXC_K_SLICE, st);
    z_slice<<<(unsigned)nt, TILE, z_slice_smem(ch.max_group), st>>>(a, ma);
    P.end(GBXC_K_SLICE, st);
    run_vgemm(a, ma, q, c, s, st);
    ChunkArgs ab = a;
    ab.Vacc = Vacc_b;
    P.begin(GBXC_K_SLICE, st);
    z_slice<<<(unsigned)nt, TILE, z_slice_smem(ch.max_group), st>>>(ab, mb);
    P.end(GBXC_K_SLICE, st);
    run_vgemm(ab, mb, q, c, s, st);
    return cudaGetLastError();
}

}  // namespace gbxc
