// Float64 form of the batched integration (Algorithm 4), one chunk of tiles at a time.
//
// Scratch layout ("slabs"): every 128-point tile t of batch j owns N_b^j rows
// (padded to a multiple of 16) of 128 doubles each, function-major, so that the
// 128 points of a row are contiguous.  Six slab arrays follow each other:
// Phi, dPhi/dx, dPhi/dy, dPhi/dz, X and Z.
//
//   k1  collocation       Phi^j and grad Phi^j (Eq. gau_cart)            thread per point
//   k3  X = P^j Phi^j     (Eq. x_mat) with P^j gathered from P on the fly  64 x 128 output tile
//   k45 rho, grad rho (Eqs. eval_local_den, eval_local_den_grad), the
//       functional (Eq. eval_xc_batch), E/N partial sums (Eq. exc_batch)
//       and Z^j (Eq. z_mat)                                                thread per point
//   k6  W^j = Z^jT Phi^j summed over the batch's points and scattered into
//       V_acc[S_j, S_j] (Eqs. vxc_batch, vxc_inc); V = V_acc + V_acc^T at the end.
//
// On this GPU float64 runs at a small fraction of float32 and tensor rates, so
// these kernels are bound by the float64 pipe; they are the precision anchor.
#include <atomic>
#include <cstdint>

#include "internal.h"
#include "solid_harmonics.cuh"
#include "group.cuh"
#include "xc_functional.cuh"

namespace gbxc {
namespace {

// planes: Phi, Phi_x, Phi_y, Phi_z, then X / Z (4), a second X / Z (5: the other spin, or Z
// of the spin-restricted form), and for the meta-GGA Y^k = (d_k Phi) P^j, later
// W^k = 1/4 w vtau d_k Phi, in planes 5, 6, 7
constexpr int NCOMP = 8;

struct Slabs {
    double *c[NCOMP];
};

__device__ __forceinline__ Slabs slabs_of(const ChunkArgs &a) {
    Slabs s;
    double *base = static_cast<double *>(a.scratch);
    for (int k = 0; k < NCOMP; ++k) s.c[k] = base + (size_t)k * a.rows * TILE;
    return s;
}

// --------------------------------------------------------------------------
// k1: collocation.  One block per tile, one thread per point; a warp walks the
// same shell list for 32 points (no divergence between shells).
// --------------------------------------------------------------------------
// A pure shell (L = 2 or 3): its Cartesian functions and gradients, then the 2L+1 real
// solid harmonics of each component (solid_harmonics.cuh), written as rows row .. row + 2L.
template <int L>
__device__ __forceinline__ void pure_shell_f64(double X, double Y, double Z, double g, double h, const Slabs &S,
                                               int64_t row0, int row, int i, bool live) {
    constexpr int NC = (L + 1) * (L + 2) / 2, NO = 2 * L + 1;
    double xp[L + 1], yp[L + 1], zp[L + 1];
    xp[0] = yp[0] = zp[0] = 1.0;
#pragma unroll
    for (int k = 1; k <= L; ++k) {
        xp[k] = xp[k - 1] * X;
        yp[k] = yp[k - 1] * Y;
        zp[k] = zp[k - 1] * Z;
    }
    double cv[4][NC];
    int f = 0;
#pragma unroll
    for (int l = L; l >= 0; --l)
#pragma unroll
        for (int m = L - l; m >= 0; --m) {
            const int n = L - l - m;
            const double mono = xp[l] * yp[m] * zp[n];
            cv[0][f] = mono * g;
            cv[1][f] = (l > 0 ? l * xp[l > 0 ? l - 1 : 0] * yp[m] * zp[n] : 0.0) * g + mono * X * h;
            cv[2][f] = (m > 0 ? m * xp[l] * yp[m > 0 ? m - 1 : 0] * zp[n] : 0.0) * g + mono * Y * h;
            cv[3][f] = (n > 0 ? n * xp[l] * yp[m] * zp[n > 0 ? n - 1 : 0] : 0.0) * g + mono * Z * h;
            ++f;
        }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double o[NO];
        sph::pure<L, sph::DoubleOps>(cv[c], o);
#pragma unroll
        for (int k = 0; k < NO; ++k) S.c[c][(size_t)(row0 + row + k) * TILE + i] = live ? o[k] : 0.0;
    }
}

__global__ void __launch_bounds__(TILE) colloc_f64(ChunkArgs a) {
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int cnt = a.plan.tile_count[t];
    int64_t row0 = a.plan.tile_row[t] - a.row0;
    Slabs S = slabs_of(a);
    bool live = i < cnt;
    int64_t p = a.plan.tile_first[t] + i;
    double px = live ? a.plan.x[p] : 0.0, py = live ? a.plan.y[p] : 0.0,
           pz = live ? a.plan.z[p] : 0.0;
    int64_t s0 = a.plan.shell_ptr[j], s1 = a.plan.shell_ptr[j + 1];
    int row = 0;
    for (int64_t si = s0; si < s1; ++si) {
        const DevShell &sh = a.shells[a.plan.shell_idx[si]];
        double X = px - sh.c[0], Y = py - sh.c[1], Z = pz - sh.c[2];
        double r2 = X * X + Y * Y + Z * Z;
        double g = 0.0, h = 0.0;
        for (int k = 0; k < sh.nprim; ++k) {
            double e = exp(-sh.alpha[k] * r2);
            g += sh.coeff[k] * e;
            h += (-2.0 * sh.alpha[k] * sh.coeff[k]) * e;
        }
        if (sh.pure) {
            if (sh.L == 2) pure_shell_f64<2>(X, Y, Z, g, h, S, row0, row, i, live);
            else pure_shell_f64<3>(X, Y, Z, g, h, S, row0, row, i, live);
            row += 2 * sh.L + 1;
            continue;
        }
        double xp[GBXC_MAX_L + 2], yp[GBXC_MAX_L + 2], zp[GBXC_MAX_L + 2];
        xp[0] = yp[0] = zp[0] = 1.0;
        for (int k = 1; k <= sh.L; ++k) {
            xp[k] = xp[k - 1] * X;
            yp[k] = yp[k - 1] * Y;
            zp[k] = zp[k - 1] * Z;
        }
        for (int l = sh.L; l >= 0; --l)
            for (int m = sh.L - l; m >= 0; --m) {
                int n = sh.L - l - m;
                double mono = xp[l] * yp[m] * zp[n];
                double dx = (l > 0 ? l * xp[l - 1] * yp[m] * zp[n] : 0.0) * g + mono * X * h;
                double dy = (m > 0 ? m * xp[l] * yp[m - 1] * zp[n] : 0.0) * g + mono * Y * h;
                double dz = (n > 0 ? n * xp[l] * yp[m] * zp[n - 1] : 0.0) * g + mono * Z * h;
                size_t o = (size_t)(row0 + row) * TILE + i;
                S.c[0][o] = live ? mono * g : 0.0;
                S.c[1][o] = live ? dx : 0.0;
                S.c[2][o] = live ? dy : 0.0;
                S.c[3][o] = live ? dz : 0.0;
                ++row;
            }
    }
}

// --------------------------------------------------------------------------
// k3: X^j (rows = functions, cols = points) = P^j Phi^j, P^j[r][k] = P[F_r][F_k].
// Block (tile t, row block rb) computes 64 rows x 128 points; 256 threads,
// each 4 rows x 8 points.  K = N_b^j in steps of 16.
// --------------------------------------------------------------------------
constexpr int XB_R = 64, XB_K = 16;

// X = P^j Phi^j from density P into slab plane `out` (4, or 5 for the second spin).
__global__ void __launch_bounds__(256) xgemm_f64(ChunkArgs a, const double *__restrict__ P, int in, int out) {
    int64_t t = a.t0 + blockIdx.x;
    int rb = blockIdx.y;
    int j = a.plan.tile_batch[t];
    int nbf = a.nbf;
    if (a.batch_mol) {   // grouped chunk: the batch's own molecule
        const MolRef r = mol_of(a, j);
        P = r.P;
        nbf = r.nbf;
    }
    int64_t f0 = a.plan.func_ptr[j];
    int n = (int)(a.plan.func_ptr[j + 1] - f0);
    int r0 = rb * XB_R;
    if (r0 >= n) return;
    const int *F = a.plan.func_idx + f0;
    Slabs S = slabs_of(a);
    int64_t row0 = a.plan.tile_row[t] - a.row0;
    const double *Phi = S.c[in] + (size_t)row0 * TILE;
    double *Xo = S.c[out] + (size_t)row0 * TILE;

    __shared__ double As[XB_K][XB_R + 1];
    __shared__ double Bs[XB_K][TILE];
    __shared__ int Frow[XB_R];
    int tid = threadIdx.x;
    if (tid < XB_R) Frow[tid] = (r0 + tid < n) ? F[r0 + tid] : -1;
    int tx = tid & 15, ty = tid >> 4;
    double acc[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.0;
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += XB_K) {
        // A tile: P[F[r0 + rr]][F[k0 + kk]]
        for (int e = tid; e < XB_K * XB_R; e += 256) {
            int kk = e / XB_R, rr = e % XB_R;
            int k = k0 + kk;
            int fr = Frow[rr];
            As[kk][rr] = (fr >= 0 && k < n) ? P[(size_t)fr * nbf + F[k]] : 0.0;
        }
        for (int e = tid; e < XB_K * TILE; e += 256) {
            int kk = e / TILE, c = e % TILE;
            int k = k0 + kk;
            Bs[kk][c] = (k < n) ? Phi[(size_t)k * TILE + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < XB_K; ++kk) {
            double av[4], bv[8];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = As[kk][ty * 4 + u];
#pragma unroll
            for (int v = 0; v < 8; ++v) bv[v] = Bs[kk][tx + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r = r0 + ty * 4 + u;
        if (r >= n) continue;
#pragma unroll
        for (int v = 0; v < 8; ++v) Xo[(size_t)r * TILE + tx + 16 * v] = acc[u][v];
    }
}

// --------------------------------------------------------------------------
// k45: rho, grad rho, functional, E/N partials, Z.  One block per tile.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE) rho_xc_z_f64(ChunkArgs a) {
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int cnt = a.plan.tile_count[t];
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int64_t row0 = a.plan.tile_row[t] - a.row0;
    Slabs S = slabs_of(a);
    size_t base = (size_t)row0 * TILE + i;
    double rho = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int r = 0; r < n; ++r) {
        size_t o = base + (size_t)r * TILE;
        double xv = S.c[4][o];
        rho = fma(S.c[0][o], xv, rho);
        gx = fma(S.c[1][o], xv, gx);
        gy = fma(S.c[2][o], xv, gy);
        gz = fma(S.c[3][o], xv, gz);
    }
    gx *= 2.0;
    gy *= 2.0;
    gz *= 2.0;
    double e = 0.0, nn = 0.0, ca = 0.0, bx = 0.0, by = 0.0, bz = 0.0;
    if (i < cnt) {
        double w = a.plan.w[a.plan.tile_first[t] + i];
        double sigma = gx * gx + gy * gy + gz * gz;
        double f, vr, vs;
        xc::evaluate<double>(mol_of(a, j).functional, rho, sigma, f, vr, vs);
        e = w * f;
        nn = w * rho;
        ca = 0.5 * w * vr;
        double b = 2.0 * w * vs;
        bx = b * gx;
        by = b * gy;
        bz = b * gz;
    }
    for (int r = 0; r < n; ++r) {
        size_t o = base + (size_t)r * TILE;
        S.c[5][o] = ca * S.c[0][o] + bx * S.c[1][o] + by * S.c[2][o] + bz * S.c[3][o];
    }
    // deterministic block reduction of the E and N partials
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

// --------------------------------------------------------------------------
// k45, spin-unrestricted (the extension of Sec. 2.1): X^a in plane 4 and X^b in plane 5 give
// rho_s and grad rho_s per spin; the spin-polarised functional; then per spin
// Z^s = 1/2 w v_s Phi + w (2 s_ss grad rho_s + s_ab grad rho_s') . grad Phi over X^s.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE) rho_xc_z_uks_f64(ChunkArgs a) {
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int cnt = a.plan.tile_count[t];
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int64_t row0 = a.plan.tile_row[t] - a.row0;
    Slabs S = slabs_of(a);
    size_t base = (size_t)row0 * TILE + i;
    double rho[2] = {0.0, 0.0}, g[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int r = 0; r < n; ++r) {
        size_t o = base + (size_t)r * TILE;
        const double p0 = S.c[0][o], p1 = S.c[1][o], p2 = S.c[2][o], p3 = S.c[3][o];
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
            const double xv = S.c[4 + sp][o];
            rho[sp] = fma(p0, xv, rho[sp]);
            g[sp][0] = fma(p1, xv, g[sp][0]);
            g[sp][1] = fma(p2, xv, g[sp][1]);
            g[sp][2] = fma(p3, xv, g[sp][2]);
        }
    }
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int d = 0; d < 3; ++d) g[sp][d] *= 2.0;
    double e = 0.0, nn = 0.0, ca[2] = {0.0, 0.0}, cb[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    if (i < cnt) {
        const double w = a.plan.w[a.plan.tile_first[t] + i];
        const double saa = g[0][0] * g[0][0] + g[0][1] * g[0][1] + g[0][2] * g[0][2];
        const double sab = g[0][0] * g[1][0] + g[0][1] * g[1][1] + g[0][2] * g[1][2];
        const double sbb = g[1][0] * g[1][0] + g[1][1] * g[1][1] + g[1][2] * g[1][2];
        double f, va, vb, s_aa, s_ab, s_bb;
        xc::evaluate_pol<double>(a.functional, rho[0], rho[1], saa, sab, sbb, f, va, vb, s_aa, s_ab, s_bb);
        e = w * f;
        nn = w * (rho[0] + rho[1]);
        ca[0] = 0.5 * w * va;
        ca[1] = 0.5 * w * vb;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cb[0][d] = w * (2.0 * s_aa * g[0][d] + s_ab * g[1][d]);
            cb[1][d] = w * (2.0 * s_bb * g[1][d] + s_ab * g[0][d]);
        }
    }
    for (int r = 0; r < n; ++r) {
        size_t o = base + (size_t)r * TILE;
        const double p0 = S.c[0][o], p1 = S.c[1][o], p2 = S.c[2][o], p3 = S.c[3][o];
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
            S.c[4 + sp][o] = ca[sp] * p0 + cb[sp][0] * p1 + cb[sp][1] * p2 + cb[sp][2] * p3;
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

// --------------------------------------------------------------------------
// k45, meta-GGA (the extension of Sec. 2.1): rho and grad rho from X (plane 4), the kinetic
// energy density tau = 1/2 sum_k sum_mu d_k Phi Y^k from Y^k = (d_k Phi) P^j (planes 5-7),
// the meta-GGA functional, then Z over X (plane 4) and W^k = 1/4 w vtau d_k Phi over Y^k,
// so that V^j = Z^T Phi + sum_k W^k^T d_k Phi plus the transpose.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE) rho_xc_z_mgga_f64(ChunkArgs a) {
    int64_t t = a.t0 + blockIdx.x;
    int i = threadIdx.x;
    int j = a.plan.tile_batch[t];
    int cnt = a.plan.tile_count[t];
    int n = (int)(a.plan.func_ptr[j + 1] - a.plan.func_ptr[j]);
    int64_t row0 = a.plan.tile_row[t] - a.row0;
    Slabs S = slabs_of(a);
    size_t base = (size_t)row0 * TILE + i;
    double rho = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, tau = 0.0;
    for (int r = 0; r < n; ++r) {
        size_t o = base + (size_t)r * TILE;
        const double xv = S.c[4][o], p1 = S.c[1][o], p2 = S.c[2][o], p3 = S.c[3][o];
        rho = fma(S.c[0][o], xv, rho);
        gx = fma(p1, xv, gx);
        gy = fma(p2, xv, gy);
        gz = fma(p3, xv, gz);
        tau = fma(p1, S.c[5][o], tau);
        tau = fma(p2, S.c[6][o], tau);
        tau = fma(p3, S.c[7][o], tau);
    }
    gx *= 2.0;
    gy *= 2.0;
    gz *= 2.0;
    tau *= 0.5;
    double e = 0.0, nn = 0.0, ca = 0.0, bx = 0.0, by = 0.0, bz = 0.0, ct = 0.0;
    if (i < cnt) {
        const double w = a.plan.w[a.plan.tile_first[t] + i];
        const double sigma = gx * gx + gy * gy + gz * gz;
        double f, vr, vs, vt;
        xc::mvs_x(rho, sigma, tau, f, vr, vs, vt);
        e = w * f;
        nn = w * rho;
        ca = 0.5 * w * vr;
        const double b = 2.0 * w * vs;
        bx = b * gx;
        by = b * gy;
        bz = b * gz;
        ct = 0.25 * w * vt;
    }
    for (int r = 0; r < n; ++r) {
        size_t o = base + (size_t)r * TILE;
        const double p1 = S.c[1][o], p2 = S.c[2][o], p3 = S.c[3][o];
        S.c[4][o] = ca * S.c[0][o] + bx * p1 + by * p2 + bz * p3;
        S.c[5][o] = ct * p1;
        S.c[6][o] = ct * p2;
        S.c[7][o] = ct * p3;
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

// --------------------------------------------------------------------------
// k6: W^j[mu][nu] = sum_i Z[mu][i] Phi[nu][i] over tiles [t0, t1) of batch j,
// 64 x 64 output block per CTA (256 threads, 4 x 4 each), then
// V_acc[F_mu][F_nu] += W (float64 atomics).
// --------------------------------------------------------------------------
constexpr int VB = 64, VK = 16;

// W = Z^T Phi from slab planes `zp` (5, or 4 for the first spin of the unrestricted form and
// the meta-GGA's Z, 5-7 for its W^k) and `pp` (Phi, or d_k Phi for the meta-GGA terms),
// scattered into Vacc.
__global__ void __launch_bounds__(256) vgemm_f64(ChunkArgs a, int zp, int pp, double *__restrict__ Vacc) {
    const int *task = a.vtasks + 5 * blockIdx.x;
    int j = task[0], mb = task[1], nb = task[2];
    int nbf = a.nbf;
    if (a.batch_mol) {   // grouped chunk: the batch's own molecule
        const MolRef r = mol_of(a, j);
        Vacc = r.Vacc;
        nbf = r.nbf;
    }
    int64_t tb = task[3], te = task[4];
    int64_t f0 = a.plan.func_ptr[j];
    int n = (int)(a.plan.func_ptr[j + 1] - f0);
    const int *F = a.plan.func_idx + f0;
    int m0 = mb * VB, n0 = nb * VB;
    Slabs S = slabs_of(a);
    __shared__ double As[VK][VB + 1];
    __shared__ double Bs[VK][VB + 1];
    int tid = threadIdx.x;
    int tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
    for (int64_t t = tb; t < te; ++t) {
        int64_t row0 = a.plan.tile_row[t] - a.row0;
        const double *Zs = S.c[zp] + (size_t)row0 * TILE;
        const double *Ps = S.c[pp] + (size_t)row0 * TILE;
        int cnt = a.plan.tile_count[t];
        for (int k0 = 0; k0 < cnt; k0 += VK) {
            for (int e = tid; e < VK * VB; e += 256) {
                int rr = e / VK, kk = e % VK;
                int k = k0 + kk;
                int mr = m0 + rr, nr = n0 + rr;
                As[kk][rr] = (mr < n && k < cnt) ? Zs[(size_t)mr * TILE + k] : 0.0;
                Bs[kk][rr] = (nr < n && k < cnt) ? Ps[(size_t)nr * TILE + k] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < VK; ++kk) {
                double av[4], bv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) av[u] = As[kk][ty * 4 + u];
#pragma unroll
                for (int v = 0; v < 4; ++v) bv[v] = Bs[kk][tx * 4 + v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int mr = m0 + ty * 4 + u;
        if (mr >= n) continue;
        size_t rowg = (size_t)F[mr] * nbf;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int nr = n0 + tx * 4 + v;
            if (nr < n) atomicAdd(&Vacc[rowg + F[nr]], acc[u][v]);
        }
    }
}

// --------------------------------------------------------------------------
// finish: V = V_acc + V_acc^T; per-batch and total E, N in a fixed order.
// --------------------------------------------------------------------------
// flag <- 1 if any of P[0 .. n) is a NaN or an infinity (a density that the functionals'
// rho >= RHO_MIN test would otherwise drop point by point without a trace)
__global__ void nonfinite_flag(const double *__restrict__ P, int64_t n, double *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(P[i])) {
            *flag = 1.0;
            return;
        }
}

// {E, N} <- NaN when the flag is set: the allocation-free call returns before its status could
// report a non-finite P, so the results themselves carry it.
__global__ void poison_if_flagged(const double *__restrict__ flag, double *EN) {
    if (threadIdx.x == 0 && *flag != 0.0) {
        EN[0] = __longlong_as_double(0x7ff8000000000000LL);
        EN[1] = __longlong_as_double(0x7ff8000000000000LL);
    }
}

__global__ void symmetrize(const double *__restrict__ Vacc, double *__restrict__ V, int nbf) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nbf * nbf) return;
    int r = (int)(e / nbf), c = (int)(e % nbf);
    V[e] = Vacc[e] + Vacc[(size_t)c * nbf + r];
}

__global__ void batch_sums(FinishArgs a) {
    int j = a.b0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.b1) return;
    double e = 0.0, n = 0.0;
    for (int64_t t = a.batch_tile[j]; t < a.batch_tile[j + 1]; ++t) {
        e += a.tileE[t];
        n += a.tileN[t];
    }
    a.Eb[j] = e;
    a.Nb[j] = n;
}

__global__ void total_sums(FinishArgs a) {
    __shared__ double se[256], sn[256];
    double e = 0.0, n = 0.0;
    for (int j = a.b0 + threadIdx.x; j < a.b1; j += 256) {
        e += a.Eb[j];
        n += a.Nb[j];
    }
    se[threadIdx.x] = e;
    sn[threadIdx.x] = n;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sn[threadIdx.x] += sn[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.tot[0] = se[0];
        a.tot[1] = sn[0];
    }
}

// --------------------------------------------------------------------------
// Allocation-free variant (gbxc_integrate_fp64_noalloc).  Its slab scratch is this
// file-scope device array, which every GPU that loads the library holds until exit.
// Host code may not use the array's name as a device address: the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
// --------------------------------------------------------------------------
constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;
constexpr size_t kNoallocFlagBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// W^j over one tile (K = its 128 points) for the 64 x 64 block (blockIdx.y, blockIdx.z),
// scattered into V_acc with float64 atomics.
__global__ void __launch_bounds__(256) vgemm_f64_tile(ChunkArgs a) {
    int64_t t = a.t0 + blockIdx.x;
    int mb = blockIdx.y, nb = blockIdx.z;
    int j = a.plan.tile_batch[t];
    int64_t f0 = a.plan.func_ptr[j];
    int n = (int)(a.plan.func_ptr[j + 1] - f0);
    int m0 = mb * VB, n0 = nb * VB;
    if (m0 >= n || n0 >= n) return;
    const int *F = a.plan.func_idx + f0;
    Slabs S = slabs_of(a);
    int64_t row0 = a.plan.tile_row[t] - a.row0;
    const double *Zs = S.c[5] + (size_t)row0 * TILE;
    const double *Ps = S.c[0] + (size_t)row0 * TILE;
    int cnt = a.plan.tile_count[t];
    __shared__ double As[VK][VB + 1];
    __shared__ double Bs[VK][VB + 1];
    int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < cnt; k0 += VK) {
        for (int e = tid; e < VK * VB; e += 256) {
            int rr = e / VK, kk = e % VK, k = k0 + kk;
            As[kk][rr] = (m0 + rr < n && k < cnt) ? Zs[(size_t)(m0 + rr) * TILE + k] : 0.0;
            Bs[kk][rr] = (n0 + rr < n && k < cnt) ? Ps[(size_t)(n0 + rr) * TILE + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < VK; ++kk)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(As[kk][ty * 4 + u], Bs[kk][tx * 4 + v], acc[u][v]);
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u) {
        int mr = m0 + ty * 4 + u;
        if (mr >= n) continue;
        for (int v = 0; v < 4; ++v) {
            int nr = n0 + tx * 4 + v;
            if (nr < n) atomicAdd(&a.Vacc[(size_t)F[mr] * a.nbf + F[nr]], acc[u][v]);
        }
    }
}

// V <- V + V^T in place: the thread of pair (r, c), r < c, owns both entries.
__global__ void symmetrize_inplace(double *V, int nbf) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nbf * nbf) return;
    int r = (int)(e / nbf), c = (int)(e % nbf);
    if (r > c) return;
    double s = V[e] + V[(size_t)c * nbf + r];
    V[e] = s;
    V[(size_t)c * nbf + r] = s;
}

}  // namespace

cudaError_t launch_fp64_chunk(const ChunkArgs &a, cudaStream_t s) {
    int64_t nt = a.t1 - a.t0;
    if (nt <= 0) return cudaSuccess;
    Profiler &P = *a.prof;
    P.begin(GBXC_K_COLLOC, s);
    colloc_f64<<<(unsigned)nt, TILE, 0, s>>>(a);
    P.end(GBXC_K_COLLOC, s);
    dim3 xg((unsigned)nt, (unsigned)((a.max_nfunc + XB_R - 1) / XB_R));
    P.begin(GBXC_K_XGEMM, s);
    xgemm_f64<<<xg, 256, 0, s>>>(a, a.P, 0, 4);
    P.end(GBXC_K_XGEMM, s);
    P.begin(GBXC_K_RHO_Z, s);
    rho_xc_z_f64<<<(unsigned)nt, TILE, 0, s>>>(a);
    P.end(GBXC_K_RHO_Z, s);
    if (a.nvtasks > 0) {
        P.begin(GBXC_K_VGEMM, s);
        vgemm_f64<<<(unsigned)a.nvtasks, 256, 0, s>>>(a, 5, 0, a.Vacc);
        P.end(GBXC_K_VGEMM, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_fp64_chunk_uks(const ChunkArgs &a, const double *Pb, double *Vacc_b, cudaStream_t s) {
    int64_t nt = a.t1 - a.t0;
    if (nt <= 0) return cudaSuccess;
    Profiler &P = *a.prof;
    P.begin(GBXC_K_COLLOC, s);
    colloc_f64<<<(unsigned)nt, TILE, 0, s>>>(a);
    P.end(GBXC_K_COLLOC, s);
    dim3 xg((unsigned)nt, (unsigned)((a.max_nfunc + XB_R - 1) / XB_R));
    P.begin(GBXC_K_XGEMM, s);
    xgemm_f64<<<xg, 256, 0, s>>>(a, a.P, 0, 4);
    xgemm_f64<<<xg, 256, 0, s>>>(a, Pb, 0, 5);
    P.end(GBXC_K_XGEMM, s, 2);
    P.begin(GBXC_K_RHO_Z, s);
    rho_xc_z_uks_f64<<<(unsigned)nt, TILE, 0, s>>>(a);
    P.end(GBXC_K_RHO_Z, s);
    if (a.nvtasks > 0) {
        P.begin(GBXC_K_VGEMM, s);
        vgemm_f64<<<(unsigned)a.nvtasks, 256, 0, s>>>(a, 4, 0, a.Vacc);
        vgemm_f64<<<(unsigned)a.nvtasks, 256, 0, s>>>(a, 5, 0, Vacc_b);
        P.end(GBXC_K_VGEMM, s, 2);
    }
    return cudaGetLastError();
}

cudaError_t launch_fp64_chunk_mgga(const ChunkArgs &a, cudaStream_t s) {
    int64_t nt = a.t1 - a.t0;
    if (nt <= 0) return cudaSuccess;
    Profiler &P = *a.prof;
    P.begin(GBXC_K_COLLOC, s);
    colloc_f64<<<(unsigned)nt, TILE, 0, s>>>(a);
    P.end(GBXC_K_COLLOC, s);
    dim3 xg((unsigned)nt, (unsigned)((a.max_nfunc + XB_R - 1) / XB_R));
    P.begin(GBXC_K_XGEMM, s);
    for (int k = 0; k < 4; ++k) xgemm_f64<<<xg, 256, 0, s>>>(a, a.P, k, 4 + k);   // X, then Y^x, Y^y, Y^z
    P.end(GBXC_K_XGEMM, s, 4);
    P.begin(GBXC_K_RHO_Z, s);
    rho_xc_z_mgga_f64<<<(unsigned)nt, TILE, 0, s>>>(a);
    P.end(GBXC_K_RHO_Z, s);
    if (a.nvtasks > 0) {
        P.begin(GBXC_K_VGEMM, s);
        for (int k = 0; k < 4; ++k) vgemm_f64<<<(unsigned)a.nvtasks, 256, 0, s>>>(a, 4 + k, k, a.Vacc);
        P.end(GBXC_K_VGEMM, s, 4);
    }
    return cudaGetLastError();
}

cudaError_t noalloc_scratch(void **ptr, size_t *bytes, double **flag) {
    // one cached address per device, kept for the life of the process; the first call on a
    // device resolves it (threads racing on that first call store the same value)
    static std::atomic<void *> cache[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    void *p = cache[dev].load(std::memory_order_acquire);
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        cache[dev].store(p, std::memory_order_release);
    }
    // the first 256 bytes hold the non-finite-P flag, the rest the slabs
    *flag = static_cast<double *>(p);
    *ptr = static_cast<unsigned char *>(p) + kNoallocFlagBytes;
    *bytes = kNoallocScratchBytes - kNoallocFlagBytes;
    return cudaSuccess;
}

cudaError_t launch_fp64_chunk_noalloc(const ChunkArgs &a, cudaStream_t s) {
    int64_t nt = a.t1 - a.t0;
    if (nt <= 0) return cudaSuccess;
    colloc_f64<<<(unsigned)nt, TILE, 0, s>>>(a);
    dim3 xg((unsigned)nt, (unsigned)((a.max_nfunc + XB_R - 1) / XB_R));
    xgemm_f64<<<xg, 256, 0, s>>>(a, a.P, 0, 4);
    rho_xc_z_f64<<<(unsigned)nt, TILE, 0, s>>>(a);
    unsigned nblk = (unsigned)((a.max_nfunc + VB - 1) / VB);
    vgemm_f64_tile<<<dim3((unsigned)nt, nblk, nblk), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double *P, int64_t n, double *flag, bool reset, cudaStream_t s) {
    if (reset) {
        cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    if (n > 0)
        nonfinite_flag<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(P, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_poison_if_flagged(const double *flag, double *EN, cudaStream_t s) {
    poison_if_flagged<<<1, 32, 0, s>>>(flag, EN);
    return cudaGetLastError();
}

cudaError_t launch_symmetrize(const double *Vacc, double *V, int nbf, cudaStream_t s) {
    int64_t nn = (int64_t)nbf * nbf;
    if (nn > 0) symmetrize<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(Vacc, V, nbf);
    return cudaGetLastError();
}

cudaError_t launch_symmetrize_inplace(double *V, int nbf, cudaStream_t s) {
    int64_t nn = (int64_t)nbf * nbf;
    if (nn > 0) symmetrize_inplace<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(V, nbf);
    return cudaGetLastError();
}

cudaError_t launch_finish(const FinishArgs &a, cudaStream_t s) {
    int64_t nn = (int64_t)a.nbf * a.nbf;
    int n = 0;
    a.prof->begin(GBXC_K_FINISH, s);
    if (a.V && nn > 0) {
        symmetrize<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(a.Vacc, a.V, a.nbf);
        ++n;
    }
    int nb = a.b1 - a.b0;
    if (nb > 0) {
        batch_sums<<<(nb + 127) / 128, 128, 0, s>>>(a);
        ++n;
    }
    total_sums<<<1, 256, 0, s>>>(a);
    a.prof->end(GBXC_K_FINISH, s, n + 1);
    return cudaGetLastError();
}

}  // namespace gbxc
