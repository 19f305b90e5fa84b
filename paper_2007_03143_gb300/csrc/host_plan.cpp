// Molecular grid and batch plan on the host (Sec. 2.2, Eq. rcut, Algorithm 1, Algorithm 3).
//
// Compiled with -ffp-contract=off: every expression below is evaluated as
// written in IEEE double precision, so the coordinates and every comparison of
// the batching are reproducible across compilers and across the host and the
// reference CPU implementation.  The logarithms, cosines and sines of the grid and
// of the cutoffs are written out below with basic operations in a fixed order
// instead of libm calls, whose last bits differ between host architectures, so a
// seeded workload has the same coordinates and plan on every host.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <stdexcept>

#include "internal.h"

namespace gbxc {
namespace {

constexpr double kPi = 3.141592653589793;
constexpr int kMaxDepth = 16;

// ln x for finite x > 0: x = m 2^e with m in [1/sqrt 2, sqrt 2), ln m = 2 atanh(s),
// s = (m - 1)/(m + 1), by the series s + s^3/3 + ... + s^25/25 (|s| <= 0.1716); ln 2 in
// two parts, the high part with 32 significant bits so that e ln2_hi is exact.
constexpr double kLn2Hi = 6.93147180369123816490e-01;
constexpr double kLn2Lo = 1.90821492927058770002e-10;
double ln_fixed(double x) {
    int e = 0;
    double m = std::frexp(x, &e);
    if (m < 0.70710678118654752440) {
        m = m * 2.0;
        e = e - 1;
    }
    const double s = (m - 1.0) / (m + 1.0);
    const double s2 = s * s;
    double t = s, acc = s;
    for (int k = 1; k <= 12; ++k) {
        t = t * s2;
        acc = acc + t / (double)(2 * k + 1);
    }
    return (double)e * kLn2Hi + (2.0 * acc + (double)e * kLn2Lo);
}

// sin x and cos x for 0 <= x <= 8: x = q pi/2 + r with |r| <= pi/4 (pi/2 in two parts, the
// high part with 33 significant bits so that q pi2_hi is exact), Taylor series of sin r and
// cos r to r^23 and r^22, then the quadrant q mod 4.
constexpr double kTwoOverPi = 0.63661977236758134308;
constexpr double kPio2Hi = 1.57079632673412561417e+00;
constexpr double kPio2Lo = 6.07710050650619224932e-11;
void sincos_fixed(double x, double &sn, double &cs) {
    const double q = std::floor(x * kTwoOverPi + 0.5);
    const double r = (x - q * kPio2Hi) - q * kPio2Lo;
    const double r2 = r * r;
    double tc = 1.0, c = 1.0, ts = r, sv = r;
    for (int k = 1; k <= 11; ++k) {
        tc = tc * (-r2) / (double)((2 * k - 1) * (2 * k));
        c = c + tc;
        ts = ts * (-r2) / (double)((2 * k) * (2 * k + 1));
        sv = sv + ts;
    }
    switch ((int)q & 3) {
        case 0: sn = sv; cs = c; break;
        case 1: sn = c; cs = -sv; break;
        case 2: sn = -sv; cs = -c; break;
        default: sn = -c; cs = sv; break;
    }
}
double cos_fixed(double x) {
    double s, c;
    sincos_fixed(x, s, c);
    return c;
}

// Mura-Knowles radial rule, r^2 Jacobian included:
// x_k = k/(n+1), r_k = -alpha ln(1 - x_k^3), w_k = 3 alpha x_k^2 / ((1 - x_k^3)(n+1)) r_k^2.
void mura_knowles(int n, double alpha, std::vector<double> &r, std::vector<double> &w) {
    r.resize(n);
    w.resize(n);
    for (int k = 1; k <= n; ++k) {
        double x = k / (n + 1.0);
        double x3 = x * x * x;
        double rk = -alpha * ln_fixed(1.0 - x3);
        r[k - 1] = rk;
        w[k - 1] = 3.0 * alpha * x * x / ((1.0 - x3) * (n + 1.0)) * rk * rk;
    }
}

// Gauss-Legendre nodes (descending) and weights by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &t_out, std::vector<double> &w_out) {
    t_out.resize(n);
    w_out.resize(n);
    auto legendre = [n](double t, double &p1, double &p2) {
        p1 = 1.0;
        p2 = 0.0;
        for (int j = 0; j < n; ++j) {
            double p3 = p2;
            p2 = p1;
            double jf = (double)j;
            p1 = ((2.0 * jf + 1.0) * t * p2 - jf * p3) / (jf + 1.0);
        }
    };
    for (int i = 0; i < n; ++i) {
        double t = cos_fixed(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p1, p2;
            legendre(t, p1, p2);
            double pp = n * (t * p1 - p2) / (t * t - 1.0);
            double t1 = t;
            t = t1 - p1 / pp;
            if (std::fabs(t - t1) <= 1e-15) break;
        }
        double p1, p2;
        legendre(t, p1, p2);
        double pp = n * (t * p1 - p2) / (t * t - 1.0);
        t_out[i] = t;
        w_out[i] = 2.0 / ((1.0 - t * t) * pp * pp);
    }
}

struct Cell {
    double lo[3], hi[3];
};

bool contains_atom(const Cell &c, const std::vector<double> &xyz) {
    size_t na = xyz.size() / 3;
    for (size_t a = 0; a < na; ++a) {
        const double *R = &xyz[3 * a];
        if (c.lo[0] <= R[0] && R[0] <= c.hi[0] && c.lo[1] <= R[1] && R[1] <= c.hi[1] &&
            c.lo[2] <= R[2] && R[2] <= c.hi[2])
            return true;
    }
    return false;
}

// Recursive cuboid subdivision of one atom's points (indices into x/y/z, in order).
void subdivide(const std::vector<int64_t> &idx, const Cell &cell, int depth, int max_batch,
               const std::vector<double> &xyz, const double *P[3],
               std::vector<std::vector<int64_t>> &out) {
    if ((int64_t)idx.size() <= max_batch || depth >= kMaxDepth) {
        out.push_back(idx);
        return;
    }
    double cuts[3][4];
    int ncut;
    if (contains_atom(cell, xyz)) {
        ncut = 3;
        for (int d = 0; d < 3; ++d) {
            double lo = cell.lo[d], hi = cell.hi[d];
            cuts[d][0] = lo;
            cuts[d][1] = lo + (hi - lo) / 3.0;
            cuts[d][2] = lo + 2.0 * (hi - lo) / 3.0;
            cuts[d][3] = hi;
        }
    } else {
        ncut = 2;
        for (int d = 0; d < 3; ++d) {
            double lo = cell.lo[d], hi = cell.hi[d];
            cuts[d][0] = lo;
            cuts[d][1] = 0.5 * (lo + hi);
            cuts[d][2] = hi;
        }
    }
    // child index per axis = number of interior cuts <= coordinate
    std::vector<std::vector<int64_t>> child((size_t)ncut * ncut * ncut);
    for (int64_t p : idx) {
        int c[3];
        for (int d = 0; d < 3; ++d) {
            double v = P[d][p];
            int k = 0;
            for (int q = 1; q < ncut; ++q) k += (v >= cuts[d][q]) ? 1 : 0;
            c[d] = k;
        }
        child[((size_t)c[2] * ncut + c[1]) * ncut + c[0]].push_back(p);
    }
    for (int iz = 0; iz < ncut; ++iz)
        for (int iy = 0; iy < ncut; ++iy)
            for (int ix = 0; ix < ncut; ++ix) {
                const auto &sel = child[((size_t)iz * ncut + iy) * ncut + ix];
                if (sel.empty()) continue;
                Cell cc;
                cc.lo[0] = cuts[0][ix];
                cc.lo[1] = cuts[1][iy];
                cc.lo[2] = cuts[2][iz];
                cc.hi[0] = cuts[0][ix + 1];
                cc.hi[1] = cuts[1][iy + 1];
                cc.hi[2] = cuts[2][iz + 1];
                subdivide(sel, cc, depth + 1, max_batch, xyz, P, out);
            }
}

// Algorithm 1 with the printed typo (W_o) and inverted return corrected:
// keep the shell iff r_cut^2 minus the squared distance to the box is >= 0.
bool cuboid_sphere(const double *R, double rcut, const double *V, const double *W) {
    double d = rcut * rcut;
    for (int p = 0; p < 3; ++p) {
        if (R[p] < V[p])
            d = d - (R[p] - V[p]) * (R[p] - V[p]);
        else if (R[p] > W[p])
            d = d - (R[p] - W[p]) * (R[p] - W[p]);
    }
    return d >= 0.0;
}

int ncart(int L) { return (L + 1) * (L + 2) / 2; }

}  // namespace

double shell_cutoff(const double *alpha, int nprim, double eta) {
    double rc = 0.0;
    for (int k = 0; k < nprim; ++k) {
        double a = alpha[k];
        double v = std::sqrt((ln_fixed(a) / 2.0 - ln_fixed(eta)) / a);
        if (v > rc) rc = v;
    }
    return rc;
}

namespace {
struct LebedevOrbit {
    int kind;       // 0 a1, 1 a2, 2 a3, 3 b, 4 c, 5 d
    double g[3];    // generator
    double w;       // weight of each point (the rule sums to 4 pi)
};
struct LebedevRuleIndex {
    int n, degree, first, count;
};
#include "lebedev_rules.inc"

const LebedevRuleIndex *find_lebedev(int n) {
    for (const LebedevRuleIndex &r : kLebedevRules)
        if (r.n == n) return &r;
    return nullptr;
}

// The octahedral orbits of a Lebedev-Laikov rule expanded to points: for each orbit, the
// permutations of the generator's coordinates in lexicographic order and for each the sign
// patterns +++, ++-, ..., --- (a set bit negates; the first coordinate is the high bit),
// keeping the first occurrence of every point (a zero never takes a sign).
void lebedev_points(const LebedevRuleIndex &rule, GridTables &T) {
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    T.ux.clear();
    T.uy.clear();
    T.uz.clear();
    T.wa.clear();
    for (int o = rule.first; o < rule.first + rule.count; ++o) {
        const LebedevOrbit &orb = kLebedevOrbits[o];
        size_t begin = T.ux.size();
        for (const auto &pm : perms)
            for (int sg = 0; sg < 8; ++sg) {
                double v[3];
                for (int k = 0; k < 3; ++k) {
                    double c = orb.g[pm[k]];
                    v[k] = ((sg >> (2 - k)) & 1) && c != 0.0 ? -c : c;
                }
                bool seen = false;
                for (size_t q = begin; q < T.ux.size() && !seen; ++q)
                    seen = T.ux[q] == v[0] && T.uy[q] == v[1] && T.uz[q] == v[2];
                if (seen) continue;
                T.ux.push_back(v[0]);
                T.uy.push_back(v[1]);
                T.uz.push_back(v[2]);
                T.wa.push_back(orb.w);
            }
    }
}
}  // namespace

bool lebedev_supported(int n) { return find_lebedev(n) != nullptr; }

void grid_tables(const gbxc_grid_spec &spec, GridTables &T) {
    std::vector<double> t, wt;
    mura_knowles(spec.nrad, spec.mk_alpha, T.r, T.wr);
    if (spec.angular == GBXC_ANGULAR_LEBEDEV) {
        const LebedevRuleIndex *rule = find_lebedev(spec.ntheta);
        if (!rule) throw std::invalid_argument("no Lebedev rule of that many points");
        lebedev_points(*rule, T);
        return;
    }
    gauss_legendre(spec.ntheta, t, wt);
    int nt = spec.ntheta, np = spec.nphi;
    T.ux.assign((size_t)nt * np, 0.0);
    T.uy.assign((size_t)nt * np, 0.0);
    T.uz.assign((size_t)nt * np, 0.0);
    T.wa.assign((size_t)nt * np, 0.0);
    std::vector<double> cphi(np), sphi(np);
    for (int b = 0; b < np; ++b) {
        sincos_fixed(2.0 * kPi * b / np, sphi[b], cphi[b]);
    }
    double wphi = 2.0 * kPi / np;
    for (int a = 0; a < nt; ++a) {
        double st = std::sqrt(1.0 - t[a] * t[a]);
        for (int b = 0; b < np; ++b) {
            size_t k = (size_t)a * np + b;
            T.ux[k] = st * cphi[b];
            T.uy[k] = st * sphi[b];
            T.uz[k] = t[a];
            T.wa[k] = wt[a] * wphi;
        }
    }
}

void build_molecular_grid(const std::vector<double> &xyz, const gbxc_grid_spec &spec,
                          std::vector<double> &x, std::vector<double> &y, std::vector<double> &z,
                          std::vector<double> &wq, std::vector<int> &parent) {
    GridTables T;
    grid_tables(spec, T);
    const std::vector<double> &r = T.r, &wr = T.wr, &ux = T.ux, &uy = T.uy, &uz = T.uz, &wa = T.wa;
    size_t natoms = xyz.size() / 3, nang = ux.size(), npa = (size_t)spec.nrad * nang;
    x.resize(natoms * npa);
    y.resize(natoms * npa);
    z.resize(natoms * npa);
    wq.resize(natoms * npa);
    parent.resize(natoms * npa);
    for (size_t A = 0; A < natoms; ++A) {
        double cx = xyz[3 * A], cy = xyz[3 * A + 1], cz = xyz[3 * A + 2];
        for (int k = 0; k < spec.nrad; ++k)
            for (size_t q = 0; q < nang; ++q) {
                size_t i = A * npa + (size_t)k * nang + q;
                x[i] = cx + r[k] * ux[q];
                y[i] = cy + r[k] * uy[q];
                z[i] = cz + r[k] * uz[q];
                wq[i] = wr[k] * wa[q];
                parent[i] = (int)A;
            }
    }
}

void build_plan(const std::vector<double> &xyz, const std::vector<DevShell> &shells,
                const std::vector<double> &rcut, int nbf, const gbxc_grid_spec &spec,
                const std::vector<double> &x, const std::vector<double> &y,
                const std::vector<double> &z, const std::vector<double> &wq,
                const std::vector<int> &parent, HostPlan &plan) {
    (void)nbf;
    size_t natoms = xyz.size() / 3;
    size_t npts = x.size();
    const double *P[3] = {x.data(), y.data(), z.data()};
    // 1. leaf batches atom by atom (points of an atom are contiguous in generation order)
    std::vector<std::vector<int64_t>> leaves;
    size_t start = 0;
    for (size_t A = 0; A < natoms; ++A) {
        size_t end = start;
        while (end < npts && parent[end] == (int)A) ++end;
        if (end == start) continue;
        std::vector<int64_t> idx(end - start);
        std::iota(idx.begin(), idx.end(), (int64_t)start);
        Cell c;
        for (int d = 0; d < 3; ++d) {
            c.lo[d] = P[d][start];
            c.hi[d] = P[d][start];
            for (size_t i = start; i < end; ++i) {
                c.lo[d] = std::min(c.lo[d], P[d][i]);
                c.hi[d] = std::max(c.hi[d], P[d][i]);
            }
        }
        subdivide(idx, c, 0, spec.max_batch, xyz, P, leaves);
        start = end;
    }
    // 2. Algorithm 1 on each leaf's tight bounding box
    std::vector<std::vector<int>> keeps(leaves.size());
    size_t nsh = shells.size();
    for (size_t l = 0; l < leaves.size(); ++l) {
        const auto &idx = leaves[l];
        double V[3], W[3];
        for (int d = 0; d < 3; ++d) {
            V[d] = W[d] = P[d][idx[0]];
            for (int64_t p : idx) {
                V[d] = std::min(V[d], P[d][p]);
                W[d] = std::max(W[d], P[d][p]);
            }
        }
        for (size_t s = 0; s < nsh; ++s)
            if (cuboid_sphere(shells[s].c, rcut[s], V, W)) keeps[l].push_back((int)s);
    }
    plan_from_leaves(natoms, shells, leaves, keeps, x, y, z, wq, parent, plan);
}

// 3. merge equal shell lists: leaves with identical lists form one batch, batches in order
// of first occurrence, leaves in order within a batch.
void merge_leaves(const std::vector<std::vector<int>> &keeps, std::vector<std::vector<int>> &bshells,
                  std::vector<std::vector<int>> &bleaves) {
    std::map<std::vector<int>, int> key_to_batch;
    bshells.clear();
    bleaves.clear();
    for (size_t l = 0; l < keeps.size(); ++l) {
        const std::vector<int> &keep = keeps[l];
        auto it = key_to_batch.find(keep);
        if (it == key_to_batch.end()) {
            key_to_batch.emplace(keep, (int)bshells.size());
            bshells.push_back(keep);
            bleaves.push_back({(int)l});
        } else {
            bleaves[it->second].push_back((int)l);
        }
    }
}

// 4. function lists and work estimate (Eq. batch_work) per batch, 5. 128-point tiles and the
// slab row offsets of each tile (padded function count); batch sizes in batch order.
void batch_metadata(size_t natoms, const std::vector<DevShell> &shells, const std::vector<std::vector<int>> &bshells,
                    const std::vector<int64_t> &batch_size, HostPlan &plan) {
    const int nb = (int)bshells.size();
    plan.batch_ptr.assign(1, 0);
    plan.shell_ptr.assign(1, 0);
    plan.shell_idx.clear();
    plan.func_ptr.assign(1, 0);
    plan.func_idx.clear();
    plan.work.clear();
    for (int j = 0; j < nb; ++j) {
        plan.batch_ptr.push_back(plan.batch_ptr.back() + batch_size[j]);
        int64_t nfun = 0;
        for (int s : bshells[j]) {
            plan.shell_idx.push_back(s);
            for (int c = 0; c < shell_nfunc(shells[s]); ++c) plan.func_idx.push_back(shells[s].fofs + c);
            nfun += shell_nfunc(shells[s]);
        }
        plan.shell_ptr.push_back((int64_t)plan.shell_idx.size());
        plan.func_ptr.push_back((int64_t)plan.func_idx.size());
        int64_t ng = batch_size[j];
        int64_t na = (int64_t)natoms;
        plan.work.push_back((double)(ng * (na * na + 9 * nfun + 2 * nfun * nfun + 3) + nfun * nfun));
    }
    plan.npts = plan.batch_ptr.back();
    plan.tile_batch.clear(); plan.tile_first.clear(); plan.tile_count.clear();
    plan.tile_row.clear();
    plan.batch_tile.assign(1, 0);
    int64_t row = 0;
    for (int j = 0; j < nb; ++j) {
        int64_t b0 = plan.batch_ptr[j], b1 = plan.batch_ptr[j + 1];
        int64_t nfp = std::max<int64_t>(pad_funcs(plan.func_ptr[j + 1] - plan.func_ptr[j]), FBLK);
        for (int64_t p = b0; p < b1; p += TILE) {
            plan.tile_batch.push_back(j);
            plan.tile_first.push_back(p);
            plan.tile_count.push_back((int)std::min<int64_t>(TILE, b1 - p));
            plan.tile_row.push_back(row);
            row += nfp;
        }
        plan.batch_tile.push_back((int64_t)plan.tile_batch.size());
    }
    plan.tile_row.push_back(row);   // total rows (one past the last tile)
}

// Steps 3-5 with the points laid out batch by batch on the host.
void plan_from_leaves(size_t natoms, const std::vector<DevShell> &shells,
                      const std::vector<std::vector<int64_t>> &leaves, const std::vector<std::vector<int>> &keeps,
                      const std::vector<double> &x, const std::vector<double> &y, const std::vector<double> &z,
                      const std::vector<double> &wq, const std::vector<int> &parent, HostPlan &plan) {
    size_t npts = x.size();
    plan.nleaf = (int)leaves.size();
    std::vector<std::vector<int>> bshells, bleaves;
    merge_leaves(keeps, bshells, bleaves);
    plan.x.clear(); plan.y.clear(); plan.z.clear(); plan.wq.clear();
    plan.parent.clear(); plan.point_index.clear();
    plan.x.reserve(npts); plan.y.reserve(npts); plan.z.reserve(npts); plan.wq.reserve(npts);
    plan.parent.reserve(npts); plan.point_index.reserve(npts);
    std::vector<int64_t> bsize;
    for (size_t j = 0; j < bshells.size(); ++j) {
        int64_t n0 = (int64_t)plan.x.size();
        for (int l : bleaves[j])
            for (int64_t p : leaves[l]) {
                plan.x.push_back(x[p]);
                plan.y.push_back(y[p]);
                plan.z.push_back(z[p]);
                plan.wq.push_back(wq[p]);
                plan.parent.push_back(parent[p]);
                plan.point_index.push_back(p);
            }
        bsize.push_back((int64_t)plan.x.size() - n0);
    }
    batch_metadata(natoms, shells, bshells, bsize, plan);
}

}  // namespace gbxc
