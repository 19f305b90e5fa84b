"""Writes csrc/lebedev_rules.inc, the Lebedev-Laikov angular rules the library offers
beside the Gauss-Legendre x trapezoid product (Sec. 2.2: the paper's atomic grids are a
Mura-Knowles radial rule times a Lebedev-Laikov angular rule; Table "Atomic Quadrature
Sizes" lists 302 and 590 angular points for its FG and UFG grids).

The rules are built here from Lebedev's published construction rather than read from
published tables:

* A rule is invariant under the octahedral group with inversion (48 elements).  Its points
  fall in orbits: a1 (6 points, (1,0,0) and images), a2 (12, (s,s,0), s = 1/sqrt 2),
  a3 (8, (t,t,t), t = 1/sqrt 3), b (24, (l,l,m)), c (24, (p,q,0)), d (48, (r,s,u)), every
  point of an orbit carrying the same weight.
* By Sobolev's theorem an invariant rule integrates every polynomial of degree <= p on the
  sphere exactly iff it integrates the invariant ones exactly.  On the sphere these are the
  polynomials in e2 = x^2 y^2 + y^2 z^2 + z^2 x^2 and e3 = x^2 y^2 z^2, so the conditions
  are one equation per (i, j) with 4 i + 6 j <= p:
      sum over orbits o of  W_o e2(g_o)^i e3(g_o)^j  =  mean over the sphere of e2^i e3^j,
  W_o being the orbit's total weight (the rule normalised to 1) and g_o its generator.
* The orbit counts make the unknowns equal the equations (the sizes below); the split of
  the one-parameter orbits between b and c is the first, scanning from most b orbits down,
  that admits a solution with positive weights.

Solution: a Levenberg-Marquardt search in an orthonormal basis of the invariant
polynomials (built by a Stieltjes recurrence on a product rule exact to degree 2p), from
seeded guesses spread over the edges and the interior of the symmetry triangle; then Newton
in 60-digit arithmetic (mpmath) on the moment equations with exact rational right-hand
sides; every coordinate and weight is rounded once to float64 from that.

Run: python -m paper_2007_03143_gb300.gen_lebedev   (needs scipy and mpmath; minutes)
"""
from __future__ import annotations

import itertools
import math
import os
import sys
from fractions import Fraction

import numpy as np

# N -> (degree, orbits present among a1 a2 a3, number of b, c, d orbits)
RULES = {
    6: (3, ("a1",), 0, 0, 0),
    14: (5, ("a1", "a3"), 0, 0, 0),
    26: (7, ("a1", "a2", "a3"), 0, 0, 0),
    38: (9, ("a1", "a3"), 0, 1, 0),
    50: (11, ("a1", "a2", "a3"), 1, 0, 0),
    86: (15, ("a1", "a3"), 2, 1, 0),
    110: (17, ("a1", "a3"), 3, 1, 0),
    146: (19, ("a1", "a2", "a3"), 3, 0, 1),
    170: (21, ("a1", "a2", "a3"), 3, 1, 1),
    194: (23, ("a1", "a2", "a3"), 4, 1, 1),
    302: (29, ("a1", "a3"), 6, 2, 2),
    590: (41, ("a1", "a3"), 9, 3, 6),
    974: (53, ("a1", "a3"), 12, 4, 12),
}
# Rules the spread-guess search does not reach: basin hopping from the best of `starts`
# spread guesses (seeded), perturbing a random 30% of the unknowns by 10^U(-3,-1) of their
# size and keeping an LM result whenever it lowers the residual (about an hour for 974).
BASIN = {974: dict(seed=23, starts=20, iters=1000)}
ORBIT_SIZE = {"a1": 6, "a2": 12, "a3": 8, "b": 24, "c": 24, "d": 48}
NPARAM = {"a1": 0, "a2": 0, "a3": 0, "b": 1, "c": 1, "d": 2}


def invariant_pairs(p):
    return sorted(((i, j) for j in range(p // 6 + 1) for i in range((p - 6 * j) // 4 + 1)),
                  key=lambda ij: (4 * ij[0] + 6 * ij[1], ij[1]))


# ---- exact moments ------------------------------------------------------------------------
def _odd_double_factorial(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def _sphere_mean_even_monomial(a, b, c):
    """Mean over the unit sphere of x^(2a) y^(2b) z^(2c)."""
    return Fraction(_odd_double_factorial(2 * a - 1) * _odd_double_factorial(2 * b - 1)
                    * _odd_double_factorial(2 * c - 1), _odd_double_factorial(2 * (a + b + c) + 1))


def invariant_moment(i, j):
    """Mean over the sphere of e2^i e3^j (e2 expanded by the multinomial theorem)."""
    total = Fraction(0)
    for i1 in range(i + 1):
        for i2 in range(i - i1 + 1):
            i3 = i - i1 - i2
            mult = math.factorial(i) // (math.factorial(i1) * math.factorial(i2) * math.factorial(i3))
            total += mult * _sphere_mean_even_monomial(i1 + i3 + j, i1 + i2 + j, i2 + i3 + j)
    return total


# ---- orthonormal invariant basis (float64, for the search) --------------------------------
class InvariantBasis:
    """q_0 = 1, then each (i, j) in degree order as U q_(i-1,j) (or V q_(i,j-1)) made
    orthonormal to the earlier ones, U = 3 e2 - 1/2 and V = 27 e3 - 1/2; the recurrence
    coefficients are kept so the basis can be evaluated anywhere."""

    def __init__(self, p):
        n_t = p + 8
        t, wt = np.polynomial.legendre.leggauss(n_t)
        n_f = 2 * p + 8
        f = 2.0 * np.pi * np.arange(n_f) / n_f
        st = np.sqrt(1.0 - t * t)
        x = (st[:, None] * np.cos(f)[None]).ravel()
        y = (st[:, None] * np.sin(f)[None]).ravel()
        z = np.repeat(t, n_f)
        w = np.repeat(wt, n_f) / (2.0 * n_f)
        U, V = self._uv(x, y, z)
        self.pairs = invariant_pairs(p)
        self.steps = [None]
        Q = [np.ones_like(x)]
        for i, j in self.pairs[1:]:
            if i > 0:
                par, var = self.pairs.index((i - 1, j)), 0
            else:
                par, var = self.pairs.index((i, j - 1)), 1
            g = (U if var == 0 else V) * Q[par]
            coef = np.zeros(len(Q))
            for _ in range(2):
                c = np.array([np.sum(w * g * q) for q in Q])
                g = g - c @ np.array(Q)
                coef += c
            nrm = math.sqrt(np.sum(w * g * g))
            self.steps.append((par, var, coef, nrm))
            Q.append(g / nrm)

    @staticmethod
    def _uv(x, y, z):
        a, b, c = x * x, y * y, z * z
        return 3.0 * (a * b + b * c + c * a) - 0.5, 27.0 * a * b * c - 0.5

    def eval(self, x, y, z):
        """Values and derivatives (d/dx, d/dy, d/dz) of every basis function at the points."""
        a, b, c = x * x, y * y, z * z
        U = 3.0 * (a * b + b * c + c * a) - 0.5
        V = 27.0 * a * b * c - 0.5
        dU = (6.0 * x * (b + c), 6.0 * y * (a + c), 6.0 * z * (a + b))
        dV = (54.0 * x * b * c, 54.0 * y * a * c, 54.0 * z * a * b)
        K, n = len(self.steps), len(x)
        Q, QU, QV = np.zeros((K, n)), np.zeros((K, n)), np.zeros((K, n))
        Q[0] = 1.0
        for k in range(1, K):
            par, var, coef, nrm = self.steps[k]
            m = len(coef)
            X = U if var == 0 else V
            Q[k] = (X * Q[par] - coef @ Q[:m]) / nrm
            QU[k] = (X * QU[par] + (Q[par] if var == 0 else 0.0) - coef @ QU[:m]) / nrm
            QV[k] = (X * QV[par] + (Q[par] if var == 1 else 0.0) - coef @ QV[:m]) / nrm
        grads = [QU * dU[d] + QV * dV[d] for d in range(3)]
        return Q, grads


def _generator(kind, prm):
    """Generator point and its derivatives with respect to the orbit's parameters."""
    if kind == "a1":
        return (1.0, 0.0, 0.0), []
    if kind == "a2":
        s = math.sqrt(0.5)
        return (s, s, 0.0), []
    if kind == "a3":
        s = math.sqrt(1.0 / 3.0)
        return (s, s, s), []
    if kind == "b":
        l = prm[0]
        m = math.sqrt(abs(1.0 - 2.0 * l * l))
        return (l, l, m), [(1.0, 1.0, -2.0 * l / m)]
    if kind == "c":
        q = prm[0]
        m = math.sqrt(abs(1.0 - q * q))
        return (q, m, 0.0), [(1.0, -q / m, 0.0)]
    r, s = prm
    u = math.sqrt(abs(1.0 - r * r - s * s))
    return (r, s, u), [(1.0, 0.0, -r / u), (0.0, 1.0, -s / u)]


def _layout(kinds):
    idx, k = [], 0
    for kind in kinds:
        idx.append(k)
        k += 1 + NPARAM[kind]
    return idx, k


def _system(basis, kinds):
    widx, nunk = _layout(kinds)
    rhs = np.zeros(len(basis.pairs))
    rhs[0] = 1.0

    def unpack(xv):
        gens, dgens = [], []
        for kind, i in zip(kinds, widx):
            g, dg = _generator(kind, list(xv[i + 1:i + 1 + NPARAM[kind]]))
            gens.append(g)
            dgens.append(dg)
        return np.array(gens), dgens

    def F(xv):
        G, _ = unpack(xv)
        Q, _ = basis.eval(G[:, 0], G[:, 1], G[:, 2])
        return Q @ xv[widx] - rhs

    def J(xv):
        G, dG = unpack(xv)
        Q, grads = basis.eval(G[:, 0], G[:, 1], G[:, 2])
        Jm = np.zeros((len(rhs), nunk))
        for o, i in enumerate(widx):
            Jm[:, i] = Q[:, o]
            for k, dv in enumerate(dG[o]):
                Jm[:, i + 1 + k] = xv[i] * sum(dv[d] * grads[d][:, o] for d in range(3))
        return Jm

    return F, J, widx, nunk


def _slerp(a, b, t):
    a = np.asarray(a, float) / np.linalg.norm(a)
    b = np.asarray(b, float) / np.linalg.norm(b)
    om = math.acos(max(-1.0, min(1.0, float(a @ b))))
    return (math.sin((1 - t) * om) * a + math.sin(t * om) * b) / math.sin(om)


def _spread_guess(kinds, n_points, rng, jitter):
    """b orbits spread along the symmetry edges (0,0,1)-(1,1,1)-(1,1,0) (normalised), c orbits
    along (0,0,1)-(0,1,1), d orbits at random in the triangle; equal weights per point."""
    A1, A2, A3 = (0.0, 0.0, 1.0), (0.0, 1.0, 1.0), (1.0, 1.0, 1.0)
    nb, nc = kinds.count("b"), kinds.count("c")
    L1 = math.acos(1.0 / math.sqrt(3.0))
    L2 = math.pi / 2.0 - L1
    b_par = []
    for s in (np.arange(nb) + 0.5) / nb * (L1 + L2) + rng.normal(0.0, jitter, nb):
        s = min(max(s, 0.02), L1 + L2 - 0.02)
        v = _slerp(A1, A3, s / L1) if s < L1 else _slerp(A3, A2, (s - L1) / L2)
        v = np.sort(np.abs(v))
        b_par.append(v[0] if abs(v[0] - v[1]) < abs(v[1] - v[2]) else v[2])
    c_par = [min(_slerp(A1, A2, t)[1], _slerp(A1, A2, t)[2])
             for t in np.clip((np.arange(nc) + 0.5) / nc + rng.normal(0.0, jitter, nc), 0.02, 0.98)]
    x0, ib, ic = [], 0, 0
    for kind in kinds:
        x0.append(ORBIT_SIZE[kind] / n_points)
        if kind == "b":
            x0.append(b_par[ib])
            ib += 1
        elif kind == "c":
            x0.append(c_par[ic])
            ic += 1
        elif kind == "d":
            while True:
                r, s = rng.uniform(0.02, 0.7, 2)
                if r * r + s * s < 0.9:
                    break
            x0 += [r, s]
    return np.array(x0)


def _basin_search(n_points, kinds, F, J, widx, nunk, seed, starts, iters):
    from scipy.optimize import least_squares

    def run(x0):
        try:
            return least_squares(F, x0, jac=J, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15,
                                 max_nfev=100 * nunk)
        except (ValueError, np.linalg.LinAlgError):
            return None

    rng = np.random.default_rng(seed)
    best = None
    for t in range(starts):
        r = run(_spread_guess(kinds, n_points, rng, 0.05 if t else 0.0))
        if r is not None and (best is None or np.linalg.norm(r.fun) < np.linalg.norm(best.fun)):
            best = r
    for _ in range(iters):
        x = best.x.copy()
        scale = 10 ** rng.uniform(-3, -1)
        mask = rng.random(len(x)) < 0.3
        x[mask] += rng.normal(0, scale, mask.sum()) * np.maximum(np.abs(x[mask]), 0.05)
        r = run(x)
        if r is None or not np.linalg.norm(r.fun) < np.linalg.norm(best.fun):
            continue
        best = r
        if np.linalg.norm(best.fun) < 1e-10 and all(best.x[i] > 0 for i in widx):
            return kinds, best.x
    raise RuntimeError(f"basin hopping found no rule of {n_points} points")


def search(n_points, tries=400, seed=0):
    from scipy.optimize import least_squares
    p, a, nb, nc, nd = RULES[n_points]
    kinds = list(a) + ["b"] * nb + ["c"] * nc + ["d"] * nd
    basis = InvariantBasis(p)
    F, J, widx, nunk = _system(basis, kinds)
    if nunk != len(basis.pairs):
        raise ValueError(f"{n_points}: {nunk} unknowns for {len(basis.pairs)} equations")
    if n_points in BASIN:
        return _basin_search(n_points, kinds, F, J, widx, nunk, **BASIN[n_points])
    rng = np.random.default_rng(seed)
    for t in range(tries):
        x0 = _spread_guess(kinds, n_points, rng, 0.05 if t else 0.0)
        if nunk == len(a):
            x = np.linalg.solve(J(x0), -F(x0) + J(x0) @ x0)
            return kinds, x
        try:
            r = least_squares(F, x0, jac=J, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15,
                              max_nfev=200 * nunk)
        except (ValueError, np.linalg.LinAlgError):
            continue
        if np.linalg.norm(r.fun) < 1e-12 and all(r.x[i] > 0 for i in widx):
            return kinds, r.x
    raise RuntimeError(f"no rule of {n_points} points found in {tries} tries")


# ---- 60-digit Newton on the moment equations ----------------------------------------------
def polish(n_points, kinds, x, digits=60, iters=8):
    import mpmath as mp
    mp.mp.dps = digits
    p = RULES[n_points][0]
    pairs = invariant_pairs(p)
    rhs = [mp.mpf(invariant_moment(i, j).numerator) / invariant_moment(i, j).denominator
           for i, j in pairs]
    widx, nunk = _layout(kinds)
    xv = [mp.mpf(float(v)) for v in x]

    def gen(kind, prm):
        if kind == "a1":
            return [mp.mpf(1), mp.mpf(0), mp.mpf(0)], []
        if kind == "a2":
            s = mp.sqrt(mp.mpf(1) / 2)
            return [s, s, mp.mpf(0)], []
        if kind == "a3":
            s = mp.sqrt(mp.mpf(1) / 3)
            return [s, s, s], []
        if kind == "b":
            l = prm[0]
            m = mp.sqrt(1 - 2 * l * l)
            return [l, l, m], [[1, 1, -2 * l / m]]
        if kind == "c":
            q = prm[0]
            m = mp.sqrt(1 - q * q)
            return [q, m, mp.mpf(0)], [[1, -q / m, 0]]
        r, s = prm
        u = mp.sqrt(1 - r * r - s * s)
        return [r, s, u], [[1, 0, -r / u], [0, 1, -s / u]]

    for _ in range(iters):
        Fv = mp.matrix(len(pairs), 1)
        Jm = mp.matrix(len(pairs), nunk)
        for kind, i in zip(kinds, widx):
            W = xv[i]
            g, dg = gen(kind, xv[i + 1:i + 1 + NPARAM[kind]])
            a, b, c = g[0] ** 2, g[1] ** 2, g[2] ** 2
            e2 = a * b + b * c + c * a
            e3 = a * b * c
            de2 = [2 * g[0] * (b + c), 2 * g[1] * (a + c), 2 * g[2] * (a + b)]
            de3 = [2 * g[0] * b * c, 2 * g[1] * a * c, 2 * g[2] * a * b]
            for k, (ii, jj) in enumerate(pairs):
                mono = e2 ** ii * e3 ** jj
                Fv[k] += W * mono
                Jm[k, i] += mono
                if dg:
                    dmono = [(ii * e2 ** (ii - 1) * e3 ** jj if ii else 0) * de2[d]
                             + (jj * e2 ** ii * e3 ** (jj - 1) if jj else 0) * de3[d] for d in range(3)]
                    for q, dv in enumerate(dg):
                        Jm[k, i + 1 + q] += W * sum(dv[d] * dmono[d] for d in range(3))
        for k in range(len(pairs)):
            Fv[k] -= rhs[k]
        step = mp.lu_solve(Jm, Fv)
        xv = [xv[k] - step[k] for k in range(nunk)]
    res = max(abs(v) for v in Fv)
    if res > mp.mpf(10) ** (-(digits - 25)):
        raise RuntimeError(f"{n_points}: Newton polish did not converge ({res})")
    orbits = []
    for kind, i in zip(kinds, widx):
        g, _ = gen(kind, xv[i + 1:i + 1 + NPARAM[kind]])
        g = [abs(v) for v in g]
        g = sorted(g) if kind in ("c", "d") else g
        if kind == "c":
            g = [g[1], g[2], g[0]]            # (p, q, 0), p < q
        w_point = xv[i] * 4 * mp.pi / ORBIT_SIZE[kind]
        orbits.append((kind, [float(v) for v in g], float(w_point)))
    order = {"a1": 0, "a2": 1, "a3": 2, "b": 3, "c": 4, "d": 5}
    orbits.sort(key=lambda o: (order[o[0]], o[1]))
    return orbits


def write_inc(rules, path):
    kind_code = {"a1": 0, "a2": 1, "a3": 2, "b": 3, "c": 4, "d": 5}
    lines = ["// Lebedev-Laikov angular rules built from the octahedral-orbit construction",
             "// (written by gen_lebedev.py; do not edit).  Per orbit: kind (0 a1, 1 a2, 2 a3,",
             "// 3 b, 4 c, 5 d), generator (x, y, z) and the weight of each point (4 pi total).",
             "static const LebedevOrbit kLebedevOrbits[] = {"]
    index = []
    count = 0
    for n in sorted(rules):
        index.append((n, RULES[n][0], count, len(rules[n])))
        for kind, g, w in rules[n]:
            lines.append(f"    {{{kind_code[kind]}, {{{g[0].hex()}, {g[1].hex()}, {g[2].hex()}}}, {w.hex()}}},"
                         f"  // N={n}")
            count += 1
    lines.append("};")
    lines.append("static const LebedevRuleIndex kLebedevRules[] = {")
    for n, p, first, cnt in index:
        lines.append(f"    {{{n}, {p}, {first}, {cnt}}},")
    lines.append("};")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def read_inc(path):
    """The rules of an existing table (to regenerate some of them only)."""
    import re
    names = ["a1", "a2", "a3", "b", "c", "d"]
    txt = open(path).read()
    orb = [(names[int(k)], [float.fromhex(x), float.fromhex(y), float.fromhex(z)], float.fromhex(w))
           for k, x, y, z, w in re.findall(r"\{(\d), \{(\S+), (\S+), (\S+)\}, (\S+)\}", txt)]
    idx = re.findall(r"\{(\d+), (\d+), (\d+), (\d+)\},", txt)
    return {int(n): orb[int(f):int(f) + int(c)] for n, _, f, c in idx}


def main():
    """python -m paper_2007_03143_gb300.gen_lebedev [N ...]: solve every rule, or only the
    listed ones (the others are kept from the existing table)."""
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "lebedev_rules.inc")
    only = [int(v) for v in sys.argv[1:]]
    rules = read_inc(out) if only and os.path.exists(out) else {}
    for n in sorted(RULES):
        if only and n not in only and n in rules:
            continue
        kinds, x = search(n)
        rules[n] = polish(n, kinds, x, digits=80, iters=10)
        print(n, "orbits", len(rules[n]), file=sys.stderr, flush=True)
    write_inc(rules, out)


if __name__ == "__main__":
    main()
