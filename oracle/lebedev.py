"""Lebedev-Laikov angular quadrature, computed from its construction (Sec. 2.2: the atomic
grids are a Mura-Knowles radial rule times a Lebedev-Laikov angular rule; Table "Atomic
Quadrature Sizes": 302 points in FG, 590 in UFG; the oracle builds the rules up to 302).

ORACLE -- test infrastructure.  Only tests/, the smoke check and the bench's CPU baseline may
import this module; the library never does.

Definition.  A rule {u_k, w_k} on the unit sphere has degree p when it integrates every real
spherical harmonic Y_lm with l <= p exactly:  sum_k w_k Y_lm(u_k) = sqrt(4 pi) delta_l0.
Lebedev's rules are invariant under the octahedral group with inversion; their points fall
in orbits of one weight each:
    a1  6 points  (1, 0, 0)              a2  12 points (1/sqrt2, 1/sqrt2, 0)
    a3  8 points  (1/sqrt3, ...)         b   24 points (l, l, m),  2 l^2 + m^2 = 1
    c   24 points (p, q, 0), p < q       d   48 points (r, s, t),  r < s < t
The orbit counts of each size are fixed by making the number of unknowns equal to the
number of conditions left once the symmetry is used (one per octahedral invariant
e2^i e3^j with 4 i + 6 j <= p, e2 = x^2 y^2 + y^2 z^2 + z^2 x^2, e3 = x^2 y^2 z^2); the
split between b and c orbits is listed below (the first that admits positive weights when
scanning from the most b orbits down).

Computation, in two steps:
1. search: least squares on the definition itself -- every Y_lm with l <= p that an
   invariant rule can fail (l even, m = 0 mod 4, cosine type; from the orthonormal
   associated Legendre recurrence) summed
   over the explicitly listed points of every orbit -- from a deterministic spread of the
   orbits over the symmetry triangle (seeded jitter on retries);
2. polish: Newton in 60-digit arithmetic on the invariant moment conditions
   sum_o W_o e2(g_o)^i e3(g_o)^j = mean of e2^i e3^j over the sphere (exact rationals from
   mean(x^2a y^2b z^2c) = (2a-1)!!(2b-1)!!(2c-1)!!/(2a+2b+2c+1)!!), then one rounding to
   float64.

Point order (a convention): orbits in the order a1 a2 a3 b c d, each kind by ascending
generator; within an orbit the images (s0 g[i0], s1 g[i1], s2 g[i2]) for the permutations
(i0 i1 i2) in lexicographic order, and for each the sign patterns +++ ++- +-+ +-- -++ ...
in that order, keeping the first occurrence of every distinct point.  Weights sum to 4 pi.
"""
from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

import numpy as np

SIZE = {"a1": 6, "a2": 12, "a3": 8, "b": 24, "c": 24, "d": 48}
KIND_ORDER = ("a1", "a2", "a3", "b", "c", "d")

# points -> (degree p, fixed orbits, number of b, c and d orbits)
STRUCTURE = {
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
}
# The library also carries the 590-point rule (degree 41: a1, a3, 9 b, 3 c, 6 d orbits); the
# search above does not reach it from its starting points in the time a golden run allows, so
# the oracle has none and that table is pinned directly (exactness on every Y_lm, l <= 41).


def orbit_points(g):
    """The distinct images of generator g under coordinate permutations and sign changes,
    in the order stated in the module docstring."""
    pts = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((False, True), repeat=3):
            v = tuple((-g[perm[k]] if signs[k] else g[perm[k]]) + 0.0 for k in range(3))
            if v not in pts:
                pts.append(v)
    return pts


def expand(orbits):
    """(orbits as (kind, generator, weight per point)) -> ux, uy, uz, w arrays."""
    u, w = [], []
    for kind, g, wp in orbits:
        pts = orbit_points(g)
        if len(pts) != SIZE[kind]:
            raise ValueError(f"orbit {kind} with generator {g} has {len(pts)} points")
        u += pts
        w += [wp] * len(pts)
    u = np.array(u)
    return u[:, 0].copy(), u[:, 1].copy(), u[:, 2].copy(), np.array(w)


# ---- step 1: search on the harmonic conditions ---------------------------------------------
def _unknowns(kinds):
    n = 0
    for k in kinds:
        n += 1 + {"b": 1, "c": 1, "d": 2}.get(k, 0)
    return n


def _generators(kinds, xv):
    """Generators and total orbit weights from the unknown vector (W, params...) per orbit."""
    out, i = [], 0
    for k in kinds:
        W = xv[i]
        i += 1
        if k == "a1":
            g = (1.0, 0.0, 0.0)
        elif k == "a2":
            g = (math.sqrt(0.5), math.sqrt(0.5), 0.0)
        elif k == "a3":
            g = (math.sqrt(1 / 3),) * 3
        elif k == "b":
            l = xv[i]
            i += 1
            g = (l, l, math.sqrt(abs(1 - 2 * l * l)))
        elif k == "c":
            q = xv[i]
            i += 1
            g = (q, math.sqrt(abs(1 - q * q)), 0.0)
        else:
            r, s = xv[i], xv[i + 1]
            i += 2
            g = (r, s, math.sqrt(abs(1 - r * r - s * s)))
        out.append((k, g, W))
    return out


def _harmonic_list(p):
    return [(l, m) for l in range(0, p + 1, 2) for m in range(0, l + 1, 4)]


_IMAGES = [(perm, signs) for perm in itertools.permutations(range(3))
           for signs in itertools.product((1.0, -1.0), repeat=3)]


def _legendre_table(lmax, x):
    """Orthonormal associated Legendre values p[l][m](x), m <= l <= lmax, so that
    Y_lm = p_lm(cos theta) e^(i m phi) (Condon-Shortley phase): p_00 = 1/sqrt(4 pi),
    p_mm = -sqrt((2m+1)/(2m)) sin(theta) p_(m-1)(m-1), p_(m+1)m = sqrt(2m+3) x p_mm and
    p_lm = a (x p_(l-1)m - b p_(l-2)m), a = sqrt((4l^2-1)/(l^2-m^2)),
    b = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1))."""
    st = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    p = {(0, 0): np.full_like(x, 1.0 / math.sqrt(4.0 * math.pi))}
    for m in range(1, lmax + 1):
        p[(m, m)] = -math.sqrt((2 * m + 1) / (2 * m)) * st * p[(m - 1, m - 1)]
    for m in range(0, lmax):
        p[(m + 1, m)] = math.sqrt(2 * m + 3) * x * p[(m, m)]
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4 * l * l - 1) / (l * l - m * m))
            b = math.sqrt(((l - 1) ** 2 - m * m) / (4 * (l - 1) ** 2 - 1))
            p[(l, m)] = a * (x * p[(l - 1, m)] - b * p[(l - 2, m)])
    return p


_IMAGES = [(perm, signs) for perm in itertools.permutations(range(3))
           for signs in itertools.product((1.0, -1.0), repeat=3)]


def _harmonic_residual(kinds, xv, harmonics):
    """4 pi * sum over orbits of W_o * (mean of Re Y_lm over the orbit's points), minus
    sqrt(4 pi) delta_l0.  The mean over an orbit's distinct points equals the mean over all
    48 images of its generator (each distinct point recurs 48/|orbit| times)."""
    gens = _generators(kinds, xv)
    pts = np.array([[sg[k] * g[pm[k]] for k in range(3)] for _, g, _ in gens for pm, sg in _IMAGES])
    wts = np.repeat([W / 48.0 for _, _, W in gens], 48)
    ct = np.clip(pts[:, 2] / np.linalg.norm(pts, axis=1), -1.0, 1.0)
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    leg = _legendre_table(max(l for l, _ in harmonics), ct)
    rows = np.array([np.sum(wts * leg[(l, m)] * np.cos(m * phi)) for l, m in harmonics])
    rows *= 4.0 * math.pi
    rows[0] -= math.sqrt(4.0 * math.pi)
    return rows


def _initial(kinds, n_points, rng, jitter):
    """Orbits spread evenly: b along the edge (0,0,1)-(1,1,1)-(1,1,0), c along the edge
    (0,0,1)-(0,1,1) (both by arc length), d at seeded points of the triangle."""
    nb, nc = kinds.count("b"), kinds.count("c")
    edge1 = math.acos(1 / math.sqrt(3))            # (0,0,1) to (1,1,1)/sqrt3
    total = math.pi / 2                            # ... and on to (1,1,0)/sqrt2
    xv = []
    ib = ic = 0
    for k in kinds:
        xv.append(SIZE[k] / n_points)
        if k == "b":
            s = (ib + 0.5) / nb * total + rng.normal(0, jitter)
            s = min(max(s, 0.02), total - 0.02)
            if abs(s - edge1) < 0.02:
                s = edge1 + 0.02
            xv.append(math.sin(s) / math.sqrt(2))     # angle s from the pole on x = y
            ib += 1
        elif k == "c":
            t = (ic + 0.5) / nc * (math.pi / 4) + rng.normal(0, jitter)
            xv.append(math.sin(min(max(t, 0.02), math.pi / 4 - 0.02)))
            ic += 1
        elif k == "d":
            while True:
                r, s = rng.uniform(0.02, 0.7, 2)
                if r * r + s * s < 0.9:
                    break
            xv += [r, s]
    return np.array(xv)


def search(n_points, tries=200, seed=1):
    from scipy.optimize import least_squares
    p, fixed, nb, nc, nd = STRUCTURE[n_points]
    kinds = list(fixed) + ["b"] * nb + ["c"] * nc + ["d"] * nd
    harmonics = _harmonic_list(p)
    rng = np.random.default_rng(seed)
    for t in range(tries):
        x0 = _initial(kinds, n_points, rng, 0.05 if t else 0.0)
        r = least_squares(lambda x: _harmonic_residual(kinds, x, harmonics), x0, method="lm",
                          xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=200 * len(x0))
        ok = all(W > 0 for _, _, W in _generators(kinds, r.x))
        if np.max(np.abs(r.fun)) < 1e-9 and ok:     # the polish below takes it the rest of the way
            return kinds, r.x
    raise RuntimeError(f"no {n_points}-point rule found")


# ---- step 2: 60-digit Newton on the moment conditions ----------------------------------------
def _dfact(n):
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


def sphere_mean(a, b, c):
    """Exact mean of x^(2a) y^(2b) z^(2c) over the unit sphere."""
    return Fraction(_dfact(2 * a - 1) * _dfact(2 * b - 1) * _dfact(2 * c - 1), _dfact(2 * (a + b + c) + 1))


def invariant_mean(i, j):
    """Exact mean of e2^i e3^j over the unit sphere."""
    s = Fraction(0)
    for i1 in range(i + 1):
        for i2 in range(i - i1 + 1):
            i3 = i - i1 - i2
            coef = math.factorial(i) // (math.factorial(i1) * math.factorial(i2) * math.factorial(i3))
            s += coef * sphere_mean(i1 + i3 + j, i1 + i2 + j, i2 + i3 + j)
    return s


def polish(n_points, kinds, xv, dps=60, iters=8):
    import mpmath as mp
    mp.mp.dps = dps
    p = STRUCTURE[n_points][0]
    conds = [(i, j) for i in range(p // 4 + 1) for j in range(p // 6 + 1) if 4 * i + 6 * j <= p]
    target = [mp.mpf(invariant_mean(i, j).numerator) / invariant_mean(i, j).denominator for i, j in conds]
    x = [mp.mpf(float(v)) for v in xv]
    n = len(x)

    def residual(x):
        f = [mp.mpf(0)] * len(conds)
        i = 0
        for k in kinds:
            W = x[i]
            i += 1
            if k == "a1":
                g = [mp.mpf(1), mp.mpf(0), mp.mpf(0)]
            elif k == "a2":
                g = [mp.sqrt(mp.mpf(1) / 2)] * 2 + [mp.mpf(0)]
            elif k == "a3":
                g = [mp.sqrt(mp.mpf(1) / 3)] * 3
            elif k == "b":
                g = [x[i], x[i], mp.sqrt(1 - 2 * x[i] ** 2)]
                i += 1
            elif k == "c":
                g = [x[i], mp.sqrt(1 - x[i] ** 2), mp.mpf(0)]
                i += 1
            else:
                g = [x[i], x[i + 1], mp.sqrt(1 - x[i] ** 2 - x[i + 1] ** 2)]
                i += 2
            a, b, c = g[0] ** 2, g[1] ** 2, g[2] ** 2
            e2, e3 = a * b + b * c + c * a, a * b * c
            for q, (ii, jj) in enumerate(conds):
                f[q] += W * e2 ** ii * e3 ** jj
        return [f[q] - target[q] for q in range(len(conds))]

    for _ in range(iters):
        f0 = residual(x)
        J = mp.matrix(len(conds), n)
        for col in range(n):           # central differences at 1e-25 in 60 digits
            h = mp.mpf(10) ** -25
            xp = list(x)
            xm = list(x)
            xp[col] += h
            xm[col] -= h
            fp, fm = residual(xp), residual(xm)
            for q in range(len(conds)):
                J[q, col] = (fp[q] - fm[q]) / (2 * h)
        step = mp.lu_solve(J, mp.matrix(f0))
        x = [x[k] - step[k] for k in range(n)]
    if max(abs(v) for v in residual(x)) > mp.mpf(10) ** -40:
        raise RuntimeError(f"{n_points}: polish did not converge")
    orbits = []
    i = 0
    for k in kinds:
        W = x[i]
        i += 1
        if k == "a1":
            g = [mp.mpf(1), mp.mpf(0), mp.mpf(0)]
        elif k == "a2":
            g = [mp.sqrt(mp.mpf(1) / 2)] * 2 + [mp.mpf(0)]
        elif k == "a3":
            g = [mp.sqrt(mp.mpf(1) / 3)] * 3
        elif k == "b":
            l = abs(x[i])
            g = [l, l, mp.sqrt(1 - 2 * l ** 2)]
            i += 1
        elif k == "c":
            pq = sorted([abs(x[i]), mp.sqrt(1 - x[i] ** 2)])
            g = [pq[0], pq[1], mp.mpf(0)]
            i += 1
        else:
            g = sorted([abs(x[i]), abs(x[i + 1]), mp.sqrt(1 - x[i] ** 2 - x[i + 1] ** 2)])
            i += 2
        orbits.append((k, tuple(float(v) for v in g), float(W * 4 * mp.pi / SIZE[k])))
    orbits.sort(key=lambda o: (KIND_ORDER.index(o[0]), o[1]))
    return orbits


def lebedev_orbits(n_points):
    """Solve for the rule of n_points points: orbits as (kind, generator, weight per point)."""
    if n_points not in STRUCTURE:
        raise ValueError(f"no Lebedev rule of {n_points} points here: {sorted(STRUCTURE)}")
    kinds, xv = search(n_points)
    return polish(n_points, kinds, xv)


def read_orbits(path):
    """Orbits from a text file of lines 'kind gx gy gz w' (float.hex values)."""
    out = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, gx, gy, gz, w = line.split()
                out.append((k, (float.fromhex(gx), float.fromhex(gy), float.fromhex(gz)), float.fromhex(w)))
    return out


def write_orbits(orbits, path, header=""):
    with open(path, "w") as f:
        if header:
            f.write("".join("# " + h + "\n" for h in header.splitlines()))
        for k, g, w in orbits:
            f.write(f"{k} {g[0].hex()} {g[1].hex()} {g[2].hex()} {w.hex()}\n")


CACHE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def angular_rule(n_points):
    """(ux, uy, uz, w) of the n-point rule.  lebedev_orbits' results are kept as text in
    tests/golden/lebedev_<n>.txt (written by tests/golden/make_lebedev.py); a kept result is
    read instead of solving again."""
    path = os.path.join(CACHE_DIR, f"lebedev_{n_points}.txt")
    orbits = read_orbits(path) if os.path.exists(path) else lebedev_orbits(n_points)
    return expand(orbits)
