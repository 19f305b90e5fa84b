"""Seeded synthetic inputs for the exchange-correlation integration path.

This module produces only *inputs*: molecular geometries (water clusters),
Cartesian Gaussian basis sets, the AO overlap matrix used to normalise the
density matrix, and seeded density matrices.  It holds none of the quadrature,
partitioning, screening, collocation or functional arithmetic of the method;
both the CPU oracle and the CUDA library consume what it returns.

Recipe (stated once, used everywhere):

* Water: O at the origin, H at (+-0.757, 0.587, 0) Angstrom, converted to bohr
  with 1/0.529177210903.
* A cluster of ``n`` waters: oxygen positions uniform in a cube of edge
  ``L = 10 * (n/16)**(1/3)`` Angstrom, any O-O distance below 2.6 Angstrom is
  rejected and redrawn; every molecule gets a uniform random rotation
  (Shoemake's quaternion construction).  Atom order is O, H, H per water.
  Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64).
* Basis (Cartesian shells, 3 primitives each): O = 3s 2p 1d, H = 2s 1p.  For an
  element and angular momentum L with k shells, 3k exponents are taken as a
  geometric sequence from 1e3 down to 0.1 and handed out in consecutive
  triples, tightest shell first.  Contraction coefficients are U(0.1, 1.0)
  from ``default_rng(100 + Z)``, multiplied by the primitive normalisation, and
  the contracted function is then rescaled so that its x^L component has unit
  norm.  Shell order on an atom: s shells, p shells, d shells; function order
  is atom-major, then shell order, then the Cartesian components
  (l, m, n) with l descending, then m descending.
* Density: C ~ N(0, 1) of shape (N_b, 5 n_waters) from ``default_rng(seed)``,
  made S-orthonormal through a Cholesky factor of C^T S C, then P = 2 C C^T, so
  that Tr(P S) = 10 n_waters and P is symmetric positive semi-definite.

Everything that decides a plan (atom positions, exponents) is computed with basic IEEE
operations in a fixed order: the rotations' sines and cosines, the box edge's cube root and
the exponents' powers by the fixed-operation functions below instead of the platform libm,
and the rotation of each water as explicit sums, so a seed gives the same geometry and basis
exponents, bit for bit, on every host architecture.  (Contraction coefficients and P, which
change values only at rounding level, use numpy as is.)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903

# Fixed-operation elementary functions (see the module docstring): ln by 2 atanh((m-1)/(m+1))
# on the frexp mantissa in [1/sqrt2, sqrt2); exp by exp(r) 2^k with r = y - k ln2 (ln 2 in two
# parts) and the Taylor series of exp(r) to r^27; sin and cos by x = q pi/2 + r and the Taylor
# series of sin r and cos r; cube root by Newton's iteration c <- (2c + x/c^2)/3.
_LN2_HI, _LN2_LO = 6.93147180369123816490e-01, 1.90821492927058770002e-10
_PIO2_HI, _PIO2_LO = 1.57079632673412561417e+00, 6.07710050650619224932e-11


def _fixed_ln(x: float) -> float:
    m, e = math.frexp(x)
    if m < 0.70710678118654752440:
        m, e = m * 2.0, e - 1
    s = (m - 1.0) / (m + 1.0)
    s2, t, acc = s * s, s, s
    for k in range(1, 13):
        t = t * s2
        acc = acc + t / float(2 * k + 1)
    return float(e) * _LN2_HI + (2.0 * acc + float(e) * _LN2_LO)


def _fixed_exp(y: float) -> float:
    k = math.floor(y / (_LN2_HI + _LN2_LO) + 0.5)
    r = (y - float(k) * _LN2_HI) - float(k) * _LN2_LO
    t, acc = 1.0, 1.0
    for j in range(1, 28):
        t = t * r / float(j)
        acc = acc + t
    return math.ldexp(acc, k)


def _fixed_sincos(x: float):
    q = float(math.floor(x * 0.63661977236758134308 + 0.5))
    r = (x - q * _PIO2_HI) - q * _PIO2_LO
    r2 = r * r
    tc, c, ts, sn = 1.0, 1.0, r, r
    for k in range(1, 12):
        tc = tc * (-r2) / float((2 * k - 1) * (2 * k))
        c = c + tc
        ts = ts * (-r2) / float((2 * k) * (2 * k + 1))
        sn = sn + ts
    return [(sn, c), (c, -sn), (-sn, -c), (-c, sn)][int(q) & 3]


def _fixed_cbrt(x: float) -> float:
    c = 1.0
    for _ in range(60):
        c = (2.0 * c + x / (c * c)) / 3.0
    return c

# element -> list of (L, number of shells)
_SHELL_RULES = {
    8: [(0, 3), (1, 2), (2, 1)],   # O: 3s 2p 1d
    1: [(0, 2), (1, 1)],           # H: 2s 1p
}


def cart_components(L: int):
    """Cartesian exponent triples (l, m, n) of a shell, l descending then m descending."""
    out = []
    for l in range(L, -1, -1):
        for m in range(L - l, -1, -1):
            out.append((l, m, L - l - m))
    return out


# Pure (spherical) shells, L >= 2: the 2L+1 functions m = -L..L are the real solid harmonics
# S_Lm in Racah normalisation (sphere norm equal to that of x^L) written in the Cartesian
# components of the shell (order of cart_components).  This table defines the pure functions
# of the synthetic workloads; it serves only the input generation here (the overlap matrix
# that normalises the density).
_S3, _S15 = math.sqrt(3.0), math.sqrt(15.0)
_A, _B = math.sqrt(5.0 / 8.0), math.sqrt(3.0 / 8.0)
PURE_TABLE = {
    # xx, xy, xz, yy, yz, zz
    2: [[0, _S3, 0, 0, 0, 0],                      # m = -2: sqrt3 xy
        [0, 0, 0, 0, _S3, 0],                      # m = -1: sqrt3 yz
        [-0.5, 0, 0, -0.5, 0, 1.0],                # m =  0: z^2 - (x^2 + y^2)/2
        [0, 0, _S3, 0, 0, 0],                      # m =  1: sqrt3 xz
        [_S3 / 2, 0, 0, -_S3 / 2, 0, 0]],          # m =  2: sqrt3/2 (x^2 - y^2)
    # xxx, xxy, xxz, xyy, xyz, xzz, yyy, yyz, yzz, zzz
    3: [[0, 3 * _A, 0, 0, 0, 0, -_A, 0, 0, 0],     # m = -3
        [0, 0, 0, 0, _S15, 0, 0, 0, 0, 0],         # m = -2
        [0, -_B, 0, 0, 0, 0, -_B, 0, 4 * _B, 0],   # m = -1
        [0, 0, -1.5, 0, 0, 0, 0, -1.5, 0, 1.0],    # m =  0
        [-_B, 0, 0, -_B, 0, 4 * _B, 0, 0, 0, 0],   # m =  1
        [0, 0, _S15 / 2, 0, 0, 0, 0, -_S15 / 2, 0, 0],   # m =  2
        [_A, 0, 0, -3 * _A, 0, 0, 0, 0, 0, 0]],    # m =  3
}


def nfunc(L: int, pure: int = 0) -> int:
    """Functions of a shell: (L+1)(L+2)/2 Cartesian, or 2L+1 for a pure shell with L >= 2."""
    return 2 * L + 1 if (pure and L >= 2) else ncart(L)


def ncart(L: int) -> int:
    return (L + 1) * (L + 2) // 2


def _dfact(n: int) -> float:
    """(n)!! with (-1)!! = 0!! = 1."""
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


@dataclass
class Basis:
    """Contracted Cartesian Gaussian shells with coefficients ready to use."""
    atom: np.ndarray      # (nshell,) int32 atom index of each shell
    L: np.ndarray         # (nshell,) int32
    nprim: np.ndarray     # (nshell,) int32
    alpha: np.ndarray     # (nshell, maxprim) float64, zero padded
    coeff: np.ndarray     # (nshell, maxprim) float64, normalisation folded in
    center: np.ndarray    # (nshell, 3) float64, bohr (copy of the atom position)
    func_offset: np.ndarray = field(default=None)  # (nshell+1,) first function of each shell
    pure: np.ndarray = field(default=None)         # (nshell,) int32: 1 = spherical shell (L >= 2)

    def __post_init__(self):
        if self.pure is None:
            self.pure = np.zeros(len(self.L), dtype=np.int32)
        if self.func_offset is None:
            off = np.zeros(len(self.L) + 1, dtype=np.int64)
            off[1:] = np.cumsum([nfunc(int(l), int(p)) for l, p in zip(self.L, self.pure)])
            self.func_offset = off

    @property
    def nshell(self) -> int:
        return len(self.L)

    @property
    def nbf(self) -> int:
        return int(self.func_offset[-1])


@dataclass
class Molecule:
    Z: np.ndarray         # (natoms,) int32
    xyz: np.ndarray       # (natoms, 3) float64 bohr
    n_waters: int = 0

    @property
    def natoms(self) -> int:
        return len(self.Z)


def _rotation_from_uniform(u1: float, u2: float, u3: float) -> np.ndarray:
    """Uniform random rotation matrix from three U(0,1) numbers (Shoemake 1992)."""
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    s2, c2 = _fixed_sincos(2.0 * math.pi * u2)
    s3, c3 = _fixed_sincos(2.0 * math.pi * u3)
    qx = a * s2
    qy = a * c2
    qz = b * s3
    qw = b * c3
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ])


_WATER_LOCAL = np.array([[0.0, 0.0, 0.0], [0.757, 0.587, 0.0], [-0.757, 0.587, 0.0]])


def water_cluster(n_waters: int, seed: int, box_angstrom: float | None = None,
                  min_oo_angstrom: float = 2.6, rotate: bool = True) -> Molecule:
    """Seeded cluster of rigid waters in a cube (see module docstring)."""
    rng = np.random.default_rng(seed)
    if box_angstrom is None:
        box_angstrom = 10.0 * _fixed_cbrt(n_waters / 16.0)
    if n_waters == 1:
        centers = [np.zeros(3)]
    else:
        centers = []
        tries = 0
        while len(centers) < n_waters:
            tries += 1
            if tries > 200000:
                raise RuntimeError("could not place waters; box too small")
            c = rng.uniform(0.0, box_angstrom, size=3)
            if all(math.sqrt((c[0] - o[0]) * (c[0] - o[0]) + (c[1] - o[1]) * (c[1] - o[1])
                             + (c[2] - o[2]) * (c[2] - o[2])) >= min_oo_angstrom for o in centers):
                centers.append(c)
    xyz, Z = [], []
    for c in centers:
        R = _rotation_from_uniform(*rng.uniform(size=3)) if (rotate and n_waters > 1) else np.eye(3)
        for k, z in enumerate((8, 1, 1)):
            v = _WATER_LOCAL[k]
            xyz.append([float(c[r]) + ((float(R[r, 0]) * v[0] + float(R[r, 1]) * v[1]) + float(R[r, 2]) * v[2])
                        for r in range(3)])
            Z.append(z)
    return Molecule(Z=np.array(Z, dtype=np.int32),
                    xyz=np.array(xyz, dtype=np.float64) * ANGSTROM_TO_BOHR,
                    n_waters=n_waters)


def single_atom(Z: int = 8) -> Molecule:
    return Molecule(Z=np.array([Z], dtype=np.int32), xyz=np.zeros((1, 3)), n_waters=0)


def _element_shells(Z: int):
    """[(L, alphas(3), raw_coeffs(3))] for one element, shell order s, p, d."""
    rng = np.random.default_rng(100 + int(Z))
    shells = []
    for L, k in _SHELL_RULES[int(Z)]:
        nexp = 3 * k
        if nexp == 1:
            exps = np.array([1e3])
        else:
            l4 = _fixed_ln(1e-4)
            exps = np.array([1e3 * _fixed_exp(l4 * (i / (nexp - 1))) for i in range(nexp)])
        for s in range(k):
            a = exps[3 * s:3 * s + 3].copy()
            d = rng.uniform(0.1, 1.0, size=3)
            shells.append((L, a, d))
    return shells


def _normalise(L: int, a: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Fold primitive normalisation into d, then scale so the x^L component has unit norm."""
    df = _dfact(2 * L - 1)
    prim = (2.0 * a / math.pi) ** 0.75 * (4.0 * a) ** (L / 2.0) / math.sqrt(df)
    c = d * prim
    norm2 = 0.0
    for i in range(len(a)):
        for j in range(len(a)):
            p = a[i] + a[j]
            norm2 += c[i] * c[j] * df / (2.0 * p) ** L * (math.pi / p) ** 1.5
    return c / math.sqrt(norm2)


def make_basis(mol: Molecule, single_shell: tuple | None = None, pure: bool = False) -> Basis:
    """Basis for a molecule from the element rules above.

    ``single_shell=(L, alphas, coeffs)`` instead puts exactly one shell with
    the given raw coefficients (normalised as above) on every atom, used by
    closed-form tests.  ``pure=True`` makes every shell with L >= 2 spherical.
    """
    atom, Ls, nprim, alpha, coeff, center = [], [], [], [], [], []
    for A in range(mol.natoms):
        if single_shell is not None:
            L, a, d = single_shell
            shells = [(L, np.asarray(a, float), np.asarray(d, float))]
        else:
            shells = _element_shells(mol.Z[A])
        for L, a, d in shells:
            atom.append(A)
            Ls.append(L)
            nprim.append(len(a))
            alpha.append(a)
            coeff.append(_normalise(L, a, d))
            center.append(mol.xyz[A])
    maxp = max(nprim)
    al = np.zeros((len(Ls), maxp))
    co = np.zeros((len(Ls), maxp))
    for s in range(len(Ls)):
        al[s, :nprim[s]] = alpha[s]
        co[s, :nprim[s]] = coeff[s]
    Ls = np.array(Ls, dtype=np.int32)
    return Basis(atom=np.array(atom, dtype=np.int32), L=Ls,
                 nprim=np.array(nprim, dtype=np.int32), alpha=al, coeff=co,
                 center=np.array(center, dtype=np.float64),
                 pure=((Ls >= 2) & bool(pure)).astype(np.int32))


def _overlap_1d_table(a, b, A, B, lmax: int):
    """1-D overlaps int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) dx for i, j <= lmax.

    ``a``/``A`` are scalars, ``b``/``B`` arrays; the result has shape
    ``b.shape + (lmax+1, lmax+1)``.  Gaussian product theorem plus the even
    Gaussian moments (k-1)!! / (2p)^(k/2) sqrt(pi/p).
    """
    p = a + b
    P = (a * A + b * B) / p
    pre = np.exp(-a * b / p * (A - B) ** 2)
    PA, PB = P - A, P - B
    mom = [np.sqrt(math.pi / p) * (_dfact(k - 1) / (2.0 * p) ** (k // 2) if k % 2 == 0 else 0.0)
           for k in range(2 * lmax + 1)]
    out = np.zeros(np.shape(b) + (lmax + 1, lmax + 1))
    for la in range(lmax + 1):
        for lb in range(lmax + 1):
            s = 0.0
            for i in range(la + 1):
                for j in range(lb + 1):
                    if (i + j) % 2:
                        continue
                    s = s + (math.comb(la, i) * math.comb(lb, j)) * PA ** (la - i) * PB ** (lb - j) * mom[i + j]
            out[..., la, lb] = pre * s
    return out


def overlap_matrix(basis: Basis) -> np.ndarray:
    """Closed-form AO overlap S (used only to normalise the seeded density); pure shells
    through PURE_TABLE applied to the Cartesian overlap."""
    if np.any(basis.pure):
        cart = Basis(atom=basis.atom, L=basis.L, nprim=basis.nprim, alpha=basis.alpha, coeff=basis.coeff,
                     center=basis.center)
        Sc = overlap_matrix(cart)
        T = np.zeros((basis.nbf, cart.nbf))
        for s in range(basis.nshell):
            o, oc = basis.func_offset[s], cart.func_offset[s]
            L = int(basis.L[s])
            if basis.pure[s]:
                T[o:o + 2 * L + 1, oc:oc + ncart(L)] = PURE_TABLE[L]
            else:
                T[o:o + ncart(L), oc:oc + ncart(L)] = np.eye(ncart(L))
        S = T @ Sc @ T.T
        return 0.5 * (S + S.T)
    nbf = basis.nbf
    lmax = int(basis.L.max())
    maxp = basis.alpha.shape[1]
    fshell = np.repeat(np.arange(basis.nshell), [ncart(int(l)) for l in basis.L])
    fexp = np.array([c for L in basis.L for c in cart_components(int(L))], dtype=np.int64)
    alpha = basis.alpha.copy()
    alpha[alpha == 0.0] = 1.0            # padded primitives carry zero coefficients
    S = np.zeros((nbf, nbf))
    for s1 in range(basis.nshell):
        o1 = basis.func_offset[s1]
        comps = cart_components(int(basis.L[s1]))
        acc = np.zeros((len(comps), nbf))
        for p1 in range(basis.nprim[s1]):
            a = basis.alpha[s1, p1]
            T = [_overlap_1d_table(a, alpha, basis.center[s1, d], basis.center[:, d][:, None], lmax)
                 for d in range(3)]                      # each (nshell, maxp, l+1, l+1)
            cq = basis.coeff[fshell]                    # (nbf, maxp)
            for i1, (l1, m1, n1) in enumerate(comps):
                v = (T[0][fshell, :, l1, fexp[:, 0]] * T[1][fshell, :, m1, fexp[:, 1]]
                     * T[2][fshell, :, n1, fexp[:, 2]])  # (nbf, maxp)
                acc[i1] += basis.coeff[s1, p1] * np.sum(cq * v, axis=1)
        S[o1:o1 + len(comps)] = acc
    return 0.5 * (S + S.T)


def density_matrix(S: np.ndarray, n_occ: int, seed: int) -> np.ndarray:
    """P = 2 C C^T with C^T S C = I (n_occ doubly occupied orbitals)."""
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((S.shape[0], n_occ))
    M = C.T @ S @ C
    Lc = np.linalg.cholesky(M)
    C = np.linalg.solve(Lc, C.T).T          # C L^{-T}
    P = 2.0 * C @ C.T
    return 0.5 * (P + P.T)


# ---------------------------------------------------------------------------
# workload configurations (sizes and rules of the five workloads)
# ---------------------------------------------------------------------------
@dataclass
class GridSpec:
    nrad: int
    ntheta: int
    nphi: int
    partition: str          # "becke" | "ssf"
    max_batch: int
    eta: float = 1e-10
    mk_alpha: float = 5.0
    angular: str = "product"  # "product": ntheta x nphi; "lebedev": the rule of ntheta points


@dataclass
class Workload:
    name: str
    mol: Molecule
    basis: Basis
    grid: GridSpec
    functional: str
    P: np.ndarray
    S: np.ndarray


WORKLOADS = {
    # one water, Slater exchange, Becke partition, 50 x 12 x 24, batches <= 256
    "water1_slater": dict(n_waters=1, grid=GridSpec(50, 12, 24, "becke", 256), functional="slater"),
    # 16-water cluster in a 10 Angstrom box, PBE, SSF, 75 x 16 x 32, batches <= 512
    "water16_pbe": dict(n_waters=16, grid=GridSpec(75, 16, 32, "ssf", 512), functional="pbe"),
    # 64-water cluster, PBE, same grid rules
    "water64_pbe": dict(n_waters=64, grid=GridSpec(75, 16, 32, "ssf", 512), functional="pbe"),
    # small cases that the oracle finishes in seconds
    "water2_pbe_small": dict(n_waters=2, grid=GridSpec(20, 8, 16, "ssf", 128), functional="pbe"),
    "water3_pbe_small": dict(n_waters=3, grid=GridSpec(24, 10, 20, "ssf", 200), functional="pbe"),
    "water1_pbe_small": dict(n_waters=1, grid=GridSpec(30, 10, 20, "becke", 256), functional="pbe"),
    # spherical d shells (O 3s2p1d: 14 functions; 24 per water)
    "water2_pbe_small_sph": dict(n_waters=2, grid=GridSpec(20, 8, 16, "ssf", 128), functional="pbe", pure=True),
    "water16_pbe_sph": dict(n_waters=16, grid=GridSpec(75, 16, 32, "ssf", 512), functional="pbe", pure=True),
    # Lebedev-Laikov angular rules: a small case, and the paper's FG grid (75 x 302)
    "water2_pbe_small_leb": dict(n_waters=2, grid=GridSpec(20, 110, 0, "ssf", 128, angular="lebedev"),
                                 functional="pbe"),
    "water16_pbe_fg": dict(n_waters=16, grid=GridSpec(75, 302, 0, "ssf", 512, angular="lebedev"),
                           functional="pbe"),
    # the paper's UFG (99 x 590) and SFG (175 x 974) grids on the 16-water cluster
    "water16_pbe_ufg": dict(n_waters=16, grid=GridSpec(99, 590, 0, "ssf", 512, angular="lebedev"),
                            functional="pbe"),
    "water16_pbe_sfg": dict(n_waters=16, grid=GridSpec(175, 974, 0, "ssf", 512, angular="lebedev"),
                            functional="pbe"),
    # the 974-point rule (the paper's SFG angular grid) on a small radial grid
    "water2_pbe_small_974": dict(n_waters=2, grid=GridSpec(20, 974, 0, "ssf", 128, angular="lebedev"),
                                 functional="pbe"),
}

_WORKLOAD_SEEDS = {"water1_slater": 1000, "water16_pbe": 2000, "water64_pbe": 3000,
                   "water2_pbe_small": 9100, "water3_pbe_small": 9200, "water1_pbe_small": 9300,
                   "water2_pbe_small_sph": 9100, "water16_pbe_sph": 2000,
                   "water2_pbe_small_leb": 9100, "water16_pbe_fg": 2000, "water2_pbe_small_974": 9100,
                   "water16_pbe_ufg": 2000, "water16_pbe_sfg": 2000}


def make_workload(name: str, n_waters: int | None = None, seed: int | None = None) -> Workload:
    cfg = WORKLOADS[name]
    nw = cfg["n_waters"] if n_waters is None else n_waters
    sd = _WORKLOAD_SEEDS[name] if seed is None else seed
    mol = water_cluster(nw, sd)
    basis = make_basis(mol, pure=cfg.get("pure", False))
    S = overlap_matrix(basis)
    P = density_matrix(S, 5 * nw, sd + 1)
    return Workload(name=name, mol=mol, basis=basis, grid=cfg["grid"], functional=cfg["functional"],
                    P=P, S=S)
