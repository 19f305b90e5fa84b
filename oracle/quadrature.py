"""Atomic product quadrature (Sec. 2.2, Eqs. atomic_partition and num_int).

The paper pairs a Mura-Knowles radial rule with Lebedev-Laikov spheres.  The
Lebedev tables are not available here, so the angular factor is a product rule:
Gauss-Legendre in cos(theta) times the trapezoid rule in phi, which integrates
every spherical harmonic of degree l <= 2*n_theta - 1 with |m| < n_phi / 2
exactly.

Floating-point contract: the coordinates produced here must be bit-identical
to the library's host-side grid builder, because batch membership is decided by
exact comparisons.  So every logarithm, sine and cosine is the fixed-operation
version of ``elementary`` (not the platform libm, whose last bits differ between
hosts), every combination is an explicit IEEE operation in a fixed order (no FMA,
no pairwise sums), and the order of operations is spelled out in each docstring.
"""
from __future__ import annotations

import math

import numpy as np

from . import elementary as el


def mura_knowles(n: int, alpha: float):
    """Mura-Knowles radial rule with the r^2 Jacobian folded into the weights.

    Reading of the paper (which only cites the rule): x_k = k/(n+1),
    r_k = -alpha*ln(1 - x_k^3), w_k = 3*alpha*x_k^2 / ((1 - x_k^3)(n+1)) * r_k^2,
    k = 1..n.  Order of operations: x3 = (x*x)*x; r = (-alpha)*log(1 - x3);
    w = ((((3*alpha)*x)*x) / ((1 - x3)*(n+1))) * r * r.
    """
    r = np.empty(n)
    w = np.empty(n)
    for k in range(1, n + 1):
        x = k / (n + 1.0)
        x3 = x * x * x
        rk = -alpha * el.ln(1.0 - x3)
        r[k - 1] = rk
        w[k - 1] = 3.0 * alpha * x * x / ((1.0 - x3) * (n + 1.0)) * rk * rk
    return r, w


def gauss_legendre(n: int):
    """Gauss-Legendre nodes t_i (descending) and weights on [-1, 1] by Newton iteration.

    Start t = cos(pi*(i + 0.75)/(n + 0.5)); evaluate P_n by the three-term
    recurrence P_{j+1} = ((2j+1) t P_j - j P_{j-1})/(j+1); P_n' = n (t P_n - P_{n-1})/(t^2 - 1);
    step t <- t - P_n/P_n' until the step is below 1e-15 in magnitude (at most
    100 steps).  Weight 2/((1 - t^2) P_n'(t)^2) at the final t.
    """
    t_out = np.empty(n)
    w_out = np.empty(n)
    for i in range(n):
        t = el.cos(math.pi * (i + 0.75) / (n + 0.5))
        for _ in range(100):
            p1, p2 = 1.0, 0.0
            for j in range(n):
                p3 = p2
                p2 = p1
                jf = float(j)
                p1 = ((2.0 * jf + 1.0) * t * p2 - jf * p3) / (jf + 1.0)
            pp = n * (t * p1 - p2) / (t * t - 1.0)
            t1 = t
            t = t1 - p1 / pp
            if abs(t - t1) <= 1e-15:
                break
        p1, p2 = 1.0, 0.0
        for j in range(n):
            p3 = p2
            p2 = p1
            jf = float(j)
            p1 = ((2.0 * jf + 1.0) * t * p2 - jf * p3) / (jf + 1.0)
        pp = n * (t * p1 - p2) / (t * t - 1.0)
        t_out[i] = t
        w_out[i] = 2.0 / ((1.0 - t * t) * pp * pp)
    return t_out, w_out


def angular_product(ntheta: int, nphi: int):
    """Unit vectors and weights of the GL(cos theta) x trapezoid(phi) rule.

    Point (a, b): cos(theta) = t_a, sin(theta) = sqrt(1 - t_a*t_a),
    phi_b = ((2*pi)*b)/n_phi; u = (sin*cos(phi), sin*sin(phi), cos(theta));
    weight = w_a * ((2*pi)/n_phi).  Ordered theta-major.  Weights sum to 4*pi.
    """
    t, wt = gauss_legendre(ntheta)
    cphi = np.array([el.cos(2.0 * math.pi * b / nphi) for b in range(nphi)])
    sphi = np.array([el.sin(2.0 * math.pi * b / nphi) for b in range(nphi)])
    st = np.array([math.sqrt(1.0 - x * x) for x in t])
    ux = st[:, None] * cphi[None, :]
    uy = st[:, None] * sphi[None, :]
    uz = np.broadcast_to(t[:, None], (ntheta, nphi))
    wphi = 2.0 * math.pi / nphi
    w = np.broadcast_to((wt * wphi)[:, None], (ntheta, nphi))
    return (ux.reshape(-1), uy.reshape(-1), np.ascontiguousarray(uz).reshape(-1),
            np.ascontiguousarray(w).reshape(-1))


def atom_grid(center, nrad: int, ntheta: int, nphi: int, mk_alpha: float, angular=None):
    """Quadrature points of one atom, ordered radial-major then angular point.

    Coordinate = R + r_k * u (product first, then the sum); weight =
    w_rad_k * w_ang (the unmodified weights w^q of Eq. num_int).  The angular rule is the
    product rule (theta-major) unless `angular` = (ux, uy, uz, wa) gives another one.
    Returns x, y, z, wq as float64 arrays of length nrad * (angular points).
    """
    r, wr = mura_knowles(nrad, mk_alpha)
    ux, uy, uz, wa = angular if angular is not None else angular_product(ntheta, nphi)
    x = center[0] + r[:, None] * ux[None, :]
    y = center[1] + r[:, None] * uy[None, :]
    z = center[2] + r[:, None] * uz[None, :]
    wq = wr[:, None] * wa[None, :]
    return x.reshape(-1), y.reshape(-1), z.reshape(-1), wq.reshape(-1)


def molecular_grid(xyz, nrad: int, ntheta: int, nphi: int, mk_alpha: float, angular=None):
    """Union of the atomic grids (the total quadrature Q), atom-major.

    Returns x, y, z, wq (float64) and the parent atom index (int32) per point.
    """
    xs, ys, zs, ws, par = [], [], [], [], []
    for A in range(len(xyz)):
        x, y, z, wq = atom_grid(xyz[A], nrad, ntheta, nphi, mk_alpha, angular)
        xs.append(x)
        ys.append(y)
        zs.append(z)
        ws.append(wq)
        par.append(np.full(len(x), A, dtype=np.int32))
    return (np.concatenate(xs), np.concatenate(ys), np.concatenate(zs), np.concatenate(ws),
            np.concatenate(par))
