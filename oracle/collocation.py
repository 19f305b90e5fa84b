"""Contracted Cartesian Gaussians and their gradients (Eq. gau_cart).

phi_mu(r) = (x-R_x)^l (y-R_y)^m (z-R_z)^n sum_xi d_xi exp(-alpha_xi |r - R|^2).

With g(r) = sum_xi d_xi exp(-alpha_xi r^2) and h(r) = sum_xi (-2 alpha_xi d_xi)
exp(-alpha_xi r^2), the gradient is, e.g. for x,
d phi / dx = l x^(l-1) y^m z^n g + x^(l+1) y^m z^n h.

Shell size is (L+1)(L+2)/2 Cartesian functions (the paper prints L(L+1), a
misprint: an L = 1 shell has 3 functions and an L = 2 shell 6).  Component
order: (l, m, n) with l descending, then m descending.
"""
from __future__ import annotations

import numpy as np


def cart_components(L: int):
    out = []
    for l in range(L, -1, -1):
        for m in range(L - l, -1, -1):
            out.append((l, m, L - l - m))
    return out


def shell_values(pts, center, L, alphas, coeffs):
    """phi and its gradient for one shell at points ``pts`` (m x 3).

    Returns (phi, dx, dy, dz), each of shape (m, ncart(L)).
    """
    X = pts[:, 0] - center[0]
    Y = pts[:, 1] - center[1]
    Z = pts[:, 2] - center[2]
    r2 = X * X + Y * Y + Z * Z
    g = np.zeros(len(pts))
    h = np.zeros(len(pts))
    for a, d in zip(alphas, coeffs):
        e = np.exp(-a * r2)
        g += d * e
        h += (-2.0 * a * d) * e
    comps = cart_components(L)
    phi = np.empty((len(pts), len(comps)))
    gx = np.empty_like(phi)
    gy = np.empty_like(phi)
    gz = np.empty_like(phi)

    def pw(v, k):
        return v ** k if k > 0 else np.ones_like(v)

    for c, (l, m, n) in enumerate(comps):
        xl, ym, zn = pw(X, l), pw(Y, m), pw(Z, n)
        mono = xl * ym * zn
        phi[:, c] = mono * g
        gx[:, c] = (l * pw(X, l - 1) * ym * zn if l > 0 else 0.0) * g + mono * X * h
        gy[:, c] = (m * xl * pw(Y, m - 1) * zn if m > 0 else 0.0) * g + mono * Y * h
        gz[:, c] = (n * xl * ym * pw(Z, n - 1) if n > 0 else 0.0) * g + mono * Z * h
    return phi, gx, gy, gz


def collocate(pts, basis, shells=None):
    """Collocation matrix Phi (m x n) and gradients over the functions of ``shells``.

    ``shells`` is a list of shell indices (default: all).  Columns follow the
    shells' function order, so for a sorted shell list they are the sorted
    global function indices.
    """
    if shells is None:
        shells = range(basis.nshell)
    blocks = [shell_values(pts, basis.center[s], int(basis.L[s]), basis.alpha[s, :basis.nprim[s]],
                           basis.coeff[s, :basis.nprim[s]]) for s in shells]
    if not blocks:
        z = np.zeros((len(pts), 0))
        return z, z, z, z
    return tuple(np.concatenate([b[k] for b in blocks], axis=1) for k in range(4))
