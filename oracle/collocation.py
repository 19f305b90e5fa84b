"""Contracted Cartesian Gaussians and their gradients (Eq. gau_cart).

phi_mu(r) = (x-R_x)^l (y-R_y)^m (z-R_z)^n sum_xi d_xi exp(-alpha_xi |r - R|^2).

With g(r) = sum_xi d_xi exp(-alpha_xi r^2) and h(r) = sum_xi (-2 alpha_xi d_xi)
exp(-alpha_xi r^2), the gradient is, e.g. for x,
d phi / dx = l x^(l-1) y^m z^n g + x^(l+1) y^m z^n h.

Shell size is (L+1)(L+2)/2 Cartesian functions (the paper prints L(L+1), a
misprint: an L = 1 shell has 3 functions and an L = 2 shell 6).  Component
order: (l, m, n) with l descending, then m descending.

Pure (spherical) shells, as the paper runs cc-pVDZ (Sec. 3): the 2L+1 functions
m = -L..L are the real solid harmonics S_Lm in Racah normalisation, sqrt(4 pi/(2L+1))
r^L Y_Lm, whose norm on the sphere equals that of x^L, expanded in the shell's Cartesian
components by the closed form of Helgaker, Jorgensen and Olsen, "Molecular
Electronic-Structure Theory" (2000), Sec. 6.4.2 (solid_harmonic_matrix below).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def cart_components(L: int):
    out = []
    for l in range(L, -1, -1):
        for m in range(L - l, -1, -1):
            out.append((l, m, L - l - m))
    return out


def solid_harmonic_matrix(L: int) -> np.ndarray:
    """(2L+1) x ncart(L) coefficients of S_Lm, m = -L..L, in the cart_components order.

    S_Lm = N_Lm sum_{t,u,v} C_tuv x^(2t+|m|-2(u+v)) y^(2(u+v)) z^(L-2t-|m|), with
    C_tuv = (-1)^(t+v-v_m) (1/4)^t binom(L,t) binom(L-t,|m|+t) binom(t,u) binom(|m|,2v),
    v_m = 0 (m >= 0) or 1/2 (m < 0), t = 0..(L-|m|)/2, u = 0..t, v = v_m .. floor(|m|/2 - v_m) + v_m,
    N_Lm = sqrt(2 (L+|m|)! (L-|m|)! / 2^delta(m,0)) / (2^|m| L!).
    """
    comps = cart_components(L)
    col = {c: k for k, c in enumerate(comps)}
    T = np.zeros((2 * L + 1, len(comps)))
    for m in range(-L, L + 1):
        am = abs(m)
        vm = Fraction(0) if m >= 0 else Fraction(1, 2)
        norm = math.sqrt(2.0 * math.factorial(L + am) * math.factorial(L - am) / (2.0 if m == 0 else 1.0)) \
            / (2 ** am * math.factorial(L))
        for t in range((L - am) // 2 + 1):
            for u in range(t + 1):
                v = vm
                vmax = math.floor(Fraction(am, 2) - vm) + vm
                while v <= vmax:
                    two_v = int(2 * v)
                    sign = -1 if (t + v - vm) % 2 else 1
                    c = sign * Fraction(1, 4) ** t * math.comb(L, t) * math.comb(L - t, am + t) \
                        * math.comb(t, u) * math.comb(am, two_v)
                    ex = 2 * t + am - 2 * (u + v)
                    ey = 2 * (u + v)
                    ez = L - 2 * t - am
                    T[m + L, col[(int(ex), int(ey), int(ez))]] += norm * float(c)
                    v += 1
    return T


def shell_values(pts, center, L, alphas, coeffs, pure=False):
    """phi and its gradient for one shell at points ``pts`` (m x 3).

    Returns (phi, dx, dy, dz), each of shape (m, ncart(L)), or (m, 2L+1) for a pure
    shell (L >= 2): the Cartesian values times solid_harmonic_matrix(L)^T.
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
    if pure and L >= 2:
        T = solid_harmonic_matrix(L).T
        return phi @ T, gx @ T, gy @ T, gz @ T
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
                           basis.coeff[s, :basis.nprim[s]], pure=bool(basis.pure[s])) for s in shells]
    if not blocks:
        z = np.zeros((len(pts), 0))
        return z, z, z, z
    return tuple(np.concatenate([b[k] for b in blocks], axis=1) for k in range(4))
