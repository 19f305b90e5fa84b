"""Pins for the oracle's atomic quadrature (Sec. 2.2, Eq. num_int)."""
import math

import numpy as np
import pytest

from oracle import quadrature as Q


@pytest.mark.parametrize("a", [0.1, 0.5, 1.0, 10.0, 100.0])
def test_radial_gaussian_moment(a):
    # int_0^inf r^2 exp(-a r^2) dr = sqrt(pi) / (4 a^(3/2)); the error must fall as n grows
    exact = math.sqrt(math.pi) / (4.0 * a ** 1.5)
    errs = []
    for n in (25, 50, 75, 150):
        r, w = Q.mura_knowles(n, 5.0)
        errs.append(abs(np.sum(w * np.exp(-a * r * r)) - exact) / exact)
    assert errs[-1] < 1e-7
    assert errs[2] < 1e-5
    assert errs[-1] < errs[0]


def test_radial_nodes_closed_form():
    r, w = Q.mura_knowles(3, 2.0)
    x = np.array([1, 2, 3]) / 4.0
    assert np.allclose(r, -2.0 * np.log(1 - x ** 3), rtol=1e-15)
    assert np.allclose(w, 3 * 2.0 * x ** 2 / ((1 - x ** 3) * 4) * r ** 2, rtol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 12, 16, 24])
def test_gauss_legendre_matches_library(n):
    t, w = Q.gauss_legendre(n)
    tl, wl = np.polynomial.legendre.leggauss(n)
    assert np.allclose(np.sort(t), tl, atol=2e-16 * n, rtol=0)
    assert np.allclose(w[np.argsort(t)], wl, rtol=5e-13, atol=0)
    assert abs(np.sum(w) - 2.0) < 1e-14


def _sphere_monomial(a, b, c):
    # int over S^2 of x^a y^b z^c = 2 G((a+1)/2) G((b+1)/2) G((c+1)/2) / G((a+b+c+3)/2), zero if any odd
    if a % 2 or b % 2 or c % 2:
        return 0.0
    g = math.gamma
    return 2.0 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)


@pytest.mark.parametrize("nt,nphi", [(4, 8), (12, 24), (16, 32)])
def test_angular_exact_for_low_degree(nt, nphi):
    ux, uy, uz, w = Q.angular_product(nt, nphi)
    assert abs(np.sum(w) - 4 * math.pi) < 1e-13
    deg = min(2 * nt - 1, nphi - 1)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                got = np.sum(w * ux ** a * uy ** b * uz ** c)
                assert abs(got - _sphere_monomial(a, b, c)) < 1e-13, (a, b, c)


def test_angular_not_exact_beyond_degree():
    # a z^(2n) monomial is beyond Gauss-Legendre's exactness: the test above is not vacuous
    ux, uy, uz, w = Q.angular_product(4, 8)
    assert abs(np.sum(w * uz ** 8) - _sphere_monomial(0, 0, 8)) > 1e-6


def test_atom_grid_layout():
    x, y, z, wq = Q.atom_grid(np.array([1.0, -2.0, 0.5]), 5, 4, 8, 5.0)
    assert len(x) == 5 * 4 * 8
    r, wr = Q.mura_knowles(5, 5.0)
    d = np.sqrt((x - 1.0) ** 2 + (y + 2.0) ** 2 + (z - 0.5) ** 2).reshape(5, 32)
    assert np.allclose(d, r[:, None], rtol=1e-14)
    assert np.allclose(wq.reshape(5, 32).sum(1), wr * 4 * math.pi, rtol=1e-13)
