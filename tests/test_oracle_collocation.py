"""Pins for the oracle's contracted Cartesian Gaussians (Eq. gau_cart)."""
import math

import numpy as np
import pytest

import xcinputs as X
from oracle import collocation as C


def _shell(L):
    return X.make_basis(X.single_atom(), single_shell=(L, [3.0, 0.7, 0.15], [0.2, 0.5, 0.4]))


@pytest.mark.parametrize("L", [0, 1, 2, 3])
def test_gradient_matches_finite_differences(L):
    b = _shell(L)
    rng = np.random.default_rng(L)
    p = rng.normal(scale=1.2, size=(40, 3))
    phi, gx, gy, gz = C.collocate(p, b)
    h = 1e-5
    for d, g in enumerate((gx, gy, gz)):
        e = np.zeros(3)
        e[d] = h
        fd = (C.collocate(p + e, b)[0] - C.collocate(p - e, b)[0]) / (2 * h)
        assert np.max(np.abs(fd - g)) < 1e-8 * max(1.0, np.abs(g).max())


def test_values_closed_form():
    b = _shell(2)
    p = np.array([[0.3, -0.4, 0.5]])
    phi = C.collocate(p, b)[0][0]
    r2 = 0.5
    g = sum(b.coeff[0, k] * math.exp(-b.alpha[0, k] * r2) for k in range(3))
    x, y, z = p[0]
    expect = [x * x, x * y, x * z, y * y, y * z, z * z]
    assert np.allclose(phi, np.array(expect) * g, rtol=1e-15)
    assert X.ncart(2) == 6 and X.ncart(1) == 3 and X.ncart(3) == 10


@pytest.mark.parametrize("L", [0, 1, 2])
def test_xL_component_unit_norm(L):
    # int phi_{x^L}^2 d^3r = 1 by construction of the basis.  phi^2 has angular degree 2L <= 4,
    # which the 8 x 16 product rule integrates exactly; 400 Mura-Knowles radial points carry
    # the radial part well below the tolerance.
    from oracle import quadrature as Q
    b = _shell(L)
    x, y, z, wq = Q.atom_grid(np.zeros(3), 400, 8, 16, 5.0)
    phi = C.collocate(np.stack([x, y, z], 1), b)[0][:, 0]
    assert abs(np.sum(wq * phi * phi) - 1.0) < 1e-11


def test_shell_subset_columns_are_sorted_global_functions():
    w = X.make_workload("water1_slater")
    p = np.random.default_rng(0).normal(size=(5, 3))
    full = C.collocate(p, w.basis)[0]
    shells = [1, 4, 5, 8]
    cols = np.concatenate([np.arange(w.basis.func_offset[s], w.basis.func_offset[s + 1]) for s in shells])
    assert np.array_equal(C.collocate(p, w.basis, shells)[0], full[:, cols])


# ---------------------------------------------------------------- pure (spherical) shells
@pytest.mark.parametrize("L", [2, 3])
def test_solid_harmonics_match_the_workload_table(L):
    # the oracle's general closed form and the explicit table of the inputs are two
    # independent derivations of the same functions
    assert np.max(np.abs(C.solid_harmonic_matrix(L) - np.array(X.PURE_TABLE[L]))) < 1e-15


@pytest.mark.parametrize("L", [2, 3, 4])
def test_solid_harmonics_addition_theorem(L):
    # Racah normalisation: sum_m S_Lm(r)^2 = r^(2L) at every point (Unsold)
    T = C.solid_harmonic_matrix(L)
    p = np.random.default_rng(L).normal(size=(50, 3))
    mono = np.stack([p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** c for a, b, c in C.cart_components(L)], 1)
    S = mono @ T.T
    r2L = np.sum(p * p, 1) ** L
    assert np.max(np.abs(np.sum(S * S, 1) / r2L - 1.0)) < 1e-13


@pytest.mark.parametrize("L", [2, 3])
def test_pure_shell_orthonormal(L):
    # int chi_m chi_m' d^3r = delta_mm' with the x^L-normalised radial part: angular degree
    # 2L <= 6 is exact on 8 x 16, the radial part to 1e-11 on 400 points
    from oracle import quadrature as Q
    b = X.make_basis(X.single_atom(), single_shell=(L, [3.0, 0.7, 0.15], [0.2, 0.5, 0.4]), pure=True)
    assert b.nbf == 2 * L + 1
    x, y, z, wq = Q.atom_grid(np.zeros(3), 400, 8, 16, 5.0)
    phi = C.collocate(np.stack([x, y, z], 1), b)[0]
    G = phi.T @ (wq[:, None] * phi)
    assert np.max(np.abs(G - np.eye(2 * L + 1))) < 1e-10


def test_pure_gradient_matches_finite_differences():
    b = X.make_basis(X.single_atom(), single_shell=(3, [3.0, 0.7, 0.15], [0.2, 0.5, 0.4]), pure=True)
    p = np.random.default_rng(7).normal(scale=1.2, size=(40, 3))
    phi, gx, gy, gz = C.collocate(p, b)
    h = 1e-5
    for d, g in enumerate((gx, gy, gz)):
        e = np.zeros(3)
        e[d] = h
        fd = (C.collocate(p + e, b)[0] - C.collocate(p - e, b)[0]) / (2 * h)
        assert np.max(np.abs(fd - g)) < 1e-8 * max(1.0, np.abs(g).max())
