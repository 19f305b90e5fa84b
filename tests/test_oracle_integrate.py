"""Pins for the oracle's E_xc / V_xc / N_el (Eqs. exc_vvar, vxc_exact, zvec_r and the batched
Eqs. x_mat ... z_mat), against closed forms, identities and brute force."""
import math

import numpy as np
import pytest

import xcinputs as X
from oracle import collocation as C
from oracle import functionals as F
from oracle import integrate as I


def _setup(name, **kw):
    w = X.make_workload(name, **kw)
    g = I.make_grid(w.mol.xyz, w.grid)
    pl = I.make_plan(g, w.mol.xyz, w.basis, w.grid)
    return w, g, pl


@pytest.fixture(scope="module")
def water1():
    return _setup("water1_slater")


@pytest.fixture(scope="module")
def water1_pbe():
    return _setup("water1_pbe_small")


@pytest.mark.parametrize("alpha", [1.0, 0.3])
def test_slater_exchange_of_single_s_gaussian(alpha):
    # rho = N^2 exp(-2 a r^2), N^2 = (2a/pi)^(3/2):
    # E_x = C_x int rho^(4/3) = C_x (2a/pi)^2 (3 pi / (8 a))^(3/2); equals -0.38275159923863333 at a = 1
    mol = X.single_atom(8)
    b = X.make_basis(mol, single_shell=(0, [alpha], [1.0]))
    spec = X.GridSpec(75, 16, 32, "becke", 512)
    g = I.make_grid(mol.xyz, spec)
    pl = I.make_plan(g, mol.xyz, b, spec)
    exact = F.C_X * (2 * alpha / math.pi) ** 2 * (3 * math.pi / (8 * alpha)) ** 1.5
    if alpha == 1.0:
        assert abs(exact - (-0.38275159923863333)) < 1e-15
    for occ in (1.0, 2.0):
        r = I.integrate_method(g, b, np.array([[occ]]), "slater", pl)
        assert abs(r.E - occ ** (4 / 3) * exact) < 1e-9
        assert abs(r.N - occ) < 1e-10


def test_electron_count_is_trace_PS(water1):
    w, g, pl = water1
    r = I.integrate_method(g, w.basis, w.P, "slater", pl)
    assert abs(np.trace(w.P @ w.S) - 10.0) < 1e-12
    assert abs(r.N - 10.0) < 1e-4       # quadrature-limited on 50 x 12 x 24


def test_lda_trace_identity(water1):
    # f = C_x rho^(4/3): Tr(P V) = sum_i w_i rho_i vrho_i = (4/3) E_x on the same grid
    w, g, pl = water1
    r = I.integrate_method(g, w.basis, w.P, "slater", pl)
    assert abs(np.sum(w.P * r.V) - 4.0 / 3.0 * r.E) < 1e-12 * abs(r.E)


def test_gga_trace_identity(water1_pbe):
    # Tr(P V) = sum_i w_i (rho_i vrho_i + 2 sigma_i vsigma_i) for any GGA
    w, g, pl = water1_pbe
    r = I.integrate_method(g, w.basis, w.P, "pbe", pl)
    pts = np.stack([g.x, g.y, g.z], 1)
    phi, gx, gy, gz = C.collocate(pts, w.basis)
    rho = np.sum((phi @ w.P) * phi, 1)
    grad = [2 * np.sum((phi @ w.P) * d, 1) for d in (gx, gy, gz)]
    sigma = sum(q * q for q in grad)
    f, vr, vs = F.pbe(rho, sigma)
    assert abs(np.sum(w.P * r.V) - np.sum(g.w * (rho * vr + 2 * sigma * vs))) < 1e-11 * abs(r.E)


def _fd_error(w, g, pl, functional, integrate=I.integrate_method):
    rng = np.random.default_rng(4)
    d = rng.normal(size=w.P.shape)
    d = 0.5 * (d + d.T)
    h = 1e-4
    V = integrate(g, w.basis, w.P, functional, pl).V
    Ep = integrate(g, w.basis, w.P + h * d, functional, pl).E
    Em = integrate(g, w.basis, w.P - h * d, functional, pl).E
    fd = (Ep - Em) / (2 * h)
    return abs(fd - np.sum(V * d)) / abs(fd)


def test_V_is_dE_dP_slater(water1):
    assert _fd_error(*water1, "slater") < 1e-7


def test_V_is_dE_dP_pbe(water1_pbe):
    assert _fd_error(*water1_pbe, "pbe") < 1e-7


def test_V_is_dE_dP_pbe0_semilocal(water1_pbe):
    assert _fd_error(*water1_pbe, "pbe0_sl") < 1e-7


def test_pbe0_semilocal_is_linear_in_the_exchange_scale(water1_pbe):
    """E[pbe0_sl] = E[pbe] - a E_x^PBE with E_x^PBE from a separate integration of the exchange
    alone (an oracle functional made on the spot from pbe_exchange), and the same for V."""
    w, g, pl = water1_pbe
    r0 = I.integrate_method(g, w.basis, w.P, "pbe0_sl", pl)
    r1 = I.integrate_method(g, w.basis, w.P, "pbe", pl)
    F.FUNCTIONALS["_x_only"] = F.pbe_exchange
    try:
        rx = I.integrate_method(g, w.basis, w.P, "_x_only", pl)
    finally:
        del F.FUNCTIONALS["_x_only"]
    assert abs(r0.E - (r1.E - 0.25 * rx.E)) < 1e-12 * abs(r1.E)
    assert np.max(np.abs(r0.V - (r1.V - 0.25 * rx.V))) < 1e-12 * np.max(np.abs(r1.V))
    assert r0.N == r1.N


def test_planted_mistake_is_caught(water1_pbe, monkeypatch):
    # drop the factor 2 of Eq. z_mat's gradient term in the oracle: the dE/dP pin must fail
    orig = I.integrate_batch

    def wrong(pts, w, phi_args, Pj, fn):
        def fn_half(rho, sigma):
            f, vr, vs = fn(rho, sigma)
            return f, vr, 0.5 * vs
        e, n, _ = orig(pts, w, phi_args, Pj, fn)
        _, _, V = orig(pts, w, phi_args, Pj, fn_half)
        return e, n, V
    monkeypatch.setattr(I, "integrate_batch", wrong)
    assert _fd_error(*water1_pbe, "pbe") > 1e-4


def test_V_symmetric(water1_pbe):
    w, g, pl = water1_pbe
    V = I.integrate_method(g, w.basis, w.P, "pbe", pl).V
    assert np.max(np.abs(V - V.T)) <= 1e-14 * np.max(np.abs(V))


def test_definitional_equals_method_without_screening():
    w = X.make_workload("water2_pbe_small")
    spec = X.GridSpec(6, 4, 8, "ssf", 40, eta=1e-300)
    g = I.make_grid(w.mol.xyz, spec)
    pl = I.make_plan(g, w.mol.xyz, w.basis, spec)
    # at eta = 1e-300 a dropped primitive is below exp(-690) on the batch: screening error is nil
    assert sum(len(s) for s in pl.batch_shells) > 0
    D = I.integrate_definitional(g, w.basis, w.P, "pbe")
    M = I.integrate_method(g, w.basis, w.P, "pbe", pl)
    assert abs(D.E - M.E) < 1e-13 * abs(D.E)
    assert np.max(np.abs(D.V - M.V)) < 1e-13 * np.max(np.abs(D.V))


def test_screening_error_is_small(water1_pbe):
    w, g, pl = water1_pbe
    D = I.integrate_definitional(g, w.basis, w.P, "pbe")
    M = I.integrate_method(g, w.basis, w.P, "pbe", pl)
    assert abs(D.E - M.E) < 1e-9 * abs(D.E)
    assert np.max(np.abs(D.V - M.V)) < 1e-8


def test_batch_order_invariance(water1_pbe):
    w, g, pl = water1_pbe
    a = I.integrate_method(g, w.basis, w.P, "pbe", pl)
    perm = list(np.random.default_rng(0).permutation(len(pl.batch_points)))
    b = I.integrate_method(g, w.basis, w.P, "pbe", pl, batches=perm)
    assert abs(a.E - b.E) < 1e-13 * abs(a.E)
    assert np.max(np.abs(a.V - b.V)) < 1e-13 * np.max(np.abs(a.V))
    assert np.allclose(a.E_batch, b.E_batch, rtol=0, atol=0)


def test_pure_basis_V_is_dE_dP_and_traces():
    w, g, pl = _setup("water2_pbe_small_sph")
    assert w.basis.nbf == 48
    assert _fd_error(w, g, pl, "pbe") < 1e-7
    r = I.integrate_method(g, w.basis, w.P, "pbe", pl)
    # the 20-point radial grid of this case integrates rho to 0.7% (as for the Cartesian basis)
    assert abs(r.N - np.trace(w.P @ w.S)) < 1e-2 * r.N


def test_pure_basis_definitional_equals_method():
    w = X.make_workload("water2_pbe_small_sph")
    spec = X.GridSpec(6, 4, 8, "ssf", 40, eta=1e-300)
    g = I.make_grid(w.mol.xyz, spec)
    pl = I.make_plan(g, w.mol.xyz, w.basis, spec)
    D = I.integrate_definitional(g, w.basis, w.P, "pbe")
    M = I.integrate_method(g, w.basis, w.P, "pbe", pl)
    assert abs(D.E - M.E) < 1e-13 * abs(D.E)
    assert np.max(np.abs(D.V - M.V)) < 1e-13 * np.max(np.abs(D.V))


# ---------------------------------------------------------------- spin-unrestricted
def _spin_densities(w, na, nb, seed):
    # P_s = C_s C_s^T with C_s^T S C_s = I (na alpha, nb beta orbitals, separately seeded):
    # positive semidefinite, so rho_a, rho_b >= 0 everywhere
    return 0.5 * X.density_matrix(w.S, na, seed), 0.5 * X.density_matrix(w.S, nb, seed + 1)


@pytest.mark.parametrize("functional", ["slater", "pbe", "pbe0_sl"])
def test_uks_equal_spins_reduce_to_rks(water1_pbe, functional):
    w, g, pl = water1_pbe
    r = I.integrate_method(g, w.basis, w.P, functional, pl)
    u = I.integrate_method_uks(g, w.basis, 0.5 * w.P, 0.5 * w.P, functional, pl)
    assert abs(u.E - r.E) < 1e-12 * abs(r.E) and abs(u.N - r.N) < 1e-12 * r.N
    assert np.max(np.abs(u.Va - r.V)) < 1e-11 * np.max(np.abs(r.V))
    assert np.max(np.abs(u.Vb - r.V)) < 1e-11 * np.max(np.abs(r.V))


@pytest.mark.parametrize("functional", ["slater", "pbe"])
def test_uks_V_is_dE_dP_per_spin(water1_pbe, functional):
    w, g, pl = water1_pbe
    Pa, Pb = _spin_densities(w, 5, 4, 500)
    u = I.integrate_method_uks(g, w.basis, Pa, Pb, functional, pl)
    rng = np.random.default_rng(6)
    d = rng.normal(size=w.P.shape)
    d = 0.5 * (d + d.T)
    h = 1e-5   # the central difference converges as h^2 (2e-7 relative at h = 1e-4, 2e-9 at 1e-5)
    for spin in (0, 1):
        Pp = [Pa.copy(), Pb.copy()]
        Pm = [Pa.copy(), Pb.copy()]
        Pp[spin] += h * d
        Pm[spin] -= h * d
        fd = (I.integrate_method_uks(g, w.basis, *Pp, functional, pl).E
              - I.integrate_method_uks(g, w.basis, *Pm, functional, pl).E) / (2 * h)
        V = u.Va if spin == 0 else u.Vb
        assert abs(fd - np.sum(V * d)) < 1e-7 * abs(fd), spin
