"""Pins for the oracle's meta-GGA (MVS exchange with the kinetic energy density tau): its
limits (uniform gas = Slater, single orbital = (1 + kappa0) Slater at s = 0), analytic
derivatives against finite differences, tau against its definition and the iso-orbital
identity tau = tau_W for one orbital, V = dE/dP by finite differences, V symmetric, and the
trace identity Tr(P V) = sum_i w (rho vrho + 2 sigma vsigma + tau vtau)."""
import math

import numpy as np
import pytest

import xcinputs as X
from oracle import collocation as C
from oracle import functionals as F
from oracle import functionals_mgga as M
from oracle import integrate as I


def _points(n=300, seed=0):
    rng = np.random.default_rng(seed)
    rho = 10 ** rng.uniform(-4, 2, n)
    sigma = rng.uniform(0, 3, n) * rho ** 2
    tw = sigma / (8 * rho)
    tau = tw + rng.uniform(0, 2, n) * M.K_T * rho ** (5 / 3)     # alpha in [0, 2]
    return rho, sigma, tau


def test_uniform_gas_and_single_orbital_limits():
    rho = 10 ** np.linspace(-3, 2, 20)
    f_slater = F.slater(rho)[0]
    tau_unif = M.K_T * rho ** (5 / 3)
    f1 = M.mvs_exchange(rho, 0 * rho, tau_unif)[0]          # alpha = 1, s = 0
    assert np.allclose(f1, f_slater, rtol=1e-14, atol=0)
    f0 = M.mvs_exchange(rho, 0 * rho, 0 * rho)[0]            # alpha = 0, s = 0
    assert np.allclose(f0, (1 + M.KAPPA0) * f_slater, rtol=1e-14, atol=0)
    assert np.all(M.mvs_exchange(np.array([1e-16]), np.array([0.0]), np.array([1.0]))[0] == 0)


def test_derivatives_match_finite_differences():
    args = list(_points())
    out = M.mvs_exchange(*args)
    for k in range(3):
        h = 1e-6 * np.maximum(np.abs(args[k]), 1e-8)
        up = [a.copy() for a in args]
        dn = [a.copy() for a in args]
        up[k] = up[k] + h
        dn[k] = dn[k] - h
        fd = (M.mvs_exchange(*up)[0] - M.mvs_exchange(*dn)[0]) / (2 * h)
        an = out[1 + k]
        tol = 1e-7 * np.abs(an) + 1e-13 * np.abs(out[0]) / h
        assert np.all(np.abs(fd - an) <= tol), k


@pytest.fixture(scope="module")
def water1():
    w = X.make_workload("water1_pbe_small")
    g = I.make_grid(w.mol.xyz, w.grid)
    pl = I.make_plan(g, w.mol.xyz, w.basis, w.grid)
    return w, g, pl


def test_tau_is_its_definition_and_tau_W_for_one_orbital(water1):
    w, g, pl = water1
    j = max(range(len(pl.batch_points)), key=lambda k: len(pl.batch_funcs[k]))
    idx, Fj = pl.batch_points[j], pl.batch_funcs[j]
    pts = np.stack([g.x[idx], g.y[idx], g.z[idx]], 1)
    cols = C.collocate(pts, w.basis, pl.batch_shells[j])
    # definition: tau = 1/2 sum_mu,nu P grad phi_mu . grad phi_nu, written as a double loop
    Pj = w.P[np.ix_(Fj, Fj)]
    _, _, _, (rho, sigma, tau) = I.integrate_batch_mgga(pts, g.w[idx], cols, Pj, M.mvs_exchange, True)
    phi, gx, gy, gz = cols
    ref = np.zeros(len(idx))
    for a in range(len(Fj)):
        for b in range(len(Fj)):
            ref += 0.5 * Pj[a, b] * (gx[:, a] * gx[:, b] + gy[:, a] * gy[:, b] + gz[:, a] * gz[:, b])
    assert np.allclose(tau, ref, rtol=1e-12, atol=1e-300)
    # one orbital c (occupation 1): rho = psi^2, tau = |grad psi|^2 / 2 = tau_W, alpha = 0
    c = np.random.default_rng(3).normal(size=len(Fj))
    P1 = np.outer(c, c)
    _, _, _, (r1, s1, t1) = I.integrate_batch_mgga(pts, g.w[idx], cols, P1, M.mvs_exchange, True)
    ok = r1 > 1e-8 * r1.max()
    assert np.allclose(t1[ok], s1[ok] / (8 * r1[ok]), rtol=1e-9)


def test_V_is_dE_dP(water1):
    w, g, pl = water1
    rng = np.random.default_rng(4)
    d = rng.normal(size=w.P.shape)
    d = 0.5 * (d + d.T)
    h = 1e-5
    r = I.integrate_method_mgga(g, w.basis, w.P, "mvs_x", pl)
    Ep = I.integrate_method_mgga(g, w.basis, w.P + h * d, "mvs_x", pl).E
    Em = I.integrate_method_mgga(g, w.basis, w.P - h * d, "mvs_x", pl).E
    fd = (Ep - Em) / (2 * h)
    assert abs(fd - np.sum(r.V * d)) < 1e-7 * abs(fd)
    assert np.array_equal(r.V, r.V.T)


def test_trace_identity(water1):
    w, g, pl = water1
    r = I.integrate_method_mgga(g, w.basis, w.P, "mvs_x", pl)
    tot = 0.0
    for j in range(len(pl.batch_points)):
        idx, Fj = pl.batch_points[j], pl.batch_funcs[j]
        if len(Fj) == 0:
            continue
        pts = np.stack([g.x[idx], g.y[idx], g.z[idx]], 1)
        cols = C.collocate(pts, w.basis, pl.batch_shells[j])
        _, _, _, (rho, sigma, tau) = I.integrate_batch_mgga(pts, g.w[idx], cols, w.P[np.ix_(Fj, Fj)],
                                                            M.mvs_exchange, True)
        f, vr, vs, vt = M.mvs_exchange(rho, sigma, tau)
        tot += np.sum(g.w[idx] * (rho * vr + 2 * sigma * vs + tau * vt))
    assert abs(np.sum(w.P * r.V) - tot) < 1e-11 * abs(tot)
    assert math.isfinite(r.E) and r.E < 0
