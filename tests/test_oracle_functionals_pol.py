"""Pins for the oracle's spin-polarised functionals (spin-unrestricted extension, Sec. 2.1):
reduction to the spin-restricted functionals at zeta = 0, analytic derivatives against
finite differences, the fully polarised limit of PW92 and the sign of its spin stiffness."""
import numpy as np
import pytest

from oracle import functionals as F
from oracle import functionals_pol as FP


def _points(n=200, seed=0):
    rng = np.random.default_rng(seed)
    rho = 10 ** rng.uniform(-4, 2, n)
    zeta = rng.uniform(-0.9, 0.9, n)
    ra, rb = 0.5 * rho * (1 + zeta), 0.5 * rho * (1 - zeta)
    ga = rng.normal(size=(n, 3)) * ra[:, None] * rng.uniform(0.1, 3, (n, 1))
    gb = rng.normal(size=(n, 3)) * rb[:, None] * rng.uniform(0.1, 3, (n, 1))
    return ra, rb, np.sum(ga * ga, 1), np.sum(ga * gb, 1), np.sum(gb * gb, 1)


@pytest.mark.parametrize("name", ["slater", "pbe"])
def test_unpolarised_limit(name):
    rng = np.random.default_rng(1)
    rho = 10 ** rng.uniform(-4, 2, 100)
    sigma = rng.uniform(0, 3, 100) * rho ** 2
    f, vr, vs = F.FUNCTIONALS[name](rho, sigma)
    q = 0.25 * sigma
    fp, va, vb, saa, sab, sbb = FP.FUNCTIONALS_POL[name](0.5 * rho, 0.5 * rho, q, q, q)
    assert np.allclose(fp, f, rtol=1e-13, atol=0)
    assert np.allclose(va, vr, rtol=1e-12, atol=1e-300) and np.allclose(vb, vr, rtol=1e-12, atol=1e-300)
    if name == "pbe":
        # Z^sigma's gradient coefficient (2 s_aa grad rho_a + s_ab grad rho_b with grad rho_a =
        # grad rho_b = grad rho / 2) reduces to the spin-restricted 2 vsigma grad rho
        assert np.allclose(saa, sbb, rtol=1e-14)
        assert np.allclose(saa + 0.5 * sab, 2 * vs, rtol=1e-12)


@pytest.mark.parametrize("name", ["slater", "pbe"])
def test_derivatives_match_finite_differences(name):
    args = list(_points())
    fn = FP.FUNCTIONALS_POL[name]
    out = fn(*args)
    for k in range(5):
        if name == "slater" and k >= 2:
            continue
        h = 1e-6 * np.maximum(np.abs(args[k]), 1e-8)
        up = [a.copy() for a in args]
        dn = [a.copy() for a in args]
        up[k] = up[k] + h
        dn[k] = dn[k] - h
        fd = (fn(*up)[0] - fn(*dn)[0]) / (2 * h)
        an = out[1 + k]
        # central differences carry O(h^2) truncation and |f| eps / h cancellation error
        tol = 1e-7 * np.abs(an) + 1e-13 * np.abs(out[0]) / h
        assert np.all(np.abs(fd - an) <= tol), k


def test_pw92_spin_interpolation():
    rs = np.array([0.5, 1.0, 2.0, 5.0])
    rho = 3.0 / (4.0 * np.pi * rs ** 3)
    e0, _ = FP._G(rs, FP.PW_E0)
    e1, _ = FP._G(rs, FP.PW_E1)
    mac, _ = FP._G(rs, FP.PW_AC)
    z = np.zeros_like(rho)

    def eps(zeta):
        f = FP.pbe_correlation_pol(0.5 * rho * (1 + zeta), 0.5 * rho * (1 - zeta), z, z, z)[0]
        return f / rho
    # fully polarised limit (H = 0 at sigma = 0): eps_c -> e1
    assert np.allclose(eps(1.0), e1, rtol=1e-8)
    assert np.allclose(eps(0.0), e0, rtol=1e-14)
    # spin stiffness: d^2 eps / d zeta^2 at 0 equals alpha_c = -G_ac > 0
    h = 1e-3
    stiff = (eps(h) - 2 * eps(0.0) + eps(-h)) / h ** 2
    assert np.all(-mac > 0)
    assert np.allclose(stiff, -mac, rtol=1e-5)
