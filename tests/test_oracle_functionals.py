"""Pins for the oracle's Slater and PBE functionals."""
import math

import numpy as np
import pytest

from oracle import functionals as F


def _grid(seed=0, n=400):
    rng = np.random.default_rng(seed)
    rho = 10.0 ** rng.uniform(-7, 2, n)
    s2 = 10.0 ** rng.uniform(-4, 1.5, n)          # reduced gradient squared
    sigma = s2 * 4 * (3 * math.pi ** 2) ** (2 / 3) * rho ** (8 / 3)
    return rho, sigma


def test_slater_constant_and_form():
    assert abs(F.C_X - (-0.7385587663820223)) < 1e-16
    rho = np.array([0.1, 1.0, 8.0])
    f, v, s = F.slater(rho)
    assert np.allclose(f, F.C_X * rho ** (4 / 3), rtol=1e-15)
    assert np.allclose(v, 4 / 3 * F.C_X * rho ** (1 / 3), rtol=1e-15)
    assert np.all(s == 0)


def test_pbe_reduces_to_slater_plus_pw92_at_zero_gradient():
    rho = 10.0 ** np.linspace(-8, 3, 50)
    f, v, s = F.pbe(rho, np.zeros_like(rho))
    fs, vs, _ = F.slater(rho)
    fc, vc = F.pw92_lda(rho)
    assert np.allclose(f, fs + fc, rtol=1e-14, atol=0)
    assert np.allclose(v, vs + vc, rtol=1e-13, atol=0)


def test_pbe_exchange_enhancement_bounds():
    rho, sigma = _grid(1)
    f, _, _ = F.pbe_exchange(rho, sigma)
    Fx = f / (F.C_X * rho ** (4 / 3))
    assert np.all(Fx >= 1.0 - 1e-14) and np.all(Fx <= 1.0 + F.KAPPA + 1e-14)
    # large-gradient limit approaches 1 + kappa (Lieb-Oxford-motivated bound of PBE)
    f, _, _ = F.pbe_exchange(np.array([1.0]), np.array([1e12]))
    assert abs(f[0] / F.C_X - (1 + F.KAPPA)) < 1e-6


def test_pw92_known_limits():
    # high-density limit: eps_c ~ 2a ln r_s + const; low density: eps_c -> 0 from below
    eps_hi, _ = F.pw92(np.array([1e-6, 2e-6]))
    slope = (eps_hi[1] - eps_hi[0]) / math.log(2.0)
    assert abs(slope - F.PW_A) < 1e-5           # eps_c -> A ln r_s + const as r_s -> 0
    eps_lo, _ = F.pw92(np.array([1e6]))
    assert -1e-5 < eps_lo[0] < 0


def test_pbe_correlation_nonpositive_and_bounded():
    rho, sigma = _grid(2)
    f, _, _ = F.pbe_correlation(rho, sigma)
    fc0, _ = F.pw92_lda(rho)
    assert np.all(f <= 1e-300)          # H >= eps_c bound keeps f_c <= 0 ...
    assert np.all(f >= fc0 - 1e-14 * np.abs(fc0))   # ... and the gradient correction is >= 0


@pytest.mark.parametrize("name", ["slater", "pbe"])
def test_derivatives_match_finite_differences(name):
    fn = F.FUNCTIONALS[name]
    rho, sigma = _grid(3)
    keep = rho > 1e-5
    rho, sigma = rho[keep], sigma[keep]
    f, vr, vs = fn(rho, sigma)
    h = 1e-6
    fr = (fn(rho * (1 + h), sigma)[0] - fn(rho * (1 - h), sigma)[0]) / (2 * h * rho)
    # scale by |f|/rho as well: vrho can cancel to ~0 between its two terms
    assert np.max(np.abs(fr - vr) / (np.abs(vr) + np.abs(f) / rho)) < 1e-8
    if name == "pbe":
        fs = (fn(rho, sigma * (1 + h))[0] - fn(rho, sigma * (1 - h))[0]) / (2 * h * sigma)
        assert np.max(np.abs(fs - vs) / (np.abs(vs) + np.abs(f) / sigma)) < 1e-8


def test_density_threshold():
    f, v, s = F.pbe(np.array([0.0, 1e-16, 1e-15]), np.array([0.0, 1e-40, 1e-40]))
    assert f[0] == 0 and v[0] == 0 and s[0] == 0 and f[1] == 0
    assert f[2] != 0
