"""Pins of the oracle's functional constants and partition cells against facts outside the
oracle's own formulas: closed forms, design conditions of the functionals, and the hydrogen
atom, whose exact density and exact exchange energy are known in closed form.

The paper takes the functionals from a library (Sec. 2.1, Sec. 3) and the partition from
Becke and from Stratmann, Scuseria and Frisch (Sec. 2.2).  A plausible mistake in the oracle
(a wrong prefactor in the reduced gradient s or in t, a wrong mu, kappa0 or b, a dropped
factor in PW92's logarithm, two Becke iterations instead of three) fails one of these."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import functionals as F
from oracle import functionals_mgga as M
from oracle import functionals_pol as FP
from oracle import partition as PT


def _hydrogen():
    """Radial quadrature (Gauss-Legendre in x, r = -2 ln(1 - x^3)) of the exact hydrogen 1s
    density rho = exp(-2r)/pi, its gradient norm |rho'| = 2 rho and tau_W = |rho'|^2/(8 rho)."""
    x, wx = np.polynomial.legendre.leggauss(400)
    x, wx = 0.5 * (x + 1.0), 0.5 * wx
    r = -2.0 * np.log(1.0 - x ** 3)
    w = 4.0 * math.pi * r * r * (6.0 * x * x / (1.0 - x ** 3)) * wx
    rho = np.exp(-2.0 * r) / math.pi
    sigma = (2.0 * rho) ** 2
    return w, rho, sigma, sigma / (8.0 * rho)


def test_hydrogen_density_is_normalised():
    w, rho, _, _ = _hydrogen()
    assert abs(np.sum(w * rho) - 1.0) < 1e-12


def test_reduced_gradient_from_its_definition():
    """s = |grad rho| / (2 k_F rho), k_F = (3 pi^2 rho)^(1/3); the oracle's PBE F_x, inverted
    for s^2 with F_x = 1 + kappa - kappa/(1 + mu s^2/kappa), must give that s^2."""
    rng = np.random.default_rng(7)
    rho = 10.0 ** rng.uniform(-4, 2, 200)
    g = rho ** (4.0 / 3.0) * 10.0 ** rng.uniform(-2, 0.5, 200)      # |grad rho|
    kF = (3.0 * math.pi ** 2 * rho) ** (1.0 / 3.0)
    s2_def = (g / (2.0 * kF * rho)) ** 2
    f, _, _ = F.pbe_exchange(rho, g * g)
    Fx = f / (F.C_X * rho ** (4.0 / 3.0))
    mu = 0.06672455060314922 * math.pi ** 2 / 3.0
    s2 = (0.804 / mu) * (0.804 / (1.0 + 0.804 - Fx) - 1.0)
    assert np.max(np.abs(s2 / s2_def - 1.0)) < 1e-9


def test_pbe_gradient_terms_cancel_in_the_slowly_varying_limit():
    """PBE's design condition: for a slowly varying density the second-order gradient terms of
    exchange (mu s^2) and correlation (beta t^2) cancel, so d(f_x + f_c)/d sigma = 0 at
    sigma = 0 for every density.  It ties mu to beta (mu = beta pi^2 / 3) and the
    normalisations of s and t to each other."""
    rho = 10.0 ** np.linspace(-6, 3, 40)
    z = np.zeros_like(rho)
    _, _, vx = F.pbe_exchange(rho, z)
    _, _, vc = F.pbe_correlation(rho, z)
    assert np.all(vx < 0) and np.all(vc > 0)
    assert np.max(np.abs(vx + vc) / np.abs(vx)) < 1e-12


def test_pbe_correlation_vanishes_for_rapidly_varying_density():
    """PBE's H cancels the LDA correlation as t -> infinity (f_c -> 0)."""
    rho = np.array([1e-3, 1e-1, 1.0, 10.0])
    fc, _, _ = F.pbe_correlation(rho, 1e16 * rho ** (7.0 / 3.0))
    f0, _ = F.pw92_lda(rho)
    assert np.max(np.abs(fc / f0)) < 1e-6


def test_pw92_high_density_coefficient_is_gell_mann_brueckner():
    """eps_c -> A ln r_s + const as r_s -> 0 with the RPA coefficient A = (1 - ln 2)/pi^2
    (Gell-Mann and Brueckner); PW92 prints A to five digits."""
    A = (1.0 - math.log(2.0)) / math.pi ** 2
    assert abs(F.PW_A - A) < 5e-7
    eps, _ = F.pw92(np.array([1e-8, 2e-8]))
    assert abs((eps[1] - eps[0]) / math.log(2.0) - A) < 2e-5


def test_hydrogen_exchange_lsd_closed_form():
    """Fully polarised Slater exchange of the hydrogen 1s density in closed form:
    E_x = -(3/4)(6/pi)^(1/3) int rho^(4/3) = -(81/256) 6^(1/3) pi^(-2/3), through the
    oracle's spin scaling E_x[rho_a, 0] = E_x[2 rho_a] / 2."""
    w, rho, _, _ = _hydrogen()
    exact = -(81.0 / 256.0) * 6.0 ** (1.0 / 3.0) * math.pi ** (-2.0 / 3.0)
    f = FP.slater_pol(rho, np.zeros_like(rho))[0]
    assert abs(np.sum(w * f) - exact) < 1e-10


def test_hydrogen_pbe_exchange_and_correlation():
    """PBE on the hydrogen atom: exchange within 0.01 Eh of the exact -5/16 (the exact value
    is the self-interaction of the 1s orbital), and the values PBE 1996 tabulates for H to three
    decimals (exchange -0.306, correlation -0.006, against LSD's -0.268 and -0.022)."""
    w, rho, sigma, _ = _hydrogen()
    z = np.zeros_like(rho)
    ex = np.sum(w * FP.pbe_exchange_pol(rho, z, sigma, z, z)[0])
    ec = np.sum(w * FP.pbe_correlation_pol(rho, z, sigma, z, z)[0])
    ec_lsd = np.sum(w * FP.pbe_correlation_pol(rho, z, z, z, z)[0])
    assert abs(ex - (-5.0 / 16.0)) < 0.01
    assert round(ex, 3) == -0.306 and round(ec, 3) == -0.006 and round(ec_lsd, 3) == -0.022


def test_mvs_reproduces_hydrogen_exact_exchange():
    """MVS is built to give the exact exchange energy -5/16 Eh of the hydrogen atom (alpha = 0
    there: tau = tau_W for one orbital), which pins kappa0, b and the normalisation of s."""
    w, rho, sigma, tauW = _hydrogen()
    f, _, _, _ = M.mvs_exchange(2.0 * rho, 4.0 * sigma, 2.0 * tauW)
    ex = 0.5 * np.sum(w * f)
    assert abs(ex - (-5.0 / 16.0)) < 5e-6


def test_becke_cell_function_has_three_iterations():
    """Becke 1988 iterates p(x) = 3x/2 - x^3/2 three times: s(1/2) in exact rational arithmetic."""
    def p(x):
        return Fraction(3, 2) * x - Fraction(1, 2) * x ** 3

    def s(k):
        x = Fraction(1, 2)
        for _ in range(k):
            x = p(x)
        return float(Fraction(1, 2) * (1 - x))

    assert abs(s(3) - 0.012350184590559365) < 1e-17
    assert abs(s(2) - 0.012350184590559365) > 0.05
    assert abs(PT._becke_s(np.array([0.5]))[0] - s(3)) < 1e-16


@pytest.mark.parametrize("prm,A,c1", [
    (FP.PW_E0, (1.0 - math.log(2.0)) / math.pi ** 2, 0.046644),
    (FP.PW_E1, (1.0 - math.log(2.0)) / (2.0 * math.pi ** 2), 0.025599),
    (FP.PW_AC, 1.0 / (6.0 * math.pi ** 2), 0.035475)])
def test_pw92_high_density_expansion_of_every_parameter_set(prm, A, c1):
    """PW92 builds beta_1 and beta_2 of each of its three sets (unpolarised, fully polarised,
    spin stiffness -alpha_c) from the high-density expansion G(r_s) = A ln r_s - c1 + O(r_s ln r_s):
    A is the random-phase coefficient ((1 - ln 2)/pi^2, half of it for the fully polarised gas,
    1/(6 pi^2) for the stiffness), c1 the constant of the same expansion that PW92 takes from the
    electron-gas literature (0.046644, 0.025599, 0.035475), and the expansion has no r_s^(1/2)
    term, i.e. beta_2 = 2 A beta_1^2.  A beta_1 off by 0.5% moves the constant by 3e-4; a beta_2
    off by 1% gives an r_s^(1/2) coefficient above 1e-4."""
    assert abs(prm[0] - A) < 5e-7
    rs = np.array([1e-16, 1e-14])
    D = FP._G(rs, prm)[0] - prm[0] * np.log(rs)   # -c1 + a r_s^(1/2) + ...
    assert abs(-D[0] - c1) < 3e-6
    a_half = (D[1] - D[0]) / (np.sqrt(rs[1]) - np.sqrt(rs[0]))
    assert abs(a_half) < 5e-6


def test_pbe_correlation_gradient_coefficient_is_ma_brueckner():
    """For a slowly varying density PBE's correlation gradient term is n beta t^2, the
    second-order gradient expansion of the high-density gas: beta = nu C_c(0) with
    nu = (16/pi)(3 pi^2)^(1/3) and Ma and Brueckner's coefficient C_c(0) = 0.004235 (the
    relation and value PW91 and PBE use; four digits, so 1e-4 relative).  t is built here from
    its definition, t = |grad n| / (2 k_s n), k_s = (4 k_F / pi)^(1/2), k_F = (3 pi^2 n)^(1/3)."""
    beta_mb = 16.0 / math.pi * (3.0 * math.pi ** 2) ** (1.0 / 3.0) * 0.004235
    n = np.array([0.05, 0.5, 5.0])
    kf = (3.0 * math.pi ** 2 * n) ** (1.0 / 3.0)
    ks = np.sqrt(4.0 * kf / math.pi)
    t2 = 1e-8
    sigma = t2 * (2.0 * ks * n) ** 2
    f1, _, _ = F.pbe_correlation(n, sigma)
    f0, _, _ = F.pbe_correlation(n, np.zeros_like(n))
    beta_eff = (f1 - f0) / (n * t2)
    assert np.max(np.abs(beta_eff / beta_mb - 1.0)) < 1e-4
