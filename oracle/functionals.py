"""Spin-restricted LDA/GGA functionals with analytic first derivatives.

The paper writes E_xc = int eps(rho, gamma) rho d^3r (Eq. exc_vvar) and Z with
derivatives of eps (Eqs. zvec_r, z_mat).  Z reproduces V = dE/dP only when the
derivatives are taken of the energy per volume f = rho*eps with respect to rho
and sigma = grad(rho).grad(rho); that reading is used throughout:

    vrho = df/drho,  vsigma = df/dsigma,
    Z_mu = 0.5 * w * vrho * phi_mu + 2 * w * vsigma * grad(rho).grad(phi_mu).

Every function returns (f, vrho, vsigma) as float64 arrays.  Points with
rho < RHO_MIN contribute nothing (f = vrho = vsigma = 0).

Slater exchange:   f = C_x rho^(4/3),  C_x = -(3/4)(3/pi)^(1/3).
PBE exchange:      f = C_x rho^(4/3) F_x(s^2),  F_x = 1 + kappa - kappa/(1 + mu s^2/kappa),
                   s^2 = sigma / (4 (3 pi^2)^(2/3) rho^(8/3)).
PBE correlation:   f = rho (eps_c^PW92(r_s) + H(r_s, t^2)),  r_s = (3/(4 pi rho))^(1/3),
                   t^2 = pi sigma / (16 (3 pi^2)^(1/3) rho^(7/3)),
                   H = gamma ln(1 + (beta/gamma) t^2 (1 + A t^2)/(1 + A t^2 + A^2 t^4)),
                   A = (beta/gamma) / (exp(-eps_c/gamma) - 1).
PW92 (unpolarised): eps_c = -2 a (1 + a1 r_s) ln(1 + 1/(2 a Q)),
                   Q = b1 r_s^(1/2) + b2 r_s + b3 r_s^(3/2) + b4 r_s^2,
                   a = 0.031091, a1 = 0.21370, b1..b4 = 7.5957, 3.5876, 1.6382, 0.49294.
PBE parameters:    kappa = 0.804, beta = 0.06672455060314922, mu = beta pi^2 / 3,
                   gamma = (1 - ln 2)/pi^2.
"""
from __future__ import annotations

import math

import numpy as np

RHO_MIN = 1e-15

C_X = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0)
KAPPA = 0.804
BETA = 0.06672455060314922
MU = BETA * math.pi ** 2 / 3.0
GAMMA = (1.0 - math.log(2.0)) / math.pi ** 2
PW_A, PW_A1 = 0.031091, 0.21370
PW_B = (7.5957, 3.5876, 1.6382, 0.49294)


def _mask(rho):
    return rho >= RHO_MIN


def slater(rho, sigma=None):
    ok = _mask(rho)
    r = np.where(ok, rho, 1.0)
    r13 = np.cbrt(r)
    f = C_X * r * r13
    vr = (4.0 / 3.0) * C_X * r13
    z = np.zeros_like(rho)
    return np.where(ok, f, 0.0), np.where(ok, vr, 0.0), z


def pbe_exchange(rho, sigma):
    ok = _mask(rho)
    r = np.where(ok, rho, 1.0)
    s = np.where(ok, sigma, 0.0)
    r13 = np.cbrt(r)
    r43 = r * r13
    r83 = r43 * r43
    ds2_dsigma = 1.0 / (4.0 * (3.0 * math.pi ** 2) ** (2.0 / 3.0) * r83)
    s2 = s * ds2_dsigma
    den = 1.0 + MU * s2 / KAPPA
    Fx = 1.0 + KAPPA - KAPPA / den
    dFx = MU / (den * den)                      # dF_x / d(s^2)
    f = C_X * r43 * Fx
    vrho = (4.0 / 3.0) * C_X * r13 * Fx + C_X * r43 * dFx * (-8.0 / 3.0) * s2 / r
    vsig = C_X * r43 * dFx * ds2_dsigma
    return np.where(ok, f, 0.0), np.where(ok, vrho, 0.0), np.where(ok, vsig, 0.0)


def pw92(rs):
    """eps_c(r_s) and d eps_c / d r_s of PW92, unpolarised."""
    b1, b2, b3, b4 = PW_B
    srs = np.sqrt(rs)
    Q = b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs
    dQ = 0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs
    lg = np.log1p(1.0 / (2.0 * PW_A * Q))
    eps = -2.0 * PW_A * (1.0 + PW_A1 * rs) * lg
    deps = -2.0 * PW_A * PW_A1 * lg + 2.0 * PW_A * (1.0 + PW_A1 * rs) * dQ / (Q * (2.0 * PW_A * Q + 1.0))
    return eps, deps


def pbe_correlation(rho, sigma):
    ok = _mask(rho)
    r = np.where(ok, rho, 1.0)
    s = np.where(ok, sigma, 0.0)
    rs = np.cbrt(3.0 / (4.0 * math.pi * r))
    eps, deps_drs = pw92(rs)
    deps_drho = deps_drs * (-rs / (3.0 * r))
    E = np.exp(-eps / GAMMA)
    A = (BETA / GAMMA) / (E - 1.0)
    dA_deps = A * A * E / BETA
    r13 = np.cbrt(r)
    du_dsigma = math.pi / (16.0 * (3.0 * math.pi ** 2) ** (1.0 / 3.0) * r * r * r13)
    u = s * du_dsigma                          # t^2
    num = u + A * u * u
    den = 1.0 + A * u + A * A * u * u
    Y = num / den
    dY_du = ((1.0 + 2.0 * A * u) * den - num * (A + 2.0 * A * A * u)) / (den * den)
    dY_dA = (u * u * den - num * (u + 2.0 * A * u * u)) / (den * den)
    H = GAMMA * np.log1p((BETA / GAMMA) * Y)
    dH_dY = BETA / (1.0 + (BETA / GAMMA) * Y)
    du_drho = -(7.0 / 3.0) * u / r
    dH_drho = dH_dY * (dY_du * du_drho + dY_dA * dA_deps * deps_drho)
    f = r * (eps + H)
    vrho = eps + H + r * (deps_drho + dH_drho)
    vsig = r * dH_dY * dY_du * du_dsigma
    return np.where(ok, f, 0.0), np.where(ok, vrho, 0.0), np.where(ok, vsig, 0.0)


def pbe(rho, sigma):
    fx, vx, sx = pbe_exchange(rho, sigma)
    fc, vc, sc = pbe_correlation(rho, sigma)
    return fx + fc, vx + vc, sx + sc


def pw92_lda(rho):
    """PW92 correlation energy per volume and its rho derivative (PBE with sigma = 0 minus Slater)."""
    ok = _mask(rho)
    r = np.where(ok, rho, 1.0)
    rs = np.cbrt(3.0 / (4.0 * math.pi * r))
    eps, deps = pw92(rs)
    f = r * eps
    v = eps + r * deps * (-rs / (3.0 * r))
    return np.where(ok, f, 0.0), np.where(ok, v, 0.0)


PBE0_A = 0.25      # exact-exchange fraction of PBE0


def pbe0_semilocal(rho, sigma):
    """The grid part of the PBE0 hybrid: (1 - a) PBE exchange + PBE correlation, a = 1/4 (the
    paper names hybrids among the functionals its method serves, Sec. 2.1; the a E_x^HF term is
    a four-centre integral, not a quadrature over the grid)."""
    fx, vx, sx = pbe_exchange(rho, sigma)
    fc, vc, sc = pbe_correlation(rho, sigma)
    k = 1.0 - PBE0_A
    return k * fx + fc, k * vx + vc, k * sx + sc


FUNCTIONALS = {"slater": slater, "pbe": pbe, "pbe0_sl": pbe0_semilocal}
