"""Spin-polarised Slater and PBE functionals with analytic first derivatives (the paper
restricts its account to spin-restricted GGAs and notes the spin-unrestricted extension,
Sec. 2.1; the formulas below are those of the functionals' own papers).

Every function takes rho_a, rho_b, sigma_aa, sigma_ab, sigma_bb (sigma_xy = grad rho_x .
grad rho_y) and returns (f, v_a, v_b, s_aa, s_ab, s_bb): the energy per volume and its
derivatives with respect to each argument.  Then, for the unrestricted Kohn-Sham matrices,

    V^sigma = dE/dP^sigma:   Z^sigma_mu = 0.5 w v_sigma phi_mu
                                          + w (2 s_{sigma sigma} grad rho_sigma
                                               + s_ab grad rho_{sigma'}) . grad phi_mu.

Exchange by spin scaling:   E_x[rho_a, rho_b] = (E_x[2 rho_a] + E_x[2 rho_b]) / 2, i.e.
    f = f_unpol(2 rho_a, 4 sigma_aa)/2 + f_unpol(2 rho_b, 4 sigma_bb)/2.
Correlation (PBE 1996 with PW92's spin interpolation, Perdew and Wang 1992):
    rho = rho_a + rho_b, zeta = (rho_a - rho_b)/rho, sigma = sigma_aa + 2 sigma_ab + sigma_bb,
    eps_c = e0 + alpha_c f(zeta)(1 - zeta^4)/f''(0) + (e1 - e0) f(zeta) zeta^4,
    f(zeta) = ((1+zeta)^(4/3) + (1-zeta)^(4/3) - 2)/(2^(4/3) - 2), f''(0) = 8/(9 (2^(4/3) - 2)),
    e0, e1, ac = G(r_s; A, a1, b1..b4) with
        e0: 0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294
        e1: 0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517
        ac: 0.016887, 0.11125, 10.357, 3.6231, 0.88026, 0.49671   (G gives -alpha_c,
            the spin stiffness, which is positive)
    G = -2A (1 + a1 r_s) ln(1 + 1/(2A (b1 r_s^(1/2) + b2 r_s + b3 r_s^(3/2) + b4 r_s^2))),
    H = gamma phi^3 ln(1 + (beta/gamma) t^2 (1 + A t^2)/(1 + A t^2 + A^2 t^4)),
    phi = ((1+zeta)^(2/3) + (1-zeta)^(2/3))/2, t^2 = pi sigma/(16 (3 pi^2)^(1/3) rho^(7/3) phi^2),
    A = (beta/gamma)/(exp(-eps_c/(gamma phi^3)) - 1),   f = rho (eps_c + H).
Readings (the paper is silent): a spin channel with rho_sigma < RHO_MIN/2 contributes no
exchange, the correlation is cut at rho < RHO_MIN as in the spin-restricted functionals
(so the unpolarised case reduces exactly to them), and |zeta| is clamped at 1 - 1e-10, where
phi'(zeta) diverges.
"""
from __future__ import annotations

import math

import numpy as np

from . import functionals as F

ZETA_MAX = 1.0 - 1e-10
PW_E0 = (0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294)
PW_E1 = (0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517)
PW_AC = (0.016887, 0.11125, 10.357, 3.6231, 0.88026, 0.49671)
FZ_DEN = 2.0 ** (4.0 / 3.0) - 2.0
FPP0 = 8.0 / (9.0 * FZ_DEN)
T2_SCALE = math.pi / (16.0 * (3.0 * math.pi ** 2) ** (1.0 / 3.0))


def _G(rs, prm):
    """PW92's G(r_s) and dG/dr_s."""
    A, a1, b1, b2, b3, b4 = prm
    srs = np.sqrt(rs)
    Q = b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs
    dQ = 0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs
    lg = np.log1p(1.0 / (2.0 * A * Q))
    g = -2.0 * A * (1.0 + a1 * rs) * lg
    dg = -2.0 * A * a1 * lg + 2.0 * A * (1.0 + a1 * rs) * dQ / (Q * (2.0 * A * Q + 1.0))
    return g, dg


def _exchange_spin(fn, r, s):
    """One spin channel of a spin-scaled exchange: f_unpol(2 rho_s, 4 sigma_ss)/2 and its
    derivatives with respect to rho_s and sigma_ss."""
    f, vr, vs = fn(2.0 * r, 4.0 * s)
    return 0.5 * f, vr, 2.0 * vs


def slater_pol(ra, rb, saa=None, sab=None, sbb=None):
    z = np.zeros_like(ra)
    fa, va, _ = _exchange_spin(F.slater, ra, z)
    fb, vb, _ = _exchange_spin(F.slater, rb, z)
    return fa + fb, va, vb, z, z, z


def pbe_exchange_pol(ra, rb, saa, sab, sbb):
    fa, va, sa = _exchange_spin(F.pbe_exchange, ra, saa)
    fb, vb, sb = _exchange_spin(F.pbe_exchange, rb, sbb)
    return fa + fb, va, vb, sa, np.zeros_like(ra), sb


def pbe_correlation_pol(ra, rb, saa, sab, sbb):
    rho_t = ra + rb
    ok = rho_t >= F.RHO_MIN
    rho = np.where(ok, rho_t, 1.0)
    zeta = np.clip(np.where(ok, (ra - rb) / rho, 0.0), -ZETA_MAX, ZETA_MAX)
    sig = np.where(ok, saa + 2.0 * sab + sbb, 0.0)
    rs = np.cbrt(3.0 / (4.0 * math.pi * rho))
    e0, de0 = _G(rs, PW_E0)
    e1, de1 = _G(rs, PW_E1)
    mac, dmac = _G(rs, PW_AC)                    # -alpha_c and its r_s derivative
    opz, omz = 1.0 + zeta, 1.0 - zeta
    fz = (opz ** (4.0 / 3.0) + omz ** (4.0 / 3.0) - 2.0) / FZ_DEN
    dfz = (4.0 / 3.0) * (np.cbrt(opz) - np.cbrt(omz)) / FZ_DEN
    z3, z4 = zeta ** 3, zeta ** 4
    eps = e0 - mac * fz * (1.0 - z4) / FPP0 + (e1 - e0) * fz * z4
    deps_drs = de0 - dmac * fz * (1.0 - z4) / FPP0 + (de1 - de0) * fz * z4
    deps_dz = -mac * (dfz * (1.0 - z4) - 4.0 * z3 * fz) / FPP0 + (e1 - e0) * (dfz * z4 + 4.0 * z3 * fz)
    deps_drho = deps_drs * (-rs / (3.0 * rho))
    phi = 0.5 * (opz ** (2.0 / 3.0) + omz ** (2.0 / 3.0))
    dphi = (1.0 / 3.0) * (1.0 / np.cbrt(opz) - 1.0 / np.cbrt(omz))
    phi3 = phi ** 3
    E = np.exp(-eps / (F.GAMMA * phi3))
    A = (F.BETA / F.GAMMA) / (E - 1.0)
    dA_deps = A * A * E / (F.BETA * phi3)
    dA_dphi = -3.0 * A * A * E * eps / (F.BETA * phi ** 4)
    u = sig * T2_SCALE / (rho ** (7.0 / 3.0) * phi * phi)   # t^2
    num = u + A * u * u
    den = 1.0 + A * u + A * A * u * u
    Y = num / den
    dY_du = ((1.0 + 2.0 * A * u) * den - num * (A + 2.0 * A * A * u)) / (den * den)
    dY_dA = (u * u * den - num * (u + 2.0 * A * u * u)) / (den * den)
    Lg = np.log1p((F.BETA / F.GAMMA) * Y)
    dL_dY = (F.BETA / F.GAMMA) / (1.0 + (F.BETA / F.GAMMA) * Y)
    H = F.GAMMA * phi3 * Lg
    du_drho = -(7.0 / 3.0) * u / rho
    du_dphi = -2.0 * u / phi
    dH_drho = F.GAMMA * phi3 * dL_dY * (dY_du * du_drho + dY_dA * dA_deps * deps_drho)
    dH_dz = 3.0 * F.GAMMA * phi * phi * dphi * Lg + F.GAMMA * phi3 * dL_dY * (
        dY_du * du_dphi * dphi + dY_dA * (dA_deps * deps_dz + dA_dphi * dphi))
    dH_dsig = F.GAMMA * phi3 * dL_dY * dY_du * T2_SCALE / (rho ** (7.0 / 3.0) * phi * phi)
    f = rho * (eps + H)
    df_drho = eps + H + rho * (deps_drho + dH_drho)
    df_dz = rho * (deps_dz + dH_dz)
    df_dsig = rho * dH_dsig
    va = df_drho + (1.0 - zeta) / rho * df_dz
    vb = df_drho - (1.0 + zeta) / rho * df_dz
    m = lambda v: np.where(ok, v, 0.0)       # noqa: E731
    return m(f), m(va), m(vb), m(df_dsig), m(2.0 * df_dsig), m(df_dsig)


def pbe_pol(ra, rb, saa, sab, sbb):
    x = pbe_exchange_pol(ra, rb, saa, sab, sbb)
    c = pbe_correlation_pol(ra, rb, saa, sab, sbb)
    return tuple(a + b for a, b in zip(x, c))


def pbe0_semilocal_pol(ra, rb, saa, sab, sbb):
    """(1 - a) PBE exchange + PBE correlation, a = 1/4: the grid part of PBE0."""
    x = pbe_exchange_pol(ra, rb, saa, sab, sbb)
    c = pbe_correlation_pol(ra, rb, saa, sab, sbb)
    k = 1.0 - F.PBE0_A
    return tuple(k * a + b for a, b in zip(x, c))


FUNCTIONALS_POL = {"slater": slater_pol, "pbe": pbe_pol, "pbe0_sl": pbe0_semilocal_pol}
