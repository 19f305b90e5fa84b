"""A meta-GGA: MVS exchange (Sun, Perdew and Ruzsinszky 2015), spin-restricted, with analytic
first derivatives.  The paper names meta-GGAs as a direct extension of its method (Sec. 2.1);
they add the kinetic energy density

    tau = 1/2 sum_mu,nu P_mu,nu grad(phi_mu) . grad(phi_nu)

to (rho, sigma).  ORACLE -- test infrastructure only.

    f   = C_x rho^(4/3) F_x(s^2, alpha),   C_x = -(3/4)(3/pi)^(1/3)
    s^2 = sigma / (4 (3 pi^2)^(2/3) rho^(8/3))
    alpha = (tau - tau_W) / tau_unif,  tau_W = sigma / (8 rho),
            tau_unif = (3/10) (3 pi^2)^(2/3) rho^(5/3)
    F_x = (1 + kappa0 f_a(alpha)) / (1 + b s^4)^(1/8)
    f_a = (1 - alpha) / ((1 + e1 alpha^2)^2 + c1 alpha^4)^(1/4)
    kappa0 = 0.174, e1 = -1.6665, c1 = 0.7438, b = 0.0233

Returns (f, vrho, vsigma, vtau).  With them the potential matrix is
    V_mu,nu = sum_i w_i [vrho phi_mu phi_nu + 2 vsigma grad rho . (phi_mu grad phi_nu
              + grad phi_mu phi_nu) + 1/2 vtau grad phi_mu . grad phi_nu].
Readings: points with rho < RHO_MIN contribute nothing (as for the other functionals); the
constants are the functional's own (a convention here: no reference implementation is
available to pin them, only the limits below).  Limits: alpha = 1, s = 0 gives Slater exchange
exactly (the uniform gas); alpha = 0, s = 0 gives (1 + kappa0) times Slater.
"""
from __future__ import annotations

import math

import numpy as np

from .functionals import C_X, RHO_MIN

KAPPA0 = 0.174
E1 = -1.6665
C1 = 0.7438
B = 0.0233
K_S = 1.0 / (4.0 * (3.0 * math.pi ** 2) ** (2.0 / 3.0))     # s^2 = K_S sigma rho^(-8/3)
K_T = 0.3 * (3.0 * math.pi ** 2) ** (2.0 / 3.0)             # tau_unif = K_T rho^(5/3)


def alpha_of(rho, sigma, tau):
    """The iso-orbital indicator alpha (for rho >= RHO_MIN)."""
    return (tau - sigma / (8.0 * rho)) / (K_T * rho ** (5.0 / 3.0))


def mvs_exchange(rho, sigma, tau):
    ok = rho >= RHO_MIN
    r = np.where(ok, rho, 1.0)
    sg = np.where(ok, sigma, 0.0)
    ta = np.where(ok, tau, 0.0)
    r13 = np.cbrt(r)
    r53 = r * r13 * r13
    u = K_S * sg / (r53 * r)                    # s^2 (rho^(8/3) = rho^(5/3) rho)
    al = (ta - sg / (8.0 * r)) / (K_T * r53)
    D = (1.0 + E1 * al * al) ** 2 + C1 * al ** 4
    fa = (1.0 - al) * D ** -0.25
    dD = 4.0 * E1 * al * (1.0 + E1 * al * al) + 4.0 * C1 * al ** 3
    dfa = -D ** -0.25 - 0.25 * (1.0 - al) * D ** -1.25 * dD
    g = (1.0 + B * u * u) ** -0.125
    dg = -0.25 * B * u * (1.0 + B * u * u) ** -1.125
    F = (1.0 + KAPPA0 * fa) * g
    F_u = (1.0 + KAPPA0 * fa) * dg
    F_a = KAPPA0 * dfa * g
    # derivatives of u and alpha
    u_r = -(8.0 / 3.0) * u / r
    u_s = K_S / (r53 * r)
    a_t = 1.0 / (K_T * r53)
    a_s = -1.0 / (8.0 * r) * a_t
    a_r = sg / (8.0 * r * r) * a_t - (5.0 / 3.0) * al / r
    e0 = C_X * r * r13
    f = e0 * F
    vr = (4.0 / 3.0) * C_X * r13 * F + e0 * (F_u * u_r + F_a * a_r)
    vs = e0 * (F_u * u_s + F_a * a_s)
    vt = e0 * F_a * a_t
    m = lambda v: np.where(ok, v, 0.0)       # noqa: E731
    return m(f), m(vr), m(vs), m(vt)


FUNCTIONALS_MGGA = {"mvs_x": mvs_exchange}
