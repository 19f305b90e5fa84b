"""E_xc, V_xc and N_el by numerical quadrature, in two modes.

Definitional mode (D) evaluates the integrands of Eqs. exc_vvar, vxc_exact and
zvec_r at every grid point with every basis function:

    rho_i      = sum_{mu nu} P_{mu nu} phi_mu(r_i) phi_nu(r_i)
    grad rho_i = sum_{mu nu} P_{mu nu} (grad phi_mu phi_nu + phi_mu grad phi_nu)
    E_xc = sum_i w_i f(rho_i, sigma_i),   N_el = sum_i w_i rho_i
    V_{mu nu} = sum_i w_i [vrho_i phi_mu phi_nu
                + 2 vsigma_i grad rho_i . (grad phi_mu phi_nu + phi_mu grad phi_nu)].

Method-equivalent mode (M) follows the batched formulation of Sec. 2.2, batch
by batch over the screened function list S_j of each (merged) batch:

    X^j = P^j Phi^j                                   (Eq. x_mat, GEMM)
    rho_i = sum_mu Phi_{mu i} X_{mu i}                 (Eq. eval_local_den)
    grad rho_i = 2 sum_mu grad Phi_{mu i} X_{mu i}     (Eq. eval_local_den_grad)
    eps^j_i = w_i f,  d/drho, d/dsigma likewise         (Eq. eval_xc_batch)
    E += sum_i eps^j_i                                 (Eq. exc_batch)
    Z_{mu i} = 1/2 w vrho Phi_{mu i} + 2 w vsigma grad rho_i . grad Phi_{mu i}   (Eq. z_mat)
    V^j = Z^j Phi^{jT} + Phi^j Z^{jT}                  (Eq. vxc_batch, SYR2K)
    V_xc[S_j, S_j] += V^j                              (Eq. vxc_inc)

Arrays here are point-major (row i = grid point), i.e. the transposes of the
paper's Phi_{mu i}; the sums are the same.  M differs from D only by the
screening (functions outside S_j are dropped) and by rounding order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import collocation, functionals, lebedev, partition, planner, quadrature

CHUNK = 8192


@dataclass
class Grid:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    wq: np.ndarray
    w: np.ndarray
    parent: np.ndarray


@dataclass
class Result:
    E: float
    N: float
    V: np.ndarray
    E_batch: np.ndarray | None = None
    N_batch: np.ndarray | None = None


def make_grid(xyz, spec, weights: bool = True) -> Grid:
    """Total quadrature Q with partitioned weights w_i = p_A(r_i) w^q_i (Eq. num_int)."""
    angular = None
    if getattr(spec, "angular", "product") == "lebedev":
        angular = lebedev.angular_rule(spec.ntheta)
    x, y, z, wq, par = quadrature.molecular_grid(xyz, spec.nrad, spec.ntheta, spec.nphi, spec.mk_alpha,
                                                 angular)
    w = None
    if weights:
        w = np.empty_like(wq)
        for s in range(0, len(x), 1 << 16):
            e = s + (1 << 16)
            w[s:e] = wq[s:e] * partition.partition_weights(x[s:e], y[s:e], z[s:e], par[s:e], xyz,
                                                           spec.partition)
    return Grid(x, y, z, wq, w, par)


def make_plan(grid: Grid, xyz, basis, spec) -> planner.Plan:
    return planner.make_plan(grid.x, grid.y, grid.z, grid.parent, xyz, basis, spec.max_batch, spec.eta)


def integrate_definitional(grid: Grid, basis, P, functional: str) -> Result:
    fn = functionals.FUNCTIONALS[functional]
    nbf = basis.nbf
    E = 0.0
    N = 0.0
    V = np.zeros((nbf, nbf))
    for s in range(0, len(grid.x), CHUNK):
        sl = slice(s, s + CHUNK)
        pts = np.stack([grid.x[sl], grid.y[sl], grid.z[sl]], axis=1)
        w = grid.w[sl]
        phi, gx, gy, gz = collocation.collocate(pts, basis)
        rho = np.einsum("iu,uv,iv->i", phi, P, phi)
        grad = [np.einsum("iu,uv,iv->i", g, P, phi) + np.einsum("iu,uv,iv->i", phi, P, g)
                for g in (gx, gy, gz)]
        sigma = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]
        f, vr, vs = fn(rho, sigma)
        E += float(np.sum(w * f))
        N += float(np.sum(w * rho))
        # G_{i mu} = grad rho_i . grad phi_mu(r_i)
        G = grad[0][:, None] * gx + grad[1][:, None] * gy + grad[2][:, None] * gz
        V += phi.T @ ((w * vr)[:, None] * phi)
        c = (2.0 * w * vs)[:, None]
        V += (c * G).T @ phi + phi.T @ (c * G)
    return Result(E, N, V)


def integrate_batch(pts, w, phi_args, Pj, fn):
    """One batch of the method-equivalent mode; returns (E_j, N_j, V^j)."""
    phi, gx, gy, gz = phi_args
    X = phi @ Pj                                                    # Eq. x_mat
    rho = np.sum(phi * X, axis=1)                                   # Eq. eval_local_den
    grad = [2.0 * np.sum(g * X, axis=1) for g in (gx, gy, gz)]      # Eq. eval_local_den_grad
    sigma = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]
    f, vr, vs = fn(rho, sigma)
    eps_w = w * f                                                   # Eq. eval_xc_batch
    a = 0.5 * w * vr
    b = 2.0 * w * vs
    Z = a[:, None] * phi + b[:, None] * (grad[0][:, None] * gx + grad[1][:, None] * gy
                                         + grad[2][:, None] * gz)   # Eq. z_mat
    Vj = Z.T @ phi + phi.T @ Z                                      # Eq. vxc_batch
    return float(np.sum(eps_w)), float(np.sum(w * rho)), Vj


def batch_intermediates(grid: Grid, basis, P, functional: str, plan: planner.Plan, j: int):
    """Phi, grad Phi and Z (Eqs. gau_cart, x_mat ... z_mat) of merged batch j, point-major
    (points in the plan's batch order, functions in the batch's function order)."""
    fn = functionals.FUNCTIONALS[functional]
    idx = plan.batch_points[j]
    F = plan.batch_funcs[j]
    pts = np.stack([grid.x[idx], grid.y[idx], grid.z[idx]], axis=1)
    phi, gx, gy, gz = collocation.collocate(pts, basis, plan.batch_shells[j])
    X = phi @ P[np.ix_(F, F)]
    rho = np.sum(phi * X, axis=1)
    grad = [2.0 * np.sum(g * X, axis=1) for g in (gx, gy, gz)]
    sigma = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]
    f, vr, vs = fn(rho, sigma)
    w = grid.w[idx]
    Z = (0.5 * w * vr)[:, None] * phi + (2.0 * w * vs)[:, None] * (grad[0][:, None] * gx + grad[1][:, None] * gy
                                                                 + grad[2][:, None] * gz)
    return phi, gx, gy, gz, Z


def integrate_method(grid: Grid, basis, P, functional: str, plan: planner.Plan,
                     batches=None) -> Result:
    """Method-equivalent mode over the merged batches of ``plan`` (or a subset)."""
    fn = functionals.FUNCTIONALS[functional]
    nbf = basis.nbf
    V = np.zeros((nbf, nbf))
    nb = len(plan.batch_points)
    sel = range(nb) if batches is None else batches
    Eb = np.zeros(nb)
    Nb = np.zeros(nb)
    for j in sel:
        idx = plan.batch_points[j]
        F = plan.batch_funcs[j]
        if len(F) == 0:
            continue
        Pj = P[np.ix_(F, F)]
        for s in range(0, len(idx), CHUNK):
            ii = idx[s:s + CHUNK]
            pts = np.stack([grid.x[ii], grid.y[ii], grid.z[ii]], axis=1)
            cols = collocation.collocate(pts, basis, plan.batch_shells[j])
            e, n, Vj = integrate_batch(pts, grid.w[ii], cols, Pj, fn)
            Eb[j] += e
            Nb[j] += n
            V[np.ix_(F, F)] += Vj                                   # Eq. vxc_inc
    return Result(float(np.sum(Eb)), float(np.sum(Nb)), V, Eb, Nb)


# ---------------------------------------------------------------- spin-unrestricted
@dataclass
class ResultUKS:
    E: float
    N: float
    Va: np.ndarray
    Vb: np.ndarray
    E_batch: np.ndarray | None = None
    N_batch: np.ndarray | None = None


def integrate_batch_uks(pts, w, phi_args, Paj, Pbj, fn):
    """One batch of the spin-unrestricted extension (Sec. 2.1): Eqs. x_mat, eval_local_den,
    eval_local_den_grad per spin, the polarised functional, then per spin
    Z^s = 1/2 w v_s phi + w (2 s_ss grad rho_s + s_ab grad rho_s') . grad phi and
    V^s = Z^sT phi + phi^T Z^s (Eqs. z_mat, vxc_batch)."""
    phi, gx, gy, gz = phi_args
    rho, grad = [], []
    for Pj in (Paj, Pbj):
        X = phi @ Pj
        rho.append(np.sum(phi * X, axis=1))
        grad.append([2.0 * np.sum(g * X, axis=1) for g in (gx, gy, gz)])
    dot = lambda u, v: u[0] * v[0] + u[1] * v[1] + u[2] * v[2]          # noqa: E731
    saa, sab, sbb = dot(grad[0], grad[0]), dot(grad[0], grad[1]), dot(grad[1], grad[1])
    f, va, vb, s_aa, s_ab, s_bb = fn(rho[0], rho[1], saa, sab, sbb)
    V = []
    for v, s_ss, own, other in ((va, s_aa, grad[0], grad[1]), (vb, s_bb, grad[1], grad[0])):
        c = [w * (2.0 * s_ss * own[d] + s_ab * other[d]) for d in range(3)]
        Z = (0.5 * w * v)[:, None] * phi + c[0][:, None] * gx + c[1][:, None] * gy + c[2][:, None] * gz
        V.append(Z.T @ phi + phi.T @ Z)
    return float(np.sum(w * f)), float(np.sum(w * (rho[0] + rho[1]))), V[0], V[1]


def integrate_method_uks(grid: Grid, basis, Pa, Pb, functional: str, plan: planner.Plan,
                         batches=None) -> ResultUKS:
    """Spin-unrestricted method-equivalent mode over the merged batches of ``plan``."""
    from . import functionals_pol
    fn = functionals_pol.FUNCTIONALS_POL[functional]
    nbf = basis.nbf
    Va = np.zeros((nbf, nbf))
    Vb = np.zeros((nbf, nbf))
    nb = len(plan.batch_points)
    sel = range(nb) if batches is None else batches
    Eb = np.zeros(nb)
    Nb = np.zeros(nb)
    for j in sel:
        idx = plan.batch_points[j]
        F = plan.batch_funcs[j]
        if len(F) == 0:
            continue
        Paj, Pbj = Pa[np.ix_(F, F)], Pb[np.ix_(F, F)]
        for s in range(0, len(idx), CHUNK):
            ii = idx[s:s + CHUNK]
            pts = np.stack([grid.x[ii], grid.y[ii], grid.z[ii]], axis=1)
            cols = collocation.collocate(pts, basis, plan.batch_shells[j])
            e, n, Vaj, Vbj = integrate_batch_uks(pts, grid.w[ii], cols, Paj, Pbj, fn)
            Eb[j] += e
            Nb[j] += n
            Va[np.ix_(F, F)] += Vaj
            Vb[np.ix_(F, F)] += Vbj
    return ResultUKS(float(np.sum(Eb)), float(np.sum(Nb)), Va, Vb, Eb, Nb)


# ---------------------------------------------------------------- meta-GGA
def integrate_batch_mgga(pts, w, phi_args, Pj, fn, return_tau=False):
    """One batch with a meta-GGA f(rho, sigma, tau): X as in Eq. x_mat, and per gradient
    component k the contraction Y^k = (d_k Phi) P^j, so that
    tau_i = 1/2 sum_k sum_mu d_k Phi_i,mu Y^k_i,mu; V^j gains the term
    sum_k (1/4 w vtau d_k Phi)^T d_k Phi + its transpose."""
    phi, gx, gy, gz = phi_args
    X = phi @ Pj
    rho = np.sum(phi * X, axis=1)
    grad = [2.0 * np.sum(g * X, axis=1) for g in (gx, gy, gz)]
    sigma = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]
    tau = 0.5 * sum(np.sum(g * (g @ Pj), axis=1) for g in (gx, gy, gz))
    f, vr, vs, vt = fn(rho, sigma, tau)
    a = 0.5 * w * vr
    b = 2.0 * w * vs
    Z = a[:, None] * phi + b[:, None] * (grad[0][:, None] * gx + grad[1][:, None] * gy
                                         + grad[2][:, None] * gz)
    c = 0.25 * w * vt
    W = Z.T @ phi + sum((c[:, None] * g).T @ g for g in (gx, gy, gz))
    Vj = W + W.T
    out = (float(np.sum(w * f)), float(np.sum(w * rho)), Vj)
    return out + ((rho, sigma, tau),) if return_tau else out


def integrate_method_mgga(grid: Grid, basis, P, functional: str, plan: planner.Plan,
                          batches=None) -> Result:
    """Meta-GGA method-equivalent mode over the merged batches of ``plan``."""
    from . import functionals_mgga
    fn = functionals_mgga.FUNCTIONALS_MGGA[functional]
    nbf = basis.nbf
    V = np.zeros((nbf, nbf))
    nb = len(plan.batch_points)
    sel = range(nb) if batches is None else batches
    Eb = np.zeros(nb)
    Nb = np.zeros(nb)
    for j in sel:
        idx = plan.batch_points[j]
        F = plan.batch_funcs[j]
        if len(F) == 0:
            continue
        Pj = P[np.ix_(F, F)]
        for s in range(0, len(idx), CHUNK):
            ii = idx[s:s + CHUNK]
            pts = np.stack([grid.x[ii], grid.y[ii], grid.z[ii]], axis=1)
            cols = collocation.collocate(pts, basis, plan.batch_shells[j])
            e, n, Vj = integrate_batch_mgga(pts, grid.w[ii], cols, Pj, fn)
            Eb[j] += e
            Nb[j] += n
            V[np.ix_(F, F)] += Vj
    return Result(float(np.sum(Eb)), float(np.sum(Nb)), V, Eb, Nb)
