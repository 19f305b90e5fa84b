"""Atomic partition functions p_A(r) (Sec. 2.2, Eq. atomic_partition, Eq. num_int).

The paper names Becke's scheme and uses Stratmann-Scuseria-Frisch (SSF) without
printing either formula.  Readings used here:

Becke (1988), no atomic-size adjustment:
    mu_AB = (|r - R_A| - |r - R_B|) / R_AB,  p(x) = 1.5 x - 0.5 x^3,
    s(mu) = 0.5 (1 - p(p(p(mu)))),  P_A(r) = prod_{B != A} s(mu_AB),
    p_A(r) = P_A(r) / sum_B P_B(r).

SSF (1996):
    g(mu) = (35 z - 35 z^3 + 21 z^5 - 5 z^7) / 16 with z = mu / a, a = 0.64,
    g = -1 for mu <= -a and g = +1 for mu >= a; s(mu) = 0.5 (1 - g(mu)),
    plus SSF's own-atom shortcut: p_A(r) = 1 when |r - R_A| < 0.5 (1 - a) R_A^nn
    (R_A^nn = distance from A to its nearest other atom).  Inside that sphere
    every s(mu_AB) is exactly 1 and every other P_B contains an s(mu_BA) = 0, so
    the shortcut does not change the value, only the cost.

The weight of point i of atom A is w_i = p_A(r_i) w_i^q (Eq. num_int).
"""
from __future__ import annotations

import numpy as np

SSF_A = 0.64


def _dist(x, y, z, R):
    dx = x - R[0]
    dy = y - R[1]
    dz = z - R[2]
    return np.sqrt(dx * dx + dy * dy + dz * dz)


def _becke_s(mu):
    f = mu
    for _ in range(3):
        f = 1.5 * f - 0.5 * f * f * f
    return 0.5 * (1.0 - f)


def _ssf_s(mu):
    z = mu / SSF_A
    z2 = z * z
    g = z * (35.0 + z2 * (-35.0 + z2 * (21.0 - 5.0 * z2))) / 16.0
    g = np.where(mu <= -SSF_A, -1.0, np.where(mu >= SSF_A, 1.0, g))
    return 0.5 * (1.0 - g)


def partition_weights(x, y, z, parent, xyz, scheme: str):
    """p_parent(r_i) for every point (float64 array, same length as x)."""
    natoms = len(xyz)
    if natoms == 1:
        return np.ones(len(x))
    s_fn = _becke_s if scheme == "becke" else _ssf_s
    Rab = np.sqrt(((xyz[:, None, :] - xyz[None, :, :]) ** 2).sum(-1))
    dist = np.stack([_dist(x, y, z, xyz[A]) for A in range(natoms)])      # (natoms, npts)
    P = np.ones((natoms, len(x)))
    for A in range(natoms):
        for B in range(natoms):
            if A == B:
                continue
            mu = (dist[A] - dist[B]) / Rab[A, B]
            P[A] *= s_fn(mu)
    num = P[parent, np.arange(len(x))]
    p = num / P.sum(axis=0)
    if scheme == "ssf":
        Rnn = np.where(np.eye(natoms, dtype=bool), np.inf, Rab).min(axis=1)
        inner = dist[parent, np.arange(len(x))] < 0.5 * (1.0 - SSF_A) * Rnn[parent]
        p = np.where(inner, 1.0, p)
    return p
