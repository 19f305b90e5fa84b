"""Pins for the oracle's atomic partition functions (Sec. 2.2, Eq. atomic_partition)."""
import numpy as np
import pytest

import xcinputs as X
from oracle import partition as PT


def _random_points(xyz, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = xyz.min(0) - 3.0, xyz.max(0) + 3.0
    p = rng.uniform(lo, hi, size=(n, 3))
    # also points very close to the nuclei, where one atom dominates
    near = xyz[rng.integers(0, len(xyz), n // 4)] + rng.normal(scale=0.05, size=(n // 4, 3))
    return np.concatenate([p, near])


@pytest.mark.parametrize("scheme", ["becke", "ssf"])
@pytest.mark.parametrize("nw", [1, 3])
def test_partition_of_unity(scheme, nw):
    mol = X.water_cluster(nw, 11 + nw)
    p = _random_points(mol.xyz, 400, 5)
    tot = np.zeros(len(p))
    for A in range(mol.natoms):
        pa = PT.partition_weights(p[:, 0], p[:, 1], p[:, 2], np.full(len(p), A), mol.xyz, scheme)
        assert np.all(pa >= 0.0) and np.all(pa <= 1.0 + 1e-15)
        tot += pa
    assert np.max(np.abs(tot - 1.0)) < 1e-14


def test_single_atom_is_one():
    mol = X.single_atom()
    p = _random_points(mol.xyz, 50, 1)
    for scheme in ("becke", "ssf"):
        assert np.all(PT.partition_weights(p[:, 0], p[:, 1], p[:, 2], np.zeros(len(p), int), mol.xyz,
                                           scheme) == 1.0)


def test_cell_functions_limits():
    # Becke: s(-1) = 1, s(0) = 1/2, s(1) = 0; SSF: s = 1 below -a, 0 above a, 1/2 at 0, continuous at +-a
    assert PT._becke_s(np.array([-1.0, 0.0, 1.0])).tolist() == [1.0, 0.5, 0.0]
    a = PT.SSF_A
    s = PT._ssf_s(np.array([-1.0, -a, 0.0, a, 1.0]))
    assert s[0] == 1.0 and s[-1] == 0.0 and s[2] == 0.5
    eps = 1e-9
    assert abs(PT._ssf_s(np.array([a - eps]))[0] - 0.0) < 1e-12
    assert abs(PT._ssf_s(np.array([-a + eps]))[0] - 1.0) < 1e-12


def test_two_atom_midplane_symmetry():
    xyz = np.array([[0.0, 0.0, -1.0], [0.0, 0.0, 1.0]])
    pts = np.array([[0.3, -0.2, 0.0], [1.0, 2.0, 0.0]])
    for scheme in ("becke", "ssf"):
        p0 = PT.partition_weights(pts[:, 0], pts[:, 1], pts[:, 2], np.array([0, 0]), xyz, scheme)
        assert np.allclose(p0, 0.5, atol=1e-15)


def test_ssf_shortcut_changes_nothing():
    # inside 0.5 (1-a) R_nn every other atom's cell function vanishes: the shortcut is exact
    mol = X.water_cluster(2, 7)
    rng = np.random.default_rng(3)
    A = 0
    Rnn = np.sort(np.linalg.norm(mol.xyz - mol.xyz[A], axis=1))[1]
    rad = 0.5 * (1 - PT.SSF_A) * Rnn * 0.999
    d = rng.normal(size=(100, 3))
    d = d / np.linalg.norm(d, axis=1)[:, None] * rad * rng.uniform(size=(100, 1))
    p = mol.xyz[A] + d
    # evaluate without the shortcut by asking for the Becke-style product with SSF cell functions
    natoms = mol.natoms
    Rab = np.linalg.norm(mol.xyz[:, None] - mol.xyz[None], axis=-1)
    dist = np.linalg.norm(p[None] - mol.xyz[:, None], axis=-1)
    P = np.ones((natoms, len(p)))
    for a in range(natoms):
        for b in range(natoms):
            if a != b:
                P[a] *= PT._ssf_s((dist[a] - dist[b]) / Rab[a, b])
    assert np.all(P[A] / P.sum(0) == 1.0)
