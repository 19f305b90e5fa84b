"""Checks of the seeded input generators (geometry rules, basis rules, overlap, density)."""
import numpy as np

import xcinputs as X
from oracle import collocation as C
from oracle import quadrature as Q


def test_water_geometry_and_cluster_rules():
    m = X.water_cluster(16, 2000)
    assert m.natoms == 48 and list(m.Z[:3]) == [8, 1, 1]
    O = m.xyz[0::3] / X.ANGSTROM_TO_BOHR
    d = np.linalg.norm(O[:, None] - O[None], axis=-1) + np.eye(16) * 99
    assert d.min() >= 2.6
    assert O.min() >= 0 and O.max() <= 10.0
    for k in range(16):
        oh = np.linalg.norm(m.xyz[3 * k + 1:3 * k + 3] - m.xyz[3 * k], axis=1) / X.ANGSTROM_TO_BOHR
        assert np.allclose(oh, np.hypot(0.757, 0.587), rtol=1e-12)
    assert np.array_equal(m.xyz, X.water_cluster(16, 2000).xyz)     # seeded


def test_basis_rules():
    w = X.make_workload("water1_slater")
    b = w.basis
    assert b.nbf == 25 and b.nshell == 12
    assert list(b.L) == [0, 0, 0, 1, 1, 2, 0, 0, 1, 0, 0, 1]
    assert np.allclose(b.alpha[5], [1e3, 10.0, 0.1])            # single d shell
    assert np.allclose(b.alpha[0, 0], 1e3) and np.allclose(b.alpha[2, 2], 0.1)


def test_overlap_against_brute_force_quadrature():
    # S from the closed form against a molecular product quadrature of phi_mu phi_nu
    w = X.make_workload("water1_slater")
    # one fine grid centred at the molecular centroid (no partition needed)
    x, y, z, wq = Q.atom_grid(w.mol.xyz.mean(0), 300, 24, 48, 2.0)
    phi = C.collocate(np.stack([x, y, z], 1), w.basis)[0]
    S_quad = phi.T @ (wq[:, None] * phi)
    # only functions smooth enough for an off-centre grid: drop the two tightest shells per atom
    tight = w.basis.alpha.max(1) > 20
    keep = np.concatenate([np.full(X.ncart(int(w.basis.L[s])), not tight[s]) for s in range(w.basis.nshell)])
    err = np.abs(S_quad - w.S)[np.ix_(keep, keep)].max()
    assert err < 1e-6


def test_overlap_on_centre_exact():
    # for a single atom the atom-centred grid integrates every product accurately
    mol = X.single_atom(8)
    b = X.make_basis(mol)
    S = X.overlap_matrix(b)
    x, y, z, wq = Q.atom_grid(np.zeros(3), 600, 16, 32, 5.0)
    phi = C.collocate(np.stack([x, y, z], 1), b)[0]
    assert np.abs(phi.T @ (wq[:, None] * phi) - S).max() < 1e-9
    # x^L components have unit norm by the basis rule
    for s in range(b.nshell):
        assert abs(S[b.func_offset[s], b.func_offset[s]] - 1.0) < 1e-13


def test_density_matrix_properties():
    w = X.make_workload("water2_pbe_small")
    assert np.array_equal(w.P, w.P.T)
    assert abs(np.trace(w.P @ w.S) - 20.0) < 1e-11
    ev = np.linalg.eigvalsh(w.S @ w.P @ w.S)
    assert ev.min() > -1e-10
