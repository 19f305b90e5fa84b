"""Spin-unrestricted form (the extension of Sec. 2.1) through the C-ABI against the oracle:
|dE| <= 1e-9 Eh, max |dV^s_ij| <= 1e-9 per spin (float64 form), and the spin-restricted result
recovered exactly enough (1e-12 relative) when P^a = P^b = P/2.  The tensor-core (mixed) form
takes the mixed form's small-case bounds: |dE| <= 1e-7 Eh, |dN| <= 1e-8, max |dV^s| <= 1e-7,
and at full size |dE| <= 1e-6 Eh against its float64 form."""
import numpy as np
import pytest

import xcinputs as X
from oracle import integrate as I

from gpu_common import Loaded

pytestmark = pytest.mark.gpu


def _spins(w, na, nb, seed):
    return 0.5 * X.density_matrix(w.S, na, seed), 0.5 * X.density_matrix(w.S, nb, seed + 1)


@pytest.fixture(scope="module", params=["water1_slater", "water1_pbe_small", "water2_pbe_small",
                                        "water2_pbe_small_sph", "water2_pbe_small_leb"])
def loaded(request):
    L = Loaded(request.param)
    yield L
    L.close()


def _uks(L, Pa, Pb, functional, precision="fp64"):
    nbf = L.w.basis.nbf
    Va, Vb = np.zeros((nbf, nbf)), np.zeros((nbf, nbf))
    E, N = L.G.gbxc_integrate_uks(L.ctx.h, L.mid, Pa, Pb, functional, precision, Va, Vb)
    return E, N, Va, Vb


@pytest.mark.parametrize("functional", ["slater", "pbe", "pbe0_sl"])
def test_uks_matches_oracle(loaded, functional):
    nw = loaded.w.mol.n_waters
    Pa, Pb = _spins(loaded.w, 5 * nw, 5 * nw - 1, 700)
    g, pl = loaded.oracle()
    ref = I.integrate_method_uks(g, loaded.w.basis, Pa, Pb, functional, pl)
    E, N, Va, Vb = _uks(loaded, Pa, Pb, functional)
    assert abs(E - ref.E) <= 1e-9 and abs(N - ref.N) <= 1e-9
    assert np.max(np.abs(Va - ref.Va)) <= 1e-9
    assert np.max(np.abs(Vb - ref.Vb)) <= 1e-9
    assert np.array_equal(Va, Va.T) and np.array_equal(Vb, Vb.T)


def test_equal_spins_give_the_restricted_result(loaded):
    fn = loaded.w.functional
    E0, N0, V0 = loaded.integrate("fp64", functional=fn)
    E, N, Va, Vb = _uks(loaded, 0.5 * loaded.w.P, 0.5 * loaded.w.P, fn)
    assert abs(E - E0) <= 1e-12 * abs(E0) and abs(N - N0) <= 1e-12 * N0
    scale = np.max(np.abs(V0))
    assert np.max(np.abs(Va - V0)) <= 1e-12 * scale and np.max(np.abs(Vb - V0)) <= 1e-12 * scale


@pytest.mark.parametrize("functional", ["slater", "pbe", "pbe0_sl"])
def test_uks_mixed_matches_oracle(loaded, functional):
    nw = loaded.w.mol.n_waters
    Pa, Pb = _spins(loaded.w, 5 * nw, 5 * nw - 1, 700)
    g, pl = loaded.oracle()
    ref = I.integrate_method_uks(g, loaded.w.basis, Pa, Pb, functional, pl)
    E, N, Va, Vb = _uks(loaded, Pa, Pb, functional, "mixed")
    assert abs(E - ref.E) <= 1e-7 and abs(N - ref.N) <= 1e-8
    assert np.max(np.abs(Va - ref.Va)) <= 1e-7, np.max(np.abs(Va - ref.Va))
    assert np.max(np.abs(Vb - ref.Vb)) <= 1e-7, np.max(np.abs(Vb - ref.Vb))
    assert np.array_equal(Va, Va.T) and np.array_equal(Vb, Vb.T)


def test_uks_mixed_equal_spins_near_restricted_mixed(loaded):
    # equal spins through the unrestricted tensor-core path against the restricted one:
    # the same slicing of Phi, P/2 slices exactly half of P's, so only the functional
    # (float64 here, float32 above the density threshold there) and rounding differ
    fn = loaded.w.functional
    E0, N0, V0 = loaded.integrate("mixed", functional=fn)
    E, N, Va, Vb = _uks(loaded, 0.5 * loaded.w.P, 0.5 * loaded.w.P, fn, "mixed")
    assert abs(E - E0) <= 2e-7 and abs(N - N0) <= 1e-9
    assert np.max(np.abs(Va - V0)) <= 1e-7 and np.max(np.abs(Vb - V0)) <= 1e-7, (np.max(np.abs(Va - V0)), np.max(np.abs(Vb - V0)))


def test_uks_full_size_equal_spins():
    L = Loaded("water16_pbe")
    try:
        E0, N0, V0 = L.integrate("fp64")
        E, N, Va, Vb = _uks(L, 0.5 * L.w.P, 0.5 * L.w.P, "pbe")
        assert abs(E - E0) <= 1e-12 * abs(E0)
        assert np.max(np.abs(Va - V0)) <= 1e-11 * np.max(np.abs(V0))
    finally:
        L.close()


def test_uks_mixed_full_size():
    """16 waters, an open-shell-like split (P^a from 41 orbitals, P^b from 39): the tensor-core
    form against the float64 form of the same call."""
    L = Loaded("water16_pbe")
    try:
        Pa, Pb = _spins(L.w, 41, 39, 900)
        E64, N64, Va64, Vb64 = _uks(L, Pa, Pb, "pbe", "fp64")
        E, N, Va, Vb = _uks(L, Pa, Pb, "pbe", "mixed")
        assert abs(E - E64) <= 1e-6 and abs(N - N64) <= 1e-7
        assert np.max(np.abs(Va - Va64)) <= 1e-7 and np.max(np.abs(Vb - Vb64)) <= 1e-7, (np.max(np.abs(Va - Va64)), np.max(np.abs(Vb - Vb64)))
    finally:
        L.close()
