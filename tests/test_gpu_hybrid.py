"""The semi-local part of the PBE0 hybrid (3/4 PBE exchange + PBE correlation; Sec. 2.1 names
hybrids among the functionals the method serves) through the C-ABI against the oracle, in both
forms and through the many-molecule call: float64 |dE| <= 1e-9 Eh and max |dV| <= 1e-9; mixed
|dE| <= 1e-7 Eh and max |dV| <= 1e-7 (the small-case bounds of the tensor-core form)."""
import numpy as np
import pytest

from oracle import integrate as I

from gpu_common import Loaded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["water1_pbe_small", "water2_pbe_small", "water2_pbe_small_sph"])
def loaded(request):
    L = Loaded(request.param)
    yield L
    L.close()


@pytest.mark.parametrize("precision,tol_e,tol_v", [("fp64", 1e-9, 1e-9), ("mixed", 1e-7, 1e-7)])
def test_pbe0_semilocal_matches_oracle(loaded, precision, tol_e, tol_v):
    g, pl = loaded.oracle()
    ref = I.integrate_method(g, loaded.w.basis, loaded.w.P, "pbe0_sl", pl)
    E, N, V = loaded.integrate(precision, functional="pbe0_sl")
    assert abs(E - ref.E) <= tol_e
    assert abs(N - ref.N) <= tol_e
    assert np.max(np.abs(V - ref.V)) <= tol_v
    assert np.array_equal(V, V.T)


def test_pbe0_semilocal_in_the_many_molecule_call(loaded):
    """Two copies of the molecule in one graph launch, one with PBE and one with the PBE0
    semi-local part: each result equals its single-molecule call."""
    G = loaded.G
    E_pbe, _, _ = loaded.integrate("fp64", functional="pbe")
    E_h, _, _ = loaded.integrate("fp64", functional="pbe0_sl")
    mid2 = loaded.ctx.load_molecule(loaded.w.mol, loaded.w.basis, loaded.w.grid)
    E, N = G.gbxc_integrate_many(loaded.ctx.h, [loaded.mid, mid2], [loaded.w.P, loaded.w.P],
                                 ["pbe", "pbe0_sl"], "fp64")
    assert abs(E[0] - E_pbe) <= 1e-12 * abs(E_pbe)
    assert abs(E[1] - E_h) <= 1e-12 * abs(E_h)
