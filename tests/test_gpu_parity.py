"""CUDA path against the oracle, element by element (float64 form), through the C-ABI.

Tolerances: |dE_xc| <= 1e-9 Eh, max |dV_ij| <= 1e-9, |dN_el| <= 1e-9 for the float64 form;
partition weights to 1e-12 relative."""
import numpy as np
import pytest

from oracle import integrate as I
from oracle import partition as PT

from gpu_common import Loaded, need_gpu

pytestmark = pytest.mark.gpu

TOL_E = 1e-9
TOL_V = 1e-9

SMALL = ["water1_slater", "water1_pbe_small", "water2_pbe_small", "water3_pbe_small", "water2_pbe_small_sph",
         "water2_pbe_small_leb"]


@pytest.fixture(scope="module", params=SMALL)
def loaded(request):
    L = Loaded(request.param)
    yield L
    L.close()


def test_partition_weights(loaded):
    ex = loaded.export()
    w = loaded.w
    ref = ex["wq"] * PT.partition_weights(ex["x"], ex["y"], ex["z"], ex["parent"], w.mol.xyz,
                                          w.grid.partition)
    # partition value p = w / w^q compared absolutely (see the full-size test)
    assert np.max(np.abs(ex["w"] - ref) / ex["wq"]) < 1e-12


def test_fp64_matches_oracle(loaded):
    g, pl = loaded.oracle()
    ref = I.integrate_method(g, loaded.w.basis, loaded.w.P, loaded.w.functional, pl)
    E, N, V = loaded.integrate("fp64")
    assert abs(E - ref.E) <= TOL_E
    assert abs(N - ref.N) <= TOL_E
    assert np.max(np.abs(V - ref.V)) <= TOL_V
    assert np.array_equal(V, V.T)


def test_fp64_other_functional(loaded):
    other = "slater" if loaded.w.functional == "pbe" else "pbe"
    g, pl = loaded.oracle()
    ref = I.integrate_method(g, loaded.w.basis, loaded.w.P, other, pl)
    E, N, V = loaded.integrate("fp64", functional=other)
    assert abs(E - ref.E) <= TOL_E
    assert np.max(np.abs(V - ref.V)) <= TOL_V


def test_batch_subset_and_per_batch_energies(loaded):
    G = loaded.G
    g, pl = loaded.oracle()
    nb = loaded.info["nbatch"]
    b0, b1 = nb // 3, max(nb // 3 + 1, 2 * nb // 3)
    ref = I.integrate_method(g, loaded.w.basis, loaded.w.P, loaded.w.functional, pl, batches=range(b0, b1))
    nbf = loaded.w.basis.nbf
    V = np.zeros((nbf, nbf))
    Eb = np.full(nb, np.nan)
    Nb = np.full(nb, np.nan)
    E, N = G.gbxc_integrate_batches(loaded.ctx.h, loaded.mid, loaded.w.P, loaded.w.functional, "fp64",
                                    b0, b1, V, Eb, Nb)
    assert np.all(Eb[:b0] == 0) and np.all(Eb[b1:] == 0)
    assert np.max(np.abs(Eb[b0:b1] - ref.E_batch[b0:b1])) <= TOL_E
    assert np.max(np.abs(Nb[b0:b1] - ref.N_batch[b0:b1])) <= TOL_E
    assert abs(E - ref.E) <= TOL_E
    assert np.max(np.abs(V - ref.V)) <= TOL_V


def test_empty_range(loaded):
    G = loaded.G
    nbf = loaded.w.basis.nbf
    V = np.ones((nbf, nbf))
    E, N = G.gbxc_integrate_batches(loaded.ctx.h, loaded.mid, loaded.w.P, loaded.w.functional, "fp64",
                                    1, 1, V)
    assert E == 0.0 and N == 0.0 and np.all(V == 0.0)


def test_device_pointers_and_determinism(loaded):
    import torch
    G = loaded.G
    nbf = loaded.w.basis.nbf
    Pd = torch.tensor(loaded.w.P, device="cuda")
    Vd = torch.zeros((nbf, nbf), dtype=torch.float64, device="cuda")
    E1, N1 = G.gbxc_integrate(loaded.ctx.h, loaded.mid, Pd, loaded.w.functional, "fp64", Vd)
    E2, N2, V2 = loaded.integrate("fp64")
    assert E1 == E2 and N1 == N2           # fixed-order reductions: bitwise reproducible
    assert np.max(np.abs(Vd.cpu().numpy() - V2)) <= 1e-13 * np.max(np.abs(V2))


def test_small_scratch_chunking():
    # force many chunks (the device-subset loop of Algorithm 2); results must not change
    L = Loaded("water2_pbe_small", scratch_bytes=6 * 128 * 8 * 300)
    try:
        g, pl = L.oracle()
        ref = I.integrate_method(g, L.w.basis, L.w.P, "pbe", pl)
        E, N, V = L.integrate("fp64")
        assert abs(E - ref.E) <= TOL_E
        assert np.max(np.abs(V - ref.V)) <= TOL_V
    finally:
        L.close()


def test_errors_are_reported():
    G = need_gpu()
    L = Loaded("water1_slater")
    try:
        with pytest.raises(G.GbxcError) as e:
            G.gbxc_integrate_batches(L.ctx.h, L.mid, L.w.P, "pbe", "fp64", 0, 10 ** 6)
        assert e.value.code == G.GBXC_EINVAL
        with pytest.raises(G.GbxcError):
            G.gbxc_integrate(L.ctx.h, 12345, L.w.P)
        with pytest.raises(G.GbxcError):
            G.gbxc_integrate(L.ctx.h, L.mid, L.w.P, "pbe", 7)
    finally:
        L.close()
