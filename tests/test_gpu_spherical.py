"""Spherical (pure) d shells on the 16-water PBE/SSF workload (O 3s2p1d with 5 d functions:
N_b = 384), as the paper's cc-pVDZ runs (Sec. 3): float64 form against the oracle on sampled
batches, tensor-core form against float64 on the whole grid."""
import numpy as np
import pytest

from oracle import integrate as I

from gpu_common import Loaded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    L = Loaded("water16_pbe_sph")
    yield L
    L.close()


def test_spherical_sampled_batches_fp64(sph):
    G = sph.G
    assert sph.w.basis.nbf == 384
    g, pl = sph.oracle()
    nb = sph.info["nbatch"]
    rng = np.random.default_rng(11)
    sel = sorted(set(rng.choice(nb, size=min(12, nb), replace=False).tolist()) | {0, nb - 1})
    ref = I.integrate_method(g, sph.w.basis, sph.w.P, "pbe", pl, batches=sel)
    Eb = np.zeros(nb)
    Nb = np.zeros(nb)
    E, N = G.gbxc_integrate_batches(sph.ctx.h, sph.mid, sph.w.P, "pbe", "fp64", 0, nb, None, Eb, Nb)
    assert np.max(np.abs(Eb[sel] - ref.E_batch[sel])) <= 1e-9
    assert np.max(np.abs(Nb[sel] - ref.N_batch[sel])) <= 1e-9
    assert abs(N - 160.0) < 1e-2


def test_spherical_mixed_against_fp64(sph):
    E64, N64, V64 = sph.integrate("fp64")
    Em, Nm, Vm = sph.integrate("mixed")
    assert abs(Em - E64) <= 1e-6 and abs(Nm - N64) <= 1e-6
    assert np.max(np.abs(Vm - V64)) <= 1e-7, np.max(np.abs(Vm - V64))
    assert np.array_equal(Vm, Vm.T)
