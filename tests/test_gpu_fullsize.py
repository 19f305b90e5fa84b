"""Full-size 16-water PBE/SSF workload (75 x 16 x 32 grid, 1.84M points) in the launch
configuration the benchmark times: sampled batches against the oracle, plus properties that
hold at any size."""
import numpy as np
import pytest

from oracle import integrate as I
from oracle import partition as PT

from gpu_common import Loaded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    L = Loaded("water16_pbe")
    yield L
    L.close()


def _sample(nb, k=12, seed=0):
    rng = np.random.default_rng(seed)
    return sorted(set(rng.choice(nb, size=min(k, nb), replace=False).tolist()) | {0, nb - 1})


def test_sampled_weights(big):
    ex = big.export()
    rng = np.random.default_rng(1)
    idx = rng.choice(len(ex["x"]), 20000, replace=False)
    ref = ex["wq"][idx] * PT.partition_weights(ex["x"][idx], ex["y"][idx], ex["z"][idx], ex["parent"][idx],
                                               big.w.mol.xyz, "ssf")
    # compare the partition value p = w / w^q absolutely: SSF's 1 - g(mu) cancels near |mu| = a,
    # so relative errors of tiny weights only measure that cancellation
    assert np.max(np.abs(ex["w"][idx] - ref) / ex["wq"][idx]) < 1e-12


def test_sampled_batches_fp64(big):
    G = big.G
    g, pl = big.oracle()
    nb = big.info["nbatch"]
    assert nb == len(pl.batch_points)
    sel = _sample(nb)
    ref = I.integrate_method(g, big.w.basis, big.w.P, "pbe", pl, batches=sel)
    Eb = np.zeros(nb)
    Nb = np.zeros(nb)
    nbf = big.w.basis.nbf
    E, N = G.gbxc_integrate_batches(big.ctx.h, big.mid, big.w.P, "pbe", "fp64", 0, nb, None, Eb, Nb)
    assert np.max(np.abs(Eb[sel] - ref.E_batch[sel])) <= 1e-9
    assert np.max(np.abs(Nb[sel] - ref.N_batch[sel])) <= 1e-9
    # whole-grid properties: N_el close to Tr(PS) = 160, sum of batches equals the total
    assert abs(N - 160.0) < 1e-2
    assert abs(E - np.sum(Eb)) <= 1e-9


def test_whole_grid_fp64_against_oracle(big):
    """The float64 form on every batch of the workload against the oracle's method-equivalent
    mode: E_xc, N_el and every element of the 400 x 400 V_xc."""
    G = big.G
    g, pl = big.oracle()
    ref = I.integrate_method(g, big.w.basis, big.w.P, "pbe", pl)
    E, N, V = big.integrate("fp64")
    assert abs(E - ref.E) <= 1e-9
    assert abs(N - ref.N) <= 1e-9
    assert np.max(np.abs(V - ref.V)) <= 1e-9


def test_sampled_range_V_fp64(big):
    G = big.G
    g, pl = big.oracle()
    nb = big.info["nbatch"]
    b0, b1 = nb // 2, nb // 2 + 40
    ref = I.integrate_method(g, big.w.basis, big.w.P, "pbe", pl, batches=range(b0, b1))
    nbf = big.w.basis.nbf
    V = np.zeros((nbf, nbf))
    E, N = G.gbxc_integrate_batches(big.ctx.h, big.mid, big.w.P, "pbe", "fp64", b0, b1, V)
    assert abs(E - ref.E) <= 1e-9
    assert np.max(np.abs(V - ref.V)) <= 1e-9


def test_full_trace_identity_fp64(big):
    # Tr(P V) = sum_i w_i (rho vrho + 2 sigma vsigma): checked through the gradient-free Slater
    # special case, where it is (4/3) E_x exactly
    E, N, V = big.integrate("fp64", functional="slater")
    assert abs(np.sum(big.w.P * V) - 4.0 / 3.0 * E) < 1e-10 * abs(E)
    assert np.array_equal(V, V.T)


def test_mixed_full_size_against_fp64_and_oracle(big):
    # the mixed form's bound on the full workload: |E_mixed - E_fp64| <= 1e-6 Eh
    G = big.G
    E64, N64, V64 = big.integrate("fp64")
    Em, Nm, Vm = big.integrate("mixed")
    assert abs(Em - E64) <= 1e-6
    assert abs(Nm - N64) <= 1e-6
    dv = np.max(np.abs(Vm - V64))
    assert dv <= 1e-7, dv
    assert np.array_equal(Vm, Vm.T)
    # sampled batches against the oracle
    g, pl = big.oracle()
    nb = big.info["nbatch"]
    sel = _sample(nb, seed=3)
    ref = I.integrate_method(g, big.w.basis, big.w.P, "pbe", pl, batches=sel)
    Eb = np.zeros(nb)
    G.gbxc_integrate_batches(big.ctx.h, big.mid, big.w.P, "pbe", "mixed", 0, nb, None, Eb)
    assert np.max(np.abs(Eb[sel] - ref.E_batch[sel])) <= 1e-8
