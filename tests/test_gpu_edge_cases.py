"""Degenerate and edge inputs through the C-ABI against the oracle (Algorithm 4, Eqs. rho/exc/
vxc): zero density, densities straddling the rho < 1e-15 cut, single atoms (partition of unity
with one centre), batches capped at 16 points (nearly empty 128-point tiles), tiny shapes
(n = 1, 3, 6 functions; m = 1, 31, 33 points); plus the library's own edge behaviour (unload,
the 974-point grid, work-order invariance, non-finite P, plan files)."""
import numpy as np
import pytest

import xcinputs as X
from oracle import integrate as I

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _run(mol, spec, functional, P, forms=("fp64", "mixed")):
    G = need_gpu()
    basis = X.make_basis(mol)
    ctx = G.Context(0)
    try:
        mid = ctx.load_molecule(mol, basis, spec)
        out = {}
        for f in forms:
            V = np.zeros((basis.nbf, basis.nbf))
            E, N = G.gbxc_integrate(ctx.h, mid, P, functional, f, V)
            out[f] = (E, N, V)
        return basis, out
    finally:
        ctx.close()


def _oracle(mol, basis, spec, functional, P):
    g = I.make_grid(mol.xyz, spec)
    pl = I.make_plan(g, mol.xyz, basis, spec)
    return I.integrate_method(g, basis, P, functional, pl)


def _density(mol, nocc, seed):
    basis = X.make_basis(mol)
    return X.density_matrix(X.overlap_matrix(basis), nocc, seed)


SPEC_SMALL = X.GridSpec(20, 8, 16, "ssf", 128)


@pytest.mark.parametrize("functional", ["pbe", "slater"])
def test_zero_density(functional):
    mol = X.water_cluster(2, 9100)
    nbf = X.make_basis(mol).nbf
    _, out = _run(mol, SPEC_SMALL, functional, np.zeros((nbf, nbf)))
    for f, (E, N, V) in out.items():
        assert E == 0.0 and N == 0.0, f
        assert not np.any(V), f


@pytest.mark.parametrize("scale", [1e-12, 1e-6])
def test_density_near_the_cut(scale):
    # rho spans the 1e-15 threshold: points on either side of it contribute ~1e-20
    mol = X.water_cluster(2, 9100)
    P = scale * _density(mol, 10, 9101)
    basis, out = _run(mol, SPEC_SMALL, "pbe", P)
    ref = _oracle(mol, basis, SPEC_SMALL, "pbe", P)
    E, N, V = out["fp64"]
    assert abs(E - ref.E) <= 1e-9 * abs(ref.E) + 1e-18
    assert abs(N - ref.N) <= 1e-9 * abs(ref.N) + 1e-18
    assert np.max(np.abs(V - ref.V)) <= 1e-9 * np.max(np.abs(ref.V)) + 1e-18
    Em, Nm, Vm = out["mixed"]
    assert abs(Em - ref.E) <= 1e-7 * abs(ref.E) + 1e-18
    # V relative to its largest element: at scale 1e-12 the points whose density lies within
    # the form's rounding of the cut are counted on one side or the other (measured |dV| 1.7e-9,
    # above 1e-7 of max |V|)
    dv = np.max(np.abs(Vm - ref.V))
    assert dv <= 1e-6 * np.max(np.abs(ref.V)) + 1e-18, dv


@pytest.mark.parametrize("Z,partition", [(8, "ssf"), (1, "becke"), (8, "becke")])
def test_single_atom(Z, partition):
    mol = X.single_atom(Z)
    spec = X.GridSpec(30, 10, 20, partition, 256)
    P = _density(mol, 4 if Z == 8 else 1, 9400 + Z)
    basis, out = _run(mol, spec, "pbe", P)
    ref = _oracle(mol, basis, spec, "pbe", P)
    E, N, V = out["fp64"]
    assert abs(E - ref.E) <= 1e-9 and abs(N - ref.N) <= 1e-9
    assert np.max(np.abs(V - ref.V)) <= 1e-9
    Em, Nm, Vm = out["mixed"]
    dv = np.max(np.abs(Vm - ref.V))
    assert abs(Em - ref.E) <= 1e-7 and dv <= 1e-7, dv


def test_tiny_batches():
    # at most 16 points per batch: every tile is mostly padding
    mol = X.water_cluster(2, 9100)
    spec = X.GridSpec(20, 8, 16, "ssf", 16)
    P = _density(mol, 10, 9101)
    basis, out = _run(mol, spec, "pbe", P)
    ref = _oracle(mol, basis, spec, "pbe", P)
    E, N, V = out["fp64"]
    assert abs(E - ref.E) <= 1e-9 and np.max(np.abs(V - ref.V)) <= 1e-9
    Em, Nm, Vm = out["mixed"]
    dv = np.max(np.abs(Vm - ref.V))
    assert abs(Em - ref.E) <= 1e-7 and dv <= 1e-7, dv


def test_unload_releases_a_molecule_and_its_cached_graph():
    """After gbxc_unload the id is refused, the batching graph that held it is rebuilt for the
    remaining molecules, and their results do not change."""
    G = need_gpu()
    ws = [X.make_workload("water1_pbe_small"), X.make_workload("water2_pbe_small")]
    ctx = G.Context(0)
    try:
        ids = [ctx.load_molecule(w.mol, w.basis, w.grid) for w in ws]
        V1 = np.zeros((ws[1].basis.nbf,) * 2)
        E1, N1 = G.gbxc_integrate(ctx.h, ids[1], ws[1].P, "pbe", "mixed", V1)
        E, N = G.gbxc_integrate_many(ctx.h, ids, [w.P for w in ws], ["pbe", "pbe"], "mixed")
        G.gbxc_unload(ctx.h, ids[0])
        with pytest.raises(G.GbxcError):
            G.gbxc_integrate(ctx.h, ids[0], ws[0].P, "pbe", "mixed", None)
        with pytest.raises(G.GbxcError):
            G.gbxc_integrate_many(ctx.h, ids, [w.P for w in ws], ["pbe", "pbe"], "mixed")
        E2, N2 = G.gbxc_integrate_many(ctx.h, ids[1:], [ws[1].P], ["pbe"], "mixed")
        assert abs(E2[0] - E1) <= 1e-10 * abs(E1) and abs(E[1] - E1) <= 1e-10 * abs(E1)
        V2 = np.zeros_like(V1)
        E3, _ = G.gbxc_integrate(ctx.h, ids[1], ws[1].P, "pbe", "mixed", V2)
        # E is summed in a fixed order; V through float64 atomics (order-dependent rounding)
        assert E3 == E1 and np.max(np.abs(V2 - V1)) <= 1e-12 * np.max(np.abs(V1))
    finally:
        ctx.close()


def test_974_point_grid_mixed_against_float64():
    """The 974-point Lebedev-Laikov rule (pinned by exactness in the CPU tests; the oracle does
    not build it): the tensor-core form against the float64 form on it."""
    G = need_gpu()
    w = X.make_workload("water2_pbe_small_974")
    ctx = G.Context(0)
    try:
        mid = ctx.load_molecule(w.mol, w.basis, w.grid)
        nbf = w.basis.nbf
        V64, Vm = np.zeros((nbf, nbf)), np.zeros((nbf, nbf))
        E64, N64 = G.gbxc_integrate(ctx.h, mid, w.P, "pbe", "fp64", V64)
        Em, Nm = G.gbxc_integrate(ctx.h, mid, w.P, "pbe", "mixed", Vm)
        assert abs(Em - E64) <= 1e-7 and abs(Nm - N64) <= 1e-8
        dv = np.max(np.abs(Vm - V64))
        assert dv <= 1e-7, dv
    finally:
        ctx.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_work_order_invariance(form):
    """Race check by work order: the same integration with a small scratch budget (many chunks,
    a different order of the V atomics and of the launches) agrees with the one-chunk result:
    E and N bit for bit (fixed-order sums); V to 1e-12 relative in float64 (atomics order
    only), 1e-9 in the mixed form (a batch cut by a chunk boundary also gets other V-side
    slicing groups, hence other roundings)."""
    G = need_gpu()
    w = X.make_workload("water3_pbe_small")
    nbf = w.basis.nbf
    out = []
    for scratch in (0, 24 << 20):
        ctx = G.Context(0, scratch)
        try:
            mid = ctx.load_molecule(w.mol, w.basis, w.grid)
            V = np.zeros((nbf, nbf))
            E, N = G.gbxc_integrate(ctx.h, mid, w.P, "pbe", form, V)
            out.append((E, N, V))
        finally:
            ctx.close()
    (E0, N0, V0), (E1, N1, V1) = out
    assert E0 == E1 and N0 == N1
    assert np.max(np.abs(V1 - V0)) <= (1e-12 if form == "fp64" else 1e-9) * np.max(np.abs(V0))


def test_nan_in_P_is_refused_and_the_next_call_is_clean():
    """Host-side injection of a NaN (and an infinity) in P: the call is refused with
    GBXC_EINVAL after a device-side check, instead of the functionals' density test silently
    dropping the affected points; the next call with a valid P gives the normal result."""
    G = need_gpu()
    w = X.make_workload("water1_pbe_small")
    nbf = w.basis.nbf
    ctx = G.Context(0)
    try:
        mid = ctx.load_molecule(w.mol, w.basis, w.grid)
        E0, N0 = G.gbxc_integrate(ctx.h, mid, w.P, "pbe", "mixed", None)
        for bad in (np.nan, np.inf):
            Pbad = w.P.copy()
            Pbad[3, 5] = Pbad[5, 3] = bad
            for form in ("fp64", "mixed"):
                with pytest.raises(G.GbxcError):
                    G.gbxc_integrate(ctx.h, mid, Pbad, "pbe", form, None)
            with pytest.raises(G.GbxcError):
                G.gbxc_integrate_uks(ctx.h, mid, 0.5 * w.P, 0.5 * Pbad, "pbe", "fp64")
        E1, N1 = G.gbxc_integrate(ctx.h, mid, w.P, "pbe", "mixed", None)
        assert E1 == E0 and N1 == N0
    finally:
        ctx.close()


def test_plan_file_reload_integrates_identically(tmp_path):
    """A plan saved from a device-planned molecule and loaded into a fresh copy of it (no
    planning) integrates to the same E_xc and N_el bit for bit and the same V to 1e-12."""
    G = need_gpu()
    w = X.make_workload("water2_pbe_small")
    nbf = w.basis.nbf
    ctx = G.Context(0)
    try:
        a = ctx.load_molecule(w.mol, w.basis, w.grid, device_planner=True)
        path = str(tmp_path / "w2.plan")
        G.gbxc_save_plan(ctx.h, a, path)
        b, _ = G.gbxc_load_basis(ctx.h, w.mol.xyz, w.mol.Z, w.basis.atom, w.basis.L, w.basis.nprim,
                                 w.basis.alpha, w.basis.coeff)
        G.gbxc_load_plan(ctx.h, b, path)
        out = []
        for mid in (a, b):
            V = np.zeros((nbf, nbf))
            E, N = G.gbxc_integrate(ctx.h, mid, w.P, "pbe", "mixed", V)
            out.append((E, N, V))
        assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
        assert np.max(np.abs(out[0][2] - out[1][2])) <= 1e-12 * np.max(np.abs(out[0][2]))
    finally:
        ctx.close()


@pytest.mark.parametrize("L", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 31, 33])
def test_tiny_shapes(L, m):
    """Tiny shapes: one atom with one shell (n = 1, 3 or 6 functions) and a grid of m points on
    one ray (m = 1: a single point; 31 and 33: one short of and one past a 32-point warp), so
    the only batch is a nearly empty tile."""
    G = need_gpu()
    mol = X.single_atom(8)
    basis = X.make_basis(mol, single_shell=(L, [5.0, 1.0, 0.3], [0.3, 0.5, 0.4]))
    spec = X.GridSpec(m, 1, 1, "becke", 512)
    S = X.overlap_matrix(basis)
    P = X.density_matrix(S, 1, 9500 + 10 * L + m)
    ctx = G.Context(0)
    try:
        mid = ctx.load_molecule(mol, basis, spec)
        info = G.gbxc_plan_info_get(ctx.h, mid)
        assert info["npts"] == m and info["nbatch"] == 1
        out = {}
        for f in ("fp64", "mixed"):
            V = np.zeros((basis.nbf, basis.nbf))
            E, N = G.gbxc_integrate(ctx.h, mid, P, "pbe", f, V)
            out[f] = (E, N, V)
    finally:
        ctx.close()
    g = I.make_grid(mol.xyz, spec)
    pl = I.make_plan(g, mol.xyz, basis, spec)
    ref = I.integrate_method(g, basis, P, "pbe", pl)
    E, N, V = out["fp64"]
    assert abs(E - ref.E) <= 1e-9 and abs(N - ref.N) <= 1e-9 and np.max(np.abs(V - ref.V)) <= 1e-9
    Em, Nm, Vm = out["mixed"]
    assert abs(Em - ref.E) <= 1e-7 and np.max(np.abs(Vm - ref.V)) <= 1e-6
