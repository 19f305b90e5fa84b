"""Batching form (one CUDA-graph launch over many molecules) and serving form (continuous
batching) against single-molecule gbxc_integrate, through the C-ABI.  The same kernels run in
every form, so results agree to rounding order: |dE| <= 1e-10 Eh and max |dV| <= 1e-9."""
import numpy as np
import pytest

import xcinputs as X

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

SPEC = X.GridSpec(24, 10, 20, "ssf", 200)


def _molecules(G, ctx, sizes, seed0):
    out = []
    for k, nw in enumerate(sizes):
        mol = X.water_cluster(nw, seed0 + k)
        b = X.make_basis(mol)
        S = X.overlap_matrix(b)
        P = X.density_matrix(S, 5 * nw, seed0 + 100 + k)
        mid, nbf = G.gbxc_load_basis(ctx.h, mol.xyz, mol.Z, b.atom, b.L, b.nprim, b.alpha, b.coeff)
        G.gbxc_load_grid(ctx.h, mid, SPEC.nrad, SPEC.ntheta, SPEC.nphi, SPEC.partition, SPEC.max_batch)
        out.append((mid, nbf, P))
    return out


def _alone(G, ctx, mid, nbf, P, fn, prec):
    V = np.zeros((nbf, nbf))
    E, N = G.gbxc_integrate(ctx.h, mid, P, fn, prec, V)
    return E, N, V


@pytest.fixture(scope="module")
def setup():
    G = need_gpu()
    ctx = G.Context(0)
    mols = _molecules(G, ctx, SIZES, SEED0)
    yield G, ctx, mols
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_many_matches_single(setup, prec):
    G, ctx, mols = setup
    fns = ["pbe", "slater", "pbe", "pbe", "slater", "pbe"]
    ref = [_alone(G, ctx, mid, nbf, P, fn, prec) for (mid, nbf, P), fn in zip(mols, fns)]
    for call in range(2):    # the second call replays the captured graph
        Vs = [np.zeros((nbf, nbf)) for (_, nbf, _) in mols]
        E, N = G.gbxc_integrate_many(ctx.h, [m[0] for m in mols], [m[2] for m in mols], fns, prec, Vs)
        for k in range(len(mols)):
            assert abs(E[k] - ref[k][0]) <= 1e-10, (call, k)
            assert abs(N[k] - ref[k][1]) <= 1e-10, (call, k)
            assert np.max(np.abs(Vs[k] - ref[k][2])) <= 1e-9, (call, k)
    # new densities through the same graph
    P2 = [0.5 * m[2] for m in mols]
    E2, _ = G.gbxc_integrate_many(ctx.h, [m[0] for m in mols], P2, fns, prec)
    for k, (mid, nbf, P) in enumerate(mols):
        e, _, _ = _alone(G, ctx, mid, nbf, P2[k], fns[k], prec)
        assert abs(E2[k] - e) <= 1e-10


def _oracle(nw, seed, P, fn):
    from oracle import integrate as I
    mol = X.water_cluster(nw, seed)
    b = X.make_basis(mol)
    g = I.make_grid(mol.xyz, SPEC)
    pl = I.make_plan(g, mol.xyz, b, SPEC)
    return I.integrate_method(g, b, P, fn, pl)


SIZES, SEED0 = [1, 3, 2, 4, 1, 2], 7000


@pytest.mark.parametrize("prec,tol_e,tol_v", [("fp64", 1e-9, 1e-9), ("mixed", 1e-7, 1e-7)])
def test_many_against_oracle(setup, prec, tol_e, tol_v):
    """The default (grouped) launch over six molecules of 1-4 waters with LDA, PBE and the
    PBE0 semi-local part mixed, each molecule against the oracle."""
    G, ctx, mols = setup
    fns = ["slater", "pbe", "pbe0_sl", "pbe", "pbe0_sl", "slater"]
    Vs = [np.zeros((nbf, nbf)) for (_, nbf, _) in mols]
    E, N = G.gbxc_integrate_many(ctx.h, [m[0] for m in mols], [m[2] for m in mols], fns, prec, Vs)
    for k, (nw, (mid, nbf, P)) in enumerate(zip(SIZES, mols)):
        ref = _oracle(nw, SEED0 + k, P, fns[k])
        assert abs(E[k] - ref.E) <= tol_e, k
        assert abs(N[k] - ref.N) <= tol_e, k
        assert np.max(np.abs(Vs[k] - ref.V)) <= tol_v, k


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grouped_launch_over_many_chunks(prec):
    """A small scratch budget splits the combined plan into many chunks, several of which hold
    tiles of more than one molecule: each result equals its single-molecule call.  Chunk
    boundaries then split batches differently from the single calls; in the mixed form that
    changes the V-side slicing groups (their exponents and so the rounding of V, whose error
    against float64 is about 1e-7 either way), so the mixed V is held to the mixed form's
    bound against the float64 call instead (E and N come from the X side and stay equal)."""
    G = need_gpu()
    ctx = G.Context(0, 6 << 20)
    try:
        mols = _molecules(G, ctx, [2, 1, 3, 1, 2], 7100)
        fns = ["pbe", "slater", "pbe", "pbe0_sl", "pbe"]
        ids = [m[0] for m in mols]
        G.gbxc_set_schedule(ctx.h, ids, prec, 0, 128)
        Vs = [np.zeros((nbf, nbf)) for (_, nbf, _) in mols]
        E, N = G.gbxc_integrate_many(ctx.h, ids, [m[2] for m in mols], fns, prec, Vs)
        for k, ((mid, nbf, P), fn) in enumerate(zip(mols, fns)):
            e, n, V = _alone(G, ctx, mid, nbf, P, fn, prec)
            assert abs(E[k] - e) <= 1e-10 and abs(N[k] - n) <= 1e-10, k
            if prec == "mixed":
                V = _alone(G, ctx, mid, nbf, P, fn, "fp64")[2]
            assert np.max(np.abs(Vs[k] - V)) <= (1e-9 if prec == "fp64" else 1e-7), (k, np.max(np.abs(Vs[k] - V)))
    finally:
        ctx.close()


@pytest.mark.parametrize("branches", [0, 2])
def test_many_rejects_nonfinite_P(setup, branches):
    """A NaN in one molecule's P fails the call with GBXC_EINVAL in the grouped launch and in
    the branched schedule; the next call with clean densities is unaffected."""
    G, ctx, mols = setup
    ids = [m[0] for m in mols]
    G.gbxc_set_schedule(ctx.h, ids, "fp64", branches, 128)
    try:
        Ps = [m[2].copy() for m in mols]
        Ps[2][1, 1] = float("nan")
        with pytest.raises(G.GbxcError) as e:
            G.gbxc_integrate_many(ctx.h, ids, Ps, ["pbe"] * len(mols), "fp64")
        assert e.value.code == G.GBXC_EINVAL
        E, _ = G.gbxc_integrate_many(ctx.h, ids, [m[2] for m in mols], ["pbe"] * len(mols), "fp64")
        e0, _, _ = _alone(G, ctx, mols[2][0], mols[2][1], mols[2][2], "pbe", "fp64")
        assert abs(E[2] - e0) <= 1e-10
    finally:
        G.gbxc_set_schedule(ctx.h, ids, "fp64", 0, 128)


def test_serving_against_oracle_and_nonfinite_P(setup):
    """Requests served by the continuous-batching loop against the oracle (float64 at 1e-9, mixed
    at the form's small-case bounds); a request whose P holds a NaN completes with GBXC_EINVAL
    and leaves the others intact."""
    G, ctx, mols = setup
    picks = [(0, "slater", "fp64"), (2, "pbe", "fp64"), (1, "pbe0_sl", "mixed"), (4, "pbe", "mixed")]
    bad = mols[3][2].copy()
    bad[0, 0] = float("inf")
    G.gbxc_serve_start(ctx.h, 3, 1 << 30)
    try:
        tickets = [G.gbxc_submit(ctx.h, mols[k][0], mols[k][2], fn, prec) for k, fn, prec in picks]
        tbad = G.gbxc_submit(ctx.h, mols[3][0], bad, "pbe", "fp64")
        for t, (k, fn, prec) in zip(tickets, picks):
            V = np.zeros((mols[k][1], mols[k][1]))
            E, N, lat = G.gbxc_wait(ctx.h, t, 120.0, V)
            ref = _oracle(SIZES[k], SEED0 + k, mols[k][2], fn)
            tol_e, tol_v = (1e-9, 1e-9) if prec == "fp64" else (1e-7, 1e-7)
            assert abs(E - ref.E) <= tol_e and abs(N - ref.N) <= tol_e, k
            assert np.max(np.abs(V - ref.V)) <= tol_v, k
        with pytest.raises(G.GbxcError) as e:
            G.gbxc_wait(ctx.h, tbad, 120.0)
        assert e.value.code == G.GBXC_EINVAL
    finally:
        G.gbxc_serve_stop(ctx.h)


@pytest.mark.parametrize("branches,tile_n", [(1, 64), (3, 64), (2, 128), (0, 64), (0, 128)])
def test_many_schedules(setup, branches, tile_n):
    # every schedule computes the same slice products in the same K order per element: only
    # the order of the float64 V atomics changes
    G, ctx, mols = setup
    fns = ["pbe", "pbe", "slater", "pbe", "pbe", "slater"]
    ids = [m[0] for m in mols]
    G.gbxc_set_schedule(ctx.h, ids, "mixed", branches, tile_n)
    Vs = [np.zeros((nbf, nbf)) for (_, nbf, _) in mols]
    E, N = G.gbxc_integrate_many(ctx.h, ids, [m[2] for m in mols], fns, "mixed", Vs)
    for k, ((mid, nbf, P), fn) in enumerate(zip(mols, fns)):
        e, n, V = _alone(G, ctx, mid, nbf, P, fn, "mixed")
        assert abs(E[k] - e) <= 1e-10 and abs(N[k] - n) <= 1e-10, k
        assert np.max(np.abs(Vs[k] - V)) <= 1e-9, k
        e64, _, V64 = _alone(G, ctx, mid, nbf, P, fn, "fp64")
        assert abs(E[k] - e64) <= 1e-7 and np.max(np.abs(Vs[k] - V64)) <= 1e-7, (k, np.max(np.abs(Vs[k] - V64)))


def test_autotune(setup):
    G, ctx, mols = setup
    fns = ["pbe"] * len(mols)
    ids = [m[0] for m in mols]
    Ps = [m[2] for m in mols]
    w, t, ms = G.gbxc_autotune(ctx.h, ids, Ps, fns, "mixed")
    assert w in (0, 1, 2, 4, 6) and t in (64, 128) and ms > 0.0   # 0: the grouped launch
    E, _ = G.gbxc_integrate_many(ctx.h, ids, Ps, fns, "mixed")
    for k, (mid, nbf, P) in enumerate(mols):
        e, _, _ = _alone(G, ctx, mid, nbf, P, "pbe", "mixed")
        assert abs(E[k] - e) <= 1e-10
    w64, t64, ms64 = G.gbxc_autotune(ctx.h, ids, Ps, fns, "fp64")
    assert w64 in (0, 1, 2, 4, 6) and t64 == 128 and ms64 > 0.0
    with pytest.raises(G.GbxcError):
        G.gbxc_set_schedule(ctx.h, ids, "mixed", 2, 96)


def test_serving_alone_equals_in_the_mix(setup):
    G, ctx, mols = setup
    rng = np.random.default_rng(0)
    reqs = []
    for r in range(24):
        k = int(rng.integers(len(mols)))
        fn = "slater" if r % 4 == 0 else "pbe"
        prec = "mixed" if r % 3 else "fp64"
        reqs.append((k, fn, prec, mols[k][2] * (1.0 + 0.01 * r)))
    alone = []
    for k, fn, prec, P in reqs:
        mid, nbf, _ = mols[k]
        alone.append(_alone(G, ctx, mid, nbf, P, fn, prec))
    G.gbxc_serve_start(ctx.h, 3, 1 << 30)
    try:
        tickets = [G.gbxc_submit(ctx.h, mols[k][0], P, fn, prec) for k, fn, prec, P in reqs]
        for t, (k, fn, prec, P), ref in zip(tickets, reqs, alone):
            V = np.zeros_like(ref[2])
            E, N, lat = G.gbxc_wait(ctx.h, t, 120.0, V)
            assert abs(E - ref[0]) <= 1e-10
            assert abs(N - ref[1]) <= 1e-10
            assert np.max(np.abs(V - ref[2])) <= 1e-9
            assert lat > 0
        st = G.gbxc_serve_stats(ctx.h)
        assert st["completed"] == len(reqs) and st["queued"] == 0 and st["running"] == 0
        assert st["arena_free"] == st["arena_cap"]      # every region returned to the arena
        with pytest.raises(G.GbxcError) as e:
            G.gbxc_wait(ctx.h, tickets[0], 0.1)
        assert e.value.code == G.GBXC_ENOENT
    finally:
        G.gbxc_serve_stop(ctx.h)


def test_serving_large_request_overlaps_small_ones(setup):
    """A 100-water request (the top of the serving pool's 4-100 water range; 11.5M points on the
    75 x 16 x 32 grid, batches of up to about 1,600 functions) submitted between small ones:
    every result equals its own gbxc_integrate (mixed form)."""
    G, ctx, mols = setup
    w = X.make_workload("water64_pbe", n_waters=100, seed=6000)
    big = ctx.load_molecule(w.mol, w.basis, w.grid, device_planner=True)
    try:
        reqs = [(mols[1][0], mols[1][2], "pbe"), (big, w.P, "pbe"), (mols[3][0], mols[3][2], "slater"),
                (mols[0][0], mols[0][2], "pbe0_sl"), (mols[5][0], mols[5][2], "pbe")]
        alone = []
        for mid, P, fn in reqs:
            V = np.zeros(P.shape)
            E, N = G.gbxc_integrate(ctx.h, mid, P, fn, "mixed", V)
            alone.append((E, N, V))
        G.gbxc_serve_start(ctx.h, 4, 0)
        try:
            tickets = [G.gbxc_submit(ctx.h, mid, P, fn, "mixed") for mid, P, fn in reqs]
            for t, (mid, P, fn), ref in zip(tickets, reqs, alone):
                V = np.zeros(P.shape)
                E, N, lat = G.gbxc_wait(ctx.h, t, 300.0, V)
                assert abs(E - ref[0]) <= 1e-10 and abs(N - ref[1]) <= 1e-10
                assert np.max(np.abs(V - ref[2])) <= 1e-9
        finally:
            G.gbxc_serve_stop(ctx.h)
    finally:
        G.gbxc_unload(ctx.h, big)


def test_serving_admission_by_footprint(setup):
    # an arena that fits one request at a time still serves every request, in order
    G, ctx, mols = setup
    G.gbxc_serve_start(ctx.h, 4, 96 << 20)
    try:
        mid, nbf, P = mols[3]
        ts = [G.gbxc_submit(ctx.h, mid, P, "pbe", "fp64") for _ in range(5)]
        E = [G.gbxc_wait(ctx.h, t, 120.0)[0] for t in ts]
        assert max(E) - min(E) <= 1e-12
        e_alone, _, _ = _alone(G, ctx, mid, nbf, P, "pbe", "fp64")
        assert abs(E[0] - e_alone) <= 1e-10
    finally:
        G.gbxc_serve_stop(ctx.h)


def test_serving_rejects_bad_requests(setup):
    G, ctx, mols = setup
    with pytest.raises(G.GbxcError):           # not running
        G.gbxc_submit(ctx.h, mols[0][0], mols[0][2])
    G.gbxc_serve_start(ctx.h, 2, 256 << 20)
    try:
        with pytest.raises(G.GbxcError):
            G.gbxc_submit(ctx.h, 987654, mols[0][2])
        t = G.gbxc_submit(ctx.h, mols[0][0], mols[0][2], "pbe", "mixed")
        E, N, lat = G.gbxc_wait(ctx.h, t, 60.0)
        assert np.isfinite(E)
    finally:
        G.gbxc_serve_stop(ctx.h)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_many_heterogeneous_molecules(prec):
    """Cartesian and spherical bases, product and Lebedev-Laikov grids in one graph launch:
    each molecule's result equals its own gbxc_integrate."""
    G = need_gpu()
    ctx = G.Context(0)
    try:
        ws = [X.make_workload(n) for n in ("water2_pbe_small", "water2_pbe_small_sph", "water2_pbe_small_leb",
                                           "water1_slater")]
        ids = [ctx.load_molecule(w.mol, w.basis, w.grid) for w in ws]
        fns = [w.functional for w in ws]
        ref = [_alone(G, ctx, mid, w.basis.nbf, w.P, fn, prec) for mid, w, fn in zip(ids, ws, fns)]
        Vs = [np.zeros((w.basis.nbf,) * 2) for w in ws]
        E, N = G.gbxc_integrate_many(ctx.h, ids, [w.P for w in ws], fns, prec, Vs)
        for k in range(len(ws)):
            assert abs(E[k] - ref[k][0]) <= 1e-10 and abs(N[k] - ref[k][1]) <= 1e-10, k
            assert np.max(np.abs(Vs[k] - ref[k][2])) <= 1e-9, k
    finally:
        ctx.close()
