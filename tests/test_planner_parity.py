"""The library's host planner against the oracle planner: coordinates, batches and shell lists
bit for bit (Sec. 2.2, Eq. rcut, Algorithm 1, Algorithm 3).  Runs on the CPU through a host-only
context of the C-ABI library."""
import numpy as np
import pytest

import xcinputs as X
from oracle import integrate as I

G = pytest.importorskip("paper_2007_03143_gb300")


def _lib_plan(w):
    try:
        G.lib()
    except G.LibraryMissing as e:
        pytest.skip(str(e))
    ctx = G.gbxc_create(-1)
    try:
        b = w.basis
        mid, nbf = G.gbxc_load_basis(ctx, w.mol.xyz, w.mol.Z, b.atom, b.L, b.nprim, b.alpha, b.coeff, b.pure)
        assert nbf == b.nbf
        g = w.grid
        G.gbxc_load_grid(ctx, mid, g.nrad, g.ntheta, g.nphi, g.partition, g.max_batch, g.eta, g.mk_alpha,
                         g.angular)
        info = G.gbxc_plan_info_get(ctx, mid)
        n, nb = info["npts"], info["nbatch"]
        out = dict(x=np.empty(n), y=np.empty(n), z=np.empty(n), wq=np.empty(n),
                   parent=np.empty(n, np.int32), point_index=np.empty(n, np.int64),
                   batch_ptr=np.empty(nb + 1, np.int64), shell_ptr=np.empty(nb + 1, np.int64),
                   shell_idx=np.empty(info["nshell_entries"], np.int32))
        G.lib().gbxc_export_plan(ctx, mid, out["x"].ctypes.data, out["y"].ctypes.data,
                                 out["z"].ctypes.data, out["wq"].ctypes.data, None,
                                 out["parent"].ctypes.data, out["point_index"].ctypes.data,
                                 out["batch_ptr"].ctypes.data, out["shell_ptr"].ctypes.data,
                                 out["shell_idx"].ctypes.data)
        return info, out
    finally:
        G.gbxc_destroy(ctx)


@pytest.mark.parametrize("name", ["water1_slater", "water2_pbe_small", "water3_pbe_small",
                                  "water1_pbe_small", "water16_pbe", "water2_pbe_small_sph",
                                  "water2_pbe_small_leb", "water16_pbe_fg"])
def test_plan_bit_exact(name):
    w = X.make_workload(name)
    info, L = _lib_plan(w)
    g = I.make_grid(w.mol.xyz, w.grid, weights=False)
    pl = I.make_plan(g, w.mol.xyz, w.basis, w.grid)
    # coordinates and quadrature weights: identical bits, in the library's batch order
    idx = L["point_index"]
    assert np.array_equal(np.sort(idx), np.arange(len(g.x)))
    for k, ref in (("x", g.x), ("y", g.y), ("z", g.z), ("wq", g.wq)):
        assert np.array_equal(L[k], ref[idx]), k
    assert np.array_equal(L["parent"], g.parent[idx])
    # merged batches: same count, same order, same points, same shell lists
    assert info["nbatch"] == len(pl.batch_points)
    assert info["nleaf"] == len(pl.unmerged_points)
    bp = L["batch_ptr"]
    sp = L["shell_ptr"]
    for j in range(info["nbatch"]):
        assert np.array_equal(idx[bp[j]:bp[j + 1]], pl.batch_points[j])
        assert L["shell_idx"][sp[j]:sp[j + 1]].tolist() == pl.batch_shells[j]
    assert info["sum_mn2"] == float(sum(len(p) * len(f) ** 2 for p, f in zip(pl.batch_points, pl.batch_funcs)))
    assert info["work"] == pytest.approx(float(np.sum(pl.work)), rel=1e-15)


def test_host_context_rejects_integration():
    try:
        G.lib()
    except G.LibraryMissing as e:
        pytest.skip(str(e))
    w = X.make_workload("water1_slater")
    ctx = G.gbxc_create(-1)
    try:
        b = w.basis
        mid, nbf = G.gbxc_load_basis(ctx, w.mol.xyz, w.mol.Z, b.atom, b.L, b.nprim, b.alpha, b.coeff, b.pure)
        with pytest.raises(G.GbxcError):
            G.gbxc_integrate(ctx, mid, w.P)
        with pytest.raises(G.GbxcError):
            G.gbxc_load_basis(ctx, w.mol.xyz, w.mol.Z, b.atom[::-1].copy(), b.L, b.nprim, b.alpha, b.coeff)
    finally:
        G.gbxc_destroy(ctx)
