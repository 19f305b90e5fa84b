"""The C-ABI library loads and exports every function that include/*.h declares (no GPU needed)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(gbxc_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_api():
    d = declared()
    for n in ("gbxc_create", "gbxc_load_basis", "gbxc_load_grid", "gbxc_integrate", "gbxc_destroy"):
        assert n in d


def test_library_exports_every_declared_symbol():
    import paper_2007_03143_gb300 as G
    try:
        L = G.lib()
    except G.LibraryMissing as e:
        pytest.skip(str(e))
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing
    assert set(G.binding.EXPORTED) <= set(declared())


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2007_03143_gb300.binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(B.LibraryMissing):
        B.gbxc_create(0)


def test_unload_on_a_host_only_context():
    """gbxc_unload releases a molecule: its id is then unknown and not reused."""
    import numpy as np

    import paper_2007_03143_gb300 as G
    import xcinputs as X
    try:
        G.lib()
    except G.LibraryMissing as e:
        pytest.skip(str(e))
    w = X.make_workload("water2_pbe_small")
    b, g = w.basis, w.grid
    ctx = G.gbxc_create(-1)
    try:
        ids = []
        for _ in range(2):
            mid, _ = G.gbxc_load_basis(ctx, w.mol.xyz, w.mol.Z, b.atom, b.L, b.nprim, b.alpha, b.coeff)
            G.gbxc_load_grid(ctx, mid, g.nrad, g.ntheta, g.nphi, g.partition, g.max_batch, g.eta, g.mk_alpha)
            ids.append(mid)
        info = G.gbxc_plan_info_get(ctx, ids[0])
        G.gbxc_unload(ctx, ids[0])
        for call in (lambda: G.gbxc_plan_info_get(ctx, ids[0]), lambda: G.gbxc_unload(ctx, ids[0])):
            with pytest.raises(G.GbxcError):
                call()
        assert G.gbxc_plan_info_get(ctx, ids[1]) == info          # the other molecule is untouched
        mid, _ = G.gbxc_load_basis(ctx, w.mol.xyz, w.mol.Z, b.atom, b.L, b.nprim, b.alpha, b.coeff)
        assert mid not in ids
        assert np.isfinite(info["sum_mn2"])
    finally:
        G.gbxc_destroy(ctx)


def test_plan_file_round_trip_on_a_host_only_context(tmp_path):
    """gbxc_save_plan / gbxc_load_plan: the reloaded plan exports the same points, batches and
    shell lists bit for bit; a plan of another molecule, a truncated file and a foreign file
    are refused without touching the molecule's grid."""
    import numpy as np

    import paper_2007_03143_gb300 as G
    import xcinputs as X
    try:
        G.lib()
    except G.LibraryMissing as e:
        pytest.skip(str(e))

    def export(ctx, mid):
        info = G.gbxc_plan_info_get(ctx, mid)
        n, nb = info["npts"], info["nbatch"]
        out = dict(x=np.empty(n), y=np.empty(n), z=np.empty(n), wq=np.empty(n), parent=np.empty(n, np.int32),
                   point_index=np.empty(n, np.int64), batch_ptr=np.empty(nb + 1, np.int64),
                   shell_ptr=np.empty(nb + 1, np.int64), shell_idx=np.empty(info["nshell_entries"], np.int32))
        G.lib().gbxc_export_plan(ctx, mid, out["x"].ctypes.data, out["y"].ctypes.data, out["z"].ctypes.data,
                                 out["wq"].ctypes.data, None, out["parent"].ctypes.data,
                                 out["point_index"].ctypes.data, out["batch_ptr"].ctypes.data,
                                 out["shell_ptr"].ctypes.data, out["shell_idx"].ctypes.data)
        return info, out

    w = X.make_workload("water2_pbe_small")
    w2 = X.make_workload("water1_pbe_small")
    ctx = G.gbxc_create(-1)
    try:
        def load(wk, grid=True):
            b, g = wk.basis, wk.grid
            mid, _ = G.gbxc_load_basis(ctx, wk.mol.xyz, wk.mol.Z, b.atom, b.L, b.nprim, b.alpha, b.coeff)
            if grid:
                G.gbxc_load_grid(ctx, mid, g.nrad, g.ntheta, g.nphi, g.partition, g.max_batch, g.eta, g.mk_alpha)
            return mid
        a = load(w)
        path = str(tmp_path / "water2.plan")
        G.gbxc_save_plan(ctx, a, path)
        b = load(w, grid=False)
        npts, nb = G.gbxc_load_plan(ctx, b, path)
        ia, ea = export(ctx, a)
        ib, eb = export(ctx, b)
        assert (npts, nb) == (ia["npts"], ia["nbatch"])
        assert {k: ia[k] for k in ia} == {k: ib[k] for k in ib}
        for k in ea:
            assert np.array_equal(ea[k], eb[k]), k
        other = load(w2)
        with pytest.raises(G.GbxcError):
            G.gbxc_load_plan(ctx, other, path)            # another molecule
        short = str(tmp_path / "short.plan")
        open(short, "wb").write(open(path, "rb").read()[:1000])
        with pytest.raises(G.GbxcError):
            G.gbxc_load_plan(ctx, b, short)
        junk = str(tmp_path / "junk.plan")
        open(junk, "wb").write(b"not a plan" * 100)
        with pytest.raises(G.GbxcError):
            G.gbxc_load_plan(ctx, b, junk)
        assert export(ctx, b)[0] == ia                    # still the good plan
    finally:
        G.gbxc_destroy(ctx)
