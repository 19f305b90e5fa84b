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
