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
