"""Shared helpers of the GPU tests: a library context with a molecule loaded, plus oracle runs."""
import numpy as np
import pytest

import xcinputs as X
from oracle import integrate as I


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2007_03143_gb300 as G
    G.lib()          # raises LibraryMissing loudly if the extension is not built
    return G


class Loaded:
    def __init__(self, name, scratch_bytes=0, **kw):
        self.G = need_gpu()
        self.w = X.make_workload(name, **kw)
        self.ctx = self.G.Context(0, scratch_bytes)
        self.mid = self.ctx.load_molecule(self.w.mol, self.w.basis, self.w.grid)
        self.info = self.G.gbxc_plan_info_get(self.ctx.h, self.mid)
        self.plan_export = None
        self._oracle = None

    def export(self):
        if self.plan_export is None:
            self.plan_export = self.G.gbxc_export_plan(self.ctx.h, self.mid)
        return self.plan_export

    def oracle(self):
        """Oracle grid (its own coordinates and weights) and plan."""
        if self._oracle is None:
            g = I.make_grid(self.w.mol.xyz, self.w.grid)
            pl = I.make_plan(g, self.w.mol.xyz, self.w.basis, self.w.grid)
            self._oracle = (g, pl)
        return self._oracle

    def integrate(self, precision="fp64", functional=None, P=None):
        fn = functional or self.w.functional
        nbf = self.w.basis.nbf
        V = np.zeros((nbf, nbf))
        E, N = self.G.gbxc_integrate(self.ctx.h, self.mid, self.w.P if P is None else P, fn, precision, V)
        return E, N, V

    def close(self):
        self.ctx.close()
