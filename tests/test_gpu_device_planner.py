"""The planner as device kernels (gbxc_load_grid_device) against the host planner
(gbxc_load_grid): grid coordinates and weights, leaf and batch structure, point order and
screening lists identical bit for bit (Sec. 2.2 micro-batching, Algorithm 1, Algorithm 3), so
the integrations agree exactly."""
import time

import numpy as np
import pytest

import xcinputs as X

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _plan(G, ctx, w, device):
    mid = ctx.load_molecule(w.mol, w.basis, w.grid, device_planner=device)
    return mid, G.gbxc_plan_info_get(ctx.h, mid), G.gbxc_export_plan(ctx.h, mid)


@pytest.mark.parametrize("name", ["water1_slater", "water1_pbe_small", "water2_pbe_small", "water3_pbe_small",
                                  "water16_pbe", "water64_pbe", "water2_pbe_small_sph",
                                  "water2_pbe_small_leb", "water16_pbe_fg", "water2_pbe_small_974"])
def test_device_plan_identical(name):
    G = need_gpu()
    w = X.make_workload(name)
    ctx = G.Context(0)
    try:
        t0 = time.perf_counter()
        mh, ih, eh = _plan(G, ctx, w, False)
        t1 = time.perf_counter()
        md, idv, ed = _plan(G, ctx, w, True)
        t2 = time.perf_counter()
        print(f"{name}: host planner {t1 - t0:.3f} s, device planner {t2 - t1:.3f} s")
        for k in ("npts", "nbatch", "nleaf", "nshell_entries", "nfunc_entries", "ntiles", "sum_mn2", "sum_mn"):
            assert ih[k] == idv[k], k
        for k in eh:
            assert np.array_equal(eh[k], ed[k]), k
        Eh, Nh = G.gbxc_integrate(ctx.h, mh, w.P, w.functional, "fp64")
        Ed, Nd = G.gbxc_integrate(ctx.h, md, w.P, w.functional, "fp64")
        assert Eh == Ed and Nh == Nd
    finally:
        ctx.close()


def test_device_plan_small_batches_and_single_atom():
    G = need_gpu()
    ctx = G.Context(0)
    try:
        cases = [(X.water_cluster(2, 9100), X.GridSpec(20, 8, 16, "ssf", 16)),
                 (X.single_atom(8), X.GridSpec(30, 10, 20, "becke", 256)),
                 (X.water_cluster(3, 9200), X.GridSpec(24, 10, 20, "becke", 1))]
        for mol, spec in cases:
            basis = X.make_basis(mol)
            outs = []
            for device in (False, True):
                mid = ctx.load_molecule(mol, basis, spec, device_planner=device)
                outs.append(G.gbxc_export_plan(ctx.h, mid))
            for k in outs[0]:
                assert np.array_equal(outs[0][k], outs[1][k]), k
    finally:
        ctx.close()


def test_device_planner_needs_a_device():
    G = need_gpu()
    ctx = G.gbxc_create(-1)
    try:
        w = X.make_workload("water1_slater")
        b = w.basis
        mid, _ = G.gbxc_load_basis(ctx, w.mol.xyz, w.mol.Z, b.atom, b.L, b.nprim, b.alpha, b.coeff)
        with pytest.raises(G.GbxcError):
            G.gbxc_load_grid_device(ctx, mid, 20, 8, 16, "ssf", 128)
    finally:
        G.gbxc_destroy(ctx)
