"""The oracle's Lebedev-Laikov rules (oracle/lebedev.py) against what fixes them: exactness on
every real spherical harmonic up to the rule's degree (scipy's sph_harm_y, independent of the
moment conditions the rules were solved from), the closed-form weights of the 6-, 14- and
26-point rules, octahedral invariance, positive weights summing to 4 pi, and a fresh solve
reproducing the kept result.  Also the library's own table (built by the package's generator,
a separate implementation) against the oracle's, through a host-only context."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import lebedev as L

scipy_special = pytest.importorskip("scipy.special")

SIZES = sorted(L.STRUCTURE)


def _harmonic_errors(ux, uy, uz, w, lmax):
    """max over m of |sum_k w_k Y_lm(u_k) - sqrt(4 pi) delta_l0| for each l <= lmax."""
    th = np.arccos(np.clip(uz, -1, 1))
    ph = np.arctan2(uy, ux)
    out = []
    for l in range(lmax + 1):
        e = 0.0
        for m in range(0, l + 1):
            y = scipy_special.sph_harm_y(l, m, th, ph)
            ref = math.sqrt(4 * math.pi) if l == 0 else 0.0
            e = max(e, abs(np.sum(w * y.real) - ref), abs(np.sum(w * y.imag)))
        out.append(e)
    return np.array(out)


@pytest.mark.parametrize("n", SIZES)
def test_exact_to_degree(n):
    p = L.STRUCTURE[n][0]
    ux, uy, uz, w = L.angular_rule(n)
    assert len(w) == n
    err = _harmonic_errors(ux, uy, uz, w, p + 1)
    assert np.max(err[:p + 1]) < 2e-14, (n, np.max(err[:p + 1]))
    assert err[p + 1] > 1e-4                       # and not beyond its degree
    assert np.all(w > 0)
    assert abs(np.sum(w) - 4 * math.pi) < 1e-13
    assert np.max(np.abs(ux * ux + uy * uy + uz * uz - 1)) < 3e-16


@pytest.mark.parametrize("n", SIZES)
def test_octahedral_invariance(n):
    ux, uy, uz, w = L.angular_rule(n)
    pts = {(round(a, 13), round(b, 13), round(c, 13)): wk for a, b, c, wk in zip(ux, uy, uz, w)}
    assert len(pts) == n
    for perm in itertools.permutations(range(3)):
        for sg in itertools.product((1, -1), repeat=3):
            for (a, b, c), wk in pts.items():
                v = (a, b, c)
                img = tuple(round(sg[k] * v[perm[k]], 13) + 0.0 for k in range(3))
                assert img in pts and abs(pts[img] - wk) < 1e-15


def test_closed_form_small_rules():
    # degree 3: the octahedron, equal weights; degree 5: a1 1/15, a3 3/40;
    # degree 7: a1 1/21, a2 4/105, a3 27/840 (weights per point, rule normalised to 1)
    ux, uy, uz, w = L.angular_rule(6)
    assert np.allclose(w / (4 * math.pi), 1 / 6, rtol=0, atol=1e-16)
    orb = dict((k, wp / (4 * math.pi)) for k, _, wp in L.read_orbits(os.path.join(L.CACHE_DIR, "lebedev_14.txt")))
    assert abs(orb["a1"] - 1 / 15) < 1e-16 and abs(orb["a3"] - 3 / 40) < 1e-16
    orb = dict((k, wp / (4 * math.pi)) for k, _, wp in L.read_orbits(os.path.join(L.CACHE_DIR, "lebedev_26.txt")))
    assert abs(orb["a1"] - 1 / 21) < 1e-16 and abs(orb["a2"] - 4 / 105) < 1e-16
    assert abs(orb["a3"] - 27 / 840) < 1e-16


def test_exact_moments():
    # mean of x^2 over the sphere is 1/3, of x^4 1/5, of x^2 y^2 1/15; e2 has mean 1/5
    assert L.sphere_mean(1, 0, 0) == L.Fraction(1, 3)
    assert L.sphere_mean(2, 0, 0) == L.Fraction(1, 5)
    assert L.sphere_mean(1, 1, 0) == L.Fraction(1, 15)
    assert L.invariant_mean(1, 0) == L.Fraction(1, 5)
    assert L.invariant_mean(0, 1) == L.sphere_mean(1, 1, 1) == L.Fraction(1, 105)


@pytest.mark.parametrize("n", [6, 14, 26, 38, 50, 86])
def test_fresh_solve_reproduces_kept_rule(n):
    pytest.importorskip("mpmath")
    fresh = L.lebedev_orbits(n)
    kept = L.read_orbits(os.path.join(L.CACHE_DIR, f"lebedev_{n}.txt"))
    assert [(k, g, w) for k, g, w in fresh] == [(k, g, w) for k, g, w in kept]


def test_unsupported_size_raises():
    with pytest.raises(ValueError):
        L.lebedev_orbits(302 + 1)


@pytest.mark.parametrize("n", SIZES)
def test_library_table_equals_oracle(n):
    """One atom at the origin with one radial shell: the library's points are r * u."""
    G = pytest.importorskip("paper_2007_03143_gb300")
    try:
        G.lib()
    except G.LibraryMissing as e:
        pytest.skip(str(e))
    ctx = G.gbxc_create(-1)
    try:
        mid, _ = G.gbxc_load_basis(ctx, np.zeros((1, 3)), np.array([1], np.int32), np.array([0], np.int32),
                                   np.array([0], np.int32), np.array([1], np.int32), np.array([[1.0]]),
                                   np.array([[1.0]]))
        G.gbxc_load_grid(ctx, mid, 1, n, 0, "becke", 1 << 20, 1e-10, 5.0, "lebedev")
        info = G.gbxc_plan_info_get(ctx, mid)
        npts, nb = info["npts"], info["nbatch"]
        ex = dict(x=np.empty(npts), y=np.empty(npts), z=np.empty(npts), wq=np.empty(npts),
                  point_index=np.empty(npts, np.int64))
        G.lib().gbxc_export_plan(ctx, mid, ex["x"].ctypes.data, ex["y"].ctypes.data, ex["z"].ctypes.data,
                                 ex["wq"].ctypes.data, None, None, ex["point_index"].ctypes.data,
                                 None, None, None)
    finally:
        G.gbxc_destroy(ctx)
    from oracle import quadrature as Q
    r, wr = Q.mura_knowles(1, 5.0)
    ux, uy, uz, w = L.angular_rule(n)
    order = np.argsort(ex["point_index"])
    assert np.array_equal(ex["x"][order], r[0] * ux)
    assert np.array_equal(ex["y"][order], r[0] * uy)
    assert np.array_equal(ex["z"][order], r[0] * uz)
    assert np.array_equal(ex["wq"][order], wr[0] * w)


def _library_unit_rule(G, n):
    """The library's n-point rule read back through a one-atom, one-radial-point grid."""
    ctx = G.gbxc_create(-1)
    try:
        mid, _ = G.gbxc_load_basis(ctx, np.zeros((1, 3)), np.array([1], np.int32), np.array([0], np.int32),
                                   np.array([0], np.int32), np.array([1], np.int32), np.array([[1.0]]),
                                   np.array([[1.0]]))
        G.gbxc_load_grid(ctx, mid, 1, n, 0, "becke", 1 << 20, 1e-10, 5.0, "lebedev")
        npts = G.gbxc_plan_info_get(ctx, mid)["npts"]
        ex = {k: np.empty(npts) for k in ("x", "y", "z", "wq")}
        ex["point_index"] = np.empty(npts, np.int64)
        G.lib().gbxc_export_plan(ctx, mid, ex["x"].ctypes.data, ex["y"].ctypes.data, ex["z"].ctypes.data,
                                 ex["wq"].ctypes.data, None, None, ex["point_index"].ctypes.data,
                                 None, None, None)
    finally:
        G.gbxc_destroy(ctx)
    from oracle import quadrature as Q
    r, wr = Q.mura_knowles(1, 5.0)
    o = np.argsort(ex["point_index"])
    return ex["x"][o] / r[0], ex["y"][o] / r[0], ex["z"][o] / r[0], ex["wq"][o] / wr[0]


@pytest.mark.parametrize("n,p", [(590, 41), (974, 53)])
def test_library_large_rules_pinned_directly(n, p):
    """The 590- and 974-point rules (degrees 41 and 53; the paper's UFG and SFG grids), which
    the oracle does not build: every Y_lm with l <= p integrated exactly, l = p + 1 not,
    positive weights summing to 4 pi, octahedral orbits."""
    G = pytest.importorskip("paper_2007_03143_gb300")
    try:
        G.lib()
    except G.LibraryMissing as e:
        pytest.skip(str(e))
    ux, uy, uz, w = _library_unit_rule(G, n)
    assert len(w) == n and np.all(w > 0) and abs(np.sum(w) - 4 * math.pi) < 1e-13
    err = _harmonic_errors(ux, uy, uz, w, p + 1)
    assert np.max(err[:p + 1]) < 2e-14 and err[p + 1] > 1e-4
    pts = {(round(a, 12), round(b, 12), round(c, 12)) for a, b, c in zip(ux, uy, uz)}
    for a, b, c in list(pts)[:50]:
        for perm in itertools.permutations((a, b, c)):
            for sg in itertools.product((1, -1), repeat=3):
                assert tuple(round(sg[k] * perm[k], 12) + 0.0 for k in range(3)) in pts


def test_library_rejects_unknown_lebedev_size():
    G = pytest.importorskip("paper_2007_03143_gb300")
    try:
        G.lib()
    except G.LibraryMissing as e:
        pytest.skip(str(e))
    ctx = G.gbxc_create(-1)
    try:
        mid, _ = G.gbxc_load_basis(ctx, np.zeros((1, 3)), np.array([1], np.int32), np.array([0], np.int32),
                                   np.array([0], np.int32), np.array([1], np.int32), np.array([[1.0]]),
                                   np.array([[1.0]]))
        with pytest.raises(G.GbxcError):
            G.gbxc_load_grid(ctx, mid, 10, 100, 0, "becke", 128, 1e-10, 5.0, "lebedev")
    finally:
        G.gbxc_destroy(ctx)
