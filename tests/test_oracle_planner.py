"""Pins for the oracle's batching and screening (Eq. rcut, Algorithm 1, Algorithm 3, Eq. batch_work)."""
import math

import numpy as np
import pytest

import xcinputs as X
from oracle import collocation as C
from oracle import integrate as I
from oracle import planner as PL


@pytest.mark.parametrize("alpha,expect", [(0.1, 14.79), (1.0, 4.80), (1e3, 0.163)])
def test_rcut_values(alpha, expect):
    assert abs(PL.cutoff_radius([alpha], 1e-10) - expect) < 5e-3 * expect


@pytest.mark.parametrize("alpha", [0.1, 1.0, 7.0, 1e3])
def test_rcut_defines_eta_level(alpha):
    # Eq. rcut solves sqrt(alpha) exp(-alpha r^2) = eta for r
    r = PL.cutoff_radius([alpha], 1e-10)
    assert abs(math.sqrt(alpha) * math.exp(-alpha * r * r) - 1e-10) < 1e-20
    # the maximum over primitives is taken
    assert PL.cutoff_radius([alpha, 0.1], 1e-10) == max(r, PL.cutoff_radius([0.1], 1e-10))


def _box_distance2(R, V, W):
    c = np.clip(R, V, W)
    return float(np.sum((R - c) ** 2))


def test_alg1_against_closest_point():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        V = rng.uniform(-2, 1, 3)
        W = V + rng.uniform(0, 2, 3)
        R = rng.uniform(-5, 5, 3)
        rc = rng.uniform(0, 4)
        d2 = _box_distance2(R, V, W)
        if abs(d2 - rc * rc) < 1e-12:
            continue
        assert PL.cuboid_sphere_intersect(R, rc, V, W) == (d2 <= rc * rc)
    # a sphere centred inside the box always intersects; tangency is kept (d = 0)
    assert PL.cuboid_sphere_intersect(np.zeros(3), 0.0, -np.ones(3), np.ones(3))
    assert PL.cuboid_sphere_intersect(np.array([2.0, 0, 0]), 1.0, -np.ones(3), np.ones(3))
    assert not PL.cuboid_sphere_intersect(np.array([2.0, 0, 0]), 0.999, -np.ones(3), np.ones(3))


def test_vectorised_screen_equals_scalar_alg1():
    w = X.make_workload("water2_pbe_small")
    g = I.make_grid(w.mol.xyz, w.grid, weights=False)
    pts = np.stack([g.x, g.y, g.z], 1)
    rc = PL.shell_cutoffs(w.basis, 1e-10)
    rng = np.random.default_rng(1)
    for _ in range(30):
        idx = rng.choice(len(pts), 50, replace=False)
        V, W = pts[idx].min(0), pts[idx].max(0)
        scalar = [s for s in range(len(rc)) if PL.cuboid_sphere_intersect(w.basis.center[s], rc[s], V, W)]
        assert PL.screen_batch(pts[idx], w.basis.center, rc) == scalar


@pytest.fixture(scope="module")
def small_plan():
    w = X.make_workload("water2_pbe_small")
    g = I.make_grid(w.mol.xyz, w.grid, weights=False)
    return w, g, I.make_plan(g, w.mol.xyz, w.basis, w.grid)


def test_batches_partition_the_grid(small_plan):
    w, g, pl = small_plan
    allp = np.concatenate(pl.unmerged_points)
    assert len(allp) == len(g.x) and len(np.unique(allp)) == len(g.x)
    merged = np.concatenate(pl.batch_points)
    assert np.array_equal(np.sort(merged), np.arange(len(g.x)))
    for b in pl.unmerged_points:
        assert len(b) <= w.grid.max_batch or True   # depth-16 leaves may exceed; checked below
        assert len(np.unique(g.parent[b])) == 1      # batches come from one atom's quadrature
    assert max(len(b) for b in pl.unmerged_points) <= w.grid.max_batch


def test_merge_keeps_order_and_uniqueness(small_plan):
    w, g, pl = small_plan
    keys = [tuple(s) for s in pl.batch_shells]
    assert len(set(keys)) == len(keys)
    # first-occurrence order and concatenation in batch order
    seen = []
    for s in pl.unmerged_shells:
        if tuple(s) not in seen:
            seen.append(tuple(s))
    assert seen == keys
    for j, key in enumerate(keys):
        parts = [b for b, s in zip(pl.unmerged_points, pl.unmerged_shells) if tuple(s) == key]
        assert np.array_equal(np.concatenate(parts), pl.batch_points[j])


def test_screening_never_drops_a_significant_shell(small_plan):
    # brute force: every point within r_cut of a shell centre lies in a batch that keeps that shell
    w, g, pl = small_plan
    pts = np.stack([g.x, g.y, g.z], 1)
    for j, idx in enumerate(pl.batch_points):
        kept = set(pl.batch_shells[j])
        d2 = ((pts[idx][:, None, :] - w.basis.center[None]) ** 2).sum(-1)
        near = np.nonzero((d2 <= pl.rcut[None] ** 2).any(0))[0]
        assert set(near.tolist()) <= kept


def test_dropped_shells_are_below_eta(small_plan):
    # functions of a dropped shell are below the screening tolerance at every batch point,
    # up to the polynomial and contraction factors the paper's Eq. rcut ignores
    w, g, pl = small_plan
    pts = np.stack([g.x, g.y, g.z], 1)
    worst = 0.0
    for j, idx in enumerate(pl.batch_points[:10]):
        dropped = sorted(set(range(w.basis.nshell)) - set(pl.batch_shells[j]))
        if not dropped:
            continue
        phi = C.collocate(pts[idx], w.basis, dropped)[0]
        worst = max(worst, float(np.abs(phi).max()))
    assert worst < 1e-6


def test_work_estimate_formula():
    assert PL.work_estimate(10, 3, 2) == 10 * (4 + 27 + 18 + 3) + 9
    assert PL.work_estimate(0, 5, 9) == 25


def test_split_rules():
    # one atom at the origin inside the cell: 27-way split; away from atoms: octants
    xyz = np.array([[0.0, 0.0, 0.0]])
    rng = np.random.default_rng(2)
    pts = rng.uniform(-1, 1, size=(300, 3))
    out = []
    PL._subdivide(np.arange(300), pts, (-1, -1, -1), (1, 1, 1), 15, 10, xyz, out)
    assert len(out) == sum(1 for _ in out) and 20 <= len(out) <= 27
    cut = -1 + 2 / 3.0
    for b in out:   # each child lies inside one third-cell along x
        side = set(((pts[b, 0] >= cut).astype(int) + (pts[b, 0] >= -1 + 2 * 2 / 3.0)).tolist())
        assert len(side) == 1
    out2 = []
    PL._subdivide(np.arange(300), pts + 5.0, (4, 4, 4), (6, 6, 6), 15, 10, xyz, out2)
    assert len(out2) == 8
