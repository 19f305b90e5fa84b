"""Batching and basis-shell screening (Sec. 2.2, Eq. rcut, Algorithm 1, Algorithm 3).

Steps, in the paper's order:

1. Screening radius per shell (Eq. rcut):
   r_cut = max_xi sqrt((ln(alpha_xi)/2 - ln(eta)) / alpha_xi).
2. Batches from each atom's own quadrature (Algorithm 3 builds batches atom
   by atom): recursive cuboid subdivision until a cell holds at most
   ``max_batch`` points.  A cell that contains an atomic centre is cut into
   3 x 3 x 3 cuboids, any other cell into octants (grid-partition figure).
3. Shell screening of each batch by the cuboid-sphere test of Algorithm 1.
4. Work estimate W_j (Eq. batch_work) and merging of batches that share the
   same shell list (Algorithm 3's final step).

Readings where the paper is silent or its print is garbled:

* Algorithm 1 prints ``W_o`` for ``W_p`` and returns ``d < 0`` for "intersects";
  read as: d = r_cut^2 - (squared distance from the shell centre to the box),
  and the shell is kept iff d >= 0.  Computed as printed: start from r_cut*r_cut
  and subtract (R_p - V_p)^2 when R_p < V_p, else (R_p - W_p)^2 when R_p > W_p.
* Initial cell: the tight bounding box of the atom's points.  A cell "contains
  an atomic centre" when lo <= R <= hi on all three axes, for any atom.
  Cuts: lo + (hi - lo)/3 and lo + 2*(hi - lo)/3 for the 27-way split, and
  0.5*(lo + hi) for the octant split; a point goes to the upper side iff its
  coordinate is >= the cut.  Children are visited z-major, then y, then x;
  empty children are dropped; a cell at depth 16 is a leaf whatever its size.
* The cuboid used for screening is the tight bounding box of the batch's
  points (not the subdivision cell).
* Merge: batches with identical shell lists are concatenated in order of first
  occurrence (points appended in batch order), with no size cap.
* Work estimate with N_A the number of atoms, N_b^j the number of basis
  functions of the batch and N_g^j its number of points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import elementary as el

MAX_DEPTH = 16


def cutoff_radius(alphas, eta: float) -> float:
    """r_cut of one shell (Eq. rcut); natural logarithms."""
    rc = 0.0
    for a in alphas:
        v = math.sqrt((el.ln(a) / 2.0 - el.ln(eta)) / a)
        if v > rc:
            rc = v
    return rc


def shell_cutoffs(basis, eta: float) -> np.ndarray:
    return np.array([cutoff_radius(basis.alpha[s, :basis.nprim[s]], eta) for s in range(basis.nshell)])


def cuboid_sphere_intersect(R, rcut: float, V, W) -> bool:
    """Algorithm 1 (typo W_o -> W_p and inverted return corrected, see module docstring)."""
    d = rcut * rcut
    for p in range(3):
        if R[p] < V[p]:
            d = d - (R[p] - V[p]) * (R[p] - V[p])
        elif R[p] > W[p]:
            d = d - (R[p] - W[p]) * (R[p] - W[p])
    return d >= 0.0


def _contains_atom(lo, hi, xyz) -> bool:
    for A in range(len(xyz)):
        R = xyz[A]
        if lo[0] <= R[0] <= hi[0] and lo[1] <= R[1] <= hi[1] and lo[2] <= R[2] <= hi[2]:
            return True
    return False


def _subdivide(idx, pts, lo, hi, depth, max_batch, xyz, out):
    """Append leaf batches (arrays of point indices, in input order) to ``out``."""
    if len(idx) <= max_batch or depth >= MAX_DEPTH:
        out.append(idx)
        return
    if _contains_atom(lo, hi, xyz):
        cuts = [[lo[d], lo[d] + (hi[d] - lo[d]) / 3.0, lo[d] + 2.0 * (hi[d] - lo[d]) / 3.0, hi[d]]
                for d in range(3)]
    else:
        cuts = [[lo[d], 0.5 * (lo[d] + hi[d]), hi[d]] for d in range(3)]
    P = pts[idx]
    cell = []
    for d in range(3):
        c = np.zeros(len(idx), dtype=np.int64)
        for k in range(1, len(cuts[d]) - 1):
            c += (P[:, d] >= cuts[d][k]).astype(np.int64)
        cell.append(c)
    nx, ny, nz = len(cuts[0]) - 1, len(cuts[1]) - 1, len(cuts[2]) - 1
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                sel = idx[(cell[0] == ix) & (cell[1] == iy) & (cell[2] == iz)]
                if len(sel) == 0:
                    continue
                clo = (cuts[0][ix], cuts[1][iy], cuts[2][iz])
                chi = (cuts[0][ix + 1], cuts[1][iy + 1], cuts[2][iz + 1])
                _subdivide(sel, pts, clo, chi, depth + 1, max_batch, xyz, out)


def atom_batches(pts, parent, natoms, xyz, max_batch):
    """Leaf batches of every atom's quadrature, atom by atom (point indices)."""
    out = []
    for A in range(natoms):
        idx = np.nonzero(parent == A)[0]
        P = pts[idx]
        lo = tuple(P.min(axis=0))
        hi = tuple(P.max(axis=0))
        _subdivide(idx, pts, lo, hi, 0, max_batch, xyz, out)
    return out


def screen_batch(pts_b, centers, rcut):
    """Sorted shell indices kept for one batch by Algorithm 1 on its bounding box.

    Vectorised over shells; every kept value is produced by exactly the
    operations of ``cuboid_sphere_intersect`` (same order, no fusion).
    """
    V = pts_b.min(axis=0)
    W = pts_b.max(axis=0)
    d = rcut * rcut
    for p in range(3):
        R = centers[:, p]
        below = R < V[p]
        above = R > W[p]
        dv = d - (R - V[p]) * (R - V[p])
        dw = d - (R - W[p]) * (R - W[p])
        d = np.where(below, dv, np.where(above, dw, d))
    return [int(s) for s in np.nonzero(d >= 0.0)[0]]


def work_estimate(ng: int, nb: int, natoms: int) -> float:
    """W_j of Eq. batch_work."""
    return ng * (natoms * natoms + 9 * nb + 2 * nb * nb + 3) + nb * nb


@dataclass
class Plan:
    batch_points: list        # list of int arrays (global point indices), merged batches
    batch_shells: list        # list of sorted shell-index lists
    batch_funcs: list         # list of int arrays (global function indices, sorted)
    work: np.ndarray          # W_j per merged batch
    rcut: np.ndarray          # per shell
    unmerged_points: list     # leaf batches before merging
    unmerged_shells: list


def make_plan(x, y, z, parent, xyz, basis, max_batch: int, eta: float) -> Plan:
    pts = np.stack([x, y, z], axis=1)
    rcut = shell_cutoffs(basis, eta)
    leaves = atom_batches(pts, parent, len(xyz), xyz, max_batch)
    shells = [screen_batch(pts[b], basis.center, rcut) for b in leaves]
    order, groups = [], {}
    for b, s in zip(leaves, shells):
        key = tuple(s)
        if key not in groups:
            groups[key] = []
            order.append(key)
        groups[key].append(b)
    bpts, bsh, bfn, work = [], [], [], []
    for key in order:
        p = np.concatenate(groups[key])
        f = np.concatenate([np.arange(basis.func_offset[s], basis.func_offset[s + 1]) for s in key]) \
            if len(key) else np.zeros(0, dtype=np.int64)
        bpts.append(p)
        bsh.append(list(key))
        bfn.append(f.astype(np.int64))
        work.append(work_estimate(len(p), len(f), len(xyz)))
    return Plan(bpts, bsh, bfn, np.array(work), rcut, leaves, shells)
