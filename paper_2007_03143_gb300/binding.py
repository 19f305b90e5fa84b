"""ctypes binding of the gbxc C-ABI (``include/gbxc.h``).

Argument marshalling only: every step of the integration runs in the CUDA
library.  Functions keep the C names.  Arrays may be NumPy arrays (host) or
torch tensors (host or CUDA); device tensors are passed as device pointers and
the current torch CUDA stream is used unless a stream is given.

If the shared library has not been built, importing the binding succeeds but
every call raises ``LibraryMissing``: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_longlong, c_size_t, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libgbxc.so")

GBXC_OK, GBXC_EINVAL, GBXC_ENOMEM, GBXC_ECUDA, GBXC_ETIMEOUT, GBXC_ENOTREADY, GBXC_ENOENT = \
    0, -1, -2, -3, -4, -5, -6
GBXC_BECKE, GBXC_SSF = 0, 1
GBXC_SLATER, GBXC_PBE, GBXC_MVS_X, GBXC_PBE0_SL = 0, 1, 2, 3
GBXC_FP64, GBXC_MIXED = 0, 1
GBXC_ANGULAR_PRODUCT, GBXC_ANGULAR_LEBEDEV = 0, 1
GBXC_MAX_PRIM = 8
GBXC_MAX_L = 3

FUNCTIONALS = {"slater": GBXC_SLATER, "pbe": GBXC_PBE, "mvs_x": GBXC_MVS_X, "pbe0_sl": GBXC_PBE0_SL}
PARTITIONS = {"becke": GBXC_BECKE, "ssf": GBXC_SSF}
PRECISIONS = {"fp64": GBXC_FP64, "mixed": GBXC_MIXED}
ANGULAR = {"product": GBXC_ANGULAR_PRODUCT, "lebedev": GBXC_ANGULAR_LEBEDEV}

EXPORTED = ["gbxc_create", "gbxc_destroy", "gbxc_last_error", "gbxc_load_basis", "gbxc_load_grid",
            "gbxc_plan_info_get", "gbxc_export_plan", "gbxc_integrate", "gbxc_integrate_batches",
            "gbxc_profile_enable", "gbxc_profile_read", "gbxc_integrate_fp64_noalloc",
            "gbxc_integrate_many", "gbxc_serve_start", "gbxc_serve_stop", "gbxc_submit", "gbxc_wait",
            "gbxc_serve_stats", "gbxc_autotune", "gbxc_set_schedule", "gbxc_load_grid_device",
            "gbxc_load_basis_pure", "gbxc_integrate_uks", "gbxc_unload", "gbxc_save_plan", "gbxc_load_plan",
            "gbxc_debug_batch"]
KERNEL_CLASSES = ["weights", "colloc", "xgemm", "rho_z", "vgemm", "finish", "pgather", "graph", "vslice"]
GBXC_NKERNEL = len(KERNEL_CLASSES)


class LibraryMissing(ImportError):
    pass


class GbxcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gbxc error {code}: {msg}")
        self.code = code


class GridSpec(ctypes.Structure):
    _fields_ = [("nrad", c_int), ("ntheta", c_int), ("nphi", c_int), ("partition", c_int),
                ("max_batch", c_int), ("eta", c_double), ("mk_alpha", c_double), ("angular", c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("natoms", c_int), ("nshell", c_int), ("nbf", c_int), ("npts", c_longlong),
                ("nbatch", c_int), ("nleaf", c_int), ("nshell_entries", c_longlong),
                ("nfunc_entries", c_longlong), ("ntiles", c_longlong), ("sum_mn2", c_double),
                ("work", c_double), ("sum_mn", c_double), ("sum_ms", c_double), ("sum_n2", c_double),
                ("max_nfunc", c_int)]


_lib = None


def lib():
    """The loaded shared library (raises LibraryMissing if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LibraryMissing(f"{LIB_PATH} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    pd = POINTER(c_double)
    L.gbxc_create.argtypes = [POINTER(c_void_p), c_int, c_size_t]
    L.gbxc_destroy.argtypes = [c_void_p]
    L.gbxc_destroy.restype = None
    L.gbxc_last_error.argtypes = [c_void_p]
    L.gbxc_last_error.restype = ctypes.c_char_p
    L.gbxc_load_basis.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, POINTER(c_int), POINTER(c_int)]
    L.gbxc_load_basis_pure.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int), POINTER(c_int)]
    L.gbxc_load_basis_pure.restype = c_int
    L.gbxc_integrate_uks.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int, pd, c_void_p, c_void_p,
                                     pd, c_void_p]
    L.gbxc_integrate_uks.restype = c_int
    L.gbxc_load_grid.argtypes = [c_void_p, c_int, POINTER(GridSpec), POINTER(c_longlong), POINTER(c_int)]
    L.gbxc_load_grid_device.argtypes = [c_void_p, c_int, POINTER(GridSpec), POINTER(c_longlong), POINTER(c_int)]
    L.gbxc_load_grid_device.restype = c_int
    L.gbxc_unload.argtypes = [c_void_p, c_int]
    L.gbxc_unload.restype = c_int
    L.gbxc_debug_batch.argtypes = [c_void_p, c_int, c_int, c_void_p, c_int, c_int] + [c_void_p] * 5
    L.gbxc_debug_batch.restype = c_int
    L.gbxc_save_plan.argtypes = [c_void_p, c_int, ctypes.c_char_p]
    L.gbxc_save_plan.restype = c_int
    L.gbxc_load_plan.argtypes = [c_void_p, c_int, ctypes.c_char_p, POINTER(c_longlong), POINTER(c_int)]
    L.gbxc_load_plan.restype = c_int
    L.gbxc_plan_info_get.argtypes = [c_void_p, c_int, POINTER(PlanInfo)]
    L.gbxc_export_plan.argtypes = [c_void_p, c_int] + [c_void_p] * 10
    L.gbxc_integrate.argtypes = [c_void_p, c_int, c_void_p, c_int, c_int, pd, c_void_p, pd, c_void_p]
    L.gbxc_integrate_batches.argtypes = [c_void_p, c_int, c_void_p, c_int, c_int, c_int, c_int, pd,
                                         c_void_p, pd, c_void_p, c_void_p, c_void_p]
    L.gbxc_integrate_fp64_noalloc.argtypes = [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p,
                                               c_void_p]
    L.gbxc_integrate_fp64_noalloc.restype = c_int
    L.gbxc_integrate_many.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                                      c_void_p, c_void_p]
    L.gbxc_autotune.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, POINTER(c_int),
                                POINTER(c_int), POINTER(c_double)]
    L.gbxc_set_schedule.argtypes = [c_void_p, c_int, c_void_p, c_int, c_int, c_int]
    L.gbxc_serve_start.argtypes = [c_void_p, c_int, c_size_t]
    L.gbxc_serve_stop.argtypes = [c_void_p]
    L.gbxc_submit.argtypes = [c_void_p, c_int, c_void_p, c_int, c_int, POINTER(c_longlong)]
    L.gbxc_wait.argtypes = [c_void_p, c_longlong, c_double, c_void_p, c_void_p, c_void_p, c_void_p]
    L.gbxc_serve_stats.argtypes = [c_void_p] + [c_void_p] * 5
    for name in ("gbxc_integrate_many", "gbxc_serve_start", "gbxc_serve_stop", "gbxc_submit", "gbxc_wait",
                 "gbxc_serve_stats", "gbxc_autotune", "gbxc_set_schedule"):
        getattr(L, name).restype = c_int
    L.gbxc_measure_alu_peaks.argtypes = [c_int, pd, pd]
    L.gbxc_measure_alu_peaks.restype = c_int
    L.gbxc_profile_enable.argtypes = [c_void_p, c_int]
    L.gbxc_profile_read.argtypes = [c_void_p, c_void_p, c_void_p]
    for name in ("gbxc_create", "gbxc_load_basis", "gbxc_load_grid", "gbxc_plan_info_get",
                 "gbxc_export_plan", "gbxc_integrate", "gbxc_integrate_batches",
                 "gbxc_profile_enable", "gbxc_profile_read"):
        getattr(L, name).restype = c_int
    _lib = L
    return L


def _ptr(a):
    """(pointer, keepalive, is_cuda) of a NumPy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, None, False
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, a, False
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), a, a.is_cuda
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_for(stream, *arrays):
    if stream is not None:
        return stream
    for a in arrays:
        if a is not None and hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _check(ctx, rc):
    if rc != GBXC_OK:
        msg = lib().gbxc_last_error(ctx).decode() if ctx else ""
        raise GbxcError(rc, msg)


def gbxc_create(device: int = 0, scratch_bytes: int = 0):
    h = c_void_p()
    rc = lib().gbxc_create(ctypes.byref(h), device, scratch_bytes)
    if rc != GBXC_OK:
        raise GbxcError(rc, "gbxc_create failed (no CUDA device?)")
    return h


def gbxc_destroy(ctx):
    lib().gbxc_destroy(ctx)


def gbxc_last_error(ctx) -> str:
    return lib().gbxc_last_error(ctx).decode()


def gbxc_load_basis(ctx, xyz, Z, shell_atom, shell_L, shell_nprim, alpha, coeff, pure=None):
    """Register a molecule; returns (mol_id, nbf).  alpha/coeff: (nshell, <=8) arrays;
    pure: optional per-shell flags (spherical shells for L >= 2)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    sa = np.ascontiguousarray(shell_atom, dtype=np.int32)
    sL = np.ascontiguousarray(shell_L, dtype=np.int32)
    sn = np.ascontiguousarray(shell_nprim, dtype=np.int32)
    nsh = len(sL)
    al = np.zeros((nsh, GBXC_MAX_PRIM))
    co = np.zeros((nsh, GBXC_MAX_PRIM))
    alpha = np.asarray(alpha, dtype=np.float64)
    coeff = np.asarray(coeff, dtype=np.float64)
    al[:, :alpha.shape[1]] = alpha
    co[:, :coeff.shape[1]] = coeff
    mol, nbf = c_int(), c_int()
    sp = None if pure is None else np.ascontiguousarray(pure, dtype=np.int32)
    _check(ctx, lib().gbxc_load_basis_pure(ctx, len(Z), xyz.ctypes.data, Z.ctypes.data, nsh, sa.ctypes.data,
                                           sL.ctypes.data, sn.ctypes.data, None if sp is None else sp.ctypes.data,
                                           al.ctypes.data, co.ctypes.data, ctypes.byref(mol), ctypes.byref(nbf)))
    return mol.value, nbf.value


def _grid_spec(nrad, ntheta, nphi, partition, max_batch, eta, mk_alpha, angular):
    return GridSpec(nrad, ntheta, nphi, PARTITIONS.get(partition, partition), max_batch, eta, mk_alpha,
                    ANGULAR.get(angular, angular))


def gbxc_load_grid(ctx, mol, nrad, ntheta, nphi, partition, max_batch, eta=1e-10, mk_alpha=5.0,
                   angular="product"):
    """angular: "product" (ntheta x nphi) or "lebedev" (the rule of ntheta points)."""
    spec = _grid_spec(nrad, ntheta, nphi, partition, max_batch, eta, mk_alpha, angular)
    npts, nb = c_longlong(), c_int()
    _check(ctx, lib().gbxc_load_grid(ctx, mol, ctypes.byref(spec), ctypes.byref(npts), ctypes.byref(nb)))
    return npts.value, nb.value


def gbxc_load_grid_device(ctx, mol, nrad, ntheta, nphi, partition, max_batch, eta=1e-10, mk_alpha=5.0,
                          angular="product"):
    """gbxc_load_grid with the planner's kernels on the device (identical plan)."""
    spec = _grid_spec(nrad, ntheta, nphi, partition, max_batch, eta, mk_alpha, angular)
    npts, nb = c_longlong(), c_int()
    _check(ctx, lib().gbxc_load_grid_device(ctx, mol, ctypes.byref(spec), ctypes.byref(npts), ctypes.byref(nb)))
    return npts.value, nb.value


def gbxc_unload(ctx, mol):
    _check(ctx, lib().gbxc_unload(ctx, mol))


def gbxc_debug_batch(ctx, mol, batch, P, functional, precision, m, n):
    """Phi, grad Phi (3) and Z of one batch as m x n float64 arrays (see gbxc.h)."""
    out = [np.zeros((m, n)) for _ in range(5)]
    pP, kP, _ = _ptr(P)
    _check(ctx, lib().gbxc_debug_batch(ctx, mol, batch, pP, FUNCTIONALS.get(functional, functional),
                                       PRECISIONS.get(precision, precision), *[o.ctypes.data for o in out]))
    return out


def gbxc_save_plan(ctx, mol, path):
    _check(ctx, lib().gbxc_save_plan(ctx, mol, os.fsencode(path)))


def gbxc_load_plan(ctx, mol, path):
    """Make the plan file at `path` the grid of `mol`; returns (npts, nbatch)."""
    npts, nb = c_longlong(), c_int()
    _check(ctx, lib().gbxc_load_plan(ctx, mol, os.fsencode(path), ctypes.byref(npts), ctypes.byref(nb)))
    return npts.value, nb.value


def gbxc_plan_info_get(ctx, mol) -> dict:
    info = PlanInfo()
    _check(ctx, lib().gbxc_plan_info_get(ctx, mol, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in PlanInfo._fields_}


def gbxc_export_plan(ctx, mol) -> dict:
    info = gbxc_plan_info_get(ctx, mol)
    n, nb = info["npts"], info["nbatch"]
    out = dict(x=np.empty(n), y=np.empty(n), z=np.empty(n), wq=np.empty(n), w=np.empty(n),
               parent=np.empty(n, np.int32), point_index=np.empty(n, np.int64),
               batch_ptr=np.empty(nb + 1, np.int64), shell_ptr=np.empty(nb + 1, np.int64),
               shell_idx=np.empty(max(info["nshell_entries"], 1), np.int32))
    order = ["x", "y", "z", "wq", "w", "parent", "point_index", "batch_ptr", "shell_ptr", "shell_idx"]
    _check(ctx, lib().gbxc_export_plan(ctx, mol, *[out[k].ctypes.data for k in order]))
    out["shell_idx"] = out["shell_idx"][:info["nshell_entries"]]
    return out


def gbxc_integrate(ctx, mol, P, functional="pbe", precision="fp64", V=None, stream=None):
    """Returns (E_xc, N_el); fills V (nbf x nbf, host array or CUDA tensor) if given."""
    pP, kP, _ = _ptr(P)
    pV, kV, _ = _ptr(V)
    st = _stream_for(stream, P, V)
    E, N = c_double(), c_double()
    _check(ctx, lib().gbxc_integrate(ctx, mol, pP, FUNCTIONALS.get(functional, functional),
                                     PRECISIONS.get(precision, precision), ctypes.byref(E), pV,
                                     ctypes.byref(N), st))
    return E.value, N.value


def gbxc_integrate_uks(ctx, mol, Pa, Pb, functional="pbe", precision="fp64", Va=None, Vb=None, stream=None):
    """Spin-unrestricted integration; returns (E_xc, N_el); fills Va, Vb if given."""
    pA, kA, _ = _ptr(Pa)
    pB, kB, _ = _ptr(Pb)
    pVa, kVa, _ = _ptr(Va)
    pVb, kVb, _ = _ptr(Vb)
    st = _stream_for(stream, Pa, Va)
    E, N = c_double(), c_double()
    _check(ctx, lib().gbxc_integrate_uks(ctx, mol, pA, pB, FUNCTIONALS.get(functional, functional),
                                         PRECISIONS.get(precision, precision), ctypes.byref(E), pVa, pVb,
                                         ctypes.byref(N), st))
    return E.value, N.value


def gbxc_integrate_batches(ctx, mol, P, functional, precision, batch_begin, batch_end, V=None,
                           E_batch=None, N_batch=None, stream=None):
    pP, kP, _ = _ptr(P)
    pV, kV, _ = _ptr(V)
    pE, kE, _ = _ptr(E_batch)
    pN, kN, _ = _ptr(N_batch)
    st = _stream_for(stream, P, V)
    E, N = c_double(), c_double()
    _check(ctx, lib().gbxc_integrate_batches(ctx, mol, pP, FUNCTIONALS.get(functional, functional),
                                             PRECISIONS.get(precision, precision), batch_begin,
                                             batch_end, ctypes.byref(E), pV, ctypes.byref(N), pE, pN, st))
    return E.value, N.value


def gbxc_integrate_fp64_noalloc(ctx, mol, P, V, EN, functional="pbe", stream=None):
    """Float64 integration without device allocation; P, V (nbf x nbf) and EN (2) are CUDA
    tensors.  Queued on the stream (torch's current stream by default); does not wait."""
    pP, kP, cP = _ptr(P)
    pV, kV, cV = _ptr(V)
    pE, kE, cE = _ptr(EN)
    if not (cP and cV and cE):
        raise ValueError("P, V and EN must be CUDA tensors")
    st = _stream_for(stream, P)
    _check(ctx, lib().gbxc_integrate_fp64_noalloc(ctx, mol, pP, FUNCTIONALS.get(functional, functional),
                                                  pV, pE, st))


def gbxc_integrate_many(ctx, mols, Ps, functionals, precision="fp64", Vs=None):
    """One graph launch over several molecules; returns (E array, N array)."""
    n = len(mols)
    ids = np.ascontiguousarray(mols, dtype=np.int32)
    fns = np.ascontiguousarray([FUNCTIONALS.get(f, f) for f in functionals], dtype=np.int32)
    keep = [_ptr(P) for P in Ps]
    pP = (c_void_p * n)(*[k[0] for k in keep])
    vkeep = [_ptr(V) for V in Vs] if Vs is not None else None
    pV = (c_void_p * n)(*[k[0] for k in vkeep]) if vkeep else None
    E = np.zeros(n)
    N = np.zeros(n)
    _check(ctx, lib().gbxc_integrate_many(ctx, n, ids.ctypes.data, pP, fns.ctypes.data,
                                          PRECISIONS.get(precision, precision), E.ctypes.data, pV,
                                          N.ctypes.data))
    return E, N


def gbxc_autotune(ctx, mols, Ps, functionals, precision="mixed"):
    """Pick the fastest batching schedule for this molecule list; returns (branches, tile_n, ms)."""
    n = len(mols)
    ids = np.ascontiguousarray(mols, dtype=np.int32)
    fns = np.ascontiguousarray([FUNCTIONALS.get(f, f) for f in functionals], dtype=np.int32)
    keep = [_ptr(P) for P in Ps]
    pP = (c_void_p * n)(*[k[0] for k in keep])
    w, t, ms = c_int(), c_int(), c_double()
    _check(ctx, lib().gbxc_autotune(ctx, n, ids.ctypes.data, pP, fns.ctypes.data,
                                    PRECISIONS.get(precision, precision), ctypes.byref(w), ctypes.byref(t),
                                    ctypes.byref(ms)))
    return w.value, t.value, ms.value


def gbxc_set_schedule(ctx, mols, precision, branches, tile_n):
    ids = np.ascontiguousarray(mols, dtype=np.int32)
    _check(ctx, lib().gbxc_set_schedule(ctx, len(mols), ids.ctypes.data, PRECISIONS.get(precision, precision),
                                        branches, tile_n))


def gbxc_serve_start(ctx, nslots=4, arena_bytes=0):
    _check(ctx, lib().gbxc_serve_start(ctx, nslots, arena_bytes))


def gbxc_serve_stop(ctx):
    _check(ctx, lib().gbxc_serve_stop(ctx))


def gbxc_submit(ctx, mol, P, functional="pbe", precision="mixed"):
    P = np.ascontiguousarray(P, dtype=np.float64)
    t = c_longlong()
    _check(ctx, lib().gbxc_submit(ctx, mol, P.ctypes.data, FUNCTIONALS.get(functional, functional),
                                  PRECISIONS.get(precision, precision), ctypes.byref(t)))
    return t.value


def gbxc_wait(ctx, ticket, timeout_s=60.0, V=None):
    """Returns (E, N, latency_s); fills V (host array) if given."""
    E, N, lat = c_double(), c_double(), c_double()
    pV, kV, _ = _ptr(V)
    _check(ctx, lib().gbxc_wait(ctx, ticket, timeout_s, ctypes.byref(E), pV, ctypes.byref(N), ctypes.byref(lat)))
    return E.value, N.value, lat.value


def gbxc_serve_stats(ctx) -> dict:
    q, r, c = c_longlong(), c_longlong(), c_longlong()
    f, cap = c_size_t(), c_size_t()
    _check(ctx, lib().gbxc_serve_stats(ctx, ctypes.byref(q), ctypes.byref(r), ctypes.byref(c), ctypes.byref(f),
                                       ctypes.byref(cap)))
    return dict(queued=q.value, running=r.value, completed=c.value, arena_free=f.value, arena_cap=cap.value)


def gbxc_profile_enable(ctx, on=True):
    _check(ctx, lib().gbxc_profile_enable(ctx, int(bool(on))))


def gbxc_profile_read(ctx) -> dict:
    """{kernel class: (milliseconds, launches)} since the last enable/disable."""
    ms = np.zeros(GBXC_NKERNEL)
    n = np.zeros(GBXC_NKERNEL, np.int64)
    _check(ctx, lib().gbxc_profile_read(ctx, ms.ctypes.data, n.ctypes.data))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}


def gbxc_measure_alu_peaks(device=0):
    """(float32, float64) FMA throughput of the device in TFLOP/s, measured."""
    a, b = c_double(), c_double()
    rc = lib().gbxc_measure_alu_peaks(device, ctypes.byref(a), ctypes.byref(b))
    if rc != GBXC_OK:
        raise GbxcError(rc, "ALU peak measurement failed")
    return a.value, b.value


class Context:
    """Convenience owner of a gbxc context."""

    def __init__(self, device: int = 0, scratch_bytes: int = 0):
        self.h = gbxc_create(device, scratch_bytes)

    def close(self):
        if self.h is not None:
            gbxc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_molecule(self, mol, basis, grid, device_planner=False):
        """Register an ``xcinputs`` Molecule/Basis pair and build its grid; returns the id."""
        mid, nbf = gbxc_load_basis(self.h, mol.xyz, mol.Z, basis.atom, basis.L, basis.nprim,
                                   basis.alpha, basis.coeff, getattr(basis, "pure", None))
        load = gbxc_load_grid_device if device_planner else gbxc_load_grid
        load(self.h, mid, grid.nrad, grid.ntheta, grid.nphi, grid.partition, grid.max_batch, grid.eta,
             grid.mk_alpha, getattr(grid, "angular", "product"))
        return mid
