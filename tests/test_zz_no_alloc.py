"""The allocation-free float64 entry point (gbxc_integrate_fp64_noalloc) against gbxc_integrate.

Callers that cannot allocate device memory (code running inside another allocator's pool or
in a pre-reserved memory region) use this call: its scratch is a static array inside the
library, and P, V and {E, N} are the caller's device buffers.  It must give the float64
path's results, within the float64 tolerance (1e-9), on two calls in a row, since every
call reuses the same static array.  This file is collected last on purpose."""
import numpy as np
import pytest

import xcinputs as X
from gpu_common import Loaded

ROW_BYTES = 8 * 128 * 8                      # eight float64 planes of a 128-point tile row
STATIC_ROWS = ((64 << 20) - 256) // ROW_BYTES   # slab rows of the static array

pytestmark = pytest.mark.gpu


def _slab_rows(L):
    """Padded slab rows of the molecule's tiles: the sum over batches of ceil(m_j / 128)
    tiles times N_b^j rounded up to 32 (the float64 slabs' row count)."""
    plan = L.export()
    nf = np.array([X.nfunc(int(l), int(p)) for l, p in zip(L.w.basis.L, L.w.basis.pure)])
    rows = 0
    for j in range(len(plan["batch_ptr"]) - 1):
        m = int(plan["batch_ptr"][j + 1] - plan["batch_ptr"][j])
        sh = plan["shell_idx"][plan["shell_ptr"][j]:plan["shell_ptr"][j + 1]]
        n = int(nf[sh].sum())
        rows += -(-m // 128) * (-(-n // 32) * 32)
    return rows


# water3_pbe_small needs about 30,000 slab rows, against the 8,191 rows (8 KiB each) the
# 64 MiB static array holds, so its call runs the chunk loop several times.
@pytest.mark.parametrize("name", ["water2_pbe_small", "water1_slater", "water3_pbe_small"])
def test_noalloc_matches_fp64_twice(name):
    import torch
    L = Loaded(name)
    try:
        G = L.G
        nbf = L.w.basis.nbf
        E_ref, N_ref, V_ref = L.integrate("fp64")
        Pd = torch.tensor(L.w.P, device="cuda")
        for call in range(2):
            Vd = torch.full((nbf, nbf), float("nan"), dtype=torch.float64, device="cuda")
            EN = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
            G.gbxc_integrate_fp64_noalloc(L.ctx.h, L.mid, Pd, Vd, EN, L.w.functional)
            torch.cuda.synchronize()
            E, N = EN.cpu().numpy()
            V = Vd.cpu().numpy()
            assert abs(E - E_ref) <= 1e-9, call
            assert abs(N - N_ref) <= 1e-9, call
            assert np.max(np.abs(V - V_ref)) <= 1e-9, call
            assert np.array_equal(V, V.T), call
    finally:
        L.close()


def test_noalloc_rejects_host_buffers():
    import torch
    L = Loaded("water1_slater")
    try:
        G = L.G
        nbf = L.w.basis.nbf
        with pytest.raises(ValueError):
            G.gbxc_integrate_fp64_noalloc(L.ctx.h, L.mid, torch.tensor(L.w.P), torch.zeros((nbf, nbf),
                                          dtype=torch.float64), torch.zeros(2, dtype=torch.float64))
        rc = G.lib().gbxc_integrate_fp64_noalloc(L.ctx.h, L.mid, L.w.P.ctypes.data, 0,
                                                 np.zeros((nbf, nbf)).ctypes.data, np.zeros(2).ctypes.data,
                                                 None)
        assert rc == G.GBXC_EINVAL
    finally:
        L.close()


def test_noalloc_multi_chunk_workload_is_split():
    """The chunk loop of the call runs more than once on water3_pbe_small (host arithmetic
    only: the slab rows the plan needs against the rows the static array holds)."""
    L = Loaded("water3_pbe_small")
    try:
        assert _slab_rows(L) > STATIC_ROWS
    finally:
        L.close()


def test_noalloc_on_a_caller_stream():
    """Work queued on a caller-created stream, read after synchronising that stream only."""
    import torch
    L = Loaded("water2_pbe_small")
    try:
        G = L.G
        nbf = L.w.basis.nbf
        E_ref, N_ref, V_ref = L.integrate("fp64")
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            Pd = torch.tensor(L.w.P, device="cuda")
            Vd = torch.empty((nbf, nbf), dtype=torch.float64, device="cuda")
            EN = torch.empty(2, dtype=torch.float64, device="cuda")
        st.synchronize()
        for call in range(2):
            G.gbxc_integrate_fp64_noalloc(L.ctx.h, L.mid, Pd, Vd, EN, L.w.functional, stream=st.cuda_stream)
            st.synchronize()
            E, N = EN.cpu().numpy()
            assert abs(E - E_ref) <= 1e-9 and abs(N - N_ref) <= 1e-9, call
            assert np.max(np.abs(Vd.cpu().numpy() - V_ref)) <= 1e-9, call
    finally:
        L.close()


def test_noalloc_nonfinite_P_gives_nan_results():
    """A NaN (then an infinity) planted in P on the host: the call cannot return a status
    for it, so E_xc and N_el come back NaN; a clean P afterwards gives the float64 results."""
    import torch
    L = Loaded("water1_slater")
    try:
        G = L.G
        nbf = L.w.basis.nbf
        E_ref, N_ref, V_ref = L.integrate("fp64")
        Vd = torch.zeros((nbf, nbf), dtype=torch.float64, device="cuda")
        EN = torch.zeros(2, dtype=torch.float64, device="cuda")
        for bad in (float("nan"), float("inf")):
            P = L.w.P.copy()
            P[3, 7] = P[7, 3] = bad
            G.gbxc_integrate_fp64_noalloc(L.ctx.h, L.mid, torch.tensor(P, device="cuda"), Vd, EN, L.w.functional)
            torch.cuda.synchronize()
            E, N = EN.cpu().numpy()
            assert np.isnan(E) and np.isnan(N), bad
        G.gbxc_integrate_fp64_noalloc(L.ctx.h, L.mid, torch.tensor(L.w.P, device="cuda"), Vd, EN, L.w.functional)
        torch.cuda.synchronize()
        E, N = EN.cpu().numpy()
        assert abs(E - E_ref) <= 1e-9 and abs(N - N_ref) <= 1e-9
        assert np.max(np.abs(Vd.cpu().numpy() - V_ref)) <= 1e-9
    finally:
        L.close()
