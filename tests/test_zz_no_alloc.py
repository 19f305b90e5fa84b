"""The allocation-free float64 entry point (gbxc_integrate_fp64_noalloc) against gbxc_integrate.

Callers that cannot allocate device memory (code running inside another allocator's pool or
in a pre-reserved memory region) use this call: its scratch is a static array inside the
library, and P, V and {E, N} are the caller's device buffers.  It must give the float64
path's results, within the float64 tolerance (1e-9), on two calls in a row, since every
call reuses the same static array.  This file is collected last on purpose."""
import numpy as np
import pytest

from gpu_common import Loaded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["water2_pbe_small", "water1_slater"])
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
