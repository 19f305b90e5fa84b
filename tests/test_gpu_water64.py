"""Precision form on the 64-water PBE/SSF workload (192 atoms, 1,600 functions, 75 x 16 x 32
grid, 7.37M points): the tensor-core form against the float64 form of the same library on the
whole grid, plus properties that hold at any size (Sec. 2.1 Eqs. rho/exc/vxc; Algorithm 4)."""
import numpy as np
import pytest

from gpu_common import Loaded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w64():
    L = Loaded("water64_pbe")
    yield L
    L.close()


def test_plan_fits_the_kernels(w64):
    # the largest N_b^j of this workload is 1,182: the tensor-core form takes N_b^j <= 1,184
    assert w64.info["nbatch"] > 0
    assert w64.info["npts"] == 192 * 75 * 16 * 32


def test_mixed_against_fp64_whole_grid(w64):
    E64, N64, V64 = w64.integrate("fp64")
    Em, Nm, Vm = w64.integrate("mixed")
    # N_el against Tr(P S) = 10 per water (quadrature-limited)
    assert abs(N64 - 640.0) < 5e-2
    dE, dN, dV = abs(Em - E64), abs(Nm - N64), float(np.max(np.abs(Vm - V64)))
    print(f"water64 PBE: E64 {E64:.10f}  |dE| {dE:.3e}  |dN| {dN:.3e}  max|dV| {dV:.3e}")
    assert dE <= 1e-6
    assert dN <= 1e-6
    assert dV <= 1e-5
    assert np.array_equal(Vm, Vm.T) and np.array_equal(V64, V64.T)
