"""Kernel steps against their oracle steps on sampled batches (through gbxc_debug_batch):
the collocation Phi and grad Phi (Eq. gau_cart) and Z (Eq. z_mat, which folds in X, rho,
grad rho and the functional).  float64 form: Phi and grad Phi to 1e-14 of their largest
magnitude, Z to 1e-11; mixed form: Phi to 1e-11 (double-float arithmetic, whose exp(-t) error
grows with t for the tight primitives), grad Phi to 1e-9 (hi word plus a bf16 low word), Z to
1e-7 (its gradient terms take the hi words of grad Phi)."""
import numpy as np
import pytest

from oracle import integrate as I

from gpu_common import Loaded

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-14, 1e-14, 1e-11), "mixed": (1e-11, 1e-9, 1e-7)}


@pytest.fixture(scope="module", params=["water2_pbe_small", "water2_pbe_small_sph", "water1_slater"])
def loaded(request):
    L = Loaded(request.param)
    yield L
    L.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_batch_intermediates_match_oracle(loaded, form):
    g, pl = loaded.oracle()
    w = loaded.w
    nb = len(pl.batch_points)
    rng = np.random.default_rng(11)
    for j in sorted(set(rng.choice(nb, size=min(4, nb), replace=False).tolist()) | {0, nb - 1}):
        m, n = len(pl.batch_points[j]), len(pl.batch_funcs[j])
        got = loaded.G.gbxc_debug_batch(loaded.ctx.h, loaded.mid, j, w.P, w.functional, form, m, n)
        ref = I.batch_intermediates(g, w.basis, w.P, w.functional, pl, j)
        tphi, tgrad, tz = TOL[form]
        errs = [float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) for a, b in zip(got, ref)]
        print(form, j, ["%.1e" % e for e in errs])
        assert errs[0] <= tphi and max(errs[1:4]) <= tgrad and errs[4] <= tz, (j, errs)
