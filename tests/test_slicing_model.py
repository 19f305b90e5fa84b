"""Error model of the tensor-core form's contractions, on the CPU: the Ozaki-style slicing of
double-float operands into five bf16-exact slices and the level-wise float32 accumulation of
their products, restated in numpy float32 and checked against a float64 GEMM on random
operands: an error-model check of the contraction scheme, independent of the GPU (the device
arithmetic itself is checked against the same bounds in test_gpu_device_math.py).

What the mixed form relies on, each checked here:
  * a value v = (h + l) 2^-e with |v| <= 1 is cut into q_s 2^-(6+7s), s = 0..4, with integer
    q_s (|q_s| <= 64 for s <= 2, <= 72 for s = 3), so every slice is exact in bf16 and the
    reconstruction error is below 2^-34 (relative to the row scale 2^e);
  * the products of slices of level d = s + t are integer multiples of 2^-(12+7d); for
    d = 0, 1, 2 their sums over K <= 1184 stay below 2^24 such units, so a float32
    accumulator holds them exactly in any order;
  * levels 3-4 together are rounded, below 2^-21 of level 0, so the contraction's error is a
    small multiple of K 2^-34 of the product of the row scales.
"""
import numpy as np
import pytest

F32 = np.float32
NSL = 5
K_MAX = 1184   # the largest padded function count the tensor-core form takes


def exp_of(x):
    """Smallest e with |x| < 2^e (0 for x == 0), with the library's 2^-22 margin."""
    x = np.asarray(x, dtype=F32)
    _, e = np.frexp(x * F32(1.0000002))
    return np.where(x > 0, e, 0).astype(np.int32)


def slice5(h, l, e):
    """Five slices of (h + l) 2^-e, float32 arithmetic only (the library's rule)."""
    sc = np.ldexp(F32(1.0), -e).astype(F32)
    rh = (h * sc).astype(F32)
    rl = (l * sc).astype(F32)
    out = []
    for s in range(NSL):
        if s == 3:
            rh = (rh + rl).astype(F32)
        up = F32(2.0 ** (6 + 7 * s))
        q = (np.rint((rh * up).astype(F32)) / up).astype(F32)
        out.append(q)
        rh = (rh - q).astype(F32)
    return out


def split_rows(v):
    """Rows of float64 values as double-float pairs, scaled per row by 2^-e_row."""
    h = v.astype(F32)
    l = (v - h.astype(np.float64)).astype(F32)
    e = exp_of(np.max(np.abs(h), axis=1))[:, None]
    return h, l, e


def bf16_exact(x):
    """True where float32 x is exactly representable in bf16 (low 16 bits zero)."""
    return (np.asarray(x, dtype=F32).view(np.uint32) & 0xFFFF) == 0


@pytest.fixture(scope="module")
def operands():
    rng = np.random.default_rng(7)
    # rows spanning many magnitudes, like Phi at a point and P^j rows
    A = rng.standard_normal((48, K_MAX)) * 10.0 ** rng.uniform(-6, 3, size=(48, 1))
    B = rng.standard_normal((40, K_MAX)) * 10.0 ** rng.uniform(-4, 2, size=(40, 1))
    A[0, 5] = 1.0   # a row whose maximum sits exactly on a power of two
    B[1, :] = 0.0   # an all-zero row
    return A, B


def test_slices_are_bounded_integers_exact_in_bf16(operands):
    for M in operands:
        h, l, e = split_rows(M)
        qs = slice5(h, l, e)
        for s, q in enumerate(qs):
            k = (q.astype(np.float64) * 2.0 ** (6 + 7 * s))
            assert np.all(k == np.round(k)), s
            bound = 72 if s == 3 else 64
            assert np.max(np.abs(k)) <= bound, (s, np.max(np.abs(k)))
            assert np.all(bf16_exact(q)), s


def test_reconstruction_within_2_pow_minus_34(operands):
    for M in operands:
        h, l, e = split_rows(M)
        qs = slice5(h, l, e)
        rec = sum(q.astype(np.float64) for q in qs)
        target = (h.astype(np.float64) + l.astype(np.float64)) * np.ldexp(1.0, -e)
        assert np.max(np.abs(target)) <= 1.0
        assert np.max(np.abs(rec - target)) <= 2.0 ** -34


def _levels(qa, qb):
    """Per level d = s + t <= 4: the list of slice-pair products (a row of A, a row of B)."""
    lv = {d: [] for d in range(5)}
    for s in range(NSL):
        for t in range(NSL - s):
            lv[s + t].append((qa[s], qb[t]))
    return lv


def test_levels_0_to_2_exact_in_float32(operands):
    A, B = operands
    ha, la, ea = split_rows(A)
    hb, lb, eb = split_rows(B)
    qa, qb = slice5(ha, la, ea), slice5(hb, lb, eb)
    lv = _levels(qa, qb)
    for d in range(3):
        exact = sum(a.astype(np.float64) @ b.astype(np.float64).T for a, b in lv[d])
        unit = 2.0 ** -(12 + 7 * d)
        assert np.max(np.abs(exact)) / unit < 2 ** 24
        # float32 accumulation, one product at a time along K, in two different orders
        for order in (np.arange(K_MAX), np.random.default_rng(d).permutation(K_MAX)):
            acc = np.zeros((A.shape[0], B.shape[0]), dtype=F32)
            for k in order:
                for a, b in lv[d]:
                    acc = (acc + np.outer(a[:, k], b[:, k]).astype(F32)).astype(F32)
            assert np.array_equal(acc.astype(np.float64), exact), d


def test_contraction_against_float64_gemm(operands):
    A, B = operands
    ha, la, ea = split_rows(A)
    hb, lb, eb = split_rows(B)
    qa, qb = slice5(ha, la, ea), slice5(hb, lb, eb)
    lv = _levels(qa, qb)
    acc = []
    for group in ((0,), (1,), (2,), (3, 4)):
        a32 = np.zeros((A.shape[0], B.shape[0]), dtype=F32)
        for k in range(K_MAX):
            for d in group:
                for a, b in lv[d]:
                    a32 = (a32 + np.outer(a[:, k], b[:, k]).astype(F32)).astype(F32)
        acc.append(a32.astype(np.float64))
    C = sum(acc) * np.ldexp(1.0, ea) * np.ldexp(1.0, eb).T
    ref = A @ B.T
    scale = np.ldexp(1.0, ea) * np.ldexp(1.0, eb).T
    err = np.abs(C - ref) / scale
    # per K term: the reconstruction (2 x 2^-34), the omitted levels s + t >= 5 (about
    # 2^-33) and the rounding of levels 3-4; summed over K
    assert np.max(err) <= 8.0 * K_MAX * 2.0 ** -34
    # and far below what a split-bf16 x 3 product (about 2^-16 per product) would leave
    assert np.max(err) < 1e-3 * K_MAX * 2.0 ** -16


def test_w_contraction_with_phi_cut_per_point():
    """The W contraction W = Z^T Phi over K points takes Phi's slices from the X contraction,
    cut with one exponent e_i per point (Phi_i,nu 2^-e_i, |.| <= 1), and slices Z_i,mu 2^e_i with
    one exponent per function over the points, so W_mu,nu = 2^(e_mu) sum_levels (Z-slices .
    Phi-slices) needs only Z's exponents.  With K = 1,024 points (a V task's 8 tiles), levels
    0-2 accumulate exactly in float32 and W lies within 8 K 2^-34 of the float64 product in units
    of 2^(e_mu), even when the points' Phi maxima span nine decades."""
    rng = np.random.default_rng(11)
    K, M, N = 1024, 24, 20
    point_scale = 10.0 ** rng.uniform(-6, 3, size=(K, 1))
    Phi = rng.standard_normal((K, N)) * point_scale                    # points x functions
    Z = rng.standard_normal((K, M)) * point_scale * 10.0 ** rng.uniform(-3, 0, size=(1, M))
    hp, lp, ep = split_rows(Phi)                                       # one exponent per point
    qp = slice5(hp, lp, ep)                                            # K x N slices, |.| <= 1
    Zs = Z * np.ldexp(1.0, ep)                                         # Z_i,mu 2^e_i
    hz, lz, ez = split_rows(Zs.T)                                      # one exponent per function
    qz = slice5(hz, lz, ez)                                            # M x K slices
    lv = {d: [] for d in range(5)}
    for s in range(NSL):
        for t in range(NSL - s):
            lv[s + t].append((qz[s], qp[t]))
    acc = []
    for group in ((0,), (1,), (2,), (3, 4)):
        a32 = np.zeros((M, N), dtype=F32)
        for k in range(K):
            for d in group:
                for a, b in lv[d]:
                    a32 = (a32 + np.outer(a[:, k], b[k, :]).astype(F32)).astype(F32)
        acc.append(a32.astype(np.float64))
    for d in range(3):   # the exact levels: the float32 sums equal the float64 ones
        exact = sum(a.astype(np.float64) @ b.astype(np.float64) for a, b in lv[d])
        assert np.array_equal(acc[d], exact), d
    W = sum(acc) * np.ldexp(1.0, ez)
    ref = Z.T @ Phi
    err = np.abs(W - ref) / np.ldexp(1.0, ez)
    assert np.max(err) <= 8.0 * K * 2.0 ** -34
