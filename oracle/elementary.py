"""Logarithm, sine and cosine written out with basic IEEE double operations in a fixed order.
ORACLE -- test infrastructure only.

The grid (Sec. 2.2: the radial rule's ln(1 - x^3), the angular nodes and azimuths) and the
shell cutoffs (Eq. rcut) need these functions.  The platform libm's last bits differ between
host architectures, and batch membership is decided by exact comparisons, so a libm call
would make the plan of a seeded workload depend on the host; these versions give the same
bits everywhere.

    ln x:      x = m 2^e with m in [1/sqrt 2, sqrt 2) (frexp, exact); ln m = 2 atanh(s) with
               s = (m - 1)/(m + 1), summed as s + s^3/3 + ... + s^25/25 (|s| <= 0.1716, so the
               first omitted term is below 1e-20); ln x = e ln2_hi + (2 sum + e ln2_lo), where
               ln2_hi carries 32 significant bits so that e ln2_hi is exact.
    sin, cos:  x = q pi/2 + r, q = floor(2x/pi + 1/2), r = (x - q pio2_hi) - q pio2_lo
               (pio2_hi with 33 significant bits, q pio2_hi exact for the arguments used here,
               0 <= x <= 8); Taylor series of cos r and sin r to r^22 and r^23, term by term
               (t <- t (-r^2) / ((2k-1)(2k)) and t <- t (-r^2) / ((2k)(2k+1))); the quadrant
               q mod 4 picks (sin, cos) = (s, c), (c, -s), (-s, -c) or (-c, s).
"""
from __future__ import annotations

import math

LN2_HI = 6.93147180369123816490e-01
LN2_LO = 1.90821492927058770002e-10
TWO_OVER_PI = 0.63661977236758134308
PIO2_HI = 1.57079632673412561417e+00
PIO2_LO = 6.07710050650619224932e-11
INV_SQRT2 = 0.70710678118654752440


def ln(x: float) -> float:
    m, e = math.frexp(x)
    if m < INV_SQRT2:
        m = m * 2.0
        e = e - 1
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    t = s
    acc = s
    for k in range(1, 13):
        t = t * s2
        acc = acc + t / float(2 * k + 1)
    return float(e) * LN2_HI + (2.0 * acc + float(e) * LN2_LO)


def sincos(x: float):
    q = float(math.floor(x * TWO_OVER_PI + 0.5))
    r = (x - q * PIO2_HI) - q * PIO2_LO
    r2 = r * r
    tc, c, ts, s = 1.0, 1.0, r, r
    for k in range(1, 12):
        tc = tc * (-r2) / float((2 * k - 1) * (2 * k))
        c = c + tc
        ts = ts * (-r2) / float((2 * k) * (2 * k + 1))
        s = s + ts
    quadrant = int(q) & 3
    if quadrant == 0:
        return s, c
    if quadrant == 1:
        return c, -s
    if quadrant == 2:
        return -s, -c
    return -c, s


def cos(x: float) -> float:
    return sincos(x)[1]


def sin(x: float) -> float:
    return sincos(x)[0]
