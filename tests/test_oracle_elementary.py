"""The oracle's fixed-operation logarithm, sine and cosine (used for the grid and the shell
cutoffs so that plans do not depend on the host's libm) against the platform's math library:
within a few units in the last place over the arguments the grid and the cutoffs use, exact at
the special points, and the same for the input generator's own versions."""
import math

import numpy as np

import xcinputs as X
from oracle import elementary as el


def test_ln_against_libm():
    rng = np.random.default_rng(1)
    xs = list(rng.uniform(1e-12, 1.0, 3000)) + list(10.0 ** rng.uniform(-12, 4, 3000)) + [1e-10, 0.1, 1e3]
    for x in xs:
        ref = math.log(x)
        assert abs(el.ln(x) - ref) <= 4 * math.ulp(ref) + 1e-300, x
    assert el.ln(1.0) == 0.0


def test_sin_cos_against_libm():
    rng = np.random.default_rng(2)
    xs = list(rng.uniform(0.0, 2.0 * math.pi, 5000)) + [2.0 * math.pi * b / 32 for b in range(32)]
    for x in xs:
        s, c = el.sincos(x)
        assert abs(s - math.sin(x)) <= 4e-16 and abs(c - math.cos(x)) <= 4e-16, x
    assert el.sincos(0.0) == (0.0, 1.0)


def test_input_generator_functions_against_libm():
    rng = np.random.default_rng(3)
    for x in 10.0 ** rng.uniform(-8, 4, 500):
        assert abs(X._fixed_ln(x) - math.log(x)) <= 4 * math.ulp(math.log(x)) + 1e-300
    for y in rng.uniform(-30.0, 10.0, 500):
        assert abs(X._fixed_exp(y) - math.exp(y)) <= 4 * math.ulp(math.exp(y))
    for x in rng.uniform(0.0, 2.0 * math.pi, 500):
        s, c = X._fixed_sincos(x)
        assert abs(s - math.sin(x)) <= 4e-16 and abs(c - math.cos(x)) <= 4e-16
    for x in (0.0625, 1.0, 4.0, 6.25):
        assert abs(X._fixed_cbrt(x) - x ** (1.0 / 3.0)) <= 2 * math.ulp(x ** (1.0 / 3.0))
