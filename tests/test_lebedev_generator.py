"""The package's Lebedev-Laikov generator (paper_2007_03143_gb300/gen_lebedev.py) reproduces the
table the library is built with (csrc/lebedev_rules.inc) for the rules it solves in seconds."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "paper_2007_03143_gb300", "csrc", "lebedev_rules.inc")
KINDS = ["a1", "a2", "a3", "b", "c", "d"]


def _table():
    txt = open(INC).read()
    orb = [(KINDS[int(k)], [float.fromhex(x), float.fromhex(y), float.fromhex(z)], float.fromhex(w))
           for k, x, y, z, w in re.findall(r"\{(\d), \{(\S+), (\S+), (\S+)\}, (\S+)\}", txt)]
    idx = {int(n): (int(first), int(cnt)) for n, _, first, cnt in re.findall(r"\{(\d+), (\d+), (\d+), (\d+)\},", txt)}
    return {n: orb[f:f + c] for n, (f, c) in idx.items()}


@pytest.mark.parametrize("n", [6, 14, 26, 38, 50, 86, 110])
def test_generator_reproduces_the_table(n):
    pytest.importorskip("scipy")
    pytest.importorskip("mpmath")
    from paper_2007_03143_gb300 import gen_lebedev as GL
    kinds, x = GL.search(n)
    fresh = GL.polish(n, kinds, x)
    kept = _table()[n]
    assert [(k, list(g), w) for k, g, w in fresh] == [(k, g, w) for k, g, w in kept]


def test_table_lists_every_rule_once():
    t = _table()
    from paper_2007_03143_gb300 import gen_lebedev as GL
    assert sorted(t) == sorted(GL.RULES)
    for n, orbits in t.items():
        assert sum(GL.ORBIT_SIZE[k] for k, _, _ in orbits) == n
