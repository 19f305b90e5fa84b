"""Writes tests/golden/lebedev_<N>.txt: the oracle's Lebedev-Laikov rules (oracle.lebedev),
one line per orbit 'kind gx gy gz w' in float.hex, w the weight of each point (4 pi total).
Run from the repository root: python tests/golden/make_lebedev.py [N ...]"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import lebedev as L  # noqa: E402

if __name__ == "__main__":
    sizes = [int(a) for a in sys.argv[1:]] or sorted(L.STRUCTURE)
    here = os.path.dirname(os.path.abspath(__file__))
    for n in sizes:
        orb = L.lebedev_orbits(n)
        p = L.STRUCTURE[n][0]
        L.write_orbits(orb, os.path.join(here, f"lebedev_{n}.txt"),
                       f"Lebedev-Laikov rule, {n} points, degree {p} (Sec. 2.2; Table Atomic Quadrature Sizes)\n"
                       f"written by tests/golden/make_lebedev.py from oracle.lebedev")
        print(n, len(orb), flush=True)
