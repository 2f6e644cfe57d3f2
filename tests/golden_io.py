"""Readers for the text fixtures under tests/golden (values printed in the paper)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def lattice():
    """(c as (9, 2) int array, w as (9,) float array) from Eq. 20a, 20b."""
    c, w = [], []
    for i, (idx, cx, cy, wt) in enumerate(_rows("d2q9_lattice.txt")):
        assert int(idx) == i
        c.append((int(cx), int(cy)))
        w.append(float(Fraction(wt)))
    return np.array(c), np.array(w)


def moment_matrix():
    return np.array([[float(v) for v in r] for r in _rows("d2q9_moment_matrix.txt")])


def parameters():
    return {k: float(v) for k, v in _rows("parameters_eq39.txt")}


def lattice3():
    """(c as (15, 3) int array, w as (15,) float array) from Eq. 21a, 21b."""
    c, w = [], []
    for i, (idx, cx, cy, cz, wt) in enumerate(_rows("d3q15_lattice.txt")):
        assert int(idx) == i
        c.append((int(cx), int(cy), int(cz)))
        w.append(float(Fraction(wt)))
    return np.array(c), np.array(w)


def moment_matrix3():
    """Eq. 24 as printed (15 x 15)."""
    return np.array([[float(v) for v in r] for r in _rows("d3q15_moment_matrix.txt")])
