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
