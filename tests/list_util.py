"""Neighbour-list triplets in canonical form.

A list entry (a, c, code) says that atom c's image n meets atom a, with
code = (nx+2)*25 + (ny+2)*5 + (nz+2) and displacement r_c - r_a + nL. The
same pair seen from c is (c, a, code(-n)). The canonical form keeps the
lower atom index first, so lists built with any owner rule compare equal.
"""
import numpy as np


def mirror_code(code):
    code = np.asarray(code)
    nx, ny, nz = code // 25 - 2, (code // 5) % 5 - 2, code % 5 - 2
    return (-nx + 2) * 25 + (-ny + 2) * 5 + (-nz + 2)


def canonical(trip):
    """(a, c, code) rows -> (min, max, code seen from min), sorted."""
    t = np.asarray(trip, dtype=np.int64).reshape(-1, 3).copy()
    swap = t[:, 0] > t[:, 1]
    t[swap] = np.stack([t[swap, 1], t[swap, 0], mirror_code(t[swap, 2])], axis=1)
    return sort_rows(t)


def both_ways(trip):
    """Every canonical entry plus the same pair seen from its other atom."""
    t = np.asarray(trip, dtype=np.int64).reshape(-1, 3)
    rev = np.stack([t[:, 1], t[:, 0], mirror_code(t[:, 2])], axis=1)
    return sort_rows(np.concatenate([t, rev]))


def sort_rows(t):
    t = np.asarray(t, dtype=np.int64).reshape(-1, 3)
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]
