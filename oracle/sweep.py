"""The paper's cell-pair interaction loops, in plain Python (Section II-C).

TEST INFRASTRUCTURE ONLY (see the package docstring).

``naive_pair``   -- the double loop over both cells: interact when
                    r < h_i or r < h_j.
``naive_self``   -- the i < j double loop inside one cell with the same test.
``sorted_pair``  -- the sorted interaction of Fig. 3: project both cells on the
                    axis joining their centres, then
                    loop 1: every i on the left against the right-hand j in
                            ascending order, stopping once r_i + h_i < r_j,
                            interacting when r < h_i;
                    loop 2: every j on the right against the left-hand i in
                            descending order, stopping once r_i < r_j - h_j,
                            interacting when r < h_j and not r < h_i.
Readings of the printed loops: loop 2 indexes the sorted list with its own loop
variable (ind_i[ii]); its second test "rij > h_i" is taken as "not rij < h_i"
so that a pair with r exactly equal to h_i is neither lost nor counted twice.
``slack`` widens both stopping tests for inputs whose projections round.
"""
from __future__ import annotations

import numpy as np


def _r2(p, q):
    d = p - q
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]


def naive_self(p, H):
    out = set()
    n = len(p)
    for i in range(n - 1):
        for j in range(i + 1, n):
            r2 = _r2(p[i], p[j])
            if r2 < H[i] ** 2 or r2 < H[j] ** 2:
                out.add((i, j))
    return out


def naive_pair(pA, HA, pB, HB):
    out = set()
    for i in range(len(pA)):
        for j in range(len(pB)):
            r2 = _r2(pA[i], pB[j])
            if r2 < HA[i] ** 2 or r2 < HB[j] ** 2:
                out.add((i, j))
    return out


def sorted_pair(pA, HA, pB, HB, axis, slack=0.0):
    """Pairs found by the sorted two-loop interaction; also returns per-pair visit counts."""
    axis = np.asarray(axis, dtype=np.float64)
    rA = pA @ axis
    rB = pB @ axis
    ind_a = np.argsort(rA, kind="stable")
    ind_b = np.argsort(rB, kind="stable")
    hits = {}
    for i in range(len(pA)):
        for jj in range(len(pB)):
            j = ind_b[jj]
            if rA[i] + HA[i] + slack < rB[j]:
                break
            if _r2(pA[i], pB[j]) < HA[i] ** 2:
                hits[(i, int(j))] = hits.get((i, int(j)), 0) + 1
    for j in range(len(pB)):
        for ii in range(len(pA) - 1, -1, -1):
            i = ind_a[ii]
            if rA[i] + slack < rB[j] - HB[j]:
                break
            r2 = _r2(pA[i], pB[j])
            if r2 < HB[j] ** 2 and not r2 < HA[i] ** 2:
                hits[(int(i), j)] = hits.get((int(i), j), 0) + 1
    return hits
