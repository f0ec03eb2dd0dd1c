"""The paper's hierarchical cell decomposition, in plain Python (small inputs).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section II-B of the paper:

1. Split the domain into cells whose edge is at least h_max.  Reading: the
   finest power-of-two grid of the box, i.e. level k = max{k : H_max < L/2^k - delta},
   with at least 4 cells per dimension for periodic boxes (k >= 2), so that a
   cell never neighbours itself or another cell twice across the boundary.
2. Self-interactions: every non-empty cell.  Pair-interactions: every non-empty
   pair sharing a face, edge or corner, across periodic boundaries too.
3. Recursively bisect a cell in all three dimensions when (a) it holds more
   than ``leaf_max`` particles and (b) more than ``split_frac`` of its particles
   have H below half the cell edge (Section III-B: 400 particles, 87.5 %).
4. A split cell's self-interaction becomes its children's self-interactions
   and the pair-interactions between them (Fig. 2A).
5. A pair-interaction between two split cells becomes the pair-interactions of
   the children across the interface iff every particle of both cells has H
   below half the cell edge (Fig. 2B; the text's "less than" is taken).

"h" in every rule is the support radius H.  ``delta = 2^-50 L`` keeps every rule
strict by more than the rounding of a cell index, so that neighbours within H
always sit in the same or adjacent cells.  Cell membership at level d is
``floor((x / L) * 2^d)`` clamped to [0, 2^d - 1].

A pair is stored as (d, ca, cb, db): cells ca and cb at level d and
db = cb - ca + s 2^d in {-1, 0, 1}^3 (s the periodic image), oriented so that db
lies in the "positive" half: dz > 0, or dz = 0 and dy > 0, or dz = dy = 0 and
dx > 0.  The 13 such db are the 13 sort axes of Section II-C.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import product

import numpy as np


def margin(L: float) -> float:
    return L * 2.0 ** -50


def positive(db) -> bool:
    dx, dy, dz = db
    return dz > 0 or (dz == 0 and (dy > 0 or (dy == 0 and dx > 0)))


AXES = [db for db in product((-1, 0, 1), repeat=3) if positive(db)]


def top_level(H_max: float, L: float, periodic: bool, max_depth: int, headroom: float = 0.0) -> int:
    """Finest level whose cell edge exceeds H_max (1 + headroom) by the margin; raises if none."""
    k_min = 2 if periodic else 0
    dl = margin(L)
    if not H_max < L * 2.0 ** -k_min - dl:
        raise ValueError("H_max too large for the box")
    k = k_min
    while k + 1 <= max_depth and H_max * (1.0 + headroom) < L * 2.0 ** -(k + 1) - dl:
        k += 1
    return k


def cell_coords(x: np.ndarray, L: float, d: int) -> np.ndarray:
    q = np.floor((x / L) * 2.0 ** d).astype(np.int64)
    return np.clip(q, 0, 2 ** d - 1)


@dataclass
class Decomposition:
    k: int
    max_depth: int
    cells: dict = field(default_factory=dict)      # (d, (ix, iy, iz)) -> particle indices
    split: set = field(default_factory=set)        # keys of split cells
    children: dict = field(default_factory=dict)   # key -> list of child keys
    selfs: set = field(default_factory=set)        # final self-interactions (cell keys)
    pairs: set = field(default_factory=set)        # final pairs (d, ca, cb, db)
    hlim: np.ndarray | None = None                 # per particle: H must stay below this


def _orient(d, ca, cb, db):
    if positive(db):
        return (d, ca, cb, db)
    return (d, cb, ca, tuple(-c for c in db))


def decompose(x, H, L, periodic, leaf_max=400, split_frac=0.875, max_depth=20, headroom=0.0) -> Decomposition:
    """headroom > 0 (an implementation option, not the paper's): pairs split and the
    top level is chosen only when H (1 + headroom) clears the limit; 0 is the rule
    of the paper."""
    x = np.asarray(x, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    n = x.shape[0]
    dl = margin(L)
    headroom = float(np.float32(headroom))    # the library holds it in FP32
    k = top_level(float(H.max()), L, periodic, max_depth, headroom)
    frac = float(np.float32(split_frac))
    D = Decomposition(k=k, max_depth=max_depth)
    D.hlim = np.full(n, L * 2.0 ** -k - dl)

    # cell tree
    ck = cell_coords(x, L, k)
    groups = {}
    for p in range(n):
        groups.setdefault(tuple(int(c) for c in ck[p]), []).append(p)
    stack = []
    for c, idx in groups.items():
        key = (k, c)
        D.cells[key] = np.array(idx, dtype=np.int64)
        stack.append(key)
    while stack:
        key = stack.pop()
        d, c = key
        idx = D.cells[key]
        half = L * 2.0 ** -(d + 1) - dl
        n_small = int(np.count_nonzero(H[idx] < half))
        if d < max_depth and len(idx) > leaf_max and float(n_small) > frac * float(len(idx)):
            D.split.add(key)
            cc = cell_coords(x[idx], L, d + 1)
            kids = {}
            for p, q in zip(idx, cc):
                kids.setdefault(tuple(int(v) for v in q), []).append(int(p))
            D.children[key] = []
            for q, sub in sorted(kids.items()):
                ckey = (d + 1, q)
                D.cells[ckey] = np.array(sub, dtype=np.int64)
                D.children[key].append(ckey)
                stack.append(ckey)

    # interaction lists
    nside = 2 ** k
    work = [("self", (k, c)) for c in groups]
    for c in groups:
        for db in AXES:
            cb = tuple(c[i] + db[i] for i in range(3))
            if periodic:
                cb = tuple(v % nside for v in cb)
            elif any(v < 0 or v >= nside for v in cb):
                continue
            if cb in groups:
                work.append(("pair", (k, c, cb, db)))
    while work:
        kind, item = work.pop()
        if kind == "self":
            key = item
            if key not in D.split:
                D.selfs.add(key)
                continue
            kids = D.children[key]
            for a in kids:
                work.append(("self", a))
            for i in range(len(kids)):
                for j in range(i + 1, len(kids)):
                    (d1, ca), (_, cb) = kids[i], kids[j]
                    db = tuple(cb[t] - ca[t] for t in range(3))
                    work.append(("pair", _orient(d1, ca, cb, db)))
            continue
        d, ca, cb, db = item
        ka, kb = (d, ca), (d, cb)
        half = L * 2.0 ** -(d + 1) - dl
        hmax = max(H[D.cells[ka]].max(), H[D.cells[kb]].max())
        if ka in D.split and kb in D.split and hmax * (1.0 + headroom) < half:
            for p in D.cells[ka]:
                D.hlim[p] = min(D.hlim[p], half)
            for p in D.cells[kb]:
                D.hlim[p] = min(D.hlim[p], half)
            s = tuple((db[t] - (cb[t] - ca[t])) // (2 ** d) for t in range(3))
            for (_, qa) in D.children[ka]:
                for (_, qb) in D.children[kb]:
                    dd = tuple(qb[t] - qa[t] + s[t] * 2 ** (d + 1) for t in range(3))
                    if all(abs(v) <= 1 for v in dd):
                        work.append(("pair", _orient(d + 1, qa, qb, dd)))
        else:
            D.pairs.add(item)
    return D


def interacting_pairs_brute(x, H, L, periodic):
    """Unordered pairs {i < j} with r < max(H_i, H_j), canonical FP64 predicate."""
    from .sph import canonical_r2
    n = x.shape[0]
    i, j = np.triu_indices(n, 1)
    r2, _ = canonical_r2(x, i, j, L, periodic)
    keep = (r2 < H[i] ** 2) | (r2 < H[j] ** 2)
    return set(zip(i[keep].tolist(), j[keep].tolist()))


def visits(D: Decomposition, x, H, L, periodic):
    """Count, for every unordered in-range pair, the interactions that contain it."""
    from .sph import canonical_r2
    count = {}
    def add(ia, ib, same):
        if same:
            a, b = np.triu_indices(len(ia), 1)
            I, J = ia[a], ia[b]
        else:
            I = np.repeat(ia, len(ib))
            J = np.tile(ib, len(ia))
        if len(I) == 0:
            return
        r2, _ = canonical_r2(x, I, J, L, periodic)
        keep = (r2 < H[I] ** 2) | (r2 < H[J] ** 2)
        for p, q in zip(I[keep].tolist(), J[keep].tolist()):
            key = (min(p, q), max(p, q))
            count[key] = count.get(key, 0) + 1
    for key in D.selfs:
        add(D.cells[key], None, True)
    for (d, ca, cb, db) in D.pairs:
        add(D.cells[(d, ca)], D.cells[(d, cb)], False)
    return count
