"""Pins of the paper's decomposition and sorted interaction (Section II-B, II-C).

* coverage: every pair within max(H_i, H_j) lies in exactly one self- or
  pair-interaction after all splits (the property the paper states for its
  decomposition), checked by brute force;
* the split rules hold cell by cell and pair by pair;
* the sorted two-loop interaction of Fig. 3 finds exactly the pairs of the naive
  double loop, each once, on random and adversarial cell pairs (ties in the
  projections, separations exactly equal to H, mixed H).
"""
import numpy as np
import pytest

from oracle import decomposition as dc
from oracle import sph, sweep
from paper_1309_3783_gb300 import inputs


def _clustered(n, seed):
    return inputs.plummer_box(n=n, n_spheres=3, scale=0.03, seed=seed)


@pytest.mark.parametrize("seed,leaf_max,headroom", [(1, 16, 0.0), (2, 40, 0.0), (3, 400, 0.0), (1, 16, 0.1),
                                                    (4, 24, 0.1)])
def test_coverage_each_pair_exactly_once(seed, leaf_max, headroom):
    """headroom 0 is the paper's rule; 0.1 is the library's default option."""
    box = _clustered(2500, seed)
    H = sph.support_radius(box.h)
    D = dc.decompose(box.x, H, box.L, True, leaf_max=leaf_max, headroom=headroom)
    want = dc.interacting_pairs_brute(box.x, H, box.L, True)
    got = dc.visits(D, box.x, H, box.L, True)
    assert set(got) == want
    assert all(c == 1 for c in got.values())
    if leaf_max < 100:
        assert len(D.split) > 0 and any(d > D.k for (d, *_ ) in D.pairs)


def test_coverage_open_box():
    box = _clustered(1500, 7)
    H = sph.support_radius(box.h) * 0.7
    D = dc.decompose(box.x, H, box.L, False, leaf_max=24)
    want = dc.interacting_pairs_brute(box.x, H, box.L, False)
    got = dc.visits(D, box.x, H, box.L, False)
    assert set(got) == want and all(c == 1 for c in got.values())


def test_split_rules_hold():
    box = _clustered(3000, 5)
    H = sph.support_radius(box.h)
    leaf_max, frac = 32, 0.875
    D = dc.decompose(box.x, H, box.L, True, leaf_max=leaf_max, split_frac=frac)
    L = box.L
    assert H.max() < L * 2.0 ** -D.k - dc.margin(L)
    # k is the finest level whose edge still exceeds H_max
    assert D.k == D.max_depth or not H.max() < L * 2.0 ** -(D.k + 1) - dc.margin(L)
    for key, idx in D.cells.items():
        d, c = key
        half = L * 2.0 ** -(d + 1) - dc.margin(L)
        ok = d < D.max_depth and len(idx) > leaf_max and np.count_nonzero(H[idx] < half) > frac * len(idx)
        assert (key in D.split) == ok
        assert np.all(dc.cell_coords(box.x[idx], L, d) == np.array(c))
    for (d, ca, cb, db) in D.pairs:
        assert dc.positive(db)
        ka, kb = (d, ca), (d, cb)
        half = L * 2.0 ** -(d + 1) - dc.margin(L)
        hmax = max(H[D.cells[ka]].max(), H[D.cells[kb]].max())
        assert not (ka in D.split and kb in D.split and hmax < half)
    for key in D.selfs:
        assert key not in D.split
    # particles keep H below the limits their pair splits relied on
    assert np.all(H < D.hlim)


def _random_cell_pair(rng, db, n, e, h_lo, h_hi, dyadic):
    if dyadic:
        q = 64
        pa = rng.integers(0, q, size=(n, 3)) / q * e
        pb = rng.integers(0, q, size=(n, 3)) / q * e + np.asarray(db) * e
        HA = rng.integers(int(h_lo * q), int(h_hi * q) + 1, size=n) / q * e
        HB = rng.integers(int(h_lo * q), int(h_hi * q) + 1, size=n) / q * e
    else:
        pa = rng.uniform(0, e, size=(n, 3))
        pb = rng.uniform(0, e, size=(n, 3)) + np.asarray(db) * e
        HA = np.exp(rng.uniform(np.log(h_lo), np.log(h_hi), size=n)) * e
        HB = np.exp(rng.uniform(np.log(h_lo), np.log(h_hi), size=n)) * e
    return pa, HA, pb, HB


@pytest.mark.parametrize("dyadic", [True, False])
def test_sorted_interaction_equals_naive(dyadic):
    rng = np.random.default_rng(17)
    for trial in range(60):
        db = dc.AXES[trial % 13]
        n = int(rng.integers(1, 40))
        pa, HA, pb, HB = _random_cell_pair(rng, db, n, 1.0, 0.05, 1.0, dyadic)
        axis = np.asarray(db, float) / np.linalg.norm(db)
        hits = sweep.sorted_pair(pa, HA, pb, HB, axis, slack=0.0 if dyadic else 1e-12)
        want = sweep.naive_pair(pa, HA, pb, HB)
        assert set(hits) == want, (trial, db)
        assert all(c == 1 for c in hits.values())


def test_sorted_interaction_ties_and_exact_cutoffs():
    # face pair along x: both cells hold a column of particles at the same
    # projection; separations hit H exactly for some pairs
    e = 1.0
    pa = np.array([[0.75, 0.25, 0.5], [0.75, 0.5, 0.5], [0.75, 0.75, 0.5], [0.5, 0.5, 0.5]])
    pb = np.array([[1.25, 0.25, 0.5], [1.25, 0.5, 0.5], [1.25, 0.75, 0.5], [1.5, 0.5, 0.5]])
    HA = np.array([0.5, 0.25, 0.5, 0.75])
    HB = np.array([0.5, 0.5 + 1 / 64, 0.25, 0.5])
    hits = sweep.sorted_pair(pa, HA, pb, HB, np.array([1.0, 0, 0]))
    want = sweep.naive_pair(pa, HA, pb, HB)
    assert set(hits) == want and all(c == 1 for c in hits.values())
    assert (0, 0) not in want       # r = 0.5 equals both H (strict predicate)
    assert (2, 2) not in want       # r = 0.5 equals H_i, H_j smaller
    assert (3, 1) not in want       # r = 0.75 equals H_i, H_j smaller
    assert (1, 1) in want           # r = 0.5 < H_j only: found by the second loop


def test_self_interaction_loop():
    rng = np.random.default_rng(5)
    p = rng.uniform(0, 1, size=(50, 3))
    H = rng.uniform(0.05, 0.6, size=50)
    got = sweep.naive_self(p, H)
    i, j = np.triu_indices(50, 1)
    d = p[i] - p[j]
    r2 = (d[:, 0] ** 2 + d[:, 1] ** 2) + d[:, 2] ** 2
    want = set(zip(i[(r2 < H[i] ** 2) | (r2 < H[j] ** 2)].tolist(), j[(r2 < H[i] ** 2) | (r2 < H[j] ** 2)].tolist()))
    assert got == want
