"""Pin of the gathered later passes of the h iteration, on the oracle's
decomposition (Section II-B, II-D).

A later pass evaluates the particles still iterating h.  Gathered, each leaf's
iterating particles are packed into clusters of up to 32, and every interaction
runs once per packed cluster of each of its cells, from the own side only: a pair
interaction (A, B) takes A's packed clusters against B's particles and B's
against A's; a self interaction of A takes A's packed clusters against all of A's
particles, the particle itself left out.  This must take every pair (i, j) with
r < H_i of an iterating i exactly once — the property the paper states for its
decomposition (every pair within max(H_i, H_j) lies in exactly one interaction)
carried over to the own side.  Checked against brute force, with the iterating
particles spread at random, gathered around one particle, and all particles.
"""
import numpy as np
import pytest

from oracle import decomposition as dc
from oracle import sph
from paper_1309_3783_gb300 import inputs


def _leaves(D, key):
    if key not in D.split:
        return [key]
    out = []
    for c in D.children[key]:
        out.extend(_leaves(D, c))
    return out


def _packed(D, key, active):
    """The packed clusters of a cell: per leaf below it, its iterating particles
    in chunks of up to 32."""
    out = []
    for leaf in _leaves(D, key):
        idx = D.cells[leaf]
        idx = idx[active[idx]]
        out.extend(idx[s:s + 32] for s in range(0, len(idx), 32))
    return out


def _gathered_visits(D, x, H, L, periodic, active, leave_self_out=True):
    count = {}

    def run(own, partners, self_cell):
        I = np.repeat(own, len(partners))
        J = np.tile(partners, len(own))
        if self_cell and leave_self_out:
            keep = I != J
            I, J = I[keep], J[keep]
        if len(I) == 0:
            return
        r2, _ = sph.canonical_r2(x, I, J, L, periodic)
        hit = r2 < H[I] ** 2
        for p, q in zip(I[hit].tolist(), J[hit].tolist()):
            count[(p, q)] = count.get((p, q), 0) + 1

    for key in D.selfs:
        for own in _packed(D, key, active):
            run(own, D.cells[key], True)
    for (d, ca, cb, db) in D.pairs:
        ka, kb = (d, ca), (d, cb)
        for own in _packed(D, ka, active):
            run(own, D.cells[kb], False)
        for own in _packed(D, kb, active):
            run(own, D.cells[ka], False)
    return count


def _brute(x, H, L, periodic, active):
    want = set()
    n = x.shape[0]
    for i in np.nonzero(active)[0]:
        J = np.delete(np.arange(n), i)
        r2, _ = sph.canonical_r2(x, np.full(n - 1, i), J, L, periodic)
        want.update((int(i), int(j)) for j in J[r2 < H[i] ** 2])
    return want


@pytest.mark.parametrize("seed,leaf_max,mode", [(1, 16, "random"), (2, 48, "random"), (3, 48, "region"),
                                                (4, 400, "random"), (5, 24, "all")])
def test_gathered_passes_take_every_own_pair_once(seed, leaf_max, mode):
    box = inputs.plummer_box(n=2500, n_spheres=3, scale=0.03, seed=seed)
    H = sph.support_radius(box.h)
    D = dc.decompose(box.x, H, box.L, True, leaf_max=leaf_max, headroom=0.1)
    rng = np.random.default_rng(seed)
    active = np.zeros(box.n, bool)
    if mode == "random":
        active[rng.choice(box.n, box.n // 20, replace=False)] = True
    elif mode == "region":
        d = box.x - box.x[rng.integers(box.n)]
        d -= box.L * np.round(d / box.L)
        active[np.argsort((d * d).sum(axis=1))[: box.n // 20]] = True
    else:
        active[:] = True
    got = _gathered_visits(D, box.x, H, box.L, True, active)
    want = _brute(box.x, H, box.L, True, active)
    assert set(got) == want
    assert all(c == 1 for c in got.values())
    if leaf_max < 100:
        # the case exercises split cells and pair interactions below the top level
        assert len(D.split) > 0 and any(d > D.k for (d, *_) in D.pairs)


def test_the_pin_catches_a_particle_kept_in_its_self_interaction():
    """Planted mistake: without leaving the particle itself out of its self
    interaction every iterating particle gains a pair with itself (r = 0 < H_i),
    which the comparison with brute force catches."""
    box = inputs.lattice_box(16, jitter=0.2, seed=3)
    H = sph.support_radius(box.h)
    D = dc.decompose(box.x, H, box.L, True, leaf_max=16)
    active = np.zeros(box.n, bool)
    active[::7] = True
    want = _brute(box.x, H, box.L, True, active)
    assert set(_gathered_visits(D, box.x, H, box.L, True, active)) == want
    bad = _gathered_visits(D, box.x, H, box.L, True, active, leave_self_out=False)
    assert set(bad) != want and {(p, q) for (p, q) in bad if p == q} == {(i, i) for i in np.nonzero(active)[0]}
