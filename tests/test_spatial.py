"""Spatial decomposition of one periodic box over several ranks (Section IV of
the paper: distributed memory as future work), on CPU: gloo all-gathers for the
halo exchanges, the FP64 oracle as each rank's computation.

Every rank owns one slab of equal particle count and receives the particles of
the others within twice the largest support radius (a part of the box only).  Owned results must equal
the single-box oracle evaluated at the same h exactly (the same FP64 pair sums
and predicates; only the order of the sums differs), the h must equal the single-box
h iteration within its tolerance, the slabs must cover every particle once, and
the rank-summed conservation sums must equal the whole box's.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleCompute:
    """A rank's passes done by the FP64 oracle (test infrastructure)."""

    def h_iterate(self, box):
        from oracle import sph as orc
        h, conv, _, _ = orc.h_iterate(box.x, box.m, box.h, box.L, box.periodic, method="kdtree")
        return h.astype(np.float32)

    def passes(self, box, n_owned):
        from oracle import sph as orc
        out = orc.full_step(box, iterate_h=False, method="kdtree")
        k = slice(0, n_owned)
        red = orc.reductions(box.m[k], box.v[k], box.u[k], out["a"][k], out["dudt"][k])
        return {"count": out["count"], "rho": out["rho"], "a": out["a"], "dudt": out["dudt"], "vsig": out["vsig"],
                "reductions": red}


WORLD = 4


def _box():
    from paper_1309_3783_gb300 import inputs
    box = inputs.lattice_box(32, jitter=0.35, seed=5, v_sigma=0.1)
    box.h = (box.h * np.random.default_rng(6).uniform(0.8, 1.2, box.n)).astype(np.float32)
    box.u = np.random.default_rng(7).uniform(0.5, 1.5, box.n).astype(np.float32)
    return box


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1309_3783_gb300 import spatial
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        box = _box()                       # the same seeded box on every rank; each keeps its slab
        bounds = spatial.slab_bounds(box.x[:, 0], world, box.L)
        idx = np.nonzero(spatial.owners(box.x[:, 0], bounds) == rank)[0]
        res, nhalo, width = spatial.spatial_passes(dist, box.subset(idx), idx, bounds, OracleCompute(), headroom=1.2)
        out[rank] = (idx, {k: np.asarray(v) for k, v in res.items()}, nhalo, width)
    finally:
        dist.destroy_process_group()


def run_ranks(worker, world=WORLD):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(worker, args=(world, port, out), nprocs=world, join=True)
        return dict(out)


def test_slab_geometry_against_brute_force():
    from paper_1309_3783_gb300 import spatial
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, 5000)
    b = spatial.slab_bounds(x, 5, 1.0)
    own = spatial.owners(x, b)
    assert np.all(np.bincount(own, minlength=5) >= 999)
    for r in range(5):
        lo, hi = b[r], b[r + 1]
        assert np.all((x[own == r] >= lo) & (x[own == r] < hi))
        # periodic distance to the slab by brute force over images and a fine sample of the slab
        s = np.linspace(lo, hi, 2001)
        d = np.min(np.abs((x[:, None] - s[None, :] + 0.5) % 1.0 - 0.5), axis=1)
        np.testing.assert_allclose(spatial.slab_distance(x, b, r, 1.0), d, atol=(hi - lo) / 2000 + 1e-12)


def test_slabs_equal_the_single_box_oracle():
    from oracle import sph as orc
    res = run_ranks(_worker)
    box = _box()
    idx = np.concatenate([res[r][0] for r in range(WORLD)])
    assert np.array_equal(np.sort(idx), np.arange(box.n))          # every particle owned once
    for r in range(WORLD):
        assert 0 < res[r][2] < box.n - len(res[r][0])               # a halo, and only a part of the rest
    h = np.zeros(box.n, np.float32)
    for r in range(WORLD):
        h[res[r][0]] = res[r][1]["h"]
    # the h iteration: as in one box, within its tolerance
    hs, conv, _, _ = orc.h_iterate(box.x, box.m, box.h, box.L, True, method="kdtree")
    assert conv.all()
    np.testing.assert_allclose(h, hs, rtol=1e-4)
    # the passes: exactly the single-box oracle at the same h
    at = box.subset(np.arange(box.n))
    at.h = h
    ref = orc.full_step(at, iterate_h=False, method="kdtree")
    for r in range(WORLD):
        i, g = res[r][0], res[r][1]
        assert np.array_equal(g["count"], ref["count"][i])
        np.testing.assert_allclose(g["rho"], ref["rho"][i], rtol=1e-12)
        scale = np.sqrt(np.mean(np.sum(ref["a"] ** 2, axis=1)))
        assert np.max(np.abs(g["a"] - ref["a"][i])) <= 1e-10 * scale
        np.testing.assert_allclose(g["vsig"], ref["vsig"][i], rtol=1e-12)
    # the conservation sums, added over the ranks, are the whole box's
    np.testing.assert_allclose(res[0][1]["reductions"], ref["reductions"], rtol=1e-9, atol=1e-12)
    for r in range(1, WORLD):
        np.testing.assert_allclose(res[0][1]["reductions"], res[r][1]["reductions"], rtol=0, atol=0)
