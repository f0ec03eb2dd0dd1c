"""Spatial decomposition of one box over four ranks with the library as each
rank's computation (the GPU path of paper_1309_3783_gb300.spatial).

The four ranks are processes that share this one GPU, each with its own
context; their exchanges are gloo all-gathers on the host, so no kernel of one
rank waits for another's.  Owned results must equal one library box over all
particles at the same h: counts exact, densities and forces within the parity
tolerances (the FP32 sums run in another order), the conservation sums added
over ranks equal to the whole box's.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402

from tests.test_spatial import WORLD, _box, run_ranks  # noqa: E402

pytestmark = pytest.mark.gpu


def _gpu_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1309_3783_gb300 import build, spatial, sph
    build.build()
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ctx = sph.sph_ctx_create(device=0)
    try:
        box = _box()
        bounds = spatial.slab_bounds(box.x[:, 0], world, box.L)
        idx = np.nonzero(spatial.owners(box.x[:, 0], bounds) == rank)[0]
        res, nhalo, width = spatial.spatial_passes(dist, box.subset(idx), idx, bounds,
                                                   spatial.LibraryCompute(sph, ctx), headroom=1.2)
        out[rank] = (idx, {k: np.asarray(v) for k, v in res.items()}, nhalo, width)
    finally:
        sph.sph_ctx_destroy(ctx)
        dist.destroy_process_group()


def test_spatial_slabs_on_the_gpu_equal_one_box():
    from paper_1309_3783_gb300 import build, sph
    build.build()
    res = run_ranks(_gpu_worker)
    box = _box()
    idx = np.concatenate([res[r][0] for r in range(WORLD)])
    assert np.array_equal(np.sort(idx), np.arange(box.n))
    h = np.zeros(box.n, np.float32)
    for r in range(WORLD):
        h[res[r][0]] = res[r][1]["h"]
    ctx = sph.sph_ctx_create(device=0)
    try:
        b = sph.box_from(ctx, box)
        try:
            st, nu, _ = b.h_update()
            h1 = b.get("h")
            b.set_field("h", h)
            b.density()
            b.force()
            ref = {k: b.get(k) for k in ("count", "rho", "a", "vsig", "reductions")}
        finally:
            b.close()
    finally:
        sph.sph_ctx_destroy(ctx)
    np.testing.assert_allclose(h, h1, rtol=1e-4)           # the h iteration, as in one box
    rms = np.sqrt(np.mean(np.sum(ref["a"].astype(np.float64) ** 2, axis=1)))
    for r in range(WORLD):
        i, g = res[r][0], res[r][1]
        assert np.array_equal(g["count"], ref["count"][i])
        np.testing.assert_allclose(g["rho"], ref["rho"][i], rtol=1e-5)
        assert np.max(np.abs(g["a"] - ref["a"][i])) <= 1e-4 * rms
        np.testing.assert_allclose(g["vsig"], ref["vsig"][i], rtol=1e-5)
    m = box.m.astype(np.float64)
    scale_p = np.sum(m * np.linalg.norm(ref["a"], axis=1))
    red = res[0][1]["reductions"]
    assert np.all(np.abs(red[0:3] - ref["reductions"][0:3]) <= 1e-5 * scale_p)
    np.testing.assert_allclose(red[4:8], ref["reductions"][4:8], rtol=1e-6, atol=1e-9)
    print(f"[spatial] {WORLD} ranks, halos {[int(res[r][2]) for r in range(WORLD)]} of {box.n} particles, "
          f"width {res[0][3]:.3f}: counts exact")
