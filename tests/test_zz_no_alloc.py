"""The allocation-free density entry point against sph_density.

sph_density_static serves callers that cannot allocate device memory: it keeps
its working memory in one static device array instead.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_1309_3783_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1309_3783_gb300 import build, sph
    build.build()
    return sph


def _reference(api, box):
    ctx = api.sph_ctx_create(device=0)
    b = api.box_from(ctx, box)
    try:
        b.density()
        out = b.get("rho"), b.get("count")
    finally:
        b.close()
        api.sph_ctx_destroy(ctx)
    return out


@pytest.mark.parametrize("periodic", [True, False])
def test_static_density_matches_sph_density_twice(api, periodic):
    import torch
    box = inputs.lattice_box(16, jitter=0.3, seed=77, v_sigma=0.0, periodic=periodic)
    box.h = (box.h * np.random.default_rng(5).uniform(0.8, 1.2, box.n)).astype(np.float32)
    rho_ref, cnt_ref = _reference(api, box)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    x, m, h = d(box.x), d(box.m), d(box.h)
    for call in range(2):                       # the shared array keeps the last call's contents
        rho = torch.full((box.n,), -1.0, dtype=torch.float32, device="cuda")
        cnt = torch.full((box.n,), -1, dtype=torch.int32, device="cuda")
        st = api.sph_density_static(x, m, h, box.L, periodic, rho, cnt)
        assert st == 0, (call, st)
        assert np.array_equal(cnt.cpu().numpy(), cnt_ref), call
        np.testing.assert_allclose(rho.cpu().numpy(), rho_ref, rtol=1e-5)


def test_static_density_rejects_sizes_beyond_its_array(api):
    import torch
    n = api.SPH_STATIC_MAX_N + 1
    x = torch.full((3 * n,), 0.5, dtype=torch.float64, device="cuda")
    f = torch.ones(n, dtype=torch.float32, device="cuda")
    c = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert api.sph_density_static(x, f, f * 0.01, 1.0, True, f.clone(), c) == -1   # SPH_E_INVALID
