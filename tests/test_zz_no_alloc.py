"""The allocation-free density entry point against sph_density and the oracle.

sph_density_static serves callers that cannot allocate device memory: it keeps
its working memory in one static device array instead.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from oracle import sph as orc
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()


def _static(api, box, stream=0):
    import torch
    rho = torch.full((box.n,), -1.0, dtype=torch.float32, device="cuda")
    cnt = torch.full((box.n,), -1, dtype=torch.int32, device="cuda")
    st = api.sph_density_static(_dev(box.x), _dev(box.m), _dev(box.h), box.L, box.periodic, rho, cnt, stream)
    return st, rho.cpu().numpy(), cnt.cpu().numpy()


@pytest.mark.parametrize("periodic", [True, False])
def test_static_density_matches_sph_density_twice(api, periodic):
    box = inputs.lattice_box(16, jitter=0.3, seed=77, v_sigma=0.0, periodic=periodic)
    box.h = (box.h * np.random.default_rng(5).uniform(0.8, 1.2, box.n)).astype(np.float32)
    rho_ref, cnt_ref = _reference(api, box)
    ref = orc.density(box.x, box.m, orc.support_radius(box.h), box.L, periodic)
    for call in range(2):                       # the shared array keeps the last call's contents
        st, rho, cnt = _static(api, box)
        assert st == 0, (call, st)
        assert np.array_equal(cnt, cnt_ref), call
        np.testing.assert_allclose(rho, rho_ref, rtol=1e-5)
        assert np.array_equal(cnt, ref["count"]), call
        np.testing.assert_allclose(rho, ref["rho"], rtol=1e-5)


def test_static_density_sparse_box_and_side_stream(api):
    """Support radii far below L/32: the cell list stays at its 32^3 cells (cells
    wider than H_max).  The call runs on a side stream."""
    import torch
    rng = np.random.default_rng(9)
    n = 8000
    box = inputs.lattice_box(20, jitter=0.0, seed=1)            # the container; particles replaced below
    box = box.subset(np.arange(n))
    box.x = rng.uniform(0.0, 1.0, (n, 3))
    box.h = rng.uniform(0.008, 0.016, n).astype(np.float32)
    box.m = np.full(n, 1.0 / n, np.float32)
    ref = orc.density(box.x, box.m, orc.support_radius(box.h), box.L, True)
    assert ref["count"].sum() > 0
    rho_ref, cnt_ref = _reference(api, box)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    st, rho, cnt = _static(api, box, s.cuda_stream)
    assert st == 0
    assert np.array_equal(cnt, ref["count"]) and np.array_equal(cnt, cnt_ref)
    np.testing.assert_allclose(rho, ref["rho"], rtol=1e-5)


def test_static_density_rejects_invalid_inputs(api):
    box = inputs.lattice_box(8, jitter=0.2, seed=3)
    for mutate, want in (
        (lambda b: b.h.__setitem__(5, -0.01), -1),            # SPH_E_INVALID
        (lambda b: b.h.__setitem__(6, 0.0), -1),
        (lambda b: b.x.__setitem__((4, 0), b.L), -1),         # x == L is outside [0, L)
        (lambda b: b.x.__setitem__((2, 2), np.nan), -1),
        (lambda b: b.m.__setitem__(1, 0.0), -1),
        (lambda b: b.h.__setitem__(0, 0.2), -3),              # SPH_E_H_TOO_LARGE: H_max > L / 3
    ):
        bad = box.subset(np.arange(box.n))
        mutate(bad)
        st, _, _ = _static(api, bad)
        assert st == want, (st, want)
    st, _, _ = _static(api, box)                              # a valid call still works afterwards
    assert st == 0


def test_static_density_rejects_sizes_beyond_its_array(api):
    import torch
    n = api.SPH_STATIC_MAX_N + 1
    x = torch.full((3 * n,), 0.5, dtype=torch.float64, device="cuda")
    f = torch.ones(n, dtype=torch.float32, device="cuda")
    c = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert api.sph_density_static(x, f, f * 0.01, 1.0, True, f.clone(), c) == -1   # SPH_E_INVALID
