"""GPU path (through the C-ABI) against the FP64 oracle.

Bars: neighbour counts, cells and interaction lists bit-exact; rho, nw, P, c, f
within 1e-5 relative; d rho/dh within 2e-5 of 3 rho/h; accelerations and du/dt
within 1e-4 of their rms; vsig within 1e-5 relative; converged h within 1e-4
relative (the h tolerance 1e-4 on N~ bounds two converged solutions to
2/3 x 1e-4 apart); conservation sums within 1e-5 of the sum of magnitudes.
"""
import os

import numpy as np
import pytest

from oracle import decomposition as dc
from oracle import sph as orc
from paper_1309_3783_gb300 import inputs

pytestmark = pytest.mark.gpu

# axis numbering of sph_get_interactions (include/sph.h): db from cell a to cell b
GPU_AXES = [(1, 0, 0), (-1, 1, 0), (0, 1, 0), (1, 1, 0), (-1, -1, 1), (0, -1, 1), (1, -1, 1),
            (-1, 0, 1), (0, 0, 1), (1, 0, 1), (-1, 1, 1), (0, 1, 1), (1, 1, 1)]


@pytest.fixture(scope="module")
def api():
    from paper_1309_3783_gb300 import build, sph
    build.build()
    return sph


def make_ctx(api, **kw):
    p = api.sph_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    return api.sph_ctx_create(p, device=0)


@pytest.fixture(scope="module")
def ctx(api):
    c = make_ctx(api)
    yield c
    api.sph_ctx_destroy(c)


def gpu_fixed_h(api, ctx, box, force=True):
    b = api.box_from(ctx, box)
    try:
        b.density()
        out = {k: b.get(k) for k in ("count", "rho", "nw", "drho_dh", "nngb", "P", "c", "f")}
        if force:
            b.force()
            for k in ("a", "dudt", "vsig", "reductions"):
                out[k] = b.get(k)
        out["stats"] = b.stats()
    finally:
        b.close()
    return out


def _test_name():
    return os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0].split("::")[-1]


def max_rel(got, ref):
    """Largest |got - ref| / |ref| (absolute where ref is 0, e.g. v_sig of a particle without approaching pairs)."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref) / np.where(ref != 0.0, np.abs(ref), 1.0))) if ref.size else 0.0


def check_density(g, ref, box, idx=None):
    idx = np.arange(box.n) if idx is None else idx
    assert np.array_equal(g["count"][idx], ref["count"]), np.nonzero(g["count"][idx] != ref["count"])
    np.testing.assert_allclose(g["rho"][idx], ref["rho"], rtol=1e-5)
    np.testing.assert_allclose(g["nw"][idx], ref["nw"], rtol=1e-5)
    h = box.h.astype(np.float64)[idx]
    drho = orc.drho_dh(ref, h)
    dd = np.abs(g["drho_dh"][idx] - drho) / (3 * ref["rho"] / h)
    assert np.all(dd <= 2e-5)
    # measured errors against the FP64 oracle (shown with pytest -s)
    print(f"[errors vs FP64] {_test_name()}: {len(idx)} particles, counts exact; rho max rel "
          f"{max_rel(g['rho'][idx], ref['rho']):.1e}, sum W {max_rel(g['nw'][idx], ref['nw']):.1e}, "
          f"drho/dh {float(dd.max()):.1e} of 3 rho/h")


def check_force(g, ref, idx=None, ref_all=None, floor=0.0):
    """floor: a force scale for configurations whose exact forces vanish (lattices at rest)."""
    idx = slice(None) if idx is None else idx
    scale_src = ref if ref_all is None else ref_all
    rms = max(np.sqrt(np.mean(np.sum(scale_src["a"] ** 2, axis=1))), floor)
    ea = np.max(np.abs(g["a"][idx] - ref["a"]))
    assert ea <= 1e-4 * rms
    rms_u = max(np.sqrt(np.mean(scale_src["dudt"] ** 2)), floor)
    eu = np.max(np.abs(g["dudt"][idx] - ref["dudt"]))
    assert eu <= 1e-4 * rms_u
    np.testing.assert_allclose(g["vsig"][idx], ref["vsig"], rtol=1e-5)
    print(f"[errors vs FP64] {_test_name()}: {len(ref['vsig'])} particles; a max {ea / rms:.1e} of rms, "
          f"du/dt max {eu / rms_u:.1e} of rms, v_sig max rel {max_rel(g['vsig'][idx], ref['vsig']):.1e}")


# ------------------------------------------------------------------ fixed h
def test_c1_lattice_4096_fixed_h(api, ctx):
    """4096 particles, 16^3 lattice jittered by +-0.1 spacing, h = 1.2348 spacing."""
    box = inputs.lattice_box(16, jitter=0.1, seed=1)
    g = gpu_fixed_h(api, ctx, box)
    ref = orc.full_step(box, iterate_h=False)
    check_density(g, ref, box)
    np.testing.assert_allclose(g["P"], ref["P"], rtol=1e-5)
    np.testing.assert_allclose(g["c"], ref["c"], rtol=1e-5)
    np.testing.assert_allclose(g["f"], ref["f"], rtol=1e-5)
    check_force(g, ref)
    m = box.m.astype(np.float64)
    red = g["reductions"]
    assert np.all(np.abs(red[0:3]) <= 1e-5 * np.sum(m * np.linalg.norm(ref["a"], axis=1)))
    assert abs(red[3]) <= 1e-5 * np.sum(m * np.abs(ref["dudt"])) + 1e-5 * np.sum(m * np.abs((box.v * ref["a"]).sum(1)))
    np.testing.assert_allclose(red[4:8], ref["reductions"][4:8], rtol=1e-6, atol=1e-9)


def test_perfect_lattice_56_neighbours(api, ctx):
    box = inputs.lattice_box(16, jitter=0.0, v_sigma=0.0)
    g = gpu_fixed_h(api, ctx, box)
    assert np.all(g["count"] == 56)
    ref = orc.full_step(box, iterate_h=False)
    np.testing.assert_allclose(g["rho"], ref["rho"], rtol=1e-6)
    scale = np.max(ref["P"] / ref["rho"]) * 16
    assert np.max(np.abs(g["a"])) < 1e-4 * scale       # a lattice at rest feels no force


def _h_for_support(H):
    """An FP32 h whose support radius rounds to exactly H."""
    h = np.float32(H / float(orc.GAMMA_K))
    for _ in range(64):
        got = np.float32(orc.GAMMA_K * h)
        if got == np.float32(H):
            return h
        h = np.nextafter(h, np.float32(np.inf) if got < H else np.float32(0))
    raise AssertionError("no FP32 h maps to H")


def test_exact_ties_at_the_cutoff(api, ctx):
    """H = 2 spacing exactly on a perfect lattice: the 6 neighbours at distance 2a are out."""
    box = inputs.lattice_box(16, jitter=0.0, v_sigma=0.0)
    box.h[:] = _h_for_support(2.0 / 16)
    g = gpu_fixed_h(api, ctx, box, force=True)
    assert np.all(g["count"] == 6 + 12 + 8)
    assert g["stats"]["n_pairs"] > 0
    ref = orc.full_step(box, iterate_h=False)
    check_density(g, ref, box)
    # the lattice is at rest: forces vanish; bound the error by the pressure force scale P / (rho H)
    check_force(g, ref, floor=float(np.max(ref["P"] / ref["rho"] / ref["H"])))


def test_ragged_sizes_and_tiny_boxes(api, ctx):
    for n_side, jit in ((3, 0.3), (5, 0.2), (11, 0.45)):
        box = inputs.lattice_box(n_side, jitter=jit, seed=n_side)
        box.h[:] = np.minimum(box.h, np.float32(0.12))    # periodic boxes need H < L/4
        g = gpu_fixed_h(api, ctx, box)
        ref = orc.full_step(box, iterate_h=False)
        check_density(g, ref, box)
        check_force(g, ref)


def test_single_particle(api, ctx):
    box = inputs.lattice_box(1, jitter=0.0)
    box.h[:] = 0.1
    g = gpu_fixed_h(api, ctx, box)
    assert g["count"][0] == 0
    np.testing.assert_allclose(g["rho"][0], box.m[0] * orc.kernel_w(0.0, orc.support_radius(box.h)[0]), rtol=1e-6)
    assert np.all(g["a"] == 0)


def test_plummer_variable_h_with_splits(api):
    box = inputs.plummer_box(n=20000, n_spheres=4, scale=0.05, seed=3)
    api_ctx = make_ctx(api, leaf_max=48)
    try:
        g = gpu_fixed_h(api, api_ctx, box)
    finally:
        api.sph_ctx_destroy(api_ctx)
    assert g["stats"]["n_cells"] > g["stats"]["n_selfs"]      # the tree was split
    ref = orc.full_step(box, iterate_h=False, method="kdtree")
    check_density(g, ref, box)
    check_force(g, ref)


def test_open_box_and_box_length(api, ctx):
    box = inputs.plummer_box(n=6000, n_spheres=2, scale=0.06, seed=8)
    L = 3.7
    box.x *= L
    box.x[box.x >= L] = 0.0
    box.h *= np.float32(L)
    box.m *= np.float32(L ** 3)
    box.L = L
    for periodic in (True, False):
        box.periodic = periodic
        g = gpu_fixed_h(api, ctx, box)
        ref = orc.full_step(box, iterate_h=False, method="kdtree")
        check_density(g, ref, box)
        check_force(g, ref)


# ------------------------------------------------------------------ interacting pair sets
def _pair_set_case(name):
    if name == "lattice4096":
        return inputs.lattice_box(16, jitter=0.1, seed=1), 400
    box = inputs.plummer_box(n=20000, n_spheres=4, scale=0.05, seed=3)
    return box, (4800 if name.endswith("leaf4800") else 48)


@pytest.mark.parametrize("case", ["lattice4096", "plummer20000", "plummer20000_leaf4800"])
def test_interacting_pair_sets_equal_brute_force(api, case):
    """Section II-B: every pair within max(H_i, H_j) lies in exactly one self- or
    pair-interaction.  The density kernel's pair and side counters and the force
    kernel's pair counter and per-particle partner counts equal brute force: a
    pair dropped or visited twice changes them (its force term can be below the
    force tolerance, dW/dr vanishing at the cutoff)."""
    box, leaf = _pair_set_case(case)
    c = make_ctx(api, leaf_max=leaf)
    try:
        b = api.box_from(c, box)
        try:
            b.count_pairs(True)
            b.density()
            sd = b.stats()
            cnt = b.get("count")
            b.force()
            sf = b.stats()
            fcnt = b.get("force_count")
        finally:
            b.close()
    finally:
        api.sph_ctx_destroy(c)
    H = orc.support_radius(box.h)
    method = "brute" if box.n <= 4096 else "kdtree"
    t, j, _, _ = orc.neighbour_pairs(box.x, None, box.L, True, None, "force", Hall=H, method=method)
    per = np.bincount(t, minlength=box.n)
    n_unordered = len(t) // 2
    if box.n <= 4096:
        assert len(dc.interacting_pairs_brute(box.x, H, box.L, True)) == n_unordered
    ref = orc.density(box.x, box.m, H, box.L, True, method=method)
    assert np.array_equal(cnt, ref["count"])
    assert sd["density_pairs"] == n_unordered
    assert sd["density_sides"] == int(ref["count"].sum())
    assert sf["force_pairs"] == n_unordered
    assert np.array_equal(fcnt, per), np.nonzero(fcnt != per)[0][:10]
    print(f"[pair sets] {case}: {n_unordered} unordered pairs within max(H_i, H_j), "
          f"{sd['density_candidates']} density and {sf['force_candidates']} force candidates evaluated")


# ------------------------------------------------------------------ decomposition
@pytest.mark.parametrize("headroom", [0.0, 0.1])
def test_decomposition_matches_the_paper_rules(api, headroom):
    """Cells, selfs and pairs equal the oracle's; headroom 0 is the paper's rule."""
    box = inputs.plummer_box(n=8000, n_spheres=3, scale=0.04, seed=5)
    leaf = 32
    c = make_ctx(api, leaf_max=leaf, split_headroom=headroom)
    try:
        b = api.box_from(c, box)
        b.build()
        cells = b.cells()
        items = b.interactions()
        b.close()
    finally:
        api.sph_ctx_destroy(c)
    D = dc.decompose(box.x, orc.support_radius(box.h), box.L, True, leaf_max=leaf, headroom=headroom)
    keys = [(int(l), tuple(int(v) for v in ijk)) for l, ijk in zip(cells["level"], cells["ijk"])]
    assert set(keys) == set(D.cells)
    for k, cnt, sp in zip(keys, cells["count"], cells["split"]):
        assert cnt == len(D.cells[k]) and bool(sp) == (k in D.split)
    selfs = {keys[a] for kd, a in zip(items["kind"], items["a"]) if kd == 0}
    assert selfs == D.selfs
    pairs = set()
    for kd, a, bb, ax in zip(items["kind"], items["a"], items["b"], items["axis"]):
        if kd == 1:
            (d, ca), (_, cb) = keys[a], keys[bb]
            pairs.add((d, ca, cb, GPU_AXES[ax]))
    assert pairs == D.pairs


# ------------------------------------------------------------------ h iteration
def _gpu_iterate(api, ctx, box):
    b = api.box_from(ctx, box)
    st, nu, it = b.h_update()
    out = {"h": b.get("h"), "rho": b.get("rho"), "nngb": b.get("nngb"), "conv": b.get("converged"),
           "iters": it, "unconverged": nu, "stats": b.stats()}
    b.force()
    out["a"] = b.get("a")
    b.close()
    return out


def test_h_iteration_matches_oracle(api, ctx):
    box = inputs.lattice_box(16, jitter=0.3, seed=4)
    box.h = (box.h * np.random.default_rng(2).uniform(0.7, 1.4, box.n)).astype(np.float32)
    g = _gpu_iterate(api, ctx, box)
    assert g["unconverged"] == 0 and g["conv"].all()
    assert np.all(np.abs(g["nngb"] - 48) <= 1e-4 * 48 * 1.01)
    h, conv, it, dens = orc.h_iterate(box.x, box.m, box.h, box.L, True, tol=1e-4)
    assert conv.all()
    np.testing.assert_allclose(g["h"], h, rtol=1e-4)


def test_h_iteration_variable_h_with_rebuild(api):
    box = inputs.plummer_box(n=20000, n_spheres=4, scale=0.03, seed=6)
    box.h = (box.h * np.float32(0.6)).astype(np.float32)   # forces h to grow past the cell splits
    c = make_ctx(api, leaf_max=64)
    try:
        g = _gpu_iterate(api, c, box)
    finally:
        api.sph_ctx_destroy(c)
    assert g["unconverged"] == 0
    h, conv, it, dens = orc.h_iterate(box.x, box.m, box.h, box.L, True, tol=1e-4, method="kdtree")
    assert conv.all()
    np.testing.assert_allclose(g["h"], h, rtol=1e-4)
    np.testing.assert_allclose(g["rho"], dens["rho"], rtol=3e-4)


# ------------------------------------------------------------------ inputs and errors
def test_invalid_inputs_are_rejected(api, ctx):
    box = inputs.lattice_box(6, jitter=0.2)
    for mutate, status in (
        (lambda b: b.x.__setitem__((3, 1), np.nan), "SPH_E_INVALID"),
        (lambda b: b.x.__setitem__((4, 0), b.L), "SPH_E_INVALID"),
        (lambda b: b.h.__setitem__(5, 0.0), "SPH_E_INVALID"),
        (lambda b: b.m.__setitem__(2, -1.0), "SPH_E_INVALID"),
        (lambda b: b.h.__setitem__(0, 0.3), "SPH_E_H_TOO_LARGE"),
    ):
        bad = box.subset(np.arange(box.n))
        mutate(bad)
        b = api.box_from(ctx, bad)
        with pytest.raises(api.SphError) as e:
            b.density()
        assert status in str(e.value)
        b.close()
    with pytest.raises(api.SphError):
        api.sph_box_create(ctx, 0, 1.0, True)


def test_device_pointers_match_host_path(api, ctx):
    torch = pytest.importorskip("torch")
    box = inputs.lattice_box(10, jitter=0.3, seed=12, v_sigma=0.1)
    host = gpu_fixed_h(api, ctx, box)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    b = api.Box(ctx, box.n, box.L, True)
    b.set(d(box.x), d(box.v), d(box.m), d(box.u), d(box.h))
    b.density()
    b.force()
    rho = torch.empty(box.n, dtype=torch.float32, device="cuda")
    b.get("rho", out=rho)
    torch.cuda.synchronize()
    np.testing.assert_allclose(rho.cpu().numpy(), host["rho"], rtol=1e-6)
    np.testing.assert_array_equal(b.get("count"), host["count"])
    b.close()


# ------------------------------------------------------------------ full-size workload, sampled
@pytest.mark.slow
def test_plummer_262144_sampled(api, ctx):
    """The 262,144-particle variable-h box (16 Plummer spheres + background): sampled parity."""
    box = inputs.plummer_box()
    g = gpu_fixed_h(api, ctx, box)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(box.n, 2000, replace=False))
    H = orc.support_radius(box.h)
    ref = orc.density(box.x, box.m, H, box.L, True, targets=idx, method="kdtree")
    check_density(g, ref, box, idx)
    # force on a smaller sample needs every neighbour's density: take it for all
    dens = orc.density(box.x, box.m, H, box.L, True, method="kdtree")
    gh = orc.ghost(dens["rho"], dens["Sr_m"], box.u)
    fi = idx[:500]
    fo = orc.force(box.x, box.v, box.m, H, dens["rho"], gh["P"], gh["c"], gh["f"], box.L, True,
                   targets=fi, method="kdtree")
    check_force(g, fo, fi)
    # h iteration from the same start: every particle's iteration is independent
    gi = _gpu_iterate(api, ctx, box)
    assert gi["unconverged"] == 0
    hs, conv, _, _ = orc.h_iterate(box.x, box.m, box.h, box.L, True, tol=1e-4, targets=idx[:300],
                                   method="kdtree")
    assert conv.all()
    np.testing.assert_allclose(gi["h"][idx[:300]], hs, rtol=1e-4)


def test_h_iteration_limit_reports_unconverged_particles(api):
    """With the iteration limit reached, the particles still off the target are
    reported (SPH_E_NOT_CONVERGED and their count) and keep the h of their last
    iteration, as in the oracle."""
    box = inputs.lattice_box(16, jitter=0.3, seed=12)
    box.h = (box.h * np.float32(0.7)).astype(np.float32)
    c = make_ctx(api, h_max_iter=2)
    try:
        b = api.box_from(c, box)
        try:
            st, nu, it = b.h_update()
            conv = b.get("converged")
            h = b.get("h")
        finally:
            b.close()
    finally:
        api.sph_ctx_destroy(c)
    assert it == 2 and nu > 0 and st == api.SPH_E_NOT_CONVERGED
    assert nu == int(np.count_nonzero(conv == 0))
    ho, convo, _, _ = orc.h_iterate(box.x, box.m, box.h, box.L, True, tol=1e-4, max_iter=2)
    np.testing.assert_allclose(h, ho, rtol=1e-4)
    assert abs(int(np.count_nonzero(~convo)) - nu) <= max(2, nu // 100)


def test_h_iteration_results_exact_at_the_final_h(api, ctx):
    """Every particle's count and density come from the pass in which its h
    converged; growing and shrinking h over several later passes (which evaluate
    only the particles still iterating, culled against their clusters' current
    largest H) must leave them equal to the oracle at the final h."""
    box = inputs.plummer_box(n=20000, n_spheres=4, scale=0.03, seed=12)
    box.h = (box.h * np.random.default_rng(3).uniform(0.75, 1.3, box.n)).astype(np.float32)
    b = api.box_from(ctx, box)
    try:
        st, nu, it = b.h_update()
        g = {k: b.get(k) for k in ("h", "count", "rho", "converged")}
    finally:
        b.close()
    assert nu == 0 and g["converged"].all() and it >= 3
    H = orc.support_radius(g["h"])
    ref = orc.density(box.x, box.m, H, box.L, True, method="kdtree")
    assert np.array_equal(g["count"], ref["count"])
    np.testing.assert_allclose(g["rho"], ref["rho"], rtol=1e-5)


def _perturbed_run(api, box, h, **kw):
    c = make_ctx(api, **kw)
    try:
        b = api.box_from(c, box)
        try:
            b.set_field("h", h)
            st, nu, it = b.h_update()
            out = {k: b.get(k) for k in ("h", "count", "rho")}
            out["stats"], out["it"] = b.stats(), it
        finally:
            b.close()
    finally:
        api.sph_ctx_destroy(c)
    return out


@pytest.mark.parametrize("leaf,mode", [(48, "random"), (48, "region"), (4800, "random")])
def test_gathered_later_passes_equal_the_symmetric_passes(api, leaf, mode):
    """Section II-D: a later pass of the h iteration evaluates the particles still
    iterating.  With at most an eighth of them iterating it gathers
    (sph_params.h_gather): each leaf's iterating particles packed into clusters,
    every interaction run for them from their own side.  Every run, with one
    later pass (h_max_iter 2) or iterated to convergence, in either mode, has
    counts exact and densities within the bar against the oracle at its final h;
    the two modes evaluate the same h after one later pass and converge to the
    same h.  5 % of the particles iterate, spread at random or gathered around
    one particle."""
    box = inputs.plummer_box(n=20000, n_spheres=4, scale=0.05, seed=5)
    c0 = make_ctx(api, leaf_max=leaf)
    try:
        b = api.box_from(c0, box)
        try:
            b.h_update()
            h0 = b.get("h")
        finally:
            b.close()
    finally:
        api.sph_ctx_destroy(c0)
    rng = np.random.default_rng(7)
    if mode == "random":
        k = rng.choice(box.n, box.n // 20, replace=False)
    else:
        d = box.x - box.x[rng.integers(box.n)]
        d -= box.L * np.round(d / box.L)
        k = np.argsort((d * d).sum(axis=1))[: box.n // 20]
    h1 = h0.copy()
    h1[k] *= rng.uniform(0.97, 1.03, k.size).astype(np.float32)   # within the split headroom: no rebuild
    res = {(g, mi): _perturbed_run(api, box, h1, leaf_max=leaf, h_gather=g, h_max_iter=mi)
           for g in (0, 1) for mi in (2, 30)}
    for key, r in res.items():
        assert r["stats"]["rebuilds"] == 0, key
    assert res[(1, 2)]["stats"]["h_gathered_passes"] == 1
    assert res[(0, 2)]["stats"]["h_gathered_passes"] == 0
    assert res[(1, 30)]["stats"]["h_gathered_passes"] >= 1
    assert res[(0, 30)]["stats"]["h_gathered_passes"] == 0
    # each run exact against the oracle at its own final h (the density sums are
    # float atomics in no fixed order, so two runs' h may differ in the last bits)
    refs = {}
    for key, r in res.items():
        ref = orc.density(box.x, box.m, orc.support_radius(r["h"]), box.L, True, method="kdtree")
        assert np.array_equal(r["count"], ref["count"]), key
        np.testing.assert_allclose(r["rho"], ref["rho"], rtol=1e-5, err_msg=str(key))
        refs[key] = ref
    g1, s1, g30, s30 = res[(1, 2)], res[(0, 2)], res[(1, 30)], res[(0, 30)]
    # one later pass: both modes evaluate the h of the first pass's Newton step
    np.testing.assert_allclose(g1["h"], s1["h"], rtol=1e-6)
    np.testing.assert_allclose(g1["rho"], s1["rho"], rtol=1e-5)
    # the full iteration converges to the same h
    np.testing.assert_allclose(g30["h"], s30["h"], rtol=1e-4)
    print(f"[gather] leaf {leaf} {mode}: {g30['it']} passes, {g30['stats']['h_gathered_passes']} gathered; "
          f"rho max rel: one later pass to the symmetric pass {max_rel(g1['rho'], s1['rho']):.1e}, "
          f"the full iteration to FP64 {max_rel(g30['rho'], refs[(1, 30)]['rho']):.1e}")


def test_compensated_sums_at_high_neighbour_counts(api):
    """With about 400 neighbours per particle the FP32 density sums carry ~20x
    more rounding than at 48; compensated summation (sph_params.compensated)
    brings them back to the error of the terms themselves."""
    box = inputs.lattice_box(24, jitter=0.3, seed=21)
    box.h = (box.h * np.float32((400.0 / 48.0) ** (1.0 / 3.0))).astype(np.float32)
    H = orc.support_radius(box.h)
    ref = orc.density(box.x, box.m, H, box.L, True, method="kdtree")
    err = {}
    for comp in (0, 1):
        c = make_ctx(api, compensated=comp)
        try:
            b = api.box_from(c, box)
            try:
                b.density()
                got = {k: b.get(k) for k in ("count", "rho", "nw")}
            finally:
                b.close()
        finally:
            api.sph_ctx_destroy(c)
        assert np.array_equal(got["count"], ref["count"])
        err[comp] = max(np.max(np.abs(got["rho"] / ref["rho"] - 1.0)), np.max(np.abs(got["nw"] / ref["nw"] - 1.0)))
        np.testing.assert_allclose(got["rho"], ref["rho"], rtol=1e-5)
    print(f"mean neighbours {ref['count'].mean():.0f}; max relative error of rho and sum W: plain {err[0]:.2e}, "
          f"compensated {err[1]:.2e}")
    assert err[1] < err[0]


# ------------------------------------------------------------------ position precision
def test_plain_fp32_positions_keep_counts_but_lose_accuracy(api):
    """Plain FP32 positions (sph_params.precision = 1: x / L rounded to FP32 in the
    box frame) against the default offsets from each cell's centre, on a box with
    dense cores (support radii down to ~1e-4 L).  Both keep the neighbour counts
    and the force pair sets exact (the guard band covers each rounding, and pairs
    inside it are decided in FP64), but plain FP32 positions carry an absolute
    error of up to 2^-25 L, a large relative error at small separations: the
    densities and forces drift from the FP64 oracle by far more than with offsets
    whose rounding scales with the cell.  The dense cores here straddle cell
    boundaries inside pairs of large cells that cannot split (their other
    particles have large H): pair tasks take the own leaf's frame, so that those
    positions are still rounded at the leaf's scale."""
    box = inputs.plummer_box(n=20000, n_spheres=2, scale=0.002, seed=7)
    # both modes at the same converged h (N~ = 48), taken from one h iteration
    c = make_ctx(api)
    try:
        b = api.box_from(c, box)
        try:
            st, nu, _ = b.h_update()
            box.h = b.get("h")
        finally:
            b.close()
    finally:
        api.sph_ctx_destroy(c)
    assert nu == 0
    H = orc.support_radius(box.h)
    ref = orc.full_step(box, iterate_h=False, method="kdtree")
    print(f"[precision] neighbour counts up to {int(ref['count'].max())} (median {int(np.median(ref['count']))})")
    t, _, _, _ = orc.neighbour_pairs(box.x, None, box.L, True, None, "force", Hall=H, method="kdtree")
    per = np.bincount(t, minlength=box.n)
    rms = np.sqrt(np.mean(np.sum(ref["a"] ** 2, axis=1)))
    err, rechecks = {}, {}
    for prec in (0, 1):
        c = make_ctx(api, precision=prec, leaf_max=48)
        try:
            b = api.box_from(c, box)
            try:
                b.count_pairs(True)
                b.density()
                g = {k: b.get(k) for k in ("count", "rho")}
                b.force()
                g["a"], g["fc"] = b.get("a"), b.get("force_count")
                rechecks[prec] = b.stats()["guard_rechecks"]
            finally:
                b.close()
        finally:
            api.sph_ctx_destroy(c)
        assert np.array_equal(g["count"], ref["count"]), prec
        assert np.array_equal(g["fc"], per), prec
        err[prec] = (max_rel(g["rho"], ref["rho"]), float(np.max(np.abs(g["a"] - ref["a"])) / rms))
    print(f"[precision] H in [{H.min():.1e}, {H.max():.1e}]: cell offsets rho {err[0][0]:.1e}, a {err[0][1]:.1e} of rms, "
          f"{rechecks[0]} FP64 decisions; plain FP32 rho {err[1][0]:.1e}, a {err[1][1]:.1e} of rms, "
          f"{rechecks[1]} FP64 decisions")
    assert err[0][0] <= 1e-5 and err[0][1] <= 1e-4
    assert err[1][0] > 10 * err[0][0]
    assert rechecks[1] > rechecks[0]
