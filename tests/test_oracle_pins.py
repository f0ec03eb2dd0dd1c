"""Pins of the FP64 oracle against mathematics it does not itself compute.

Each test checks one property that a plausible mistake in the oracle (a dropped
term, a wrong sign, a wrong support radius, a transposed operand, a broken
periodic wrap) would violate: kernel normalisation and its derivative, the
perfect-lattice neighbour count and closed-form density, finite differences of
density in h, the variational (Lagrangian) derivation of the pressure force and
of du/dt with grad-h terms, conservation of momentum and energy, two-particle
closed forms, the h-iteration's fixed point, and agreement of two independent
neighbour searches.
"""
import numpy as np
import pytest
from scipy import integrate, optimize

from oracle import sph
from paper_1309_3783_gb300 import inputs


# ---------------------------------------------------------------- kernel
@pytest.mark.parametrize("H", [0.1, 1.0, 3.7])
def test_kernel_normalisation(H):
    val, err = integrate.quad(lambda r: 4 * np.pi * r * r * sph.kernel_w(r, H), 0, H,
                              points=[0.5 * H], epsabs=1e-14, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


def test_kernel_values_and_continuity():
    H = 0.7
    assert np.isclose(sph.kernel_w(0.0, H), 8 / (np.pi * H ** 3), rtol=1e-15)
    assert np.isclose(sph.kernel_w(0.5 * H, H), 2 / (np.pi * H ** 3), rtol=1e-15)
    assert sph.kernel_w(H, H) == 0.0 and sph.kernel_w(1.5 * H, H) == 0.0
    assert sph.kernel_dwdr(0.0, H) == 0.0 and sph.kernel_dwdr(H, H) == 0.0
    eps = 1e-12
    for f in (sph.kernel_w, sph.kernel_dwdr):
        assert np.isclose(f((0.5 - eps) * H, H), f((0.5 + eps) * H, H), rtol=1e-9)


def test_kernel_derivative_matches_finite_difference():
    H = 1.3
    r = np.linspace(0.01, 0.99, 97) * H
    r = r[np.abs(r / H - 0.5) > 1e-3]
    dr = 1e-6 * H
    fd = (sph.kernel_w(r + dr, H) - sph.kernel_w(r - dr, H)) / (2 * dr)
    np.testing.assert_allclose(sph.kernel_dwdr(r, H), fd, rtol=1e-7, atol=1e-9)


# ---------------------------------------------------------------- lattice closed forms
def _lattice_shell_sum(H, a, fn):
    n = np.arange(-4, 5)
    v = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3)
    r = np.sqrt((v * v).sum(1)) * a
    r = r[r < H]
    return fn(r)


def test_perfect_lattice_count_and_density():
    box = inputs.lattice_box(16, jitter=0.0, v_sigma=0.0)
    H = sph.support_radius(box.h)
    d = sph.density(box.x, box.m, H, box.L, box.periodic)
    # shells |n|^2 = 1..5 lie inside H = 2.2544 a, |n|^2 = 6 outside: 6+12+8+6+24
    assert np.all(d["count"] == 56)
    a = box.meta["spacing"]
    Hs = float(H[0])
    rho_cf = float(box.m[0]) * _lattice_shell_sum(Hs, a, lambda r: sph.kernel_w(r, Hs).sum())
    np.testing.assert_allclose(d["rho"], rho_cf, rtol=1e-13)
    assert abs(rho_cf - 1.0039807835807686) < 2e-6     # value quoted for this lattice
    Nw = 4 * np.pi / 3 * Hs ** 3 * _lattice_shell_sum(Hs, a, lambda r: sph.kernel_w(r, Hs).sum())
    np.testing.assert_allclose(d["Nw"], Nw, rtol=1e-13)
    g = _lattice_shell_sum(Hs, a, lambda r: (3 * sph.kernel_w(r, Hs) + r * sph.kernel_dwdr(r, Hs)).sum())
    np.testing.assert_allclose(d["S"], g, rtol=1e-12)


def test_h_iteration_fixed_point_on_lattice():
    box = inputs.lattice_box(8, jitter=0.0, v_sigma=0.0)
    a = box.meta["spacing"]
    gk = float(sph.GAMMA_K)

    def Nw(h):
        H = gk * h
        return 4 * np.pi / 3 * H ** 3 * _lattice_shell_sum(H, a, lambda r: sph.kernel_w(r, H).sum()) - 48.0

    h_star = optimize.brentq(Nw, 1.0 * a, 1.6 * a, xtol=1e-15 * a)
    h0 = np.full(box.n, 1.1 * a)
    h, conv, it, _ = sph.h_iterate(box.x, box.m, h0, box.L, True, tol=1e-12, max_iter=50)
    assert conv.all()
    np.testing.assert_allclose(h, h_star, rtol=1e-10)


# ---------------------------------------------------------------- density derivatives
def test_density_h_derivative_matches_finite_difference():
    box = inputs.lattice_box(8, jitter=0.3, seed=3)
    h = box.h.astype(np.float64) * np.random.default_rng(0).uniform(0.9, 1.1, box.n)
    gk = float(sph.GAMMA_K)
    eps = 1e-6
    dp = sph.density(box.x, box.m, gk * h * (1 + eps), box.L, True)
    dm = sph.density(box.x, box.m, gk * h * (1 - eps), box.L, True)
    d0 = sph.density(box.x, box.m, gk * h, box.L, True)
    fd_rho = (dp["rho"] - dm["rho"]) / (2 * eps * h)
    np.testing.assert_allclose(sph.drho_dh(d0, h), fd_rho, rtol=1e-6)
    fd_n = (dp["nw"] - dm["nw"]) / (2 * eps * gk * h)     # d n / dH = -S / H
    np.testing.assert_allclose(-d0["S"] / (gk * h), fd_n, rtol=1e-6)


def test_h_iteration_is_self_consistent():
    box = inputs.lattice_box(10, jitter=0.4, seed=5)
    h0 = box.h.astype(np.float64) * np.random.default_rng(1).uniform(0.6, 1.6, box.n)
    tol = 1e-4
    h, conv, it, dens = sph.h_iterate(box.x, box.m, h0, box.L, True, tol=tol)
    assert conv.all() and it.max() < 30
    d = sph.density(box.x, box.m, float(sph.GAMMA_K) * h, box.L, True)
    assert np.all(np.abs(d["Nw"] - 48.0) <= tol * 48.0)
    np.testing.assert_allclose(d["rho"], dens["rho"], rtol=1e-14)


# ---------------------------------------------------------------- force
def _prepare(box, alpha=sph.ALPHA_VISC, tol=1e-12):
    h, conv, _, dens = sph.h_iterate(box.x, box.m, box.h, box.L, box.periodic, tol=tol, max_iter=60)
    assert conv.all()
    H = float(sph.GAMMA_K) * h
    g = sph.ghost(dens["rho"], dens["Sr_m"], box.u)
    fo = sph.force(box.x, box.v, box.m, H, dens["rho"], g["P"], g["c"], g["f"], box.L, box.periodic,
                   alpha=alpha)
    return h, dens, g, fo


def test_lattice_at_rest_has_no_force():
    box = inputs.lattice_box(8, jitter=0.0, v_sigma=0.0)
    _, dens, g, fo = _prepare(box)
    scale = np.max(g["P"] / dens["rho"]) / box.meta["spacing"]
    assert np.max(np.abs(fo["a"])) < 1e-11 * scale
    assert np.max(np.abs(fo["dudt"])) < 1e-11 * scale


def test_momentum_and_energy_conservation():
    """Pairwise antisymmetry: sum m a = 0 and sum m (v.a + du/dt) = 0 to rounding.
    The masses differ by up to a factor 3, so that the same sums without the mass
    factor (in the force or in the reductions) are far from zero."""
    box = inputs.lattice_box(8, jitter=0.45, seed=11, v_sigma=0.3)
    rng = np.random.default_rng(2)
    box.u[:] = rng.uniform(0.5, 2.0, box.n).astype(np.float32)
    box.m = (box.m * rng.uniform(0.5, 1.5, box.n)).astype(np.float32)
    _, dens, g, fo = _prepare(box, tol=1e-6)
    m = box.m.astype(np.float64)
    red = sph.reductions(m, box.v, box.u, fo["a"], fo["dudt"])
    scale_p = np.sum(m * np.linalg.norm(fo["a"], axis=1))
    scale_e = np.sum(m * np.abs(fo["dudt"])) + np.sum(m * np.abs((box.v * fo["a"]).sum(1)))
    assert np.all(np.abs(red[0:3]) < 1e-12 * scale_p)
    assert abs(red[3]) < 1e-12 * scale_e
    # the unweighted sums do not vanish: the mass factor is what cancels them
    ones = np.ones(box.n)
    unweighted = sph.reductions(ones, box.v, box.u, fo["a"], fo["dudt"])
    assert np.linalg.norm(unweighted[0:3]) > 1e-3 * np.sum(np.linalg.norm(fo["a"], axis=1))
    # viscosity is on for approaching pairs: some particle must heat
    assert np.any(fo["dudt"] > 0) and np.all(fo["vsig"] > 0)


def test_reductions_momentum_and_energy_closed_form():
    """sum m v and E = sum m (v^2/2 + u) of a box moving at one velocity v0 with
    u_i = i and masses m_i = 2 i / (n (n + 1)) (i = 1..n): total mass 1, so
    sum m v = v0 and E = |v0|^2 / 2 + (2 n + 1) / 3 exactly.  A dropped mass
    factor, a missing 1/2 in the kinetic term or a transposed v fails it."""
    n = 1000
    i = np.arange(1, n + 1, dtype=np.float64)
    m = 2.0 * i / (n * (n + 1))
    v0 = np.array([0.3, -1.25, 2.0])
    v = np.tile(v0, (n, 1))
    u = i.copy()
    zero3 = np.zeros((n, 3))
    red = sph.reductions(m, v, u, zero3, np.zeros(n))
    np.testing.assert_allclose(red[4:7], v0, rtol=1e-13)
    np.testing.assert_allclose(red[7], 0.5 * float(v0 @ v0) + (2 * n + 1) / 3.0, rtol=1e-13)
    assert np.all(red[0:4] == 0.0)


def test_reductions_rates_are_time_derivatives():
    """Entries 0-3 are the time derivatives of entries 4-7 along v(t) = v + a t,
    u(t) = u + du/dt t: sum m a = d/dt sum m v and sum m (v.a + du/dt) =
    d/dt sum m (v^2/2 + u).  Both are polynomials of degree <= 2 in t, so a
    centred difference is exact up to rounding; arbitrary unequal masses and
    rates make every term count."""
    rng = np.random.default_rng(31)
    n = 500
    m = rng.uniform(0.1, 3.0, n)
    v = rng.normal(0.0, 1.0, (n, 3))
    u = rng.uniform(0.0, 2.0, n)
    a = rng.normal(0.0, 5.0, (n, 3))
    dudt = rng.normal(0.0, 3.0, n)
    red = sph.reductions(m, v, u, a, dudt)
    eps = 1e-3
    rp = sph.reductions(m, v + eps * a, u + eps * dudt, a, dudt)
    rm = sph.reductions(m, v - eps * a, u - eps * dudt, a, dudt)
    fd = (rp[4:8] - rm[4:8]) / (2 * eps)
    scale = np.sum(m * (np.linalg.norm(a, axis=1) * (1 + np.linalg.norm(v, axis=1)) + np.abs(dudt)))
    np.testing.assert_allclose(red[0:4], fd, rtol=0, atol=1e-11 * scale)


def test_two_particle_closed_form():
    L = 1.0
    r = 0.3
    H = 0.5
    x = np.array([[0.25, 0.5, 0.5], [0.25 + r, 0.5, 0.5]])
    r = x[1, 0] - x[0, 0]
    m = np.array([0.7, 0.7], np.float32)
    mm = float(m[0])
    u = np.array([1.0, 1.0], np.float32)
    Hv = np.array([H, H])
    d = sph.density(x, m, Hv, L, periodic=False)
    rho = mm * (sph.kernel_w(0, H) + sph.kernel_w(r, H))
    np.testing.assert_allclose(d["rho"], rho, rtol=1e-14)
    g = sph.ghost(d["rho"], d["Sr_m"], u)
    v = np.zeros((2, 3), np.float32)
    fo = sph.force(x, v, m, Hv, d["rho"], g["P"], g["c"], g["f"], L, False)
    Fk = g["f"][0] * g["P"][0] / rho ** 2
    ax = -mm * (2 * Fk) * sph.kernel_dwdr(r, H) * (-1.0)   # x_1 - x_2 = -r along x
    np.testing.assert_allclose(fo["a"][0], [ax, 0, 0], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(fo["a"][1], [-ax, 0, 0], rtol=1e-13, atol=1e-15)
    assert ax < 0          # pressure pushes particle 1 away from particle 2
    # approaching pair: viscosity heats both and brakes the approach
    v = np.array([[0.5, 0, 0], [-0.5, 0, 0]], np.float32)
    fo2 = sph.force(x, v, m, Hv, d["rho"], g["P"], g["c"], g["f"], L, False)
    w = -1.0
    vsig = 2 * g["c"][0] - 3 * w
    Pi = -2.0 * vsig * w / (2 * rho)
    Wp = sph.kernel_dwdr(r, H)
    ax2 = -mm * (2 * Fk * Wp + Pi * Wp) * (-1.0)
    np.testing.assert_allclose(fo2["a"][0, 0], ax2, rtol=1e-13)
    du = mm * (Fk * Wp + 0.5 * Pi * Wp) * w
    np.testing.assert_allclose(fo2["dudt"], [du, du], rtol=1e-13)
    assert du > 0 and np.allclose(fo2["vsig"], vsig)


def _thermal_energy(box, x, A, gamma=sph.GAMMA_GAS):
    h, conv, _, dens = sph.h_iterate(x, box.m, box.h, box.L, True, tol=1e-13, max_iter=80)
    assert conv.all()
    return np.sum(box.m.astype(np.float64) * A * dens["rho"] ** (gamma - 1) / (gamma - 1)), dens


def test_pressure_force_is_the_gradient_of_thermal_energy():
    """Lagrangian pin: with alpha = 0, m_i a_i = -dE_th/dx_i at fixed entropy."""
    box = inputs.lattice_box(6, jitter=0.35, seed=21, v_sigma=0.0)
    gamma = sph.GAMMA_GAS
    h, dens, g, fo = _prepare(box, alpha=0.0, tol=1e-13)
    A = box.u.astype(np.float64) * (gamma - 1) / dens["rho"] ** (gamma - 1)
    eps = 1e-6 * box.meta["spacing"]
    for p in (0, 37, 101):
        for k in range(3):
            xp = box.x.copy(); xp[p, k] += eps
            xm = box.x.copy(); xm[p, k] -= eps
            Ep, _ = _thermal_energy(box, xp, A)
            Em, _ = _thermal_energy(box, xm, A)
            grad = (Ep - Em) / (2 * eps)
            ma = float(box.m[p]) * fo["a"][p, k]
            assert abs(ma + grad) < 2e-6 * np.abs(box.m[0] * fo["a"]).max(), (p, k, ma, -grad)


def test_dudt_is_the_adiabatic_density_rate():
    """du_i/dt = P_i/rho_i^2 d rho_i/dt with rho_i at converged h, alpha = 0."""
    box = inputs.lattice_box(6, jitter=0.35, seed=23, v_sigma=0.2)
    h, dens, g, fo = _prepare(box, alpha=0.0, tol=1e-13)
    dt = 1e-6
    xp = np.mod(box.x + dt * box.v.astype(np.float64), box.L)
    xm = np.mod(box.x - dt * box.v.astype(np.float64), box.L)
    _, dp = _thermal_energy(box, xp, np.ones(box.n))
    _, dm = _thermal_energy(box, xm, np.ones(box.n))
    drho = (dp["rho"] - dm["rho"]) / (2 * dt)
    pred = g["P"] / dens["rho"] ** 2 * drho
    np.testing.assert_allclose(fo["dudt"], pred, rtol=1e-5, atol=1e-6 * np.abs(pred).max())


# ---------------------------------------------------------------- search agreement
def test_brute_force_and_tree_search_agree():
    box = inputs.plummer_box(n=3000, n_spheres=2, scale=0.05, seed=4)
    H = sph.support_radius(box.h)
    a = sph.density(box.x, box.m, H, box.L, True, method="brute")
    b = sph.density(box.x, box.m, H, box.L, True, method="kdtree")
    assert np.array_equal(a["count"], b["count"])
    np.testing.assert_allclose(a["rho"], b["rho"], rtol=1e-13)
    g = sph.ghost(a["rho"], a["Sr_m"], box.u)
    fa = sph.force(box.x, box.v, box.m, H, a["rho"], g["P"], g["c"], g["f"], box.L, True, method="brute")
    fb = sph.force(box.x, box.v, box.m, H, a["rho"], g["P"], g["c"], g["f"], box.L, True, method="kdtree")
    np.testing.assert_allclose(fa["a"], fb["a"], rtol=1e-10, atol=1e-12 * np.abs(fa["a"]).max())
    np.testing.assert_allclose(fa["vsig"], fb["vsig"], rtol=1e-14)


def test_permutation_invariance():
    box = inputs.lattice_box(8, jitter=0.4, seed=9, v_sigma=0.1)
    perm = np.random.default_rng(3).permutation(box.n)
    out = sph.full_step(box, iterate_h=False)
    outp = sph.full_step(box.subset(perm), iterate_h=False)
    assert np.array_equal(out["count"][perm], outp["count"])
    np.testing.assert_allclose(out["rho"][perm], outp["rho"], rtol=1e-14)
    np.testing.assert_allclose(out["a"][perm], outp["a"], rtol=1e-11, atol=1e-13)


def test_periodic_wrap_matches_explicit_images():
    """Neighbours across the boundary equal those of an explicitly replicated open box."""
    box = inputs.lattice_box(6, jitter=0.4, seed=13)
    H = sph.support_radius(box.h)
    d = sph.density(box.x, box.m, H, box.L, True)
    shifts = np.stack(np.meshgrid(*[[-1, 0, 1]] * 3, indexing="ij"), -1).reshape(-1, 3)
    xr = np.concatenate([box.x + s * box.L for s in shifts])
    mr = np.tile(box.m, len(shifts))
    Hr = np.tile(H, len(shifts))
    centre = int(np.nonzero((shifts == 0).all(1))[0][0]) * box.n
    e = sph.density(xr, mr, Hr, 3 * box.L, False, targets=np.arange(centre, centre + box.n))
    assert np.array_equal(d["count"], e["count"])
    np.testing.assert_allclose(d["rho"], e["rho"], rtol=1e-12)


def test_sound_speed_is_the_adiabatic_pressure_derivative():
    """c^2 = dP/drho at fixed entropy.  The adiabat is followed with the first
    law alone, du/drho = P / rho^2 (integrated with RK4, P from the oracle), and
    the pressure change along it is compared with the oracle's c^2: a wrong factor
    in P (gamma for gamma - 1) or in c (a missing 1/rho or gamma) fails it."""
    zero = np.zeros(4)
    rho0 = np.array([0.3, 1.0, 2.5, 40.0])
    u0 = np.array([0.2, 1.0, 3.0, 0.05])
    P = lambda rho, u: sph.ghost(rho, zero, u)["P"]
    dudr = lambda rho, u: P(rho, u) / rho ** 2

    def along_adiabat(rho_to, steps=200):
        rho, u = rho0.copy(), u0.copy()
        dr = (rho_to - rho0) / steps
        for _ in range(steps):
            k1 = dudr(rho, u)
            k2 = dudr(rho + dr / 2, u + dr / 2 * k1)
            k3 = dudr(rho + dr / 2, u + dr / 2 * k2)
            k4 = dudr(rho + dr, u + dr * k3)
            u = u + dr / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            rho = rho + dr
        return P(rho, u)

    eps = 1e-4
    dPdrho = (along_adiabat(rho0 * (1 + eps)) - along_adiabat(rho0 * (1 - eps))) / (2 * eps * rho0)
    c = sph.ghost(rho0, zero, u0)["c"]
    np.testing.assert_allclose(c ** 2, dPdrho, rtol=1e-7)
