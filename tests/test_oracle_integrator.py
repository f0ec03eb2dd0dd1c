"""Pins of the oracle's fixed-step kick-drift-kick integration (Section III-B
runs the test problems with a fixed time step and forces on every particle each
step; the leapfrog itself is a reading).  Neither test compares the oracle with
itself: one checks a motion known in closed form, the other the convergence
order that a leapfrog must have."""

import numpy as np

from oracle import sph as orc
from paper_1309_3783_gb300 import inputs


def test_moving_lattice_drifts_rigidly():
    """A perfect lattice moving at one velocity feels no force (every pair's
    terms cancel by symmetry, and no pair approaches), so every step only
    translates it: x_n = x_0 + n dt v_0 (periodic), v and u unchanged, h uniform."""
    box = inputs.lattice_box(8, jitter=0.0, seed=1)
    v0 = np.array([0.3, -0.2, 0.1], np.float32)
    box.v = np.tile(v0, (box.n, 1))
    dt, n = 0.01, 5
    x, v, u, h, _ = orc.kdk_steps(box, dt, n)
    d = x - (box.x + n * dt * v0.astype(np.float64))
    d -= box.L * np.round(d / box.L)
    assert np.max(np.abs(d)) < 1e-12
    assert np.max(np.abs(v - v0.astype(np.float64))) < 1e-12
    assert np.max(np.abs(u - box.u.astype(np.float64))) < 1e-12
    assert np.ptp(h) < 1e-9 * h.mean()


def test_leapfrog_energy_error_is_second_order():
    """Without viscosity the SPH equations with grad-h terms conserve the total
    energy sum(m v^2 / 2) + sum(m u); a kick-drift-kick leapfrog then drifts from
    it by O(dt^2) over a fixed time, so halving dt divides the drift by about 4.
    A first-order scheme (a full kick before the drift and none after, or forces
    from the previous positions) divides it by 2 and drifts ~100x more here."""
    box = inputs.lattice_box(8, jitter=0.2, seed=5)
    rng = np.random.default_rng(3)
    box.v = (0.1 * rng.standard_normal((box.n, 3))).astype(np.float32)
    m = box.m.astype(np.float64)

    def energy(v, u):
        return float(np.sum(0.5 * m * np.sum(v * v, axis=1)) + np.sum(m * u))

    e0 = energy(box.v.astype(np.float64), box.u.astype(np.float64))
    drift = []
    for dt, n in ((0.004, 10), (0.002, 20)):          # the same time, about a tenth of the Courant step
        _, v, u, _, _ = orc.kdk_steps(box, dt, n, tol=1e-10, max_iter=60, alpha=0.0)
        drift.append(energy(v, u) - e0)
    assert 3.0 < drift[0] / drift[1] < 5.0
    assert abs(drift[1]) < 1e-6 * e0
