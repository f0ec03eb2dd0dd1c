"""Pins of the Sedov-Taylor similarity solution used as the blast reference."""
import numpy as np

from oracle import sedov
from paper_1309_3783_gb300 import inputs


def test_textbook_shock_constants():
    """xi0 in R = xi0 (E t^2 / rho0)^(1/5): 1.033 for gamma = 1.4 (Sedov, Taylor)
    and 1.152 for gamma = 5/3."""
    assert abs(sedov.SedovProfile(1.4).xi0 - 1.033) < 5e-4
    assert abs(sedov.SedovProfile(5.0 / 3.0).xi0 - 1.152) < 5e-4


def test_swept_mass_and_centre_limit():
    """The gas inside the shock is the gas the shock swept up (the ODEs do not
    impose it), and the flow at the centre moves with V -> 1/gamma."""
    for g in (1.4, 5.0 / 3.0, 1.2):
        s = sedov.SedovProfile(g)
        assert abs(s.mass - 1.0) < 1e-4, g
        assert abs(s.V[0] - 1.0 / g) < 1e-5, g
        assert np.all(np.diff(s.G) > 0)           # density rises monotonically to the shock


def test_jump_conditions_and_energy_of_the_sampled_profile():
    """At the shock: rho = rho0 (g+1)/(g-1), v = 2D/(g+1), P = 2 rho0 D^2/(g+1); and
    the sampled profile holds the released energy (checks the scalings in E, rho0, t)."""
    g = 5.0 / 3.0
    s = sedov.SedovProfile(g)
    E, rho0, t = 100.0, 2.0, 0.15
    R = s.shock_radius(E, rho0, t)
    D = 0.4 * R / t
    rho, v, P = s.sample(np.array([R * (1 - 1e-12)]), E, rho0, t)
    np.testing.assert_allclose(rho[0], rho0 * (g + 1) / (g - 1), rtol=1e-6)
    np.testing.assert_allclose(v[0], 2 * D / (g + 1), rtol=1e-6)
    np.testing.assert_allclose(P[0], 2 * rho0 * D * D / (g + 1), rtol=1e-6)
    r = np.linspace(0.0, R, 200001)
    rho, v, P = s.sample(r, E, rho0, t)
    e = np.trapezoid(4 * np.pi * r * r * (0.5 * rho * v * v + P / (g - 1)), r)
    np.testing.assert_allclose(e, E, rtol=2e-4)


def test_sedov_input_recipe():
    box = inputs.sedov_box(n=21, L=1.0)
    meta = box.meta
    assert box.n == 21 ** 3
    m = float(box.m[0])
    np.testing.assert_allclose(m * 21 ** 3, 1.0, rtol=1e-6)
    hot = meta["hot"]
    assert len(hot) == 33
    # the hot particles are the centre and the shells |n|^2 <= 4 of the lattice
    d = (box.x[hot] - meta["centre"]) / meta["spacing"]
    n2 = np.round(np.sum(d * d, axis=1)).astype(int)
    assert sorted(np.bincount(n2, minlength=5)[:5].tolist()) == sorted([1, 6, 12, 8, 6])
    np.testing.assert_allclose(np.sum(box.m[hot].astype(np.float64) * box.u[hot]), 100.0, rtol=1e-5)
