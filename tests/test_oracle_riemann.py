"""Pins of the exact Riemann solution used as the Sod-shock reference."""
import numpy as np

from oracle import riemann


def test_textbook_sod_star_state():
    """The classic Sod problem (gamma 1.4; rho 1 / 0.125, p 1 / 0.1, at rest): the
    star state of Toro's Table 4.3 (test 1), p* = 0.30313, u* = 0.92745,
    rho*_L = 0.42632, rho*_R = 0.26557."""
    p, u, rl, rr = riemann.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert abs(p - 0.30313) < 5e-5 and abs(u - 0.92745) < 5e-5
    assert abs(rl - 0.42632) < 5e-5 and abs(rr - 0.26557) < 5e-5


def test_rankine_hugoniot_and_isentropy_for_the_papers_sod_states():
    """The paper's Sod states (gamma 5/3): mass, momentum and energy fluxes match
    across the right shock in its frame, and the left rarefaction is isentropic."""
    g = 5.0 / 3.0
    rl, pl, rr, pr = 1.0, 1.0, 0.25, 0.1795
    p, u, rsl, rsr = riemann.star_state(rl, 0.0, pl, rr, 0.0, pr, g)
    assert pr < p < pl and u > 0
    S = riemann.shock_speed(rr, 0.0, pr, p, g, right=True)
    # fluxes in the shock frame
    w0, w1 = 0.0 - S, u - S
    e0 = pr / ((g - 1) * rr) + 0.5 * w0 * w0
    e1 = p / ((g - 1) * rsr) + 0.5 * w1 * w1
    np.testing.assert_allclose(rr * w0, rsr * w1, rtol=1e-12)
    np.testing.assert_allclose(rr * w0 * w0 + pr, rsr * w1 * w1 + p, rtol=1e-12)
    np.testing.assert_allclose(rr * w0 * (e0 + pr / rr), rsr * w1 * (e1 + p / rsr), rtol=1e-12)
    np.testing.assert_allclose(p / rsl ** g, pl / rl ** g, rtol=1e-12)


def test_sampled_profile_limits_and_mirror_symmetry():
    g = 5.0 / 3.0
    xi = np.linspace(-3, 3, 601)
    rho, u, p = riemann.sample(xi, 1.0, 0.0, 1.0, 0.25, 0.0, 0.1795, g)
    assert rho[0] == 1.0 and p[0] == 1.0 and rho[-1] == 0.25 and p[-1] == 0.1795
    assert np.all(np.diff(p) <= 1e-15)            # pressure falls monotonically left to right
    # the mirrored problem gives the mirrored solution
    rho2, u2, p2 = riemann.sample(-xi, 0.25, 0.0, 0.1795, 1.0, 0.0, 1.0, g)
    np.testing.assert_allclose(rho2, rho, rtol=1e-12)
    np.testing.assert_allclose(p2, p, rtol=1e-12)
    np.testing.assert_allclose(u2, -u, atol=1e-12)
    # equal states: nothing happens
    r3, u3, p3 = riemann.sample(xi, 0.7, 0.2, 0.5, 0.7, 0.2, 0.5, g)
    assert np.allclose(r3, 0.7) and np.allclose(u3, 0.2) and np.allclose(p3, 0.5)
