"""Sedov-Taylor similarity solution of a point explosion in a uniform gas.

TEST INFRASTRUCTURE ONLY: the analytical reference that the Sedov blast run of
the full solver is compared against (Section III: radial density, pressure and
velocity profiles of the blast are compared with the analytical solution of
Sedov 1959).  Written from the gas-dynamics definitions, spherical symmetry:

  an energy E released at r = 0 in gas of density rho0 and zero pressure drives
  a strong shock at R(t) = xi0 (E t^2 / rho0)^(1/5), moving at D = 2 R / (5 t).
  Inside, with xi = r / R, the flow is self-similar:
      v = D xi V(xi),   rho = rho0 G(xi),   c^2 = gamma P / rho = D^2 xi^2 Z(xi).
  Continuity, momentum and the adiabatic condition reduce, with ' = d / d ln xi, to
      V' = [3 Z (V - 1/gamma) - V (V - 1)(V - 5/2)] / [(V - 1)^2 - Z]
      G'/G = -(V' + 3 V) / (V - 1)
      Z'/Z = 3 / (V - 1) - 2 - (1 - gamma) G'/G
  and the strong-shock (Rankine-Hugoniot) conditions fix the values at xi = 1:
      V = 2 / (gamma + 1),  G = (gamma + 1) / (gamma - 1),  Z = 2 gamma (gamma - 1) / (gamma + 1)^2.
  The ODEs are integrated from the shock inwards; xi0 follows from the energy:
      E = 4 pi rho0 D^2 R^3 int_0^1 xi^4 G [V^2 / 2 + Z / (gamma (gamma - 1))] dxi,
  with D^2 R^3 = (4/25) xi0^5 E / rho0.

Pinned by tests/test_oracle_sedov.py: the textbook xi0 for gamma = 1.4 and 5/3,
the swept-up mass (int_0^1 3 xi^2 G dxi = 1, which the ODEs do not impose), the
limit V -> 1/gamma at the centre, and the shock jump conditions.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp


def _rhs(x, y, gamma):
    V, lnG, lnZ = y
    Z = np.exp(lnZ)
    dV = (3.0 * Z * (V - 1.0 / gamma) - V * (V - 1.0) * (V - 2.5)) / ((V - 1.0) ** 2 - Z)
    dlnG = -(dV + 3.0 * V) / (V - 1.0)
    dlnZ = 3.0 / (V - 1.0) - 2.0 - (1.0 - gamma) * dlnG
    return [dV, dlnG, dlnZ]


class SedovProfile:
    """The similarity functions V, G, Z on a grid of xi in (0, 1], and xi0."""

    def __init__(self, gamma: float, xi_min: float = 0.03, n: int = 4000):
        self.gamma = g = float(gamma)
        y0 = [2.0 / (g + 1.0), np.log((g + 1.0) / (g - 1.0)), np.log(2.0 * g * (g - 1.0) / (g + 1.0) ** 2)]
        xs = np.linspace(0.0, np.log(xi_min), n)
        sol = solve_ivp(_rhs, (0.0, np.log(xi_min)), y0, t_eval=xs, args=(g,), method="DOP853",
                        rtol=1e-11, atol=1e-13)
        if not sol.success:
            raise RuntimeError(sol.message)
        self.xi = np.exp(sol.t)[::-1]                  # ascending
        self.V = sol.y[0][::-1]
        self.G = np.exp(sol.y[1][::-1])
        self.Z = np.exp(sol.y[2][::-1])
        # energy integral; below xi_min (where the fixed point V = 1/gamma makes the
        # inward integration ill-conditioned) the gas is at rest to within G -> 0 and
        # its pressure, G Z xi^2 / gamma in units of rho0 D^2, is uniform: that part
        # adds xi_min^3 / 3 times the thermal term's xi^2-free factor
        f = self.xi ** 4 * self.G * (0.5 * self.V ** 2 + self.Z / (g * (g - 1.0)))
        p_c = self.G[0] * self.Z[0] * self.xi[0] ** 2
        I = np.trapezoid(f, self.xi) + p_c / (g * (g - 1.0)) * self.xi[0] ** 3 / 3.0
        self.xi0 = (25.0 / (16.0 * np.pi * I)) ** 0.2
        self.mass = np.trapezoid(3.0 * self.xi ** 2 * self.G, self.xi)

    def shock_radius(self, E, rho0, t):
        return self.xi0 * (E * t * t / rho0) ** 0.2

    def sample(self, r, E, rho0, t, p0=0.0):
        """(rho, v_r, P) at radii r (array) and time t; the undisturbed gas outside R."""
        r = np.asarray(r, dtype=np.float64)
        R = self.shock_radius(E, rho0, t)
        D = 0.4 * R / t
        xi = r / R
        inside = xi <= 1.0
        xq = np.clip(xi, self.xi[0], 1.0)
        V = np.interp(xq, self.xi, self.V)
        G = np.interp(xq, self.xi, self.G)
        # G Z xi^2 is smooth down to the centre (uniform pressure there)
        GZ = np.interp(xq, self.xi, self.G * self.Z * self.xi ** 2)
        core = xi < self.xi[0]
        G = np.where(core, 0.0, G)
        V = np.where(core, 1.0 / self.gamma, V)
        rho = np.where(inside, rho0 * G, rho0)
        v = np.where(inside, D * xi * V, 0.0)
        P = np.where(inside, rho0 * D * D * GZ / self.gamma, p0)
        return rho, v, P
