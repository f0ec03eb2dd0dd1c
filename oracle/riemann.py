"""Exact solution of the 1-D Riemann problem for an ideal gas (shock tubes).

TEST INFRASTRUCTURE ONLY: the analytical reference that the Sod-shock run of
the full solver is compared against (Section III: the shock-tube profiles are
compared with Sod's analytical solution, Sod 1978).  The solution is the
classical one: the star-region pressure p* solves f_L(p*) + f_R(p*) + (u_R - u_L) = 0,
f_K being the shock (Rankine-Hugoniot) branch for p* > p_K and the rarefaction
(isentropic) branch otherwise; u* follows, and the self-similar solution is
sampled at x / t.  Written from the gas-dynamics definitions; pinned by
tests/test_oracle_riemann.py (textbook star states, Rankine-Hugoniot jump
conditions across the computed shock, isentropy across the rarefaction).
"""
from __future__ import annotations

import numpy as np


def _f(p, rho, pk, gamma):
    """Velocity jump across the wave of state (rho, pk) to pressure p, and its derivative."""
    c = np.sqrt(gamma * pk / rho)
    if p > pk:    # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** e - 1.0), 1.0 / (rho * c) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))


def star_state(rl, ul, pl, rr, ur, pr, gamma):
    """(p*, u*, rho*_L, rho*_R) of the Riemann problem."""
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _f(p, rl, pl, gamma)
        fr, dr = _f(p, rr, pr, gamma)
        g = fl + fr + (ur - ul)
        step = g / (dl + dr)
        p_new = max(p - step, 1e-12 * p)
        if abs(p_new - p) <= 1e-14 * max(p, p_new):
            p = p_new
            break
        p = p_new
    fl, _ = _f(p, rl, pl, gamma)
    fr, _ = _f(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    g1 = (gamma - 1.0) / (gamma + 1.0)

    def rho_star(rk, pk):
        if p > pk:
            return rk * (p / pk + g1) / (g1 * p / pk + 1.0)
        return rk * (p / pk) ** (1.0 / gamma)

    return p, u, rho_star(rl, pl), rho_star(rr, pr)


def sample(xi, rl, ul, pl, rr, ur, pr, gamma):
    """(rho, u, p) of the self-similar solution at xi = (x - x0) / t (array)."""
    xi = np.asarray(xi, dtype=np.float64)
    ps, us, rsl, rsr = star_state(rl, ul, pl, rr, ur, pr, gamma)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    g = gamma
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    for k, s in enumerate(xi):
        if s <= us:      # left of the contact
            if ps > pl:  # left shock
                S = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                st = (rl, ul, pl) if s < S else (rsl, us, ps)
            else:        # left rarefaction
                head, tail = ul - cl, us - cl * (ps / pl) ** ((g - 1) / (2 * g))
                if s < head:
                    st = (rl, ul, pl)
                elif s > tail:
                    st = (rsl, us, ps)
                else:
                    uu = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    cc = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    rr_ = rl * (cc / cl) ** (2 / (g - 1))
                    st = (rr_, uu, pl * (cc / cl) ** (2 * g / (g - 1)))
        else:            # right of the contact
            if ps > pr:  # right shock
                S = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                st = (rr, ur, pr) if s > S else (rsr, us, ps)
            else:        # right rarefaction
                head, tail = ur + cr, us + cr * (ps / pr) ** ((g - 1) / (2 * g))
                if s > head:
                    st = (rr, ur, pr)
                elif s < tail:
                    st = (rsr, us, ps)
                else:
                    uu = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    cc = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    rr_ = rr * (cc / cr) ** (2 / (g - 1))
                    st = (rr_, uu, pr * (cc / cr) ** (2 * g / (g - 1)))
        rho[k], u[k], p[k] = st
    return rho, u, p


def shock_speed(rk, uk, pk, ps, gamma, right=True):
    """Speed of the shock moving into state (rk, uk, pk) with post-shock pressure ps."""
    c = np.sqrt(gamma * pk / rk)
    m = np.sqrt((gamma + 1) / (2 * gamma) * ps / pk + (gamma - 1) / (2 * gamma))
    return uk + c * m if right else uk - c * m
