"""Seeded synthetic particle boxes for the SPH density/force path.

This module only draws inputs: positions, velocities, masses, internal
energies and a first guess of the smoothing length.  It holds none of the
method's arithmetic (no kernel, no neighbour search, no density) and is the one
module that both the FP64 oracle (tests) and the CUDA path (bench, tests)
import.

The workloads follow the particle distributions the paper uses to motivate the
method (Section III-B: uniform lattices, strongly clustered volumes whose
smoothing lengths span orders of magnitude):

* ``lattice_box``   -- cubic lattice with uniform jitter (16^3 = 4096 particles by
  default), equal masses, Gaussian velocities, u = 1, h = 1.2348 x spacing.
* ``plummer_box``   -- uniform background plus Plummer spheres (262,144 particles
  by default: 50 % background, 16 spheres of scale radius 0.02).
* ``lognormal_box`` -- particles drawn from a log-normal density field built on a
  Gaussian random field with power-law spectrum (8,388,608 particles by default).
* ``clustered_box`` -- 30 % background plus 4096 Plummer spheres with log-uniform
  scale radii (33,554,432 particles by default).
* ``served_boxes``  -- a stream of independent jittered lattices with log-uniform
  particle counts, for the batched/served form.

The first-guess smoothing length of every recipe is ``h0 = 1.2348 * s`` where
``s = n(x)^(-1/3)`` is the local mean interparticle spacing of the distribution
the particles were drawn from (analytic for lattices and Plummer spheres, the
grid-cell density for the log-normal field).  The method then iterates h.

All generators use ``numpy.random.default_rng(seed)`` (PCG64), which gives the
same stream on x86-64 and aarch64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

#: h = ETA x mean interparticle spacing (the lattice recipe's constant).
ETA = 1.2348


@dataclass
class ParticleBox:
    """One periodic (or open) cubic box of particles.

    Arrays are in the layout the C-ABI takes: ``x`` float64 (n, 3), ``v`` float32
    (n, 3), ``m``, ``u``, ``h`` float32 (n,).  Positions lie in [0, L)^3.
    """

    x: np.ndarray
    v: np.ndarray
    m: np.ndarray
    u: np.ndarray
    h: np.ndarray
    L: float = 1.0
    periodic: bool = True
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def subset(self, idx: np.ndarray) -> "ParticleBox":
        return ParticleBox(self.x[idx].copy(), self.v[idx].copy(), self.m[idx].copy(),
                           self.u[idx].copy(), self.h[idx].copy(), self.L, self.periodic,
                           self.name + "[subset]", dict(self.meta))


def _wrap(x: np.ndarray, L: float) -> np.ndarray:
    """Fold positions into [0, L); values that round up to L are folded to 0."""
    x = np.mod(x, L)
    x[x >= L] = 0.0
    return x


def lattice_box(n_side: int = 16, jitter: float = 0.1, seed: int = 1, L: float = 1.0,
                v_sigma: float = 0.01, u: float = 1.0, eta: float = ETA,
                periodic: bool = True) -> ParticleBox:
    """Cubic lattice of n_side^3 particles, x = (i + 1/2 + U(-jitter, jitter)) * a.

    Equal masses L^3 / N (mean density 1), v ~ N(0, v_sigma) per component,
    u constant, h = eta * a.  ``jitter=0`` gives the perfect lattice.
    """
    rng = np.random.default_rng(seed)
    a = L / n_side
    idx = np.indices((n_side, n_side, n_side)).reshape(3, -1).T.astype(np.float64)
    off = rng.uniform(-jitter, jitter, size=idx.shape) if jitter > 0 else 0.0
    x = (idx + 0.5 + off) * a
    x = _wrap(x, L) if periodic else np.clip(x, 0.0, np.nextafter(L, 0.0))
    n = x.shape[0]
    v = rng.normal(0.0, v_sigma, size=(n, 3)).astype(np.float32) if v_sigma > 0 else np.zeros((n, 3), np.float32)
    m = np.full(n, L ** 3 / n, dtype=np.float32)
    uu = np.full(n, u, dtype=np.float32)
    h = np.full(n, eta * a, dtype=np.float32)
    return ParticleBox(x, v, m, uu, h, L, periodic, f"lattice{n_side}^3 jitter={jitter}",
                       {"spacing": a, "seed": seed})


def _plummer_radii(rng, count: int, a: float, r_max: float) -> np.ndarray:
    """Radii drawn from a Plummer sphere of scale radius a, truncated at r_max.

    Inverse of the enclosed-mass fraction X = r^3 / (r^2 + a^2)^(3/2).
    """
    out = np.empty(0)
    while out.size < count:
        X = rng.uniform(0.0, 1.0, size=2 * (count - out.size) + 16)
        X = X[X > 0]
        r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        out = np.concatenate([out, r[r < r_max]])
    return out[:count]


def _isotropic(rng, count: int) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0, size=count)
    phi = rng.uniform(0.0, 2 * np.pi, size=count)
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _plummer_number_density(r: np.ndarray, n_sphere: float, a: float) -> np.ndarray:
    return 3.0 * n_sphere / (4.0 * np.pi * a ** 3) * (1.0 + (r / a) ** 2) ** (-2.5)


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def plummer_box(n: int = 262_144, frac_uniform: float = 0.5, n_spheres: int = 16,
                scale: float = 0.02, seed: int = 1, L: float = 1.0, v_sigma: float = 0.1,
                u: float = 1.0, r_max: float = 0.5, eta: float = ETA) -> ParticleBox:
    """Uniform background plus ``n_spheres`` equal Plummer spheres, periodic box.

    Sphere centres are U(0, L)^3; radii follow the Plummer enclosed-mass inverse,
    truncated at ``r_max``; directions are isotropic; positions are wrapped.
    h0 = eta * n(x)^(-1/3) with n the analytic number density (background plus
    the minimum-image Plummer profiles).
    """
    rng = np.random.default_rng(seed)
    n_bg = int(round(n * frac_uniform))
    n_sph = n - n_bg
    per = np.full(n_spheres, n_sph // n_spheres)
    per[: n_sph - per.sum()] += 1
    centres = rng.uniform(0.0, L, size=(n_spheres, 3))
    parts = [rng.uniform(0.0, L, size=(n_bg, 3))]
    for s in range(n_spheres):
        r = _plummer_radii(rng, int(per[s]), scale, r_max)
        parts.append(centres[s] + r[:, None] * _isotropic(rng, int(per[s])))
    x = _wrap(np.concatenate(parts, axis=0), L)
    dens = np.full(n, n_bg / L ** 3)
    for s in range(n_spheres):
        d = _min_image(x - centres[s], L)
        dens += _plummer_number_density(np.sqrt((d * d).sum(1)), per[s], scale)
    h = (eta * dens ** (-1.0 / 3.0)).astype(np.float32)
    v = rng.normal(0.0, v_sigma, size=(n, 3)).astype(np.float32)
    m = np.full(n, L ** 3 / n, dtype=np.float32)
    return ParticleBox(x, v, m, np.full(n, u, np.float32), h, L, True,
                       f"plummer n={n} spheres={n_spheres} a={scale}",
                       {"seed": seed, "centres": centres})


def gaussian_random_field(n_grid: int, index: float, rng) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian field with P(k) ~ k^index."""
    white = rng.normal(size=(n_grid,) * 3)
    fk = np.fft.rfftn(white)
    k1 = np.fft.fftfreq(n_grid) * n_grid
    kz = np.fft.rfftfreq(n_grid) * n_grid
    k2 = k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (index / 4.0)  # sqrt(P) with P ~ k^index
    g = np.fft.irfftn(fk * amp, s=(n_grid,) * 3, axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_box(n: int = 2 ** 23, n_grid: int = 256, sigma: float = 2.0, index: float = -2.0,
                  seed: int = 1, L: float = 1.0, v_sigma: float = 0.1, u: float = 1.0,
                  eta: float = ETA) -> ParticleBox:
    """Particles drawn from a mean-one log-normal field delta = exp(sigma g - sigma^2/2).

    g is a Gaussian random field on an n_grid^3 mesh (P(k) ~ k^index); particle
    counts per mesh cell are multinomial with probabilities ~ delta and positions
    are uniform inside each cell.  h0 = eta * (local number density)^(-1/3).
    """
    rng = np.random.default_rng(seed)
    g = gaussian_random_field(n_grid, index, rng)
    delta = np.exp(sigma * g - 0.5 * sigma * sigma).ravel()
    p = delta / delta.sum()
    counts = rng.multinomial(n, p)
    cell = np.repeat(np.arange(p.size, dtype=np.int64), counts)
    ijk = np.stack(np.unravel_index(cell, (n_grid,) * 3), axis=1).astype(np.float64)
    x = _wrap((ijk + rng.uniform(0.0, 1.0, size=ijk.shape)) * (L / n_grid), L)
    dens = n * p[cell] * (n_grid ** 3) / L ** 3
    h = (eta * dens ** (-1.0 / 3.0)).astype(np.float32)
    v = rng.normal(0.0, v_sigma, size=(n, 3)).astype(np.float32)
    m = np.full(n, L ** 3 / n, dtype=np.float32)
    return ParticleBox(x, v, m, np.full(n, u, np.float32), h, L, True,
                       f"lognormal n={n} grid={n_grid} sigma={sigma}", {"seed": seed})


def clustered_box(n: int = 2 ** 25, frac_uniform: float = 0.3, n_spheres: int = 4096,
                  scale_range=(1e-4, 1e-2), seed: int = 1, L: float = 1.0, v_sigma: float = 0.1,
                  u: float = 1.0, r_max: float = 0.5, eta: float = ETA) -> ParticleBox:
    """Background plus many Plummer spheres with log-uniform scale radii.

    h0 uses the background density plus each particle's own sphere profile
    (a first guess only; the method iterates h).
    """
    rng = np.random.default_rng(seed)
    n_bg = int(round(n * frac_uniform))
    n_sph = n - n_bg
    per = np.full(n_spheres, n_sph // n_spheres)
    per[: n_sph - per.sum()] += 1
    centres = rng.uniform(0.0, L, size=(n_spheres, 3))
    scales = np.exp(rng.uniform(np.log(scale_range[0]), np.log(scale_range[1]), size=n_spheres))
    x = np.empty((n, 3))
    dens = np.full(n, n_bg / L ** 3)
    x[:n_bg] = rng.uniform(0.0, L, size=(n_bg, 3))
    o = n_bg
    for s in range(n_spheres):
        c = int(per[s])
        r = _plummer_radii(rng, c, scales[s], r_max)
        x[o:o + c] = centres[s] + r[:, None] * _isotropic(rng, c)
        dens[o:o + c] += _plummer_number_density(r, c, scales[s])
        o += c
    x = _wrap(x, L)
    h = (eta * dens ** (-1.0 / 3.0)).astype(np.float32)
    v = rng.normal(0.0, v_sigma, size=(n, 3)).astype(np.float32)
    m = np.full(n, L ** 3 / n, dtype=np.float32)
    return ParticleBox(x, v, m, np.full(n, u, np.float32), h, L, True,
                       f"clustered n={n} spheres={n_spheres}", {"seed": seed})


def sod_box(n_left: tuple = (58, 116, 116), n_right: tuple = (37, 73, 73), L: float = 1.0,
            rho_left: float = 1.0, p_left: float = 1.0, p_right: float = 0.1795, gamma: float = 5.0 / 3.0,
            eta: float = ETA) -> ParticleBox:
    """The Sod shock of Section III: a periodic cube whose half x < L/2 holds the
    dense gas (rho 1, P 1) and the other half the thin gas (P 0.1795, a quarter of
    the density), at rest, as two cubic lattices of equal-mass particles (so the
    dense half holds about four times as many).  The default sizes give about
    780,000 + 197,000 particles (the paper: 800,000 + 200,000 on its own grid).
    Masses follow from rho_left on the dense lattice; u is set from the target
    pressures and each lattice's actual density; h = eta x the lattice spacing.
    """
    def lattice(n, x0, ax, a):
        idx = np.indices(n).reshape(3, -1).T.astype(np.float64)
        x = np.empty_like(idx)
        x[:, 0] = x0 + (idx[:, 0] + 0.5) * ax
        x[:, 1] = (idx[:, 1] + 0.5) * a
        x[:, 2] = (idx[:, 2] + 0.5) * a
        return x
    half = 0.5 * L
    aL = L / n_left[1]
    aR = L / n_right[1]
    xl = lattice(n_left, 0.0, half / n_left[0], aL)
    xr = lattice(n_right, half, half / n_right[0], aR)
    nl, nr = xl.shape[0], xr.shape[0]
    m = rho_left * half * L * L / nl
    rho_right = m * nr / (half * L * L)
    u = np.concatenate([np.full(nl, p_left / ((gamma - 1.0) * rho_left)),
                        np.full(nr, p_right / ((gamma - 1.0) * rho_right))]).astype(np.float32)
    h = np.concatenate([np.full(nl, eta * aL), np.full(nr, eta * aR)]).astype(np.float32)
    x = _wrap(np.concatenate([xl, xr]), L)
    n = nl + nr
    return ParticleBox(x, np.zeros((n, 3), np.float32), np.full(n, m, np.float32), u, h, L, True,
                       f"sod {nl}+{nr}", {"rho_left": rho_left, "rho_right": rho_right, "p_left": p_left,
                                          "p_right": p_right, "gamma": gamma, "n_left": nl})


def sedov_box(n: int = 101, L: float = 4.0, rho0: float = 1.0, p0: float = 1e-5, energy: float = 100.0,
              n_hot: int = 33, gamma: float = 5.0 / 3.0, eta: float = ETA) -> ParticleBox:
    """The Sedov blast of Section III: an n^3 cubic lattice of particles at rest
    with rho0 = 1 and P = 1e-5, the n_hot particles nearest the centre holding the
    energy (u_i = E / n_hot / m_i, E = 100).  The paper does not give the box: the
    lattice fills a periodic cube of edge L = 4, which keeps the blast (radius 1.72
    at t = 0.275) clear of its periodic images.  n odd puts a particle at the
    centre; the 33 nearest are the centre and its shells |n|^2 <= 4 (6 + 12 + 8 + 6)."""
    a = L / n
    idx = np.indices((n, n, n)).reshape(3, -1).T.astype(np.float64)
    x = (idx + 0.5) * a
    N = x.shape[0]
    m = rho0 * L ** 3 / N
    u = np.full(N, p0 / ((gamma - 1.0) * rho0), np.float64)
    c = 0.5 * L
    d2 = np.sum((x - c) ** 2, axis=1)
    hot = np.argsort(d2, kind="stable")[:n_hot]
    u[hot] = energy / n_hot / m
    return ParticleBox(x, np.zeros((N, 3), np.float32), np.full(N, m, np.float32), u.astype(np.float32),
                       np.full(N, eta * a, np.float32), L, True, f"sedov {n}^3",
                       {"rho0": rho0, "p0": p0, "energy": energy, "gamma": gamma, "centre": c, "spacing": a,
                        "hot": hot})


def served_box_sizes(n_boxes: int = 512, n_min: int = 1000, n_max: int = 262_144,
                     seed: int = 1) -> np.ndarray:
    """Lattice side lengths n_b with n_b^3 log-uniform in [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    nb = np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_boxes)) ** (1.0 / 3.0)
    return np.clip(np.round(nb), 10, 64).astype(np.int64)


def served_boxes(n_boxes: int = 512, n_min: int = 1000, n_max: int = 262_144, seed: int = 1,
                 jitter: float = 0.1, v_sigma: float = 0.01) -> list[ParticleBox]:
    """Independent jittered lattices (per-box seed 1000 + b) for the served batch."""
    sides = served_box_sizes(n_boxes, n_min, n_max, seed)
    return [lattice_box(int(s), jitter=jitter, seed=1000 + b, v_sigma=v_sigma)
            for b, s in enumerate(sides)]


def poisson_arrivals(n: int, rate: float, seed: int = 1) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
