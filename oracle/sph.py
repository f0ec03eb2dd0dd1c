"""FP64 oracle: SPH density, smoothing-length iteration, ghost and force.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What the paper fixes and what is read into it
---------------------------------------------
The paper (Section II) fixes the two passes and who interacts with whom:

* density: particle i gathers every j within its own smoothing length h_i;
* force:   particle i interacts with every j within max(h_i, h_j).

It prints no kernel, density sum, force law or h rule; the constants it names
are N_ngb = 48, gamma = 5/3, alpha = 2.0 (viscosity), C_CFL = 0.3 (Section
III-B).  The formulation below is the textbook one of Gadget-2 (Springel
2005), the code the paper compares against, with the grad-h terms of Springel &
Hernquist (2002) in thermal-energy form:

* "within h" means within the kernel support H = gamma_K * h with
  gamma_K = 1.825742 (FP32 constant), which gives ~48 neighbours for
  h = 1.2348 x spacing;
* kernel: cubic spline with compact support H (``kernel_w``, ``kernel_dwdr``);
* density: rho_i = sum_{j: r_ij < H_i} m_j W(r_ij, H_i) including j = i;
  d rho_i / d h_i = -(1/h_i) sum_j m_j (3 W + r dW/dr);
  number density n_i = sum_j W(r_ij, H_i); weighted neighbour number
  N~_i = (4 pi / 3) H_i^3 n_i; integer count excludes j = i;
* h: Newton iteration on N~_i(h) = N_ngb, steps clamped to [h/2, 2h], bisection
  on the bracket when Newton leaves it (``h_iterate``);
* ghost: P = (gamma - 1) rho u, c = sqrt(gamma P / rho),
  f = [1 + h/(3 rho) d rho/d h]^-1;
* force: symmetric pressure term with grad-h factors and Monaghan viscosity
  (``force``).

Neighbour predicate.  The decision "r_ij < H" is an integer outcome, so it is
fixed here as one FP64 evaluation in a fixed order, which the CUDA path
reproduces exactly for every pair near the cutoff:
``d = x_i - x_j`` (each component), wrapped by +-L when |d| > L/2 for periodic
boxes, ``r2 = (d0*d0 + d1*d1) + d2*d2`` with every operation correctly rounded
and no fused multiply-add, and ``r2 < H*H`` with H the FP64 value of the FP32
support radius (``support_radius``).
"""
from __future__ import annotations

import numpy as np

GAMMA_K = np.float32(1.825742)   # support radius / smoothing length (cubic spline)
N_NGB = 48.0                     # target weighted neighbour number (Section III-B)
GAMMA_GAS = 5.0 / 3.0            # adiabatic index (Section III-B)
ALPHA_VISC = 2.0                 # artificial viscosity alpha (Section III-B)
C_CFL = 0.3                      # Courant factor (Section III-B)

_KNORM = 8.0 / np.pi             # 3D cubic-spline normalisation with support H


# --------------------------------------------------------------------------- kernel
def kernel_w(r, H):
    """Cubic spline W(r, H) with compact support H (3D), FP64.

    W = 8/(pi H^3) * {1 - 6 q^2 + 6 q^3 (q < 1/2); 2 (1 - q)^3 (1/2 <= q < 1); 0}.
    """
    r = np.asarray(r, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    q = r / H
    inner = 1.0 - 6.0 * q * q + 6.0 * q * q * q
    outer = 2.0 * (1.0 - q) ** 3
    w = np.where(q < 0.5, inner, np.where(q < 1.0, outer, 0.0))
    return _KNORM / H ** 3 * w


def kernel_dwdr(r, H):
    """dW/dr of the cubic spline, FP64 (zero for r >= H).

    dW/dr = 8/(pi H^4) * {-12 q + 18 q^2 (q < 1/2); -6 (1 - q)^2 (1/2 <= q < 1); 0}.
    """
    r = np.asarray(r, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    q = r / H
    inner = -12.0 * q + 18.0 * q * q
    outer = -6.0 * (1.0 - q) ** 2
    w = np.where(q < 0.5, inner, np.where(q < 1.0, outer, 0.0))
    return _KNORM / H ** 4 * w


def support_radius(h):
    """H = gamma_K * h rounded once to FP32 (the value both paths compare against), as FP64."""
    h32 = np.asarray(h, dtype=np.float32)
    return (GAMMA_K * h32).astype(np.float32).astype(np.float64)


# ------------------------------------------------------------------- pair geometry
def canonical_r2(x, i, j, L, periodic):
    """Squared separation of pairs (i, j) in the fixed FP64 evaluation order."""
    d = x[i] - x[j]
    if periodic:
        half = 0.5 * L
        d = np.where(d > half, d - L, np.where(d < -half, d + L, d))
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2], d


def _kdtree(x, L, periodic):
    from scipy.spatial import cKDTree
    return cKDTree(x, boxsize=L if periodic else None)


def _ball_candidates(tree, x, targets, radius, index=None):
    """(target position, j) for every j within radius[t] (slightly inflated) of target t."""
    lists = tree.query_ball_point(x[targets], r=radius * (1.0 + 1e-9) + 1e-300,
                                  workers=-1, return_sorted=False)
    lens = np.fromiter((len(a) for a in lists), dtype=np.int64, count=len(lists))
    ti = np.repeat(np.arange(len(targets), dtype=np.int64), lens)
    j = np.concatenate([np.asarray(a, dtype=np.int64) for a in lists]) if lens.sum() else np.zeros(0, np.int64)
    if index is not None:
        j = index[j]
    return ti, j


def _filter(x, targets, t, j, H, L, periodic, mode):
    keep = targets[t] != j
    t, j = t[keep], j[keep]
    r2, d = canonical_r2(x, targets[t], j, L, periodic)
    Hi2 = H[targets[t]] ** 2
    keep = (r2 < Hi2) if mode == "density" else ((r2 < Hi2) | (r2 < H[j] ** 2))
    return t[keep], j[keep], r2[keep], d[keep]


def neighbour_pairs(x, Hreach, L, periodic, targets=None, mode="density", Hall=None, method="auto"):
    """Ordered pairs (t, j), j != targets[t], that satisfy the canonical predicate.

    mode="density": r < Hreach[targets[t]] (the gather set of the density pass).
    mode="force":   r < max(H_i, H_j) with H = ``Hall`` for every particle.
    ``method="brute"`` tests every j (all pairs); ``"kdtree"`` takes candidates from a
    k-d tree ball search with a slightly inflated radius and then applies the same
    predicate.  Returns (t, j, r2, d) with d = x_i - x_j after the periodic wrap.
    """
    n = x.shape[0]
    targets = np.arange(n) if targets is None else np.asarray(targets, dtype=np.int64)
    if method == "auto":
        method = "brute" if n * len(targets) <= 16_000_000 else "kdtree"
    H = np.asarray(Hreach if mode == "density" else Hall, dtype=np.float64)
    parts = []
    if method == "brute":
        chunk = max(1, 2_000_000 // max(n, 1))
        for s in range(0, len(targets), chunk):
            nt = min(chunk, len(targets) - s)
            t = np.repeat(np.arange(s, s + nt, dtype=np.int64), n)
            j = np.tile(np.arange(n, dtype=np.int64), nt)
            parts.append(_filter(x, targets, t, j, H, L, periodic, mode))
    else:
        tree = _kdtree(x, L, periodic)
        cand_t, cand_j = _ball_candidates(tree, x, targets, H[targets])
        ts, js = [cand_t], [cand_j]
        if mode == "force":
            # every j whose own support reaches the target: bucket j by H and query
            # each bucket with its largest H.
            lo, hi = H.min(), H.max()
            edges = hi * 2.0 ** -np.arange(0, 64)
            edges = edges[edges >= lo * 0.5]
            for b in range(len(edges)):
                upper = edges[b]
                lower = edges[b + 1] if b + 1 < len(edges) else 0.0
                sel = np.nonzero((H <= upper) & (H > lower))[0]
                if sel.size == 0:
                    continue
                sub = _kdtree(x[sel], L, periodic)
                t, j = _ball_candidates(sub, x, targets, np.full(len(targets), upper), index=sel)
                ts.append(t)
                js.append(j)
            key = np.unique(np.concatenate(ts) * np.int64(n) + np.concatenate(js))
            cand_t, cand_j = key // n, key % n
        parts.append(_filter(x, targets, cand_t, cand_j, H, L, periodic, mode))
    if not parts:
        z = np.zeros(0, np.int64)
        return z, z, np.zeros(0), np.zeros((0, 3))
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(4))


# ------------------------------------------------------------------------ density
def density(x, m, H, L, periodic, targets=None, method="auto"):
    """Density pass for ``targets`` (default: all) at fixed support radii H (FP64 array).

    Returns a dict of FP64 arrays over the targets:
    rho, S_m = sum m_j (3W + r dW/dr), Sr_m = sum_{j != i} m_j r dW/dr,
    nw = sum W, S = sum (3W + r dW/dr), count (int64, j != i), Nw = (4 pi/3) H^3 nw.
    """
    n = x.shape[0]
    targets = np.arange(n) if targets is None else np.asarray(targets, dtype=np.int64)
    H = np.asarray(H, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    t, j, r2, _ = neighbour_pairs(x, H, L, periodic, targets, "density", method=method)
    Ht = H[targets]
    r = np.sqrt(r2)
    Hi = Ht[t]
    w = kernel_w(r, Hi)
    dw = kernel_dwdr(r, Hi)
    g = 3.0 * w + r * dw
    nt = len(targets)
    w0 = kernel_w(0.0, Ht)
    mt = m[targets]
    out = {
        "rho": np.bincount(t, weights=m[j] * w, minlength=nt) + mt * w0,
        "S_m": np.bincount(t, weights=m[j] * g, minlength=nt) + mt * 3.0 * w0,
        "Sr_m": np.bincount(t, weights=m[j] * r * dw, minlength=nt),
        "nw": np.bincount(t, weights=w, minlength=nt) + w0,
        "S": np.bincount(t, weights=g, minlength=nt) + 3.0 * w0,
        "count": np.bincount(t, minlength=nt).astype(np.int64),
    }
    out["Nw"] = 4.0 * np.pi / 3.0 * Ht ** 3 * out["nw"]
    return out


def drho_dh(dens, h):
    """d rho / d h = -(1/h) sum_j m_j (3 W + r dW/dr)."""
    return -dens["S_m"] / np.asarray(h, dtype=np.float64)


# -------------------------------------------------------------------- h iteration
def h_iterate(x, m, h0, L, periodic, n_ngb=N_NGB, tol=1e-4, max_iter=30, targets=None,
              method="auto", gamma_k=float(GAMMA_K)):
    """Solve N~_i(h_i) = n_ngb per particle (FP64 throughout, H = gamma_k * h).

    For iteration it = 1..max_iter on every still-active particle:
      1. density at the current h;
      2. F = N~ - n_ngb; converged when |F| <= tol * n_ngb (h kept, stop);
      3. on the last iteration the particle stops unconverged with h unchanged;
      4. otherwise bracket: F < 0 -> lo = h, else hi = h;
         Newton h' = h - F / (dN~/dh) with dN~/dh = gamma_k (4 pi/3) H^2 (3 nw - S)
         (h' = 2h when the derivative is not positive), clamped to [h/2, 2h];
         when both bracket ends are known and h' is not strictly inside them,
         h' = (lo + hi) / 2.
    Every particle's iteration is independent of the others' (its density at its
    own h depends on positions only).  Returns (h, converged, iterations, dens)
    with dens the density dict at the returned h.
    """
    n = x.shape[0]
    targets = np.arange(n) if targets is None else np.asarray(targets, dtype=np.int64)
    h = np.asarray(h0, dtype=np.float64)[targets].copy()
    lo = np.zeros_like(h)
    hi = np.full_like(h, np.inf)
    conv = np.zeros(len(h), dtype=bool)
    iters = np.zeros(len(h), dtype=np.int64)
    final = {k: np.zeros(len(h)) for k in ("rho", "S_m", "Sr_m", "nw", "S", "Nw")}
    final["count"] = np.zeros(len(h), dtype=np.int64)
    active = np.arange(len(h))
    for it in range(1, max_iter + 1):
        if active.size == 0:
            break
        Hall = np.zeros(n)
        Hall[targets[active]] = gamma_k * h[active]
        d = density(x, m, Hall, L, periodic, targets=targets[active], method=method)
        for k in final:
            final[k][active] = d[k]
        iters[active] = it
        F = d["Nw"] - n_ngb
        done = np.abs(F) <= tol * n_ngb
        conv[active[done]] = True
        if it == max_iter:
            break
        upd = active[~done]
        Fu = F[~done]
        hu = h[upd]
        H = gamma_k * hu
        dN = gamma_k * (4.0 * np.pi / 3.0) * H * H * (3.0 * d["nw"][~done] - d["S"][~done])
        lo[upd] = np.where(Fu < 0, hu, lo[upd])
        hi[upd] = np.where(Fu < 0, hi[upd], hu)
        with np.errstate(divide="ignore", invalid="ignore"):
            hn = np.where(dN > 0, hu - Fu / dN, np.where(Fu < 0, 2.0 * hu, 0.5 * hu))
        hn = np.clip(hn, 0.5 * hu, 2.0 * hu)
        both = (lo[upd] > 0) & np.isfinite(hi[upd])
        outside = both & ~((hn > lo[upd]) & (hn < hi[upd]))
        hn = np.where(outside, 0.5 * (lo[upd] + hi[upd]), hn)
        h[upd] = hn
        active = upd
    return h, conv, iters, final


# -------------------------------------------------------------------------- ghost
def ghost(rho, Sr_m, u, gamma=GAMMA_GAS):
    """Derived per-particle quantities between the passes.

    P = (gamma - 1) rho u; c = sqrt(gamma P / rho);
    f = [1 + h/(3 rho) d rho/d h]^-1.  With h d rho/dh = -(3 rho + sum_j m_j r dW/dr)
    this is f = 3 rho / (-sum_{j != i} m_j r dW/dr) (``Sr_m``), the same quantity
    without the cancellation of 1 - S_m/(3 rho).  Reading: f is undefined when no
    other particle lies inside the support (rho then does not depend on h beyond
    the self term); it is taken as 1 there.
    """
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    Sr_m = np.asarray(Sr_m, dtype=np.float64)
    P = (gamma - 1.0) * rho * u
    c = np.sqrt(gamma * P / rho)
    f = np.where(Sr_m < 0, 3.0 * rho / np.where(Sr_m < 0, -Sr_m, 1.0), 1.0)
    return {"P": P, "c": c, "f": f}


# -------------------------------------------------------------------------- force
def force(x, v, m, H, rho, P, c, f, L, periodic, alpha=ALPHA_VISC, targets=None, method="auto"):
    """Force pass over pairs with r < max(H_i, H_j), r > 0.

    With x_ij = x_i - x_j, r = |x_ij|, W'_k = dW/dr(r, H_k), F_k = f_k P_k / rho_k^2,
    v_ij = v_i - v_j, w = v_ij . x_ij / r, mu = min(w, 0):
      v_sig = c_i + c_j - 3 mu,  Pi = -alpha v_sig mu / (rho_i + rho_j),
      a_i   -= m_j [F_i W'_i + F_j W'_j + Pi (W'_i + W'_j)/2] x_ij / r,
      du_i  += m_j [F_i W'_i + Pi (W'_i + W'_j)/4] v_ij . x_ij / r,
      vsig_i = max_j v_sig (0 when i has no partner).
    Returns dict a (t, 3), dudt (t,), vsig (t,).
    """
    n = x.shape[0]
    targets = np.arange(n) if targets is None else np.asarray(targets, dtype=np.int64)
    H = np.asarray(H, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    t, j, r2, d = neighbour_pairs(x, None, L, periodic, targets, "force", Hall=H, method=method)
    pos = r2 > 0
    t, j, r2, d = t[pos], j[pos], r2[pos], d[pos]
    i = targets[t]
    r = np.sqrt(r2)
    Wi = kernel_dwdr(r, H[i])
    Wj = kernel_dwdr(r, H[j])
    Fi = f[i] * P[i] / rho[i] ** 2
    Fj = f[j] * P[j] / rho[j] ** 2
    vij = v[i] - v[j]
    vdx = (vij * d).sum(1)
    w = vdx / r
    mu = np.minimum(w, 0.0)
    vsig = c[i] + c[j] - 3.0 * mu
    Pi = -alpha * vsig * mu / (rho[i] + rho[j])
    Wbar = 0.5 * (Wi + Wj)
    coef = Fi * Wi + Fj * Wj + Pi * Wbar
    nt = len(targets)
    acc = np.zeros((nt, 3))
    for k in range(3):
        acc[:, k] = -np.bincount(t, weights=m[j] * coef * d[:, k] / r, minlength=nt)
    dudt = np.bincount(t, weights=m[j] * (Fi * Wi + 0.5 * Pi * Wbar) * w, minlength=nt)
    vs = np.zeros(nt)
    np.maximum.at(vs, t, vsig)
    return {"a": acc, "dudt": dudt, "vsig": vs}


# ------------------------------------------------------------------- reductions
def reductions(m, v, u, a, dudt):
    """[sum m a (3), sum m (v.a + du/dt), sum m v (3), sum m (v^2/2 + u)] in FP64."""
    m = np.asarray(m, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    dudt = np.asarray(dudt, dtype=np.float64)
    out = np.zeros(8)
    out[0:3] = (m[:, None] * a).sum(0)
    out[3] = (m * ((v * a).sum(1) + dudt)).sum()
    out[4:7] = (m[:, None] * v).sum(0)
    out[7] = (m * (0.5 * (v * v).sum(1) + u)).sum()
    return out


# ------------------------------------------------------------------ full pass
def full_step(box, n_ngb=N_NGB, tol=1e-4, max_iter=30, alpha=ALPHA_VISC, gamma=GAMMA_GAS,
              iterate_h=True, method="auto"):
    """Density (with h iteration), ghost, force and reductions for a whole box.

    With ``iterate_h=False`` the given h is used as is (H = FP32 support radius);
    with ``iterate_h=True`` h is iterated in FP64 from the given h.
    Returns a dict of FP64 arrays in the box's particle order.
    """
    x, m = box.x, box.m.astype(np.float64)
    if iterate_h:
        h, conv, iters, dens = h_iterate(x, m, box.h, box.L, box.periodic, n_ngb, tol, max_iter,
                                         method=method)
        H = float(GAMMA_K) * h
    else:
        h = box.h.astype(np.float64)
        H = support_radius(box.h)
        dens = density(x, m, H, box.L, box.periodic, method=method)
        conv = np.ones(box.n, dtype=bool)
        iters = np.ones(box.n, dtype=np.int64)
    g = ghost(dens["rho"], dens["Sr_m"], box.u, gamma)
    fo = force(x, box.v, m, H, dens["rho"], g["P"], g["c"], g["f"], box.L, box.periodic,
               alpha, method=method)
    red = reductions(m, box.v, box.u, fo["a"], fo["dudt"])
    out = dict(dens)
    out.update(g)
    out.update(fo)
    out.update({"h": h, "H": H, "drho_dh": drho_dh(dens, h), "converged": conv,
                "iterations": iters, "reductions": red})
    return out


# ------------------------------------------------------------- time stepping
def kdk_steps(box, dt, n_steps, n_ngb=N_NGB, tol=1e-4, max_iter=30, alpha=ALPHA_VISC, gamma=GAMMA_GAS,
              method="auto"):
    """Fixed-step kick-drift-kick integration (Section III-B: fixed time step,
    forces on every particle each step; the integrator itself is a reading).

    Starting forces come from an h iteration and a force pass at the initial
    positions; every step then does v += a dt/2, u += du/dt dt/2 (u >= 0),
    x += v dt in FP64 wrapped into [0, L), h iteration from the previous h,
    force pass, and the closing half kick.  v, u are held in FP64.  The force
    pass of a step takes v and u predicted to the end of the step with the
    previous forces, v + a dt/2 and max(u + du/dt dt/2, 0) (as the drift of the
    force-relevant quantities in Springel 2005), so that its velocity- and
    u-dependent terms are taken at the time of the positions.
    Returns (x, v, u, h, last full_step dict).
    """
    from copy import deepcopy
    b = deepcopy(box)
    x = b.x.astype(np.float64).copy()
    v = b.v.astype(np.float64).copy()
    u = b.u.astype(np.float64).copy()
    m = b.m.astype(np.float64)

    def passes(h0, vp, up):
        h, conv, _, dens = h_iterate(x, m, h0, b.L, b.periodic, n_ngb, tol, max_iter, method=method)
        H = float(GAMMA_K) * h
        g = ghost(dens["rho"], dens["Sr_m"], up, gamma)
        fo = force(x, vp, m, H, dens["rho"], g["P"], g["c"], g["f"], b.L, b.periodic, alpha, method=method)
        out = dict(dens)
        out.update(g)
        out.update(fo)
        out["h"] = h
        return h, out

    h, out = passes(b.h.astype(np.float64), v, u)
    for _ in range(n_steps):
        v += 0.5 * dt * out["a"]
        u = np.maximum(u + 0.5 * dt * out["dudt"], 0.0)
        x = x + v * dt
        if b.periodic:
            x = np.mod(x, b.L)
            x[x >= b.L] = 0.0
        h, out = passes(h, v + 0.5 * dt * out["a"], np.maximum(u + 0.5 * dt * out["dudt"], 0.0))
        v += 0.5 * dt * out["a"]
        u = np.maximum(u + 0.5 * dt * out["dudt"], 0.0)
    return x, v, u, h, out
