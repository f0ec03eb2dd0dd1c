"""Spatial decomposition of one periodic box over several ranks (Section IV of
the paper names a hybrid shared/distributed-memory version as future work).

Each rank owns the particles of one slab of the box along x (slabs of equal
particle count) and computes their density, smoothing length and forces with
the single-box library on its own GPU.  What a rank needs from the others is a
halo: every particle within ``width`` of its slab (periodic distance along x).
With ``width`` at least twice the largest support radius H_max, the halo holds

* every neighbour j of an owned particle i (r < max(H_i, H_j) <= H_max), and
* every neighbour of those neighbours within their own support (their densities
  enter i's force),

so owned results equal the single-box results (up to the order of FP32 sums).
One step:

1. halo exchange of positions, velocities, masses, internal energies and h;
2. the h iteration over owned + halo particles: an owned particle's density
   depends only on its own support, so its h converges exactly as in one box
   (halo particles at the outer edge converge to wrong values, which step 3
   replaces);
3. exchange of the converged h of every halo particle from its owner (the one
   exchange of results the passes need);
4. density, ghost and force passes at those fixed h over owned + halo particles:
   the owned particles' forces;
5. the FP64 conservation sums of the owned particles (the library sums only a
   box's owned particles, sph_box_set_owned), added over ranks.

The exchanges use ``torch.distributed`` all-gathers of the boundary particles
(each rank keeps what falls in its halo): NCCL on GPUs, gloo on CPUs.  The width
is checked after the h iteration against the largest final H of all ranks and
the step is redone with a wider halo when it was too narrow.

The per-rank computation is an object (``compute``) with two methods:
``h_iterate(box) -> h`` and ``passes(box, n_owned) -> dict`` (fields ``count``,
``rho``, ``a``, ``dudt``, ``vsig`` of every particle of the box, and
``reductions``, the 8 conservation sums of its first n_owned particles).
``LibraryCompute`` runs them through the C-ABI on the rank's GPU.
"""
from __future__ import annotations

import numpy as np

from . import inputs

# --------------------------------------------------------------------- geometry
def slab_bounds(x0: np.ndarray, nranks: int, L: float) -> np.ndarray:
    """Slab boundaries b_0 = 0 < b_1 < ... < b_R = L along x with (about) equal
    particle counts, from the x coordinates of every particle."""
    q = np.quantile(np.asarray(x0, dtype=np.float64), np.arange(1, nranks) / nranks)
    return np.concatenate([[0.0], q, [float(L)]])


def owners(x0: np.ndarray, bounds: np.ndarray) -> np.ndarray:
    """Rank owning each particle: slab r holds b_r <= x < b_{r+1}."""
    r = np.searchsorted(bounds, np.asarray(x0, dtype=np.float64), side="right") - 1
    return np.clip(r, 0, len(bounds) - 2)


def slab_distance(x0: np.ndarray, bounds: np.ndarray, r: int, L: float) -> np.ndarray:
    """Periodic distance along x from each position to slab r (0 inside)."""
    lo, hi = float(bounds[r]), float(bounds[r + 1])
    x0 = np.asarray(x0, dtype=np.float64)
    best = np.full(x0.shape, np.inf)
    for s in (-L, 0.0, L):
        y = x0 + s
        best = np.minimum(best, np.maximum(0.0, np.maximum(lo - y, y - hi)))
    return best


def halo_mask(x0: np.ndarray, bounds: np.ndarray, r: int, width: float, L: float, own: np.ndarray) -> np.ndarray:
    """Particles of other ranks within `width` of slab r."""
    return (own != r) & (slab_distance(x0, bounds, r, L) < width)


# --------------------------------------------------------------------- exchange
def _device(dist):
    import torch
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def all_gather_rows(dist, arr: np.ndarray) -> list[np.ndarray]:
    """Every rank's 2-D float64 array (rows of equal width), gathered on every rank."""
    import torch
    dev = _device(dist)
    arr = np.ascontiguousarray(arr, dtype=np.float64)
    n = torch.tensor([arr.shape[0]], dtype=torch.int64, device=dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(dist.get_world_size())]
    dist.all_gather(sizes, n)
    sizes = [int(s.item()) for s in sizes]
    width = arr.shape[1]
    pad = max(max(sizes), 1)
    buf = torch.zeros((pad, width), dtype=torch.float64, device=dev)
    buf[: arr.shape[0]] = torch.from_numpy(arr).to(dev)
    out = [torch.zeros((pad, width), dtype=torch.float64, device=dev) for _ in sizes]
    dist.all_gather(out, buf)
    return [o[:s].cpu().numpy() for o, s in zip(out, sizes)]


def _pack(box, gid) -> np.ndarray:
    """Rows of (global id, x(3), v(3), m, u, h) in FP64 (FP32 fields exactly)."""
    return np.column_stack([gid.astype(np.float64), box.x, box.v.astype(np.float64), box.m.astype(np.float64),
                            box.u.astype(np.float64), box.h.astype(np.float64)])


def _unpack(rows: np.ndarray, L: float, periodic: bool, name: str) -> tuple[inputs.ParticleBox, np.ndarray]:
    gid = rows[:, 0].astype(np.int64)
    box = inputs.ParticleBox(rows[:, 1:4].copy(), rows[:, 4:7].astype(np.float32), rows[:, 7].astype(np.float32),
                             rows[:, 8].astype(np.float32), rows[:, 9].astype(np.float32), L, periodic, name, {})
    return box, gid


def exchange_halo(dist, owned, gid, bounds, width):
    """The halo of this rank: other ranks' particles within `width` of its slab,
    as (ParticleBox, global ids), ordered by global id."""
    r = dist.get_rank()
    L = owned.L
    # each rank sends the particles within `width` of any other slab
    near = np.zeros(owned.n, dtype=bool)
    for q in range(dist.get_world_size()):
        if q != r:
            near |= slab_distance(owned.x[:, 0], bounds, q, L) < width
    parts = all_gather_rows(dist, _pack(owned.subset(np.nonzero(near)[0]), gid[near]))
    rows = [p for q, p in enumerate(parts) if q != r and len(p)]
    if not rows:
        return _unpack(np.zeros((0, 10)), L, owned.periodic, "halo")
    rows = np.concatenate(rows)
    keep = slab_distance(rows[:, 1], bounds, r, L) < width
    rows = rows[keep]
    rows = rows[np.argsort(rows[:, 0], kind="stable")]
    return _unpack(rows, L, owned.periodic, "halo")


def _concat(a, b, name):
    return inputs.ParticleBox(np.concatenate([a.x, b.x]), np.concatenate([a.v, b.v]), np.concatenate([a.m, b.m]),
                              np.concatenate([a.u, b.u]), np.concatenate([a.h, b.h]), a.L, a.periodic, name, {})


# --------------------------------------------------------------------- one step
def spatial_passes(dist, owned, gid, bounds, compute, width_factor=2.0, headroom=1.5, max_widen=4):
    """Density with the h iteration, then force, for this rank's owned particles
    (ParticleBox ``owned`` with global ids ``gid``), slab ``bounds`` shared by all
    ranks.  The halo starts at width_factor x headroom x the largest first-guess
    support radius (headroom: room for h to grow while it iterates) and is widened
    when the converged supports need more.  Returns (results of the owned
    particles in their order, halo size, width used) with ``h`` and the
    rank-summed ``reductions`` among the results."""
    import torch
    dev = _device(dist)

    def allmax(v):
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    H0 = allmax(float(inputs_support_max(owned)))
    width = width_factor * headroom * H0
    for _ in range(max_widen):
        halo, hgid = exchange_halo(dist, owned, gid, bounds, width)
        local = _concat(owned, halo, "owned+halo")
        h = np.asarray(compute.h_iterate(local), dtype=np.float32)
        Hmax = allmax(float(np.max(support_radius32(h[: owned.n]))) if owned.n else 0.0)
        if width_factor * Hmax <= width:
            break
        width = width_factor * 1.25 * Hmax     # too narrow for the converged supports: again, wider
    # the converged h of every halo particle, from its owner
    own_rows = np.column_stack([gid.astype(np.float64), h[: owned.n].astype(np.float64)])
    table = np.concatenate(all_gather_rows(dist, own_rows))
    order = np.argsort(table[:, 0], kind="stable")
    ids, hs = table[order, 0].astype(np.int64), table[order, 1].astype(np.float32)
    pos = np.searchsorted(ids, hgid)
    assert np.all(ids[pos] == hgid), "a halo particle has no owner"
    local.h = np.concatenate([h[: owned.n], hs[pos]]).astype(np.float32)
    res = compute.passes(local, owned.n)
    out = {k: np.asarray(v)[: owned.n] for k, v in res.items() if k != "reductions"}
    out["h"] = local.h[: owned.n]
    red = torch.tensor(np.asarray(res["reductions"], dtype=np.float64), device=dev)
    dist.all_reduce(red)
    out["reductions"] = red.cpu().numpy()
    return out, halo.n, width


def support_radius32(h):
    """H = gamma_K h rounded to FP32 (the support radius every pass compares against)."""
    return (np.float32(1.825742) * np.asarray(h, dtype=np.float32)).astype(np.float32)


def inputs_support_max(box) -> float:
    return float(np.max(support_radius32(box.h))) if box.n else 0.0


# --------------------------------------------------------------------- per-rank compute on the GPU
class LibraryCompute:
    """The per-rank passes through the C-ABI on the current GPU (one context)."""

    def __init__(self, sph_module, ctx):
        self.sph, self.ctx = sph_module, ctx

    def h_iterate(self, box):
        b = self.sph.box_from(self.ctx, box)
        try:
            b.h_update()            # halo particles at the outer edge may stop unconverged
            return b.get("h")
        finally:
            b.close()

    def passes(self, box, n_owned):
        b = self.sph.box_from(self.ctx, box)
        try:
            b.set_owned(n_owned)
            b.density()
            b.force()
            return {"count": b.get("count"), "rho": b.get("rho"), "a": b.get("a"), "dudt": b.get("dudt"),
                    "vsig": b.get("vsig"), "reductions": b.get("reductions")}
        finally:
            b.close()
