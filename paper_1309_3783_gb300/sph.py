"""Python binding of libsph (include/sph.h): the same entry points, marshalling only.

Every computation runs in the library's CUDA kernels.  The binding loads the
in-tree ``_build/libsph.so`` and raises if it is missing -- there is no
fallback.  Host arguments are numpy arrays; device arguments are CUDA torch
tensors (their data pointers are passed with ``SPH_MEM_DEVICE``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsph.so")

SPH_OK = 0
STATUS = {0: "SPH_OK", -1: "SPH_E_INVALID", -2: "SPH_E_OOM", -3: "SPH_E_H_TOO_LARGE", -4: "SPH_E_NOT_BUILT",
          -5: "SPH_E_NOT_CONVERGED", -6: "SPH_E_TIMEOUT", -7: "SPH_E_CUDA", -8: "SPH_E_BUSY"}
SPH_E_NOT_CONVERGED = -5
SPH_MEM_HOST, SPH_MEM_DEVICE = 0, 1

FIELDS = {"rho": 0, "drho_dh": 1, "nw": 2, "nngb": 3, "count": 4, "h": 5, "P": 6, "c": 7, "f": 8, "a": 9,
          "dudt": 10, "vsig": 11, "converged": 12, "x": 13, "v": 14, "u": 15, "reductions": 16,
          "force_count": 17}
_FIELD_TYPE = {0: (np.float32, 1), 1: (np.float32, 1), 2: (np.float32, 1), 3: (np.float32, 1), 4: (np.int32, 1),
               5: (np.float32, 1), 6: (np.float32, 1), 7: (np.float32, 1), 8: (np.float32, 1), 9: (np.float32, 3),
               10: (np.float32, 1), 11: (np.float32, 1), 12: (np.int32, 1), 13: (np.float64, 3),
               14: (np.float32, 3), 15: (np.float32, 1), 16: (np.float64, 1), 17: (np.int32, 1)}


class sph_params(C.Structure):
    _fields_ = [("gamma_kernel", C.c_float), ("n_ngb", C.c_float), ("gamma_gas", C.c_float),
                ("alpha_visc", C.c_float), ("c_cfl", C.c_float), ("h_tol", C.c_float),
                ("h_max_iter", C.c_int32), ("leaf_max", C.c_int32), ("split_frac", C.c_float),
                ("max_depth", C.c_int32), ("split_headroom", C.c_float), ("reuse", C.c_int32),
                ("sort_merge", C.c_int32), ("cluster_max", C.c_int32), ("compensated", C.c_int32),
                ("precision", C.c_int32), ("graphs", C.c_int32),
                ("pair_cache", C.c_int32), ("h_gather", C.c_int32)]


class sph_stats(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("n_cells", C.c_int64), ("n_leaves", C.c_int64),
                ("n_selfs", C.c_int64), ("n_pairs", C.c_int64), ("n_sort_segments", C.c_int64),
                ("n_sorted_entries", C.c_int64), ("top_level", C.c_int32), ("depth", C.c_int32),
                ("h_iterations", C.c_int32), ("rebuilds", C.c_int32), ("n_unconverged", C.c_int64),
                ("density_pairs", C.c_int64), ("density_sides", C.c_int64), ("density_candidates", C.c_int64),
                ("density_pairs_cellpair", C.c_int64), ("density_sides_cellpair", C.c_int64),
                ("density_candidates_cellpair", C.c_int64), ("force_pairs", C.c_int64),
                ("force_candidates", C.c_int64), ("force_pairs_cellpair", C.c_int64),
                ("force_candidates_cellpair", C.c_int64), ("guard_rechecks", C.c_int64),
                ("builds", C.c_int64), ("reuses", C.c_int64), ("h_active_after_first", C.c_int64),
                ("leaf_max", C.c_int64), ("cluster_max", C.c_int64), ("graph_steps", C.c_int64),
                ("host_steps", C.c_int64), ("host_syncs", C.c_int64),
                ("force_tasks_replayed", C.c_int64), ("force_tasks_culled", C.c_int64),
                ("h_gathered_passes", C.c_int64)]


class sph_profile_entry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("calls", C.c_int64), ("launches", C.c_int64), ("ms", C.c_double)]


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_P = C.c_void_p
_SIGS = {
    "sph_params_default": (None, [C.POINTER(sph_params)]),
    "sph_ctx_create": (C.c_int, [C.POINTER(sph_params), C.c_int, C.POINTER(_P)]),
    "sph_ctx_set_stream": (C.c_int, [_P, _P]),
    "sph_ctx_stream": (_P, [_P]),
    "sph_ctx_destroy": (C.c_int, [_P]),
    "sph_last_error": (C.c_char_p, [_P]),
    "sph_box_create": (C.c_int, [_P, C.c_int64, C.c_double, C.c_int, C.POINTER(_P)]),
    "sph_box_set": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int]),
    "sph_box_count_pairs": (C.c_int, [_P, C.c_int]),
    "sph_box_set_owned": (C.c_int, [_P, C.c_int64]),
    "sph_box_set_field": (C.c_int, [_P, C.c_int, _P, C.c_int64, C.c_int]),
    "sph_box_destroy": (C.c_int, [_P]),
    "sph_build": (C.c_int, [_P]),
    "sph_density": (C.c_int, [_P]),
    "sph_h_update": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "sph_force": (C.c_int, [_P]),
    "sph_step": (C.c_int, [_P, C.c_double]),
    "sph_cfl_dt": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "sph_get": (C.c_int, [_P, C.c_int, _P, C.c_int64, C.c_int]),
    "sph_get_stats": (C.c_int, [_P, C.POINTER(sph_stats)]),
    "sph_box_profile": (C.c_int, [_P, C.c_int]),
    "sph_get_profile": (C.c_int, [_P, C.c_int32, C.POINTER(sph_profile_entry), C.POINTER(C.c_int32)]),
    "sph_launch_count": (C.c_int64, []),
    "sph_measure_fp32_peak": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "sph_get_fields": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_void_p),
                                 C.POINTER(C.c_int64), C.c_int]),
    "sph_box_tune": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "sph_box_set_cluster_max": (C.c_int, [_P, C.c_int32]),
    "sph_box_set_leaf_max": (C.c_int, [_P, C.c_int32]),
    "sph_get_cells": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, C.POINTER(C.c_int64)]),
    "sph_get_interactions": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, C.POINTER(C.c_int64)]),
    "sph_server_create": (C.c_int, [_P, C.c_int64, C.c_int32, C.POINTER(_P)]),
    "sph_server_submit": (C.c_int, [_P, C.c_int64, C.c_double, C.c_int, _P, _P, _P, _P, _P, C.c_int32,
                                    C.c_double, C.POINTER(C.c_int64)]),
    "sph_server_tick": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "sph_server_set_tick_budget": (C.c_int, [_P, C.c_int64]),
    "sph_server_intake_ms": (C.c_int, [_P, C.c_int64, C.POINTER(C.c_float)]),
    "sph_server_poll": (C.c_int, [_P, C.c_int64, C.POINTER(C.c_int32), _P, C.c_int32]),
    "sph_server_get": (C.c_int, [_P, C.c_int64, C.c_int, _P, C.c_int64]),
    "sph_server_release": (C.c_int, [_P, C.c_int64]),
    "sph_server_destroy": (C.c_int, [_P]),
    "sph_density_static": (C.c_int, [_P, _P, _P, C.c_int64, C.c_double, C.c_int, _P, _P, _P]),
}

SPH_STATIC_MAX_N = 16384

_lib = None


def load(path: str | None = None):
    """Load libsph.so (built by ``paper_1309_3783_gb300.build``).  Raises when absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libsph.so not found at {p}: run __graft_entry__.build() first")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _err(ctx):
    if not ctx:
        return ""
    s = load().sph_last_error(ctx)
    return s.decode() if s else ""


def _check(status, ctx, allow=()):
    if status != SPH_OK and status not in allow:
        raise SphError(status, _err(ctx))
    return status


# ---------------------------------------------------------------- marshalling
def _arg(a, dtype, count):
    """(pointer, mem, keepalive) for a numpy array or a CUDA torch tensor."""
    if hasattr(a, "is_cuda") and a.is_cuda:
        import torch
        want = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous() or a.numel() != count:
            raise ValueError(f"device tensor must be contiguous {want} with {count} elements")
        return C.c_void_p(a.data_ptr()), SPH_MEM_DEVICE, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.size != count:
        raise ValueError(f"expected {count} elements, got {arr.size}")
    return arr.ctypes.data_as(C.c_void_p), SPH_MEM_HOST, arr


# ---------------------------------------------------------------- entry points
def sph_params_default() -> sph_params:
    p = sph_params()
    load().sph_params_default(C.byref(p))
    return p


def sph_ctx_create(params: sph_params | None = None, device: int = 0):
    h = C.c_void_p()
    st = load().sph_ctx_create(C.byref(params) if params is not None else None, device, C.byref(h))
    if st != SPH_OK:
        raise SphError(st, "sph_ctx_create failed")
    return h


def sph_ctx_set_stream(ctx, stream: int | None):
    _check(load().sph_ctx_set_stream(ctx, C.c_void_p(stream) if stream else None), ctx)


def sph_ctx_stream(ctx) -> int:
    return load().sph_ctx_stream(ctx) or 0


def sph_ctx_destroy(ctx):
    _check(load().sph_ctx_destroy(ctx), None)


def sph_last_error(ctx) -> str:
    return _err(ctx)


def sph_box_create(ctx, n: int, box_len: float, periodic: bool = True):
    h = C.c_void_p()
    _check(load().sph_box_create(ctx, int(n), float(box_len), 1 if periodic else 0, C.byref(h)), ctx)
    return h


def sph_box_set(box, ctx, x, v, m, u, h, n: int):
    px, mx, kx = _arg(x, np.float64, 3 * n)
    pv, mv, kv = _arg(v, np.float32, 3 * n)
    pm, mm, km = _arg(m, np.float32, n)
    pu, mu, ku = _arg(u, np.float32, n)
    ph, mh, kh = _arg(h, np.float32, n)
    mems = {mx, mv, mm, mu, mh}
    if len(mems) != 1:
        raise ValueError("all inputs must be on the host or all on the device")
    _check(load().sph_box_set(box, px, pv, pm, pu, ph, mems.pop()), ctx)


def sph_box_set_field(box, ctx, field, src, n: int):
    f = FIELDS[field] if isinstance(field, str) else int(field)
    dtype, per = _FIELD_TYPE[f]
    p, mem, keep = _arg(src, dtype, n * per)
    _check(load().sph_box_set_field(box, f, p, n, mem), ctx)


def sph_box_set_owned(box, ctx, n_owned: int):
    _check(load().sph_box_set_owned(box, int(n_owned)), ctx)


def sph_box_count_pairs(box, ctx, on: bool):
    _check(load().sph_box_count_pairs(box, 1 if on else 0), ctx)


def sph_box_destroy(box):
    _check(load().sph_box_destroy(box), None)


def sph_build(box, ctx):
    _check(load().sph_build(box), ctx)


def sph_density(box, ctx):
    _check(load().sph_density(box), ctx)


def sph_h_update(box, ctx):
    """Returns (status, n_unconverged, iterations); SPH_E_NOT_CONVERGED is not raised."""
    nu = C.c_int64()
    it = C.c_int32()
    st = _check(load().sph_h_update(box, C.byref(nu), C.byref(it)), ctx, allow=(SPH_E_NOT_CONVERGED,))
    return st, nu.value, it.value


def sph_force(box, ctx):
    _check(load().sph_force(box), ctx)


def sph_step(box, ctx, dt: float = 0.0):
    return _check(load().sph_step(box, float(dt)), ctx, allow=(SPH_E_NOT_CONVERGED,))


def sph_cfl_dt(box, ctx) -> float:
    d = C.c_double()
    _check(load().sph_cfl_dt(box, C.byref(d)), ctx)
    return d.value


def sph_get(box, ctx, field, n: int, out=None):
    """Copy a field into a new numpy array (or into ``out``: numpy or CUDA tensor)."""
    f = FIELDS[field] if isinstance(field, str) else int(field)
    dtype, per = _FIELD_TYPE[f]
    count = 8 if f == 16 else n * per
    if out is None:
        out = np.empty(count, dtype=dtype)
    p, mem, keep = _arg(out, dtype, count) if (hasattr(out, "is_cuda") and out.is_cuda) else (
        out.ctypes.data_as(C.c_void_p), SPH_MEM_HOST, out)
    _check(load().sph_get(box, f, p, 8 if f == 16 else n, mem), ctx)
    if isinstance(out, np.ndarray) and per == 3:
        return out.reshape(n, 3)
    return out


def sph_get_fields(box, ctx, outs: dict, n: int):
    """Copy several fields at once into host numpy arrays (``outs``: name -> array),
    with one synchronisation."""
    names = list(outs)
    k = len(names)
    fields = (C.c_int32 * k)(*[FIELDS[f] for f in names])
    ptrs = (C.c_void_p * k)(*[outs[f].ctypes.data_as(C.c_void_p).value for f in names])
    cnt = (C.c_int64 * k)(*[8 if FIELDS[f] == 16 else n for f in names])
    _check(load().sph_get_fields(box, k, fields, ptrs, cnt, SPH_MEM_HOST), ctx)
    return outs


def sph_get_stats(box, ctx) -> dict:
    s = sph_stats()
    _check(load().sph_get_stats(box, C.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in sph_stats._fields_}


def sph_box_profile(box, ctx, on: bool = True):
    _check(load().sph_box_profile(box, 1 if on else 0), ctx)


def sph_get_profile(box, ctx) -> dict:
    """{phase: {"calls", "launches", "ms"}} recorded since sph_box_profile(box, True)."""
    arr = (sph_profile_entry * 32)()
    n = C.c_int32()
    _check(load().sph_get_profile(box, 32, arr, C.byref(n)), ctx)
    return {arr[k].name.decode(): {"calls": arr[k].calls, "launches": arr[k].launches, "ms": arr[k].ms}
            for k in range(n.value)}


def sph_launch_count() -> int:
    return int(load().sph_launch_count())


def sph_measure_fp32_peak(ctx) -> float:
    """Measured FP32 FMA throughput of the context's device (TFLOP/s)."""
    v = C.c_double(0.0)
    _check(load().sph_measure_fp32_peak(ctx, C.byref(v)), ctx)
    return float(v.value)


def sph_box_tune(box, ctx) -> int:
    v = C.c_int32()
    _check(load().sph_box_tune(box, C.byref(v)), ctx)
    return v.value


def sph_box_set_leaf_max(box, ctx, leaf_max: int):
    _check(load().sph_box_set_leaf_max(box, int(leaf_max)), ctx)


def sph_box_set_cluster_max(box, ctx, cluster_max: int):
    _check(load().sph_box_set_cluster_max(box, int(cluster_max)), ctx)


def sph_get_cells(box, ctx) -> dict:
    n = C.c_int64()
    _check(load().sph_get_cells(box, 0, None, None, None, None, C.byref(n)), ctx)
    k = n.value
    lv = np.empty(k, np.int32); ijk = np.empty(3 * k, np.int32); ct = np.empty(k, np.int32); sp = np.empty(k, np.int32)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(load().sph_get_cells(box, k, ptr(lv), ptr(ijk), ptr(ct), ptr(sp), C.byref(n)), ctx)
    return {"level": lv, "ijk": ijk.reshape(k, 3), "count": ct, "split": sp}


def sph_get_interactions(box, ctx) -> dict:
    n = C.c_int64()
    _check(load().sph_get_interactions(box, 0, None, None, None, None, C.byref(n)), ctx)
    k = n.value
    kd = np.empty(k, np.int32); a = np.empty(k, np.int32); b = np.empty(k, np.int32); ax = np.empty(k, np.int32)
    ptr = lambda z: z.ctypes.data_as(C.c_void_p)
    _check(load().sph_get_interactions(box, k, ptr(kd), ptr(a), ptr(b), ptr(ax), C.byref(n)), ctx)
    return {"kind": kd, "a": a, "b": b, "axis": ax}


def sph_server_create(ctx, budget_bytes: int = 0, max_boxes: int = 0):
    h = C.c_void_p()
    _check(load().sph_server_create(ctx, int(budget_bytes), int(max_boxes), C.byref(h)), ctx)
    return h


def sph_server_submit(srv, x, v, m, u, h, box_len: float, periodic: bool, n_steps: int, dt: float) -> int:
    n = len(m)
    keep = [_arg(x, np.float64, 3 * n), _arg(v, np.float32, 3 * n), _arg(m, np.float32, n),
            _arg(u, np.float32, n), _arg(h, np.float32, n)]
    rid = C.c_int64()
    st = load().sph_server_submit(srv, n, float(box_len), 1 if periodic else 0, *[k[0] for k in keep],
                                  int(n_steps), float(dt), C.byref(rid))
    if st != SPH_OK:
        raise SphError(st, "sph_server_submit failed")
    return rid.value


def sph_server_set_tick_budget(srv, max_particles: int) -> None:
    st = load().sph_server_set_tick_budget(srv, int(max_particles))
    if st != SPH_OK:
        raise SphError(st, "sph_server_set_tick_budget failed")


def sph_server_intake_ms(srv, rid: int) -> float:
    ms = C.c_float(0.0)
    st = load().sph_server_intake_ms(srv, int(rid), C.byref(ms))
    if st != SPH_OK:
        raise SphError(st, "sph_server_intake_ms failed")
    return float(ms.value)


def sph_server_tick(srv) -> int:
    n = C.c_int32()
    st = load().sph_server_tick(srv, C.byref(n))
    if st != SPH_OK:
        raise SphError(st, "sph_server_tick failed")
    return n.value


def sph_server_poll(srv, rid: int, max_steps: int = 0):
    done = C.c_int32()
    ms = np.zeros(max(max_steps, 1), np.float32)
    st = load().sph_server_poll(srv, int(rid), C.byref(done), ms.ctypes.data_as(C.c_void_p), int(max_steps))
    if st != SPH_OK:
        raise SphError(st, "sph_server_poll failed")
    return bool(done.value), ms[:max_steps]


def sph_server_get(srv, rid: int, field, n: int):
    f = FIELDS[field] if isinstance(field, str) else int(field)
    dtype, per = _FIELD_TYPE[f]
    count = 8 if f == 16 else n * per
    out = np.empty(count, dtype=dtype)
    st = load().sph_server_get(srv, int(rid), f, out.ctypes.data_as(C.c_void_p), 8 if f == 16 else n)
    if st != SPH_OK:
        raise SphError(st, "sph_server_get failed")
    return out.reshape(n, 3) if per == 3 else out


def sph_server_release(srv, rid: int):
    st = load().sph_server_release(srv, int(rid))
    if st != SPH_OK:
        raise SphError(st, "sph_server_release failed")


def sph_server_destroy(srv):
    load().sph_server_destroy(srv)


# ---------------------------------------------------------------- convenience
class Box:
    """One box on one context: create, set, run the passes, read fields."""

    def __init__(self, ctx, n, box_len=1.0, periodic=True):
        self.ctx, self.n = ctx, int(n)
        self.h = sph_box_create(ctx, n, box_len, periodic)

    def set(self, x, v, m, u, h):
        sph_box_set(self.h, self.ctx, x, v, m, u, h, self.n)
        return self

    def set_field(self, field, src):
        sph_box_set_field(self.h, self.ctx, field, src, self.n)
        return self

    def set_owned(self, n_owned):
        sph_box_set_owned(self.h, self.ctx, n_owned)

    def count_pairs(self, on=True):
        sph_box_count_pairs(self.h, self.ctx, on)

    def build(self):
        sph_build(self.h, self.ctx)

    def density(self):
        sph_density(self.h, self.ctx)

    def h_update(self):
        return sph_h_update(self.h, self.ctx)

    def force(self):
        sph_force(self.h, self.ctx)

    def step(self, dt=0.0):
        return sph_step(self.h, self.ctx, dt)

    def cfl_dt(self):
        return sph_cfl_dt(self.h, self.ctx)

    def get(self, field, out=None):
        return sph_get(self.h, self.ctx, field, self.n, out)

    def get_many(self, outs: dict):
        """Fill several host arrays at once (name -> numpy array), one synchronisation."""
        return sph_get_fields(self.h, self.ctx, outs, self.n)

    def stats(self):
        return sph_get_stats(self.h, self.ctx)

    def tune(self):
        return sph_box_tune(self.h, self.ctx)

    def set_leaf_max(self, leaf_max):
        sph_box_set_leaf_max(self.h, self.ctx, leaf_max)

    def set_cluster_max(self, cluster_max):
        sph_box_set_cluster_max(self.h, self.ctx, cluster_max)

    def profile(self, on=True):
        sph_box_profile(self.h, self.ctx, on)

    def get_profile(self):
        return sph_get_profile(self.h, self.ctx)

    def cells(self):
        return sph_get_cells(self.h, self.ctx)

    def interactions(self):
        return sph_get_interactions(self.h, self.ctx)

    def close(self):
        if self.h:
            sph_box_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def box_from(ctx, pb) -> Box:
    """A Box holding a ParticleBox of ``paper_1309_3783_gb300.inputs``."""
    b = Box(ctx, pb.n, pb.L, pb.periodic)
    return b.set(pb.x, pb.v, pb.m, pb.u, pb.h)


def sph_density_static(x, m, h, box_len: float, periodic: bool, rho, count, stream: int = 0):
    """The allocation-free density pass (all arguments CUDA tensors); returns the status."""
    n = len(m)
    px, mx, _ = _arg(x, np.float64, 3 * n)
    pm, mm, _ = _arg(m, np.float32, n)
    ph, mh, _ = _arg(h, np.float32, n)
    pr, mr, _ = _arg(rho, np.float32, n)
    pc, mc, _ = _arg(count, np.int32, n)
    if {mx, mm, mh, mr, mc} != {SPH_MEM_DEVICE}:
        raise ValueError("sph_density_static takes device tensors only")
    import torch
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in (x, m, h, rho, count)):
        raise ValueError(f"sph_density_static runs on the current device (cuda:{dev}): every tensor must be there")
    return load().sph_density_static(px, pm, ph, n, float(box_len), 1 if periodic else 0, pr, pc,
                                     C.c_void_p(stream) if stream else None)
