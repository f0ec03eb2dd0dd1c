#!/usr/bin/env python
"""Throughput of the SPH density + force step on GB300 (one JSON line).

Workload (default): the large high-contrast box -- 33,554,432 particles, 30 %
uniform background plus 70 % in 4096 Plummer spheres with scale radii
log-uniform in [1e-4, 1e-2], periodic unit box, equal masses, u = 1,
v ~ N(0, 0.1), h iterated to 48 neighbours (H spans three orders of magnitude),
leaf size and cluster size autotuned.  ``--workload`` selects another:
``plummer-262144`` (262,144 particles, 50 % uniform plus 16 Plummer spheres) or
``lognormal-8388608`` (2^23 particles drawn from a log-normal field).

The run follows the paper's protocol (fixed time step, forces on every particle
every step): one step is a half kick, a drift, the whole decomposition build
(keys, sort, cell tree, interaction lists, particle offsets, axis sorts), density
with the h iteration (started from the last four steps' roots of N~(h) = 48,
extrapolated with a cubic), ghost, force, FP64 conservation reductions and the
closing half kick.  dt is the Courant step of the initial state (C_CFL = 0.3).

value : particle-updates/s of a run resident in device memory.
e2e   : the same through the C-ABI with host buffers: every step uploads the full
        state (x, v, m, u, h, a, du/dt) from pinned host memory and reads the new
        state back (x, v, u, h, a, du/dt, one multi-field read) inside the timed
        region.

step_control: per timed step, steps run as one captured CUDA graph, steps
        sequenced from the host (the fallback when a captured build's shape no
        longer holds) and host synchronisations; gpu_launches counts the kernels
        of the timed steps, those inside graphs included.

amortised: the same run with the decomposition kept over steps while it stays
        valid (sph_params.reuse, Section II-C: sorted indices re-used until the
        decomposition must be rebuilt); builds and reuses over the timed steps.

workloads: the other two single-box workloads, a shorter run each.

precision: the headline workload and the 262,144-particle box run again from the
        same state with plain FP32 positions (sph_params.precision = 1) beside the
        default offsets from each cell's centre: throughput, FP64 re-decisions per
        pass and the largest relative density difference between the two.

serving: the served batch -- 512 independent jittered-lattice boxes with
        particle counts log-uniform in [1k, 262k] (per-box seeds), each request
        advancing 10 kick-drift-kick steps -- through the continuous-batching
        server, which admits boxes while a tick steps at most 2^19 particles
        (sph_server_set_tick_budget).  A saturated run (every request submitted at
        once) measures the capacity; a run with Poisson arrivals at 80 % of that
        capacity gives the p50/p99 step latency (CUDA events around every batched
        step, one sample per box and step), the request latency and the aggregate
        throughput; the same arrivals again without the tick budget for
        comparison.  Boxes admitted in a tick first go through a batched intake
        pass (h iterated from the submitted h, starting forces; its device time
        reported apart, p50/p99_intake_ms) and take their first step in the same
        tick.  The same requests on a 1-in-8 subset also run one box at a
        time through the plain single-box path for comparison with the batched
        server.

``--workload clustered-4194304`` runs one octant of the headline recipe (the same
densities in a box of half the edge), the case the counter captures use.

``--impl reference`` times the FP64 oracle (the only reference this method has:
the paper publishes no code) on the host cores, each step on a bounded sample of
the same workload.  Under torchrun (N > 1) every rank runs an independent replica
on its own GPU ("replicas only": the path has no exchange step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1309_3783_gb300 import inputs  # noqa: E402

METRIC = "SPH density+force particle-updates/s"
UNIT = "particle-updates/s"


def _clustered(seed):
    return inputs.clustered_box(seed=seed)


def _plummer(seed):
    return inputs.plummer_box(seed=seed)


def _lognormal(seed):
    return inputs.lognormal_box(seed=seed)


def _clustered_octant(seed):
    return inputs.clustered_box(n=2 ** 22, n_spheres=512, L=0.5, seed=seed)


WORKLOADS = {
    "clustered-33554432": (_clustered, "33,554,432 particles: 30 % uniform, 70 % in 4096 Plummer spheres with "
                                       "scale radii log-uniform in [1e-4, 1e-2]"),
    "plummer-262144": (_plummer, "262,144 particles: 50 % uniform, 50 % in 16 Plummer spheres of scale 0.02"),
    "lognormal-8388608": (_lognormal, "8,388,608 particles drawn from a log-normal field (sigma 2, P(k) ~ k^-2, "
                                      "256^3 mesh)"),
}
# profiling only (never among the extra workloads): one octant of the headline
# recipe -- the same background density, sphere populations and scale radii in a
# box of half the edge -- small enough for multi-pass counter captures
PROFILE_WORKLOADS = {
    "clustered-4194304": (_clustered_octant, "4,194,304 particles: one octant of the 33,554,432-particle recipe "
                                             "(L = 0.5, 512 Plummer spheres: the same densities and sphere "
                                             "profiles)"),
}
DEFAULT_WORKLOAD = "clustered-33554432"
SAMPLE_K = 4096             # the oracle's bounded sample per step: particles nearest a drawn centre

# Algorithmic FP32 operations per interacting pair, counted from the formulas
# the kernels evaluate (mul/add = 1, FMA = 2, sqrt/rsqrt/div = 1; one branch of
# the piecewise kernel):
#   density: per unordered pair 11 (separation 3, r^2 5, two guard-band tests 2,
#            r 1) plus 16 per side that accumulates (q 1, w and w' 8, q w' 1,
#            four sums 6);
#   force:   per unordered pair 75 (separation 3, r^2 5, guard bands 2, 1/r and r
#            2, two kernel derivatives 10, v.x 8, w 1, min 1, v_sig 3, Pi 4,
#            W-bar 2, coefficient 6, half-viscosity 2, both sides' a, du/dt and
#            v_sig 26).
# bytes a force pass must move per particle: its position/offset, cell offset and
# mass, velocity and u, ghost quantities (4 x 16 B read), its a, du/dt and v_sig
# (20 B written)
FORCE_BYTES_PER_PARTICLE = 84
FLOPS_DENSITY_PAIR = 11
FLOPS_DENSITY_SIDE = 16
FLOPS_FORCE_PAIR = 75

# FP32 ALU peak of GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.070 GHz
SM_COUNT, FP32_LANES, MAX_SM_GHZ = 152, 128, 2.070
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * MAX_SM_GHZ / 1e3


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def host_threads():
    """Host cores this process may run on (the oracle's k-d tree searches use them all)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ replicas
def max_over_ranks(dist, value, device="cpu"):
    """The largest of every rank's value (the whole job ends with its slowest
    replica); the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput of independent replicas: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


def replica_seed(rank):
    """Every replica draws its own instance of the workload recipe."""
    return 1 + rank


# ------------------------------------------------------------------ timed runs
def timed_steps(torch, b, dt, stream, steps, flush=None):
    """Device time (ms) of each of `steps` steps, CUDA events on the library's stream."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            if flush is not None:
                flush.zero_()                       # L2 flush between steps (outside the events)
            evs[k][0].record(stream)
        b.step(dt)
        with torch.cuda.stream(stream):
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in evs]


def prepare_box(sph, ctx, box, tune, leaf=None):
    """Resident input state: h converged once (a simulation's previous step), the
    split threshold and cluster size tuned for the workload (or the split
    threshold given), dt from the CFL rule."""
    b = sph.Box(ctx, box.n, box.L, True)
    b.set(box.x, box.v, box.m, box.u, box.h)
    leaf_max = 400
    if leaf:
        b.set_leaf_max(leaf)
        leaf_max = leaf
        tune = False
    b.h_update()
    if tune:
        leaf_max = b.tune()                           # untimed
        b.h_update()
    b.force()
    return b, leaf_max, b.stats()["cluster_max"], b.cfl_dt()


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1309_3783_gb300 import build as libbuild
    from paper_1309_3783_gb300 import sph

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    make, recipe = {**WORKLOADS, **PROFILE_WORKLOADS}[args.workload]
    box = make(replica_seed(rank))
    n = box.n
    params = sph.sph_params_default()
    if getattr(args, "host_steps", False):
        params.graphs = 0
    ctx = sph.sph_ctx_create(params, device=local_rank)
    stream = torch.cuda.Stream()
    sph.sph_ctx_set_stream(ctx, stream.cuda_stream)
    b, leaf_max, cluster_max, dt = prepare_box(sph, ctx, box, not args.no_tune, args.leaf_max_set)
    args.leaf_max, args.cluster_max = leaf_max, cluster_max
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        b.step(dt)
    torch.cuda.synchronize()

    # algorithmic work of one step (the same for every step): exact pair counts
    # over the step's density passes and its force pass (untimed, after the warm-up
    # so that the h iteration starts as in the timed steps)
    b.count_pairs(True)
    b.step(dt)
    st = b.stats()
    b.count_pairs(False)
    flops_step = {"density": FLOPS_DENSITY_PAIR * st["density_pairs"] + FLOPS_DENSITY_SIDE * st["density_sides"],
                  "force": FLOPS_FORCE_PAIR * st["force_pairs"]}

    # inputs far larger than L2 need no flush; small ones get a 256 MB write between steps
    big = n * 520 > 4 * 129 * 2 ** 20
    flush = None if big else torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local_rank}")
    l0 = sph.sph_launch_count()
    st_first = b.stats()
    b.profile(True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.profiler.start()                 # ncu --profile-from-start off captures from here
        ms = timed_steps(torch, b, dt, stream, args.steps, flush)
        barrier()
        torch.cuda.profiler.stop()
    launches = sph.sph_launch_count() - l0
    st_last = b.stats()
    prof = b.get_profile()
    b.profile(False)
    total_ms = max_over_ranks(dist, sum(ms), f"cuda:{local_rank}")
    value = job_rate(world, n * args.steps, total_ms / 1e3)

    # e2e through the C-ABI: the state lives in pinned host buffers between steps
    pinned = lambda shape, dt_: torch.empty(shape, dtype=dt_).pin_memory().numpy()
    xh, vh, ah = pinned((n, 3), torch.float64), pinned((n, 3), torch.float32), pinned((n, 3), torch.float32)
    mh, uh, hh, duh = (pinned(n, torch.float32) for _ in range(4))
    b.get_many({"x": xh, "v": vh, "a": ah, "u": uh, "h": hh, "dudt": duh})
    mh[:] = box.m
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        b.set(xh, vh, mh, uh, hh)
        b.set_field("a", ah)
        b.set_field("dudt", duh)
        b.step(dt)
        b.get_many({"x": xh, "v": vh, "u": uh, "h": hh, "a": ah, "dudt": duh})
    barrier()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0, f"cuda:{local_rank}")
    e2e = job_rate(world, n * e2e_steps, e2e_s)

    # roofline of the dominant kernel (FP32 ALU bound), the force kernel: the largest
    # single launch of a step (the density phase of a captured step spans the whole h
    # iteration, several kernels); the FMA throughput measured beside it
    fp32_measured = sph.sph_measure_fp32_peak(ctx)
    dom = "force"
    calls = max(prof[dom]["calls"], 1)
    avg_ms = prof[dom]["ms"] / calls
    flops = flops_step[dom] * args.steps / calls
    achieved = flops / (avg_ms / 1e3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            tj = json.load(open(tpath)).get(args.workload, {})
            # counters taken on another decomposition do not describe this launch
            if dom in tj and tj.get("leaf_max") == leaf_max and tj.get("cluster_max") == cluster_max:
                traffic = tj[dom]
        except (OSError, ValueError, AttributeError):
            traffic = None

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "recipe": recipe, "particles_per_gpu": n,
                   "h": "iterated to N~ = 48 each step, from the last four steps' roots extrapolated (cubic)",
                   "protocol": "fixed-step kick-drift-kick run, forces on all particles every step, decomposition "
                               "rebuilt every step",
                   "dt": dt, "leaf_max": leaf_max, "cluster_max": cluster_max,
                   "leaf_max_source": ("set" if args.leaf_max_set else
                                       "autotuned" if not args.no_tune else "paper"),
                   "l2": ("inputs larger than L2 (about 540 B per particle resident)" if big
                          else "flushed between timed steps (256 MB write)"),
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": n * (24 + 12 + 4 + 4 + 4 + 12 + 4),
                "d2h_bytes_per_step": n * (24 + 12 + 4 + 4 + 12 + 4), "steps": e2e_steps},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "flops_per_launch": flops, "avg_launch_ms": avg_ms,
                     "algorithmic_bytes": n * FORCE_BYTES_PER_PARTICLE,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.070 GHz (nominal max clock)",
                     "peak_measured": fp32_measured,
                     "frac_of_measured": achieved / fp32_measured if fp32_measured else None,
                     "peak_measured_source": "independent FMA chains on every SM (sph_measure_fp32_peak), this run"},
        "gpu_launches": launches,
        "step_control": {k: (st_last[k] - st_first[k]) / args.steps for k in ("graph_steps", "host_steps", "host_syncs")},
        "clocks": clk.summary(),
        "phases_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in prof.items() if v["calls"]},
        "pairs": {"density": st["density_pairs"], "density_candidates": st["density_candidates"],
                  "force": st["force_pairs"], "force_candidates": st["force_candidates"],
                  "guard_rechecks": st["guard_rechecks"]},
        "decomposition": {"cells": st_last["n_cells"], "leaves": st_last["n_leaves"], "depth": st_last["depth"],
                          "pair_interactions": st_last["n_pairs"]},
        "h_iterations_last_step": st_last["h_iterations"],
        "h_unconverged_after_first_pass": st_last["h_active_after_first"] / box.n,
    }
    out["amortised"] = run_reuse_leg(sph, torch, b, box, dt, stream, args, flush)
    out["axis_sorts"] = run_sort_leg(sph, torch, b, box, stream, args)
    state = {k: b.get(k) for k in ("x", "v", "u", "h", "a", "dudt")}
    b.close()
    if not args.no_precision:
        out["precision"] = {args.workload: run_precision_leg(sph, torch, box, state, dt, stream, args)}
    if not args.no_extra_workloads:
        out["workloads"] = run_other_workloads(sph, torch, ctx, stream, args, rank,
                                               None if args.no_precision else out.setdefault("precision", {}))
    if not args.no_serving:
        out["serving"] = run_serving(sph, ctx)
    sph.sph_ctx_destroy(ctx)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(box, args.workload)
    if dist is not None:
        dist.destroy_process_group()
    return out


# ------------------------------------------------------------------ other legs
def run_other_workloads(sph, torch, ctx, stream, args, rank, precision=None, steps=10, warmup=3):
    """The other single-box workloads, a shorter run each (leaf and cluster size
    autotuned for each box); the 262,144-particle box also in both position
    precisions (into `precision`)."""
    out = {}
    for name, (make, recipe) in WORKLOADS.items():
        if name == args.workload:
            continue
        box = make(replica_seed(rank))
        b, leaf, cmax, dt = prepare_box(sph, ctx, box, tune=True)
        try:
            for _ in range(warmup):
                b.step(dt)
            torch.cuda.synchronize()
            flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
            ms = timed_steps(torch, b, dt, stream, steps, flush)
            del flush
            out[name] = {"value": box.n * steps / (sum(ms) / 1e3), "unit": UNIT, "ms_per_step": sum(ms) / steps,
                         "steps": steps, "leaf_max": leaf, "cluster_max": cmax, "recipe": recipe}
            if precision is not None and name == "plummer-262144":
                state = {k: b.get(k) for k in ("x", "v", "u", "h", "a", "dudt")}
                args_small = argparse.Namespace(leaf_max=leaf, cluster_max=cmax, warmup=warmup, steps=steps)
                precision[name] = run_precision_leg(sph, torch, box, state, dt, stream, args_small)
        finally:
            b.close()
    return out


def run_precision_leg(sph, torch, box, state, dt, stream, args):
    """The same state in both position precisions (sph_params.precision): offsets
    from each cell's centre taken from the FP64 positions (0, the default) and plain
    FP32 positions x / L (1).  Per mode: throughput of the stepping run, FP64
    re-decisions of one density and force pass, and the largest relative
    difference of the densities of that pass from the default mode's (the default
    mode is within 1e-6 of the FP64 oracle in the parity tests)."""
    out, rho = {}, {}
    for prec, name in ((0, "cell_offsets"), (1, "plain_fp32")):
        p = sph.sph_params_default()
        p.precision = prec
        ctx = sph.sph_ctx_create(p, device=torch.cuda.current_device())
        sph.sph_ctx_set_stream(ctx, stream.cuda_stream)
        b = sph.Box(ctx, box.n, box.L, True)
        try:
            b.set(state["x"], state["v"], box.m, state["u"], state["h"])
            b.set_leaf_max(args.leaf_max)
            b.set_cluster_max(args.cluster_max)
            b.count_pairs(True)
            b.density()
            rho[prec] = b.get("rho").astype(np.float64)
            b.force()
            st = b.stats()
            b.count_pairs(False)
            b.set_field("a", state["a"])
            b.set_field("dudt", state["dudt"])
            for _ in range(args.warmup):
                b.step(dt)
            torch.cuda.synchronize()
            ms = sum(timed_steps(torch, b, dt, stream, args.steps))
            out[name] = {"value": box.n * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
                         "fp64_decisions_per_pass": st["guard_rechecks"],
                         "pairs_per_pass": st["force_pairs"]}
        finally:
            b.close()
            sph.sph_ctx_destroy(ctx)
    out["plain_fp32"]["rho_max_rel_diff_from_cell_offsets"] = float(np.max(np.abs(rho[1] - rho[0]) / rho[0]))
    return out


def run_sort_leg(sph, torch, b, box, stream, args, builds=10):
    """Device time of the axis-sort phase per build, the cell lists sorted directly
    and built by merging the leaves' sorted runs (sph_params.sort_merge), on the
    timed run's state."""
    out = {}
    for name, merge in (("direct_ms", 0), ("merged_ms", 1)):
        p = sph.sph_params_default()
        p.sort_merge = merge
        ctx = sph.sph_ctx_create(p, device=torch.cuda.current_device())
        sph.sph_ctx_set_stream(ctx, stream.cuda_stream)
        bs = sph.Box(ctx, box.n, box.L, True)
        try:
            bs.set(b.get("x"), b.get("v"), box.m, b.get("u"), b.get("h"))
            bs.set_leaf_max(args.leaf_max)
            bs.set_cluster_max(args.cluster_max)
            bs.build()
            bs.profile(True)
            for _ in range(builds):
                bs.build()
            pr = bs.get_profile()
            out[name] = pr["axis_sort"]["ms"] / builds
            st = bs.stats()
            out["segments"], out["entries"] = st["n_sort_segments"], st["n_sorted_entries"]
        finally:
            bs.close()
            sph.sph_ctx_destroy(ctx)
    return out


def run_reuse_leg(sph, torch, b, box, dt, stream, args, flush):
    """The timed run again, on a box whose context keeps the decomposition over steps."""
    p = sph.sph_params_default()
    p.reuse = 1
    ctx = sph.sph_ctx_create(p, device=torch.cuda.current_device())
    sph.sph_ctx_set_stream(ctx, stream.cuda_stream)
    br = sph.Box(ctx, box.n, box.L, True)
    try:
        br.set(b.get("x"), b.get("v"), box.m, b.get("u"), b.get("h"))
        br.set_field("a", b.get("a"))
        br.set_field("dudt", b.get("dudt"))
        br.set_leaf_max(args.leaf_max)
        br.set_cluster_max(args.cluster_max)
        for _ in range(args.warmup):
            br.step(dt)
        torch.cuda.synchronize()
        s0 = br.stats()
        ms = sum(timed_steps(torch, br, dt, stream, args.steps, flush))
        s1 = br.stats()
        return {"value": box.n * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
                "builds": s1["builds"] - s0["builds"], "reuses": s1["reuses"] - s0["reuses"]}
    finally:
        br.close()
        sph.sph_ctx_destroy(ctx)


# ------------------------------------------------------------------ serving
SERVE_STEPS = 10
SERVE_LOAD = 0.8
SERVE_TICK_BUDGET = 2 ** 19     # particles a tick may step: two of the largest served boxes


def _served_requests(n_boxes):
    """(box, dt) per request: C_CFL x min H / (2 c) at the initial state (u = 1)."""
    out = []
    for bx in inputs.served_boxes(n_boxes):
        c = np.sqrt(5.0 / 3.0 * (5.0 / 3.0 - 1.0) * float(bx.u.max()))
        out.append((bx, 0.3 * 1.825742 * float(bx.h.min()) / (2.0 * c)))
    return out


def _serve(sph, ctx, reqs, arrivals=None, tick_budget=0):
    """Run requests through one server; returns (wall s, step ms list, request latencies s)."""
    srv = sph.sph_server_create(ctx, 0, 0)
    try:
        sph.sph_server_set_tick_budget(srv, tick_budget)
        order = np.argsort(arrivals) if arrivals is not None else np.arange(len(reqs))
        ids, t_sub = {}, {}
        k = 0
        done_t = {}
        t0 = time.perf_counter()
        while len(done_t) < len(reqs):
            now = time.perf_counter() - t0
            while k < len(reqs) and (arrivals is None or arrivals[order[k]] <= now):
                bx, dt = reqs[order[k]]
                ids[order[k]] = sph.sph_server_submit(srv, bx.x, bx.v, bx.m, bx.u, bx.h, bx.L, True, SERVE_STEPS, dt)
                t_sub[order[k]] = t0 + (arrivals[order[k]] if arrivals is not None else 0.0)
                k += 1
            active = sph.sph_server_tick(srv)
            tnow = time.perf_counter()
            for r, rid in ids.items():
                if r not in done_t and sph.sph_server_poll(srv, rid)[0]:
                    done_t[r] = tnow
            if active == 0 and k < len(reqs) and arrivals is not None:
                time.sleep(max(0.0, min(0.002, arrivals[order[k]] - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        step_ms, intake_ms = [], []
        for r, rid in ids.items():
            step_ms.extend(sph.sph_server_poll(srv, rid, SERVE_STEPS)[1].tolist())
            intake_ms.append(sph.sph_server_intake_ms(srv, rid))
            sph.sph_server_release(srv, rid)
        lat = [done_t[r] - t_sub[r] for r in ids]
        _serve.intake_ms = intake_ms
        return wall, step_ms, lat
    finally:
        sph.sph_server_destroy(srv)


def run_serving(sph, ctx, n_boxes=512):
    reqs = _served_requests(n_boxes)
    work = sum(bx.n for bx, _ in reqs) * SERVE_STEPS
    mean_n = work / SERVE_STEPS / len(reqs)
    # saturated: every request at once, the ticks as large as the budget allows
    wall_sat, _, _ = _serve(sph, ctx, reqs, tick_budget=SERVE_TICK_BUDGET)
    capacity = work / wall_sat
    rate = SERVE_LOAD * capacity / (mean_n * SERVE_STEPS)  # requests per second
    arrivals = inputs.poisson_arrivals(len(reqs), rate, seed=1)
    wall, step_ms, lat = _serve(sph, ctx, reqs, arrivals, tick_budget=SERVE_TICK_BUDGET)
    intake = [v for v in _serve.intake_ms if v >= 0.0]
    # the same arrivals without the tick budget: every waiting box admitted at once
    _, step_ms_nb, lat_nb = _serve(sph, ctx, reqs, arrivals)
    # the same requests on a 1-in-8 subset: batched server against one box at a time
    sub = reqs[::8]
    sub_work = sum(bx.n for bx, _ in sub) * SERVE_STEPS
    wall_b, _, _ = _serve(sph, ctx, sub)
    t0 = time.perf_counter()
    for bx, dt in sub:
        b = sph.box_from(ctx, bx)
        b.h_update()
        b.force()
        for _ in range(SERVE_STEPS):
            b.step(dt)
        b.get("rho")
        b.close()
    wall_1 = time.perf_counter() - t0
    pct = lambda a, q: float(np.percentile(np.asarray(a), q))
    return {
        "workload": f"{len(reqs)} jittered-lattice boxes, 1k-262k particles (mean {mean_n:.0f}), "
                    f"{SERVE_STEPS} kick-drift-kick steps each, Poisson arrivals at {SERVE_LOAD:.0%} of capacity",
        "tick_budget_particles": SERVE_TICK_BUDGET,
        "p50_step_ms": pct(step_ms, 50), "p99_step_ms": pct(step_ms, 99),
        "p99_over_p50": pct(step_ms, 99) / pct(step_ms, 50),
        "p50_request_s": pct(lat, 50), "p99_request_s": pct(lat, 99),
        "p50_intake_ms": pct(intake, 50), "p99_intake_ms": pct(intake, 99),
        "without_tick_budget": {"p50_step_ms": pct(step_ms_nb, 50), "p99_step_ms": pct(step_ms_nb, 99),
                                "p50_request_s": pct(lat_nb, 50), "p99_request_s": pct(lat_nb, 99)},
        "throughput": work / wall, "unit": UNIT, "capacity": capacity, "arrival_rate_per_s": rate,
        "step_samples": len(step_ms),
        "batched_vs_single_box": {"boxes": len(sub), "batched": sub_work / wall_b, "single_box": sub_work / wall_1,
                                  "unit": UNIT},
    }


# ------------------------------------------------------------------ oracle arm
class _Grid:
    """Particles of a periodic box binned on a g^3 mesh, for ball queries."""

    def __init__(self, x, L, g=64):
        self.x, self.L, self.g = x, L, g
        c = np.minimum((x * (g / L)).astype(np.int64), g - 1)
        cid = (c[:, 0] * g + c[:, 1]) * g + c[:, 2]
        self.order = np.argsort(cid, kind="stable")
        self.start = np.searchsorted(cid[self.order], np.arange(g ** 3 + 1))

    def ball(self, centre, R):
        g, L = self.g, self.L
        lo = np.floor((centre - R) * (g / L)).astype(np.int64)
        hi = np.floor((centre + R) * (g / L)).astype(np.int64)
        axes = [np.unique(np.arange(lo[k], hi[k] + 1) % g) if hi[k] - lo[k] + 1 < g else np.arange(g)
                for k in range(3)]
        cells = ((axes[0][:, None, None] * g + axes[1][None, :, None]) * g + axes[2][None, None, :]).ravel()
        idx = np.concatenate([self.order[self.start[c]:self.start[c + 1]] for c in cells])
        d = self.x[idx] - centre
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(1))
        keep = r <= R
        return idx[keep], r[keep]


class OracleSampler:
    """Bounded samples of a workload for the FP64 oracle: the k particles nearest to
    a randomly drawn particle (so that clumps and background are drawn in
    proportion to their mass), and around them the sub-volume that holds their
    neighbours and their partners' neighbours (3 x the largest first-guess support
    radius near them)."""

    def __init__(self, box, k=SAMPLE_K, seed=1):
        from oracle import sph as orc
        self.box, self.k = box, min(k, box.n)
        self.grid = _Grid(box.x, box.L)
        self.H0 = orc.support_radius(box.h)
        self.rng = np.random.default_rng(seed)

    def draw(self):
        box, k = self.box, self.k
        centre = box.x[self.rng.integers(box.n)]
        R = 1e-3 * box.L
        while True:
            idx, r = self.grid.ball(centre, R)
            if len(idx) >= k or R > box.L:
                break
            R *= 1.6
        part = np.argpartition(r, k - 1)[:k]
        rk = float(r[part].max())
        cand, rc = self.grid.ball(centre, rk + float(self.H0.max()))
        hloc = float(self.H0[cand[rc <= rk + self.H0[cand]]].max())
        sub, _ = self.grid.ball(centre, min(rk + 3.0 * hloc, 0.5 * box.L))
        sub = np.sort(sub)
        return sub, np.searchsorted(sub, np.sort(idx[part]))


def oracle_sample_step(box, sub, t):
    """One oracle step on a sample: the h iteration (FP64, from the first guess)
    over the sub-volume, ghost, then the force pass and the conservation sums of
    the k sampled particles.  Results at the sub-volume's edge are not used."""
    from oracle import sph as orc
    xs = box.x[sub]
    m = box.m[sub].astype(np.float64)
    h, conv, _, dens = orc.h_iterate(xs, m, box.h[sub], box.L, True, method="kdtree")
    H = float(orc.GAMMA_K) * h
    g = orc.ghost(dens["rho"], dens["Sr_m"], box.u[sub])
    fo = orc.force(xs, box.v[sub], m, H, dens["rho"], g["P"], g["c"], g["f"], box.L, True, targets=t,
                   method="kdtree")
    return orc.reductions(m[t], box.v[sub][t], box.u[sub][t], fo["a"], fo["dudt"])


def cpu_baseline(box, workload, budget_s=20.0):
    sampler = OracleSampler(box)
    t_total, cpu_total, reps = 0.0, 0.0, 0
    while t_total < budget_s and reps < 20:
        sub, t = sampler.draw()
        t0, c0 = time.perf_counter(), time.process_time()
        oracle_sample_step(box, sub, t)
        t_total += time.perf_counter() - t0
        cpu_total += time.process_time() - c0
        reps += 1
    return {"value": sampler.k * reps / t_total, "unit": UNIT, "cores": host_threads(),
            "cores_busy": round(cpu_total / t_total, 2), "kind": "oracle",
            "sample": f"{reps} oracle sample steps on the {workload} box: each the {sampler.k} particles nearest a "
                      f"randomly drawn particle, h iterated over the sub-volume around them (FP64), then their force "
                      f"pass and conservation sums; k-d tree searches on all host threads, numpy arithmetic mostly "
                      f"single-threaded; time per sampled particle"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    workload = getattr(args, "workload", DEFAULT_WORKLOAD)
    steps, warmup = getattr(args, "steps", 20), getattr(args, "warmup", 5)
    make, recipe = {**WORKLOADS, **PROFILE_WORKLOADS}[workload]
    box = make(replica_seed(0))
    sampler = OracleSampler(box)
    draws = [sampler.draw() for _ in range(warmup + steps)]
    for sub, t in draws[:warmup]:
        oracle_sample_step(box, sub, t)
    times, cpu = [], 0.0
    for sub, t in draws[warmup:]:
        t0, c0 = time.perf_counter(), time.process_time()
        oracle_sample_step(box, sub, t)
        times.append(time.perf_counter() - t0)
        cpu += time.process_time() - c0
    total = sum(times)
    value = sampler.k * steps / total
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * total / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "recipe": recipe, "particles_per_step": sampler.k,
                   "sample": f"each step the {sampler.k} particles nearest a randomly drawn particle of the box, h "
                             f"iterated over their sub-volume, their force pass and sums"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_threads(),
                         "cores_busy": round(cpu / total, 2) if total > 0 else None, "kind": "oracle",
                         "sample": f"{sampler.k} sampled particles of the {workload} box per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted({**WORKLOADS, **PROFILE_WORKLOADS}), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the timed oracle sample")
    ap.add_argument("--no-tune", action="store_true", help="keep the paper's leaf_max = 400")
    ap.add_argument("--leaf-max", dest="leaf_max_set", type=int, default=None,
                    help="use this split threshold instead of autotuning it (clusters of 32)")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-batch latency run")
    ap.add_argument("--no-extra-workloads", action="store_true", help="skip the other single-box workloads")
    ap.add_argument("--no-precision", action="store_true", help="skip the plain-FP32 position comparison")
    ap.add_argument("--host-steps", action="store_true",
                    help="launch every kernel of a step from the host instead of one captured graph "
                         "(the same kernels; for counter captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
