#!/usr/bin/env python
"""Throughput of the SPH density + force step on GB300 (one JSON line).

Workload: the variable-h single box -- 262,144 particles, 50 % uniform
background plus 16 Plummer spheres (scale radius 0.02, seeded centres),
periodic unit box, equal masses, u = 1, v ~ N(0, 0.1), h iterated to 48
neighbours.  The run follows the paper's protocol (fixed time step, forces on
every particle every step): one step is a half kick, a drift, the whole
decomposition build (keys, sort, cell tree, interaction lists, particle offsets,
axis sorts), density with the h iteration (started from the last two steps'
roots of N~(h) = 48, extrapolated), ghost,
force, FP64 conservation reductions and the closing half kick.  dt is the
Courant step of the initial state (C_CFL = 0.3).

value : particle-updates/s of a run resident in device memory.
e2e   : the same through the C-ABI with host buffers: every step uploads the full
        state (x, v, m, u, h, a, du/dt) from pinned host memory and reads the new
        state back (x, v, u, h, a, du/dt, one multi-field read) inside the timed
        region.

amortised: the same run with the decomposition kept over steps while it stays
        valid (sph_params.reuse, Section II-C: sorted indices re-used until the
        decomposition must be rebuilt); builds and reuses over the timed steps.

serving: the served batch -- 512 independent jittered-lattice boxes with
        particle counts log-uniform in [1k, 262k] (per-box seeds), each request
        advancing 10 kick-drift-kick steps -- through the continuous-batching
        server.  A saturated run (every request submitted at once) measures the
        capacity; a run with Poisson arrivals at 80 % of that capacity gives the
        p50/p99 step latency (CUDA events around every batched step, one sample
        per box and step), the request latency and the aggregate throughput.  The
        same requests on a 1-in-8 subset also run one box at a time through the
        plain single-box path for comparison with the batched server.

``--impl reference`` times the FP64 oracle (the only reference this method has:
the paper publishes no code) on the host cores, on a bounded sample of the same
workload per step.  Under torchrun (N > 1) every rank runs an independent replica
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
WORKLOAD = "plummer-262144"
SAMPLE_N = 16384            # the oracle's bounded sample: the same recipe at 1/16 of the particles

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

    box = inputs.plummer_box(seed=replica_seed(rank))
    n = box.n
    ctx = sph.sph_ctx_create(device=local_rank)
    stream = torch.cuda.Stream()
    sph.sph_ctx_set_stream(ctx, stream.cuda_stream)
    b = sph.Box(ctx, n, box.L, True)

    # resident input state: h converged once (a simulation's previous step), dt from CFL
    b.set(box.x, box.v, box.m, box.u, box.h)
    b.h_update()
    leaf_max = 400
    if not args.no_tune:
        leaf_max = b.tune()                           # split threshold for this workload (untimed)
        b.h_update()
    args.leaf_max = leaf_max
    args.cluster_max = b.stats()["cluster_max"]        # particles per cluster (tuned with it)
    b.force()
    dt = b.cfl_dt()
    torch.cuda.synchronize()

    def step_device():
        return b.step(dt)

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()

    # algorithmic work of one step (the same for every step): exact pair counts
    # over the step's density passes and its force pass (untimed, after the warm-up
    # so that the h iteration starts as in the timed steps)
    b.count_pairs(True)
    b.profile(True)
    step_device()
    st = b.stats()
    b.profile(False)
    b.count_pairs(False)
    # per step; the timed steps run the same passes (their number can differ by one
    # pass of the few particles the h extrapolation leaves), so a launch's share is
    # the step's flops over the timed launches per step
    flops_step = {"density": FLOPS_DENSITY_PAIR * st["density_pairs"] + FLOPS_DENSITY_SIDE * st["density_sides"],
                  "force": FLOPS_FORCE_PAIR * st["force_pairs"]}

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local_rank}")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = sph.sph_launch_count()
    b.profile(True)
    statuses = []
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.profiler.start()                 # ncu --profile-from-start off captures from here
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()                       # L2 flush between steps (outside the events)
                evs[k][0].record(stream)
            statuses.append(step_device())
            with torch.cuda.stream(stream):
                evs[k][1].record(stream)
        barrier()
        torch.cuda.profiler.stop()
    launches = sph.sph_launch_count() - l0
    st_last = b.stats()
    prof = b.get_profile()
    b.profile(False)
    ms = [s.elapsed_time(e) for s, e in evs]
    total_ms = max_over_ranks(dist, sum(ms), f"cuda:{local_rank}")
    value = job_rate(world, n * args.steps, total_ms / 1e3)

    # e2e through the C-ABI: the state lives in pinned host buffers between steps
    pinned = lambda shape, dt_: torch.empty(shape, dtype=dt_).pin_memory().numpy()
    xh, vh, ah = pinned((n, 3), torch.float64), pinned((n, 3), torch.float32), pinned((n, 3), torch.float32)
    mh, uh, hh, duh = (pinned(n, torch.float32) for _ in range(4))
    for name, buf in (("x", xh), ("v", vh), ("a", ah), ("u", uh), ("h", hh), ("dudt", duh)):
        b.get(name, out=buf)
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

    # roofline of the dominant kernel (FP32 ALU bound); the FMA throughput measured beside it
    fp32_measured = sph.sph_measure_fp32_peak(ctx)
    dom = max(("density", "force"), key=lambda k: prof[k]["ms"])
    calls = max(prof[dom]["calls"], 1)
    avg_ms = prof[dom]["ms"] / calls
    flops = flops_step[dom] * args.steps / calls
    achieved = flops / (avg_ms / 1e3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            traffic = json.load(open(tpath)).get(dom)
        except (OSError, ValueError):
            traffic = None

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles_per_gpu": n, "h": "iterated to N~ = 48 each step, from the last four steps' roots extrapolated (cubic)",
                   "protocol": "fixed-step kick-drift-kick run, forces on all particles every step",
                   "dt": dt, "leaf_max": leaf_max, "cluster_max": args.cluster_max,
                   "leaf_max_source": "autotuned" if not args.no_tune else "paper", "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": n * (24 + 12 + 4 + 4 + 4 + 12 + 4),
                "d2h_bytes_per_step": n * (24 + 12 + 4 + 4 + 12 + 4), "steps": e2e_steps},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "flops_per_launch": flops, "avg_launch_ms": avg_ms,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.070 GHz (nominal max clock)",
                     "peak_measured": fp32_measured,
                     "peak_measured_source": "independent FMA chains on every SM (sph_measure_fp32_peak), this run"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "phases_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in prof.items() if v["calls"]},
        "pairs": {"density": st["density_pairs"], "density_candidates": st["density_candidates"],
                  "force": st["force_pairs"], "force_candidates": st["force_candidates"],
                  "guard_rechecks": st["guard_rechecks"]},
        "h_iterations_last_step": st_last["h_iterations"],
        "h_unconverged_after_first_pass": st_last["h_active_after_first"] / box.n,
    }
    out["amortised"] = run_reuse_leg(sph, torch, b, box, dt, stream, args, flush)
    out["axis_sorts"] = run_sort_leg(sph, torch, b, box, stream, args)
    b.close()
    if not args.no_serving:
        out["serving"] = run_serving(sph, ctx)
    sph.sph_ctx_destroy(ctx)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(box)
    if dist is not None:
        dist.destroy_process_group()
    return out


# ------------------------------------------------------------------ reuse
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
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                evs[k][0].record(stream)
            br.step(dt)
            with torch.cuda.stream(stream):
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        s1 = br.stats()
        ms = sum(s_.elapsed_time(e_) for s_, e_ in evs)
        return {"value": box.n * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
                "builds": s1["builds"] - s0["builds"], "reuses": s1["reuses"] - s0["reuses"]}
    finally:
        br.close()
        sph.sph_ctx_destroy(ctx)


# ------------------------------------------------------------------ serving
SERVE_STEPS = 10
SERVE_LOAD = 0.8


def _served_requests(n_boxes):
    """(box, dt) per request: C_CFL x min H / (2 c) at the initial state (u = 1)."""
    out = []
    for bx in inputs.served_boxes(n_boxes):
        c = np.sqrt(5.0 / 3.0 * (5.0 / 3.0 - 1.0) * float(bx.u.max()))
        out.append((bx, 0.3 * 1.825742 * float(bx.h.min()) / (2.0 * c)))
    return out


def _serve(sph, ctx, reqs, arrivals=None):
    """Run requests through one server; returns (wall s, step ms list, request latencies s)."""
    srv = sph.sph_server_create(ctx, 0, 0)
    try:
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
        step_ms = []
        for r, rid in ids.items():
            step_ms.extend(sph.sph_server_poll(srv, rid, SERVE_STEPS)[1].tolist())
            sph.sph_server_release(srv, rid)
        lat = [done_t[r] - t_sub[r] for r in ids]
        return wall, step_ms, lat
    finally:
        sph.sph_server_destroy(srv)


def run_serving(sph, ctx, n_boxes=512):
    reqs = _served_requests(n_boxes)
    work = sum(bx.n for bx, _ in reqs) * SERVE_STEPS
    mean_n = work / SERVE_STEPS / len(reqs)
    wall_sat, _, _ = _serve(sph, ctx, reqs)                 # saturated: every request at once
    capacity = work / wall_sat
    rate = SERVE_LOAD * capacity / (mean_n * SERVE_STEPS)  # requests per second
    arrivals = inputs.poisson_arrivals(len(reqs), rate, seed=1)
    wall, step_ms, lat = _serve(sph, ctx, reqs, arrivals)
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
        "p50_step_ms": pct(step_ms, 50), "p99_step_ms": pct(step_ms, 99),
        "p50_request_s": pct(lat, 50), "p99_request_s": pct(lat, 99),
        "throughput": work / wall, "unit": UNIT, "capacity": capacity, "arrival_rate_per_s": rate,
        "step_samples": len(step_ms),
        "batched_vs_single_box": {"boxes": len(sub), "batched": sub_work / wall_b, "single_box": sub_work / wall_1,
                                  "unit": UNIT},
    }


# ------------------------------------------------------------------ oracle arm
def _oracle_sample_box():
    """The workload's recipe at 1/16 of the particles, with h converged by the oracle."""
    from oracle import sph as orc
    box = inputs.plummer_box(n=SAMPLE_N, seed=1)
    h, conv, _, _ = orc.h_iterate(box.x, box.m, box.h, box.L, True, method="kdtree")
    box.h = h.astype(np.float32)
    return box


def _oracle_step(box):
    from oracle import sph as orc
    return orc.full_step(box, iterate_h=True, method="kdtree")


def cpu_baseline(_box=None):
    sample = _oracle_sample_box()
    t0 = time.perf_counter()
    reps = 0
    while True:
        _oracle_step(sample)
        reps += 1
        if time.perf_counter() - t0 > 10.0 or reps >= 20:
            break
    dt = time.perf_counter() - t0
    return {"value": sample.n * reps / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} oracle steps (h iteration from converged h, force, reductions; FP64) on the "
                      f"same Plummer recipe at {sample.n} particles; k-d tree search on all cores, numpy "
                      f"arithmetic on one"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    sample = _oracle_sample_box()
    for _ in range(args.warmup):
        _oracle_step(sample)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _oracle_step(sample)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample.n * args.steps / total
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles_per_step": sample.n,
                   "sample": "same recipe at 1/16 of the particles"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{sample.n}-particle Plummer box per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the timed oracle sample")
    ap.add_argument("--no-tune", action="store_true", help="keep the paper's leaf_max = 400")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-batch latency run")
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
