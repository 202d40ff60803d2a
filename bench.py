#!/usr/bin/env python
"""Throughput and accuracy of the pore / water-vapour MD hot path on one GB300.

Default workload (the configuration the metric's mixed-vs-FP64 comparison is defined on): one
cylindrical pore of radius 10 sigma through a simple-cubic wall slab |z| < 30 (1,331,040 fixed wall
atoms) in a 150 x 150 x 300 sigma box, 200,000 vapour molecules outside the slab, reduced LJ
units, rc = 2.5, dt = 0.005, T* = 0.9 with velocity rescaling every 10 steps; the Verlet skin,
which the configuration leaves open, is chosen by the autotuner. One bench step = one MD step
(half-kick/drift/reflect, device-decided list rebuild, pair forces, half-kick, thermostat).

value: pair interactions per second of the FP64 form -- unique vapour-vapour plus vapour-wall
pairs with r < rc, counted exactly by the force kernel over the timed steps -- divided by the
summed CUDA-event durations of the steps (L2 flushed between steps, outside the timed events, by a
256 MB write and then a 256 MB read, which leaves no dirty line of the flush to be written back
inside the next step).

Also reported: MD steps/s; the mixed-precision form (FP32 pair terms) and the double-float form
with their speed-up over FP64 and their RMS force error against the FP64 oracle; the first ten
steps from the initial state without thermostat (RMS force error of each form at its own
positions after every step, total energy against the oracle's own trajectory); the NVE energy
drift of the FP64 and mixed forms; the pair kernel's roofline (timed live with CUDA events); the
rebuild chain timed alone; the FP64 CPU oracle timed on the host cores (cpu_baseline); and an
end-to-end figure through the C ABI with host buffers (state upload, one step, force read-back).

--impl reference times the FP64 CPU oracle on the same workload (one system advanced per step, in
turn) and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s & MD steps/s; mixed-FP32 vs FP64 at RMS force err ≤1e-5"
UNIT = "pair-interactions/s"
WORKLOAD = ("pore_shapes_4x20k: four 40x40x80 boxes (cylinder r5, cone r3->8, slit w6, "
            "ink-bottle neck 3 / cavity 8) through an SC wall slab |z|<10, 20,000 vapour each, "
            "rc 2.5, skin 0.3, dt 0.005, T*=1.0, rescale every 10 steps")
# FP64 operations per pair interaction counted as algorithmic work (FMA = 2): dx, dy, dz (3);
# r^2 (1 mul + 2 fma = 5); 1/r^2 (1); inv^6 (2 mul); force factor (fma + 2 mul = 4);
# accumulate (3 fma = 6)
FLOPS_PER_PAIR = 21
# peak of the FP64 CUDA-core pipe: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per launch of a pair kernel on a workload, from one ncu capture
# (the command is in profiles/), valid for the kernel source whose SHA-256 prefix is recorded:
# traffic is reported as null for any other workload, kernel or source
NCU_TRAFFIC = {
    ("cylinder_pore_200k", "k_forces_flat<0>"):
        {"bytes_per_launch": 23693056, "source_sha": "57dfe9f1543d79eb",
         "source": "profiles/flat_stream_fp64_cylinder_pore_200k.md"},
    ("pore_shapes_4x20k", "k_forces_flat<0>"):
        {"bytes_per_launch": 14651904, "source_sha": "57dfe9f1543d79eb",
         "source": "profiles/flat_stream_fp64_pore_shapes_4x20k.md"},
}

# The rebuild chain's dominant kernel -- the list build the device chose on that workload -- from
# one ncu capture (--set full) inside the bench's rebuild range: DRAM bytes per launch, its
# duration there and its DRAM throughput as a fraction of the peak. Keyed by (workload, precision,
# accumulation), valid for the recorded kernel source.
NCU_LIST_BUILD = {
    ("cylinder_pore_200k", "fp64", "atomic"):
        {"kernel": "k_list_build_mol", "dram_bytes_per_launch": 12547328, "duration_us": 83.0,
         "dram_frac_of_peak": 0.0191, "source_sha": "57dfe9f1543d79eb",
         "source": "profiles/list_builds_cylinder_pore_200k_and_pore_shapes_4x20k.md"},
    ("pore_shapes_4x20k", "fp64", "atomic"):
        {"kernel": "k_list_build", "dram_bytes_per_launch": 2978816, "duration_us": 50.4,
         "dram_frac_of_peak": 0.0075, "source_sha": "57dfe9f1543d79eb",
         "source": "profiles/list_builds_cylinder_pore_200k_and_pore_shapes_4x20k.md"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "df64"], default="fp64",
                    help="fp64; mixed (FP32 pair terms); df64 (an FP64 context whose pair terms "
                         "run in double-float on the FP32 pipe)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the comparison runs of the mixed and double-float forms")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--roofline-launches", type=int, default=50)
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cylinder_pore_200k")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--force-tpp", type=int, default=0,
                    help="pin the pair kernel's lanes per molecule (32: the packed FP64 kernels) "
                         "instead of the autotuner's choice")
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="with --force-tpp, the pair kernel's resident blocks per SM")
    ap.add_argument("--nve-steps", type=int, default=2000,
                    help="with the mixed comparison, also the NVE energy drift of both GPU forms "
                         "over this many steps (after 200 thermostatted ones); 0: skip")
    ap.add_argument("--first-steps", type=int, default=10,
                    help="with the mixed comparison, the accuracy of every form over this many "
                         "steps from the initial state without thermostat, against the oracle; "
                         "0: skip")
    ap.add_argument("--launch-mode", choices=["graph", "plain"], default="graph",
                    help="timed steps as CUDA-graph replays (default) or plain launches (for ncu "
                         "launch lists)")
    ap.add_argument("--skin", default="",
                    help="Verlet-list skin: a number, or 'auto' for the autotuner's choice of "
                         "skin and cell side (autotune.choose_geometry); default: auto for the "
                         "workloads whose "
                         "definition does not fix the skin (200k cylinder, 256-replica batch, "
                         "2M pore array), else 0.3")
    ap.add_argument("--pair-method", choices=["auto", "lists", "cells", "small"], default="auto",
                    help="the pair kernel: auto (the autotuner picks between the Verlet-list walk "
                         "and the cell-tiled kernel, atomic form, and for FP64 contexts of at most "
                         "16384 molecules the small-system method, by whole steps), lists, cells, "
                         "or small (whole steps in one persistent launch)")
    ap.add_argument("--accumulate", choices=["atomic", "deterministic"], default="atomic",
                    help="reaction forces by FP64 atomic adds (half list, both precisions), or "
                         "the bit-reproducible forms (FP64 slot-and-gather, mixed full list)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


WORKLOADS = {
    "pore_shapes_4x20k": WORKLOAD,
    "cylinder_pore_1k": "20x20x40 box, slab |z|<5, cylinder r4, 1,000 vapour, T*=1.0",
    "cylinder_pore_200k": "150x150x300 box, slab |z|<30, cylinder r10, 200,000 vapour, T*=0.9",
    "replica_batch_256": ("256 replicas: shape uniform over cylinder/cone/slit/ink-bottle, R~U[2,10], "
                          "N log-uniform [1k,50k], T*~U[0.8,1.2], density 0.02 outside |z|<8"),
    "replica_batch_32": ("32 replicas drawn as the 256-replica batch's are (461,031 vapour, "
                         "2,392,655 wall atoms): a smaller case for kernel captures"),
    "pore_array_2m": ("400x400x200 box, 4x4 pores (cylinder/cone/ink-bottle, R~U[4,10]) in slab "
                      "|z|<20, 2,000,000 vapour, T*=0.85"),
    "paper_prism_pore": ("the paper's 3D geometry in reduced units: a 5x5x50 prism pore closed on "
                         "five faces by hard reflecting walls, open into a space 9 times its "
                         "volume, 250 molecules inside and 450 outside, T*=1.0"),
    "paper_pore_2d": ("the paper's 2D geometry in reduced units: a planar 20x20 pore with "
                      "reflecting walls on three sides, outer space k=3 (21 times the pore), 84 "
                      "molecules inside and 352 outside, T*=1.0"),
    "drying_pore_6k": ("drying of a filled pore: 40x40x80 box, slab |z|<10, cylinder r8 holding "
                       "1,000 molecules, 4,800 outside at a fifth of that density, T*=1.0, "
                       "Berendsen tau_B=0.5"),
}

# workloads whose definition leaves the Verlet skin open (the 4x20k pore shapes fix it at 0.3):
# the bench lets the autotuner pick it
SKIN_BY_AUTOTUNER = ("cylinder_pore_200k", "replica_batch_256", "pore_array_2m")


def bench_skin(skin_arg: str, rank: int, world: int, choose):
    """The Verlet skin of this run and the record of its choice: a number as given (no record), or
    with "auto" the choice ``choose()`` makes on rank 0, broadcast to every rank so that all
    replicas run with one skin; 0.3 where no candidate worked."""
    if skin_arg != "auto":
        return float(skin_arg), None
    choice = choose() if rank == 0 else None
    if world > 1:
        import torch.distributed as dist
        box = [choice]
        dist.broadcast_object_list(box, src=0)
        choice = box[0]
    skin = choice["skin"] if choice and choice.get("skin") is not None else 0.3
    return skin, choice


def make_workload(name: str):
    from paper_1812_07993_gb300 import workloads as W
    if name == "cylinder_pore_1k":
        return [W.cylinder_pore_1k()], name
    if name == "cylinder_pore_200k":
        return [W.cylinder_pore_200k()], name
    if name == "replica_batch_256":
        return W.replica_batch(256), name
    if name == "replica_batch_32":
        return W.replica_batch(32), name
    if name == "pore_array_2m":
        return [W.pore_array_2m()], name
    if name == "drying_pore_6k":
        return [W.drying_cylinder_pore()], name
    if name == "paper_prism_pore":
        return [W.paper_prism_pore()], name
    if name == "paper_pore_2d":
        return [W.paper_pore_2d()], name
    return W.pore_shape_systems_20k(), "pore_shapes_4x20k"


def kernel_sha() -> str:
    p = os.path.join(ROOT, "paper_1812_07993_gb300", "csrc", "md_kernels.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


# ------------------------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ------------------------------------------------------------------------------------ oracle leg


def oracle_rate(systems, seconds: float, nthreads: int = 0):
    """Advance the systems with the FP64 CPU oracle, one MD step of one system at a time in turn,
    until ``seconds`` have passed; returns (pairs/s, steps, pairs, elapsed, threads)."""
    import oracle
    from paper_1812_07993_gb300 import workloads as W
    pot = W.Potential()
    states = [oracle.State(oracle.make_params(s, pot), s.x0, s.v0, s.wall, method=1,
                           nthreads=nthreads, pores=s.pores) for s in systems]
    steps = pairs = 0
    t0 = time.perf_counter()
    while True:
        st = states[steps % len(states)]
        st.run(1)
        pairs += st.stats["pairs_vv"] + st.stats["pairs_vw"]
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    threads = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    return pairs / el, steps, pairs, el, threads


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1812_07993_gb300 import workloads as W
    systems, wname = make_workload(args.workload)
    pot = W.Potential()
    states = [oracle.State(oracle.make_params(s, pot), s.x0, s.v0, s.wall, method=1, nthreads=0,
                           pores=s.pores) for s in systems]
    for k in range(args.warmup):
        states[k % len(states)].run(1)
    pairs = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        st = states[k % len(states)]
        st.run(1)
        pairs += st.stats["pairs_vv"] + st.stats["pairs_vw"]
    el = time.perf_counter() - t0
    value = pairs / el
    cores = os.cpu_count() or 1
    sample = (f"{args.steps} oracle MD steps, one of the {len(systems)} systems per step in turn "
              f"(FP64 cell-list oracle, OpenMP over molecules)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "description": WORKLOADS[wname],
                       "replicas": len(systems)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------ GPU leg


def nvtx_push(torch, name):
    """Mark a region for ncu's --nvtx-include filter (a no-op where NVTX is unavailable)."""
    try:
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop(torch):
    try:
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def pair_total(sim, nrep):
    return sim.observables(0)[0]["pair_evals_total"]


def current_pairs(sim, nrep):
    tot = 0
    for r in range(nrep):
        o = sim.observables(r)[0]
        tot += o["pairs_vv"] + o["pairs_vw"]
    return tot


class L2Flush:
    """Empties the L2 cache (129 MB) between timed regions, outside the timing events, on the
    current stream: a 256 MB write evicts every line the timed work could reuse, and a 256 MB read
    after it evicts the write's own dirty lines, so the next timed region neither finds its data in
    L2 nor pays for writing the flush buffer back to memory."""

    def __init__(self, torch):
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        self.r = torch.ones(32 << 20, dtype=torch.int64, device="cuda")
        self.out = torch.empty((), dtype=torch.int64, device="cuda")
        self.torch = torch

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r, dim=0, out=self.out)


def time_steps(sim, torch, stream, flush, steps):
    evs = []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(1)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def rank_barrier(world: int):
    """All ranks meet here (N > 1: a gloo barrier)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_totals(ms: float, pairs: float, world: int):
    """Whole-job figures over the ranks: the slowest rank's timed milliseconds and the pair
    interactions of every rank (each rank runs its own copy of the workload: replicas only)."""
    if world <= 1:
        return ms, float(pairs)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(pairs)], dtype=torch.float64)
    m = torch.tensor([float(ms)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(m[0]), float(t[0])


def prec_enum(md, name):
    return {"fp64": md.MD_PREC_FP64, "mixed": md.MD_PREC_MIXED, "df64": md.MD_PREC_DF64}[name]


def measure_precision(md, systems, precision, args, torch, stream, flush, world=1, potential=None):
    from paper_1812_07993_gb300 import autotune
    sim = md.Simulation(systems, potential, precision=precision, stream=stream)
    sim.method_choice = None
    sim.set_tuning(force_accumulate=2 if args.accumulate == "atomic" else 1)
    method = {"lists": 1, "cells": 3, "small": 4}.get(args.pair_method, 0)
    if (args.pair_method == "auto" and precision == md.MD_PREC_FP64 and
            sum(s.n_vapor for s in systems) <= autotune.SMALL_MAX):
        sim.method_choice = autotune.choose_step_method(systems, potential, precision,
                                                        stream=stream)
        method = 4 if sim.method_choice["pair_method"] == 4 else 0
    if method:                         # the autotuner then times that method's shapes only
        sim.set_tuning(pair_method=method)
    sim.tune_info = None
    main = precision == prec_enum(md, args.precision)
    if args.force_tpp and main:   # the pin is the headline run's; the comparison run is tuned
        sim.set_tuning(force_tpp=args.force_tpp, force_blocks_per_sm=args.blocks_per_sm)
        sim.tune_info = {"tuning": sim.tuning(), "pinned": True}
    elif not args.no_autotune:
        sim.tune_info = autotune.tune(sim, trials=9, use_cache=False)
    sim.set_tuning(use_graph=1 if args.launch_mode == "graph" else 2, steps_per_graph=1)
    for _ in range(args.warmup):
        flush()
        sim.step(1)
    sim.sync()
    p0 = pair_total(sim, len(systems))
    l0 = sim.kernel_launches()
    torch.cuda.synchronize()
    rank_barrier(world)            # the timed region starts on every rank together
    nvtx_push(torch, "timed_steps")
    ms = time_steps(sim, torch, stream, flush, args.steps)   # ends with a device synchronize
    nvtx_pop(torch)
    rank_barrier(world)
    launches = sim.kernel_launches() - l0
    p1 = pair_total(sim, len(systems))
    return sim, ms, p1 - p0, launches


def steady_state(sim, torch, stream, flush, steps, nrep, per_replay=10):
    """The same steps run back to back as CUDA-graph replays of ``per_replay`` steps each (how a
    long run executes), with the L2 flush between replays, not between steps."""
    sim.set_tuning(use_graph=1, steps_per_graph=per_replay)
    sim.step(per_replay)
    sim.sync()
    p0 = pair_total(sim, nrep)
    reps = max(1, steps // per_replay)
    evs = []
    for _ in range(reps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(per_replay)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    pairs = pair_total(sim, nrep) - p0
    sim.set_tuning(steps_per_graph=1)
    return {"value": pairs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / (reps * per_replay),
            "steps": reps * per_replay, "steps_per_replay": per_replay,
            "l2": "flushed between graph replays"}


def pair_kernel_name(sim, precision, accumulate):
    """The kernel md_pair_pass launches under the context's current tuning (with its lanes per
    molecule as the template argument, as ncu names it)."""
    tpp = sim.tuning()["force_tpp"]
    atomic = accumulate == "atomic"
    if sim.tuning()["pair_method"] == 4:
        return "k_small_steps"
    if sim.tuning()["pair_method"] == 3:
        return "k_forces_cells<%d, 0>" % {"fp64": 0, "mixed": 1, "df64": 2}[precision]
    if tpp == 64:  # the flat stream (atomic form)
        return "k_forces_flat<%d>" % {"fp64": 0, "mixed": 1, "df64": 2}[precision]
    if precision == "df64":
        return f"k_forces_df_atomic<{tpp}>" if atomic else f"k_forces_df<0, {tpp}>"
    if precision == "fp64":
        if sim.tuning()["pair_method"] == 2:
            return "k_allpairs<0, 0>"
        if tpp == 32:
            return "k_forces_atomic_packed" if atomic else "k_forces_half_packed"
        return f"k_forces_half_atomic<{tpp}>" if atomic else f"k_forces_half<{tpp}>"
    return f"k_forces_mixed_atomic<{tpp}>" if atomic else f"k_forces_mixed<0, 0, {tpp}>"


def roofline(sim, torch, stream, flush, nlaunch, pairs_per_launch, precision, accumulate,
             workload):
    evs = []
    nvtx_push(torch, "roofline")
    for _ in range(nlaunch):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.pair_pass()          # the pair kernel alone
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    nvtx_pop(torch)
    sim.compute_forces()         # complete forces again
    sim.sync()
    ms = sum(a.elapsed_time(b) for a, b in evs) / nlaunch
    flops = pairs_per_launch * FLOPS_PER_PAIR
    achieved = flops / (ms * 1e-3) / 1e12
    peak = FP64_PEAK_TFLOPS if precision == "fp64" else FP32_PEAK_TFLOPS
    kname = pair_kernel_name(sim, precision, accumulate)
    tr = NCU_TRAFFIC.get((workload, kname))
    traffic = tr["bytes_per_launch"] if tr and tr.get("source_sha") == kernel_sha() else None
    return {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "peak_source": ("derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz" if precision ==
                            "fp64" else "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"),
            "launch_ms": ms, "pairs_per_launch": pairs_per_launch,
            "flops_per_pair": FLOPS_PER_PAIR}


def list_build(sim, torch, stream, flush, nlaunch, precision, accumulate, workload):
    """The rebuild chain alone (md_rebuild_lists: cell sort, Verlet lists, processing order or
    flat stream, for every replica), timed with CUDA events on the library's stream, L2 flushed
    before each; beside it the ncu figures of the list build the device chose, the chain's
    dominant kernel. Both list builds are bound by instruction issue, not by HBM: their DRAM
    traffic is a small fraction of the peak."""
    evs = []
    nvtx_push(torch, "rebuild")
    for _ in range(nlaunch):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.rebuild_lists()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    nvtx_pop(torch)
    sim.sync()
    ms = sum(a.elapsed_time(b) for a, b in evs) / nlaunch
    cells = sim.tuning()["pair_method"] == 3
    nc = NCU_LIST_BUILD.get((workload, precision, accumulate))
    if cells or (nc and nc.get("source_sha") != kernel_sha()):
        nc = None
    kernel = ("k_cell_count" if cells else
              nc["kernel"] if nc else "k_list_build or k_list_build_mol (the device's choice)")
    return {"kernel": kernel, "bound": "issue",
            "rebuild_chain_ms": ms, "chains_timed": nlaunch,
            "chain": ("cell clear, count, scan, scatter, permute (all replicas; the cell method "
                      "builds no lists)" if cells else
                      "cell clear, count, scan, scatter, permute, list build, then the processing "
                      "order or the flat stream (all replicas)"),
            "ncu": ({"dram_bytes_per_launch": nc["dram_bytes_per_launch"],
                     "duration_us": nc["duration_us"],
                     "dram_frac_of_peak": nc["dram_frac_of_peak"],
                     "source": nc["source"]}
                    if nc else None)}


def nve_drift(md, systems, precision, stream, accumulate, equil=200, steps=2000, every=50):
    """Energy drift without the thermostat: equilibrate with it, then run ``steps`` NVE steps and
    fit a line to the total energy per molecule against time (|slope|, in eps per molecule per
    tau); also the RMS of the residuals (the fluctuation)."""
    import dataclasses
    import numpy as np
    with md.Simulation(systems, precision=precision, stream=stream) as sim:
        sim.step(equil)
        states = [sim.state(r) for r in range(len(systems))]
    nve = [dataclasses.replace(s, x0=x, v0=v, thermostat_every=0)
           for s, (x, v) in zip(systems, states)]
    n = sum(s.n_vapor for s in systems)
    t, e = [], []
    with md.Simulation(nve, precision=precision, stream=stream) as sim:
        sim.set_tuning(force_accumulate=2 if accumulate == "atomic" else 1)
        for k in range(steps // every):
            sim.step(every)
            tot = 0.0
            for r in range(len(nve)):
                o = sim.observables(r)[0]
                tot += o["ke"] + o["pe"]
            t.append((k + 1) * every * nve[0].dt)
            e.append(tot / n)
    t, e = np.array(t), np.array(e)
    fit = np.polyfit(t, e, 1)
    return {"drift": abs(float(fit[0])), "fluctuation": float(np.std(e - np.polyval(fit, t))),
            "unit": "eps per molecule per tau", "steps": steps}


def first_steps(md, systems, potential, stream, nsteps):
    """Accuracy over the first ``nsteps`` steps from the initial state with the thermostat off
    (NVE), per form: after every step, the RMS force error sqrt(sum |F - F_oracle|^2 / sum
    |F_oracle|^2) against the FP64 oracle's forces at the form's own positions, and the total
    energy per molecule against the oracle's own NVE trajectory from the same state. Reported:
    the largest of each over the steps, beside the oracle's own energy change over them."""
    import numpy as np
    import oracle
    nve = [dataclasses.replace(s, thermostat_every=0) for s in systems]
    n = sum(s.n_vapor for s in nve)
    params = [oracle.make_params(s, potential) for s in nve]
    e_or = np.zeros(nsteps)
    e0 = 0.0
    for s, p in zip(nve, params):
        st = oracle.State(p, s.x0, s.v0, s.wall, method=1, nthreads=0, pores=s.pores)
        e0 += oracle.kinetic(p, s.v0) + st.stats["pe_vv"] + st.stats["pe_vw"]
        ke, pe = st.run(nsteps)
        e_or += ke + pe
    e_or /= n
    out = {"steps": nsteps, "thermostat": "off",
           "oracle_energy_change_per_molecule": float(e_or[-1] - e0 / n)}
    for name, prec in (("fp64", md.MD_PREC_FP64), ("mixed", md.MD_PREC_MIXED),
                       ("df64", md.MD_PREC_DF64)):
        errs, dev = [], []
        with md.Simulation(nve, potential, precision=prec, stream=stream) as sim:
            sim.set_tuning(force_accumulate=2)
            for k in range(nsteps):
                sim.step(1)
                num = den = etot = 0.0
                for r, (s, p) in enumerate(zip(nve, params)):
                    x, _ = sim.state(r)
                    g, _, _ = oracle.forces(p, x, s.wall, method=1, nthreads=0)
                    f = sim.forces(r)
                    num += float(((f - g) ** 2).sum())
                    den += float((g ** 2).sum())
                    o = sim.observables(r)[0]
                    etot += o["ke"] + o["pe"]
                errs.append(math.sqrt(num / den))
                dev.append(abs(etot / n - float(e_or[k])))
        out[name] = {"rms_force_err_max": max(errs), "rms_force_err_last": errs[-1],
                     "energy_dev_per_molecule_max": max(dev)}
    return out


def e2e(sim, systems, nsteps, pairs_per_step, torch):
    """Whole-job steps through the public API with host buffers: every step uploads the state of
    every replica from pinned host memory (md_set_state, replica -1: lists rebuilt where the skin
    test asks for it, forces evaluated), runs one MD step and reads every force back
    (md_get_forces, replica -1)."""
    n = sum(s.n_vapor for s in systems)
    bufs = [torch.empty((n, 3), dtype=torch.float64).pin_memory() for _ in range(3)]
    x, v, f = (b.numpy() for b in bufs)
    sim.state(-1, out=(x, v))
    sim.set_state(-1, x, v)
    sim.step(1)
    sim.forces(-1, out=f)                      # warm-up of the same path
    h0, d0 = sim.transfer_bytes()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        sim.set_state(-1, x, v)
        sim.step(1)
        sim.forces(-1, out=f)
    el = time.perf_counter() - t0
    h1, d1 = sim.transfer_bytes()
    return {"value": pairs_per_step * nsteps / el, "unit": UNIT,
            "h2d_bytes_per_step": (h1 - h0) // nsteps, "d2h_bytes_per_step": (d1 - d0) // nsteps,
            "ms_per_step": 1e3 * el / nsteps,
            "path": "md_set_state(-1) from pinned host arrays + md_step(1) + md_get_forces(-1)"}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1812_07993_gb300 as md
    from paper_1812_07993_gb300 import build as mdbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    mdbuild.build()
    md.load_library()
    systems, wname = make_workload(args.workload)
    nrep = len(systems)
    # one non-default stream carries the library's work, the L2 flush and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    flush = L2Flush(torch)
    prec = prec_enum(md, args.precision)
    from paper_1812_07993_gb300 import workloads as W
    skin_arg = args.skin or ("auto" if args.workload in SKIN_BY_AUTOTUNER else "0.3")

    def choose():
        # the autotuner times whole MD steps on fresh contexts for each candidate skin, then each
        # cell side at the fastest skin (every candidate gives the same forces and pair counts),
        # and keeps the fastest, cached per size class
        from paper_1812_07993_gb300 import autotune
        return dict(autotune.choose_geometry(systems, precision=prec, stream=stream),
                    by="autotune.choose_geometry")

    skin, skin_choice = bench_skin(skin_arg, rank, world, choose)
    pot = dataclasses.replace(W.Potential(), skin=skin,
                              cell_size=float((skin_choice or {}).get("cell_size") or 0.0))

    clocks = ClockSampler(local)
    clocks.start()
    sim, ms, pairs, launches = measure_precision(md, systems, prec, args, torch, stream, flush,
                                                 world, potential=pot)
    clocks.stop()
    ms_job, pairs_job = job_totals(ms, pairs, world)
    value = pairs_job / (ms_job * 1e-3)
    ms_per_step = ms_job / args.steps
    pairs_per_step = pairs / args.steps

    sim_tune = sim.tune_info
    extra = {}
    if rank == 0 and args.launch_mode == "graph":
        extra["steady_state"] = steady_state(sim, torch, stream, flush, args.steps,
                                             len(systems))
    if rank == 0:
        cur = current_pairs(sim, nrep)
        extra["roofline"] = roofline(sim, torch, stream, flush, args.roofline_launches, cur,
                                     args.precision, args.accumulate, args.workload)
        if sim.tuning()["pair_method"] not in (2, 4):
            extra["list_build"] = list_build(sim, torch, stream, flush,
                                             max(3, args.roofline_launches // 5), args.precision,
                                             args.accumulate, args.workload)
        extra["e2e"] = e2e(sim, systems, args.e2e_steps, pairs_per_step, torch)
        if not args.no_mixed and args.precision == "fp64":
            import oracle
            from paper_1812_07993_gb300 import workloads as W
            simm, msm, pairsm, _ = measure_precision(md, systems, md.MD_PREC_MIXED, args, torch,
                                                     stream, flush, potential=pot)
            # RMS force error of both GPU forms against the FP64 oracle at the mixed run's state
            errs = []
            with md.Simulation(systems, stream=stream) as sim64:
                for r, s in enumerate(systems):
                    x, v = simm.state(r)
                    sim64.set_state(r, x, v)
                    g, _, _ = oracle.forces(oracle.make_params(s, W.Potential()), x, s.wall,
                                            method=1, nthreads=0)
                    fm = simm.forces(r)
                    f64 = sim64.forces(r)
                    errs.append((((fm - g) ** 2).sum(), ((f64 - g) ** 2).sum(), (g ** 2).sum()))
            den = sum(e[2] for e in errs)
            vm = pairsm / (msm * 1e-3)
            if args.first_steps > 0:
                extra["first_steps"] = first_steps(md, systems, pot, stream, args.first_steps)
            if args.nve_steps > 0:
                extra["nve_drift"] = {
                    "fp64": nve_drift(md, systems, md.MD_PREC_FP64, stream, args.accumulate,
                                      steps=args.nve_steps),
                    "mixed": nve_drift(md, systems, md.MD_PREC_MIXED, stream, args.accumulate,
                                       steps=args.nve_steps)}
            extra["mixed"] = {"value": vm, "unit": UNIT, "ms_per_step": msm / args.steps,
                              "speedup_vs_fp64": vm / value,
                              "rms_force_err": math.sqrt(sum(e[0] for e in errs) / den),
                              "fp64_rms_force_err": math.sqrt(sum(e[1] for e in errs) / den),
                              "rms_force_err_at": "the mixed run's final state (after the timed "
                                                  "steps), both GPU forms at the same positions",
                              "md_steps_per_s": args.steps / (msm * 1e-3),
                              "tuning": (simm.tune_info or {}).get("tuning")}
            simm.close()
            # double-float pair terms: the same workload, steps and timing; force error against
            # the oracle and against the FP64 GPU form at the run's final state
            simd, msd, pairsd, _ = measure_precision(md, systems, md.MD_PREC_DF64, args, torch,
                                                     stream, flush, potential=pot)
            errs, max_vs64 = [], 0.0
            with md.Simulation(systems, stream=stream) as sim64:
                sim64.set_tuning(force_accumulate=2)
                for r, s in enumerate(systems):
                    x, v = simd.state(r)
                    sim64.set_state(r, x, v)
                    g, _, _ = oracle.forces(oracle.make_params(s, W.Potential()), x, s.wall,
                                            method=1, nthreads=0)
                    fd = simd.forces(r)
                    f64 = sim64.forces(r)
                    errs.append((((fd - g) ** 2).sum(), (g ** 2).sum()))
                    rms = math.sqrt(float((f64 ** 2).sum(1).mean()))
                    max_vs64 = max(max_vs64, float(abs(fd - f64).max()) / rms)
            vd = pairsd / (msd * 1e-3)
            extra["df64"] = {"value": vd, "unit": UNIT, "ms_per_step": msd / args.steps,
                             "speedup_vs_fp64": vd / value,
                             "rms_force_err": math.sqrt(sum(e[0] for e in errs) /
                                                        sum(e[1] for e in errs)),
                             "max_force_err_vs_fp64_over_rms": max_vs64,
                             "md_steps_per_s": args.steps / (msd * 1e-3),
                             "tuning": (simd.tune_info or {}).get("tuning")}
            simd.close()
        if not args.no_cpu_baseline:
            v, st, pr, el, thr = oracle_rate(systems, args.cpu_seconds)
            v1, st1, pr1, el1, _ = oracle_rate(systems, max(1.0, args.cpu_seconds / 5), nthreads=1)
            extra["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                                     "sample": f"{st} oracle MD steps (one system per step, in "
                                               f"turn) in {el:.1f} s, {pr} pair interactions",
                                     "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                                       "sample": f"{st1} oracle MD steps in "
                                                                 f"{el1:.1f} s, {pr1} pair "
                                                                 f"interactions"}}
    sim.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "mixed": "f32+f64", "df64": "df64+f64"}[args.precision],
                "data": "synthetic",
                "config": {"workload": wname, "description": WORKLOADS[wname], "replicas": nrep,
                           "n_vapor": sum(s.n_vapor for s in systems),
                           "n_wall": sum(s.n_wall for s in systems),
                           "precision": args.precision,
                           "force_accumulate": args.accumulate,
                           "skin": pot.skin,
                           "cell_size": pot.cell_size or max(pot.rc, pot.rc_w) + pot.skin,
                           "skin_choice": skin_choice,
                           "l2": "flushed between timed steps (256 MB write, then 256 MB read, outside the events)",
                           "launch_mode": args.launch_mode,
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
                "md_steps_per_s": 1e3 / ms_per_step,
                "replica_steps_per_s": nrep * 1e3 / ms_per_step,
                "pairs_per_step": pairs_per_step,
                "gpu_launches": launches,
                "clocks": clocks.summary(),
                "autotune": sim_tune,
                "method_choice": getattr(sim, "method_choice", None)}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
