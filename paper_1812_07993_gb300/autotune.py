"""Autotuner: launch shape, Verlet skin and cell side, per size class.

The timing of launch shapes runs in the library (``md_autotune``: CUDA events around the pair-force
evaluation for every candidate shape); this module keys the result by a size class and caches it in
a small JSON file, and chooses the skin and the cell side by timing whole MD steps on fresh
contexts, cached by size class too. The paper's counterpart is its manual scan of threads per block
(Sec. 4 and Sec. 5, Figs. 7 and 12).
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
import time
from typing import Dict, Optional, Sequence

from . import MD_PREC_FP64, MDError, Simulation, workloads


def size_class(systems: Sequence["workloads.System"], precision: int) -> str:
    """Bucket a batch by precision, replica count and log2 of its molecule and wall-atom counts."""
    n = sum(s.n_vapor for s in systems)
    nw = sum(s.n_wall for s in systems)
    return (f"prec{precision}-rep{len(systems)}-n2^{round(math.log2(max(n, 1)))}"
            f"-w2^{round(math.log2(max(nw, 1)))}")


def default_cache_path() -> str:
    return os.environ.get("MD_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1812_07993_gb300", "tuning.json")


def _load(path: str) -> Dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune(sim: Simulation, trials: int = 15, cache_path: Optional[str] = None,
         use_cache: bool = True) -> Dict:
    """Apply the cached launch shape of the simulation's size class, or run ``md_autotune`` and
    cache its choice. Returns {"tuning": ..., "us": ..., "cached": bool, "seconds": ...}."""
    path = cache_path or default_cache_path()
    key = size_class(sim.systems, sim.precision) + f"-acc{sim.tuning()['force_accumulate']}"
    cache = _load(path) if use_cache else {}
    t0 = time.perf_counter()
    if key in cache:
        t = cache[key]["tuning"]
        sim.set_tuning(force_block=t["force_block"], force_blocks_per_sm=t["force_blocks_per_sm"],
                       force_tpp=t["force_tpp"], order_by_length=t["order_by_length"],
                       chunk_walk=t.get("chunk_walk", 0),
                       pair_method=t.get("pair_method", 0) if t.get("pair_method") in (1, 3)
                       else 0)
        return {"tuning": t, "us": cache[key]["us"], "cached": True,
                "seconds": time.perf_counter() - t0, "size_class": key}
    t, us = sim.autotune(trials)
    cache[key] = {"tuning": t, "us": us}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path + ".tmp", "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(path + ".tmp", path)
    except OSError:
        pass
    return {"tuning": t, "us": us, "cached": False, "seconds": time.perf_counter() - t0,
            "size_class": key}


def _time_steps(systems, pot, precision, steps, warmup, stream) -> Dict:
    """Steps per second of a fresh context with an autotuned launch shape, over ``steps`` MD steps
    after ``warmup``, with its list rebuilds; or the error of a context that is refused or whose
    lists overflow."""
    try:
        with Simulation(systems, pot, precision=precision, stream=stream) as sim:
            sim.autotune(7)
            sim.step(warmup)
            sim.sync()
            o0 = sim.observables(0)[0]
            t0 = time.perf_counter()
            sim.step(steps)
            sim.sync()
            dt = time.perf_counter() - t0
            o1 = sim.observables(0)[0]
    except MDError as e:
        return {"error": str(e)}
    return {"steps_per_s": steps / dt, "rebuilds": o1["n_rebuilds"] - o0["n_rebuilds"]}


def choose_skin(systems: Sequence["workloads.System"], potential: "workloads.Potential" = None,
                precision: int = MD_PREC_FP64, skins=(0.2, 0.3, 0.4, 0.5, 0.6, 0.8),
                steps: int = 100, warmup: int = 20, stream=None) -> Dict:
    """Time ``steps`` MD steps (after ``warmup``) for each candidate skin on a fresh context with an
    autotuned launch shape; returns the skin with the most steps per second and the table. The skin
    only trades list length against rebuild frequency: every candidate gives the same forces. A
    candidate the context refuses (box too small for its cells) or whose lists overflow their
    capacity is left out, with its error in the table."""
    pot = potential or workloads.Potential()
    table = []
    for skin in skins:
        table.append(dict(skin=skin, **_time_steps(systems, dataclasses.replace(pot, skin=skin),
                                                   precision, steps, warmup, stream)))
    ok = [r for r in table if "steps_per_s" in r]
    best = max(ok, key=lambda r: r["steps_per_s"]) if ok else None
    return {"skin": best["skin"] if best else None, "table": table}


def choose_geometry(systems: Sequence["workloads.System"], potential: "workloads.Potential" = None,
                    precision: int = MD_PREC_FP64, skins=(0.2, 0.3, 0.4, 0.5, 0.6, 0.8),
                    cell_scales=(1.0, 1.25, 1.5, 2.0), steps: int = 100, warmup: int = 20,
                    stream=None, cache_path: Optional[str] = None, use_cache: bool = True) -> Dict:
    """The Verlet skin and the cell side of a batch's size class, by whole MD steps on fresh
    contexts: every candidate skin with cells of side rc + skin (choose_skin), then, at the fastest
    skin, every cell scale (cell side = scale x (max(rc, rc_w) + skin)); the fastest pair is kept.
    Neither changes the forces or the pair counts: the skin trades list length against rebuild
    frequency, the cell side the work per cell of the sort and the list build against the number of
    cells. The choice is cached per size class (precision, replica count, log2 of the molecule and
    wall counts) beside the launch shapes. Returns {"skin", "cell_size" (0: the list radius),
    "skin_table", "cell_table", "cached", "size_class"}."""
    pot = potential or workloads.Potential()
    path = cache_path or default_cache_path()
    key = "geometry-" + size_class(systems, precision)
    cache = _load(path) if use_cache else {}
    if key in cache:
        return dict(cache[key], cached=True, size_class=key)
    sk = choose_skin(systems, pot, precision, skins, steps, warmup, stream)
    result = {"skin": sk["skin"], "cell_size": 0.0, "skin_table": sk["table"], "cell_table": []}
    if sk["skin"] is not None:
        best_rate = max(r["steps_per_s"] for r in sk["table"] if r.get("skin") == sk["skin"])
        base = dataclasses.replace(pot, skin=sk["skin"])
        rl = max(pot.rc, pot.rc_w) + sk["skin"]
        for scale in cell_scales:
            if scale == 1.0:
                continue
            cell = scale * rl
            row = dict(scale=scale, cell_size=cell,
                       **_time_steps(systems, dataclasses.replace(base, cell_size=cell),
                                     precision, steps, warmup, stream))
            result["cell_table"].append(row)
            if row.get("steps_per_s", 0.0) > best_rate:
                best_rate = row["steps_per_s"]
                result["cell_size"] = cell
    if use_cache and result["skin"] is not None:
        cache[key] = result
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path + ".tmp", "w") as fh:
                json.dump(cache, fh, indent=1, sort_keys=True)
            os.replace(path + ".tmp", path)
        except OSError:
            pass
    return dict(result, cached=False, size_class=key)


SMALL_MAX = 16384  # molecules of a context the small-system method (pair_method 4) takes


def choose_step_method(systems: Sequence["workloads.System"],
                       potential: "workloads.Potential" = None, precision: int = MD_PREC_FP64,
                       steps: int = 200, warmup: int = 20, stream=None) -> Dict:
    """For a context of at most SMALL_MAX molecules (FP64): whole MD steps with the autotuned
    Verlet-list method against the small-system method (pair_method 4: whole steps in one
    persistent launch, no lists), on fresh contexts, timed as ``steps`` single-step calls; returns
    {"pair_method": 1 or 4, "table": [...]}. Larger or non-FP64 contexts keep the lists."""
    n = sum(s.n_vapor for s in systems)
    if precision != MD_PREC_FP64 or n > SMALL_MAX:
        return {"pair_method": 1, "table": [], "reason": "not eligible for the small-system method"}
    pot = potential or workloads.Potential()
    table = []
    for method in (1, 4):
        try:
            with Simulation(systems, pot, precision=precision, stream=stream) as sim:
                sim.set_tuning(pair_method=method)
                if method == 1:
                    sim.autotune(7)
                sim.step(warmup)
                sim.sync()
                t0 = time.perf_counter()
                for _ in range(steps):
                    sim.step(1)
                sim.sync()
                table.append({"pair_method": method,
                              "steps_per_s": steps / (time.perf_counter() - t0)})
        except MDError as e:
            table.append({"pair_method": method, "error": str(e)})
    ok = [r for r in table if "steps_per_s" in r]
    best = max(ok, key=lambda r: r["steps_per_s"]) if ok else {"pair_method": 1}
    return {"pair_method": best["pair_method"], "table": table}
