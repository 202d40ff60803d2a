"""Autotuner: launch shape per size class, and the Verlet skin where a workload leaves it free.

The timing of launch shapes runs in the library (``md_autotune``: CUDA events around the pair-force
evaluation for every candidate shape); this module keys the result by a size class and caches it in
a small JSON file, and chooses the skin by timing whole MD steps on fresh contexts. The paper's
counterpart is its manual scan of threads per block (Sec. 4 and Sec. 5, Figs. 7 and 12).
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
        p = dataclasses.replace(pot, skin=skin)
        try:
            with Simulation(systems, p, precision=precision, stream=stream) as sim:
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
            table.append({"skin": skin, "error": str(e)})
            continue
        table.append({"skin": skin, "steps_per_s": steps / dt,
                      "rebuilds": o1["n_rebuilds"] - o0["n_rebuilds"]})
    ok = [r for r in table if "steps_per_s" in r]
    best = max(ok, key=lambda r: r["steps_per_s"]) if ok else None
    return {"skin": best["skin"] if best else None, "table": table}
