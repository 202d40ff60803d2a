"""GB300 (sm_103a) molecular dynamics of water vapour near atomistic pore walls.

Python binding of the C ABI in ``include/md.h`` (ctypes, argument marshalling only): every step of
the simulation runs in the CUDA kernels of ``libmd.so``. There is no CPU fallback; importing works
without a GPU, but every call that needs the library raises if ``libmd.so`` is missing.

The functions ``md_*`` mirror the C entry points one to one; ``Simulation`` wraps a context.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads

__all__ = ["Simulation", "MDError", "load_library", "library_path", "md_potential_from",
           "MD_PREC_FP64", "MD_PREC_MIXED", "MD_PREC_DF64"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmd.so")
_lib = None

MD_OK, MD_EINVAL, MD_ENOMEM, MD_ECUDA, MD_EOVERFLOW, MD_EUNSTABLE, MD_ETIMEOUT, MD_EBOUNDS = \
    range(8)
MD_PREC_FP64, MD_PREC_MIXED, MD_PREC_DF64 = 0, 1, 2
STATUS_NAMES = {0: "MD_OK", 1: "MD_EINVAL", 2: "MD_ENOMEM", 3: "MD_ECUDA", 4: "MD_EOVERFLOW",
                5: "MD_EUNSTABLE", 6: "MD_ETIMEOUT", 7: "MD_EBOUNDS"}


class md_pore(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("r0", ctypes.c_double), ("r1", ctypes.c_double), ("r_cavity", ctypes.c_double),
                ("width", ctypes.c_double)]


_DP = ctypes.POINTER(ctypes.c_double)


class md_system(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("n_vapor", ctypes.c_int64), ("x0", _DP), ("v0", _DP), ("T0", ctypes.c_double),
                ("dt", ctypes.c_double), ("tau_B", ctypes.c_double),
                ("thermostat_every", ctypes.c_int32), ("slab_half", ctypes.c_double),
                ("lattice_a", ctypes.c_double), ("wall_xyz", _DP), ("n_wall", ctypes.c_int64),
                ("pores", ctypes.POINTER(md_pore)), ("n_pores", ctypes.c_int32),
                ("dims", ctypes.c_int32), ("wall_model", ctypes.c_int32)]


class md_potential(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("mass", ctypes.c_double),
                ("rc", ctypes.c_double), ("eps_w", ctypes.c_double), ("sigma_w", ctypes.c_double),
                ("rc_w", ctypes.c_double), ("skin", ctypes.c_double),
                ("shift_energy", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("r_ads", ctypes.c_double), ("bin_width", ctypes.c_double),
                ("max_neighbors", ctypes.c_int32), ("max_wall_neighbors", ctypes.c_int32),
                ("cell_size", ctypes.c_double)]


class md_tuning(ctypes.Structure):
    _fields_ = [("force_block", ctypes.c_int32), ("force_blocks_per_sm", ctypes.c_int32),
                ("force_tpp", ctypes.c_int32), ("order_by_length", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("steps_per_graph", ctypes.c_int32),
                ("force_accumulate", ctypes.c_int32), ("pair_method", ctypes.c_int32),
                ("chunk_walk", ctypes.c_int32), ("list_build", ctypes.c_int32)]


class md_obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("n_vapor", ctypes.c_int64), ("n_wall", ctypes.c_int64),
                ("ke", ctypes.c_double), ("pe", ctypes.c_double), ("pe_vv", ctypes.c_double),
                ("pe_vw", ctypes.c_double), ("T", ctypes.c_double),
                ("virial_vv", ctypes.c_double), ("virial_vw", ctypes.c_double),
                ("pairs_vv", ctypes.c_int64), ("pairs_vw", ctypes.c_int64),
                ("occupancy", ctypes.c_int64), ("adsorbed", ctypes.c_int64),
                ("n_groups", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("n_rebuilds", ctypes.c_int64), ("pair_evals_total", ctypes.c_int64),
                ("max_list_used", ctypes.c_int32), ("list_capacity", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_CTX = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); the same names as include/md.h
_SIGNATURES = {
    "md_create": (ctypes.c_int, [ctypes.POINTER(md_system), ctypes.POINTER(md_potential),
                                 ctypes.c_void_p, ctypes.POINTER(_CTX)]),
    "md_create_batch": (ctypes.c_int, [ctypes.POINTER(md_system), ctypes.c_int32,
                                       ctypes.POINTER(md_potential), ctypes.c_void_p,
                                       ctypes.POINTER(_CTX)]),
    "md_set_tuning": (ctypes.c_int, [_CTX, ctypes.POINTER(md_tuning)]),
    "md_autotune": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.POINTER(md_tuning),
                                   ctypes.POINTER(ctypes.c_double)]),
    "md_get_tuning": (ctypes.c_int, [_CTX, ctypes.POINTER(md_tuning)]),
    "md_step": (ctypes.c_int, [_CTX, ctypes.c_int64]),
    "md_sync": (ctypes.c_int, [_CTX]),
    "md_get_state": (ctypes.c_int, [_CTX, ctypes.c_int32, _DP, _DP]),
    "md_set_state": (ctypes.c_int, [_CTX, ctypes.c_int32, _DP, _DP]),
    "md_get_forces": (ctypes.c_int, [_CTX, ctypes.c_int32, _DP]),
    "md_compute_forces": (ctypes.c_int, [_CTX]),
    "md_pair_pass": (ctypes.c_int, [_CTX]),
    "md_rebuild_lists": (ctypes.c_int, [_CTX]),
    "md_transfer_bytes": (ctypes.c_int, [_CTX, _I64P, _I64P]),
    "md_observables": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.POINTER(md_obs), _I64P, _I64P,
                                      _I64P, _DP]),
    "md_get_wall": (ctypes.c_int, [_CTX, ctypes.c_int32, _DP]),
    "md_get_sizes": (ctypes.c_int, [_CTX, ctypes.c_int32, _I64P, _I64P,
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "md_kernel_launches": (ctypes.c_int64, [_CTX]),
    "md_check_barrier_timeout": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double)]),
    "md_forces_noalloc": (ctypes.c_int, [ctypes.POINTER(md_potential), ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p,
                                         ctypes.c_int32]),
    "md_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "md_last_error": (ctypes.c_char_p, [_CTX]),
    "md_destroy": (None, [_CTX]),
}


def library_path() -> str:
    """``libmd.so`` beside this file, or the library named by the environment variable
    MD_LIBRARY (for instance the checked build, libmd_checked.so)."""
    return os.environ.get("MD_LIBRARY") or _LIB_PATH


def load_library():
    """Load the library (built by ``paper_1812_07993_gb300.build``). Raises if it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run paper_1812_07993_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class MDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int, ctx=None):
    if status != MD_OK:
        msg = load_library().md_last_error(ctx).decode(errors="replace")
        raise MDError(status, msg)


def md_potential_from(pot: "workloads.Potential", precision: int = MD_PREC_FP64,
                      max_neighbors: int = 0, max_wall_neighbors: int = 0) -> md_potential:
    return md_potential(pot.eps, pot.sigma, pot.mass, pot.rc, pot.eps_w, pot.sigma_w, pot.rc_w,
                        pot.skin, pot.shift_energy, precision, pot.r_ads, pot.bin_width,
                        max_neighbors, max_wall_neighbors, getattr(pot, "cell_size", 0.0))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # a torch.cuda.Stream


def _as3(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1, 3)
    return a


def _as_out(a, n: int) -> np.ndarray:
    """An output array must already be (n, 3) float64 and C-contiguous (it is written in place)."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.shape == (n, 3)
            and a.flags.c_contiguous and a.flags.writeable):
        raise ValueError(f"output must be a writeable C-contiguous float64 array of shape ({n}, 3)")
    return a


class Simulation:
    """One context: a batch of replicas advanced together on the GPU.

    ``systems`` are ``workloads.System`` objects (their wall arrays are passed explicitly, so the
    GPU and the oracle see the same wall atoms unless ``generate_wall`` is set)."""

    def __init__(self, systems, potential: "workloads.Potential" = None,
                 precision: int = MD_PREC_FP64, stream=None, generate_wall: bool = False,
                 max_neighbors: int = 0, max_wall_neighbors: int = 0):
        lib = load_library()
        if isinstance(systems, workloads.System):
            systems = [systems]
        self.systems = list(systems)
        self.potential = potential or workloads.Potential()
        self._keep = []
        arr = (md_system * len(self.systems))()
        for k, s in enumerate(self.systems):
            x0, v0 = _as3(s.x0), _as3(s.v0)
            wall = _as3(s.wall)
            pores = (md_pore * max(1, len(s.pores)))()
            for q, p in enumerate(s.pores):
                pores[q] = md_pore(p.kind, p.cx, p.cy, p.r0, p.r1, p.r_cavity, p.width)
            self._keep += [x0, v0, wall, pores]
            arr[k] = md_system(s.Lx, s.Ly, s.Lz, len(x0), x0.ctypes.data_as(_DP),
                               v0.ctypes.data_as(_DP), s.T0, s.dt, s.tau_B, s.thermostat_every,
                               s.slab_half, s.lattice_a,
                               None if generate_wall else wall.ctypes.data_as(_DP),
                               0 if generate_wall else len(wall), pores, len(s.pores),
                               getattr(s, "dims", 3), getattr(s, "wall_model", 0))
        pot = md_potential_from(self.potential, precision, max_neighbors, max_wall_neighbors)
        ctx = _CTX()
        st = lib.md_create_batch(arr, len(self.systems), ctypes.byref(pot),
                                 _stream_handle(stream), ctypes.byref(ctx))
        self._keep = []
        _check(st, None)
        self.ctx = ctx
        self.precision = precision

    # -- lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            load_library().md_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls
    def step(self, n: int = 1):
        _check(load_library().md_step(self.ctx, n), self.ctx)

    def sync(self):
        _check(load_library().md_sync(self.ctx), self.ctx)

    def sizes(self, r: int = 0):
        nv, nw = ctypes.c_int64(), ctypes.c_int64()
        ng, nb = ctypes.c_int32(), ctypes.c_int32()
        _check(load_library().md_get_sizes(self.ctx, r, ctypes.byref(nv), ctypes.byref(nw),
                                           ctypes.byref(ng), ctypes.byref(nb)), self.ctx)
        return nv.value, nw.value, ng.value, nb.value

    def n_molecules(self, r: int = 0) -> int:
        """Vapour molecules of replica r, or of the whole context for r = -1."""
        if r == -1:
            return sum(s.n_vapor for s in self.systems)
        return self.sizes(r)[0]

    def state(self, r: int = 0, out=None):
        """(x, v) of replica r (r = -1: every replica, concatenated in replica order). ``out`` may
        supply the two (n, 3) float64 C-contiguous arrays to fill (e.g. pinned host memory)."""
        n = self.n_molecules(r)
        x, v = out if out is not None else (np.zeros((n, 3)), np.zeros((n, 3)))
        _check(load_library().md_get_state(self.ctx, r, _as_out(x, n).ctypes.data_as(_DP),
                                           _as_out(v, n).ctypes.data_as(_DP)), self.ctx)
        return x, v

    def set_state(self, r: int, x, v):
        """Overwrite the state of replica r (r = -1: every replica, concatenated)."""
        x, v = _as3(x), _as3(v)
        n = self.n_molecules(r)
        if x.shape[0] != n or v.shape[0] != n:
            raise ValueError(f"set_state({r}): expected {n} molecules, got {x.shape[0]}, "
                             f"{v.shape[0]}")
        _check(load_library().md_set_state(self.ctx, r, x.ctypes.data_as(_DP),
                                           v.ctypes.data_as(_DP)), self.ctx)

    def forces(self, r: int = 0, out=None):
        """Forces of replica r (r = -1: every replica, concatenated), into ``out`` if given."""
        n = self.n_molecules(r)
        f = out if out is not None else np.zeros((n, 3))
        _check(load_library().md_get_forces(self.ctx, r, _as_out(f, n).ctypes.data_as(_DP)),
               self.ctx)
        return f

    def wall(self, r: int = 0):
        nw = self.sizes(r)[1]
        w = np.zeros((nw, 3))
        _check(load_library().md_get_wall(self.ctx, r, w.ctypes.data_as(_DP)), self.ctx)
        return w

    def observables(self, r: int = 0):
        """Return (dict of md_obs fields plus "pore_pressure" [n_pores], occupancy[n_pores],
        adsorbed[n_groups], profile[n_groups, n_bins])."""
        nv, nw, ng, nb = self.sizes(r)
        npores = len(self.systems[r].pores)
        occ = np.zeros(max(npores, 1), dtype=np.int64)
        ads = np.zeros(ng, dtype=np.int64)
        prof = np.zeros((ng, nb), dtype=np.int64)
        press = np.zeros(max(npores, 1))
        o = md_obs()
        _check(load_library().md_observables(self.ctx, r, ctypes.byref(o),
                                             occ.ctypes.data_as(_I64P), ads.ctypes.data_as(_I64P),
                                             prof.ctypes.data_as(_I64P),
                                             press.ctypes.data_as(_DP)), self.ctx)
        d = o.as_dict()
        d["pore_pressure"] = press[:npores]
        return d, occ[:npores], ads, prof

    def set_tuning(self, force_block=0, force_blocks_per_sm=0, force_tpp=0, order_by_length=0,
                   use_graph=0, steps_per_graph=0, force_accumulate=0, pair_method=0,
                   chunk_walk=0, list_build=0):
        """Launch-shape knobs (0 keeps a value). force_tpp: lanes per molecule's list (1..16), 32
        the FP64 packed kernel, 64 the flat stream (atomic form); use_graph: 1 graph replay, 2 plain launches;
        order_by_length: 1 longest list first, 2 cell order; force_accumulate (FP64): 1
        deterministic gather, 2 atomic reaction forces; pair_method: 1 Verlet lists, 2 all pairs
        (FP64), 3 cell-tiled kernel without lists (atomic reaction forces), 4 small systems
        (FP64, at most 16384 molecules: whole steps in one persistent launch); chunk_walk (the atomic
        list kernels): 1 dynamic, 2 static round robin with the next molecule prefetched;
        list_build: 1 the device chooses by occupancy, 2 a warp per cell, 3 a thread per
        molecule."""
        t = md_tuning(force_block, force_blocks_per_sm, force_tpp, order_by_length, use_graph,
                      steps_per_graph, force_accumulate, pair_method, chunk_walk, list_build)
        _check(load_library().md_set_tuning(self.ctx, ctypes.byref(t)), self.ctx)

    def autotune(self, trials: int = 15):
        """Time every launch shape of the pair kernel and keep the fastest (md_autotune).
        Returns (tuning dict, median microseconds)."""
        t = md_tuning()
        us = ctypes.c_double()
        _check(load_library().md_autotune(self.ctx, trials, ctypes.byref(t), ctypes.byref(us)),
               self.ctx)
        return {k: getattr(t, k) for k, _ in t._fields_}, us.value

    def tuning(self):
        t = md_tuning()
        _check(load_library().md_get_tuning(self.ctx, ctypes.byref(t)), self.ctx)
        return {k: getattr(t, k) for k, _ in t._fields_}

    def compute_forces(self):
        """Enqueue one pair-force evaluation at the current positions (asynchronous)."""
        _check(load_library().md_compute_forces(self.ctx), self.ctx)

    def pair_pass(self):
        """Enqueue the pair kernel alone, for timing it (md_pair_pass); call compute_forces
        before reading forces or stepping again."""
        _check(load_library().md_pair_pass(self.ctx), self.ctx)

    def rebuild_lists(self):
        """Enqueue the rebuild chain alone (cell sort, Verlet lists, processing order) for every
        replica at the current positions (md_rebuild_lists); forces are left as they are."""
        _check(load_library().md_rebuild_lists(self.ctx), self.ctx)

    def transfer_bytes(self):
        h, d = ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().md_transfer_bytes(self.ctx, ctypes.byref(h), ctypes.byref(d)),
               self.ctx)
        return h.value, d.value

    def check_barrier_timeout(self) -> float:
        """Make a bounded device wait run out on purpose and check that it reports MD_ETIMEOUT
        (md_check_barrier_timeout); the context goes on as before. Returns the GPU seconds until
        the wait gave up."""
        sec = ctypes.c_double(0.0)
        _check(load_library().md_check_barrier_timeout(self.ctx, ctypes.byref(sec)), self.ctx)
        return sec.value

    def kernel_launches(self) -> int:
        return int(load_library().md_kernel_launches(self.ctx))
