"""ctypes front end of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's CPU
baseline / reference legs. The CUDA library and its Python binding never import this package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (FP64, no fast-math, no FMA contraction, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", _LIB_PATH + ".tmp", src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("mass", ctypes.c_double),
                ("rc", ctypes.c_double), ("eps_w", ctypes.c_double), ("sigma_w", ctypes.c_double),
                ("rc_w", ctypes.c_double), ("shift_energy", ctypes.c_int32),
                ("thermostat_every", ctypes.c_int32), ("dt", ctypes.c_double),
                ("T0", ctypes.c_double), ("tau_B", ctypes.c_double),
                ("slab_half", ctypes.c_double), ("r_ads", ctypes.c_double),
                ("bin_width", ctypes.c_double), ("dims", ctypes.c_int32),
                ("hard_walls", ctypes.c_int32)]


class PoreC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("r0", ctypes.c_double), ("r1", ctypes.c_double), ("r_cavity", ctypes.c_double),
                ("width", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("pe_vv", ctypes.c_double), ("pe_vw", ctypes.c_double),
                ("vir_vv", ctypes.c_double), ("vir_vw", ctypes.c_double),
                ("pairs_vv", ctypes.c_int64), ("pairs_vw", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def _load(path: str):
    L = ctypes.CDLL(path)
    L.orc_lj.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D]
    L.orc_lj.restype = None
    L.orc_forces.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _D, ctypes.c_int64, _D,
                             _D, _D, ctypes.POINTER(Stats), ctypes.c_int, ctypes.c_int]
    L.orc_forces.restype = ctypes.c_int
    L.orc_forces_w.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _D, ctypes.c_int64, _D,
                               _D, _D, _D, ctypes.POINTER(Stats), ctypes.c_int, ctypes.c_int]
    L.orc_forces_w.restype = ctypes.c_int
    L.orc_pore_volume.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(PoreC)]
    L.orc_pore_volume.restype = ctypes.c_double
    L.orc_pore_pressure.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(PoreC), ctypes.c_int,
                                    ctypes.c_int64, _D, _D, _D, _D]
    L.orc_pore_pressure.restype = ctypes.c_int
    L.orc_kinetic.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _D]
    L.orc_kinetic.restype = ctypes.c_double
    L.orc_run.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _D, _D, _D, ctypes.c_int64,
                          _D, _I64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _D, _D, _D,
                          ctypes.POINTER(Stats)]
    L.orc_run.restype = ctypes.c_int
    L.orc_run_geom.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(PoreC), ctypes.c_int,
                               ctypes.c_int64, _D, _D, _D, ctypes.c_int64, _D, _I64,
                               ctypes.c_int64, ctypes.c_int, ctypes.c_int, _D, _D, _D,
                               ctypes.POINTER(Stats)]
    L.orc_run_geom.restype = ctypes.c_int
    L.orc_in_solid.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(PoreC), ctypes.c_int, _D]
    L.orc_in_solid.restype = ctypes.c_int
    L.orc_observables.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(PoreC), ctypes.c_int,
                                  ctypes.c_int64, _D, _D, _I64, _I64, _I64, ctypes.c_int]
    L.orc_observables.restype = ctypes.c_int
    L.orc_nbins.argtypes = [ctypes.POINTER(Params)]
    L.orc_nbins.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_LIB_PATH)
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of ``oracle.c`` (used by
    the mutation tests, which compile deliberately broken copies to show the pins catch them)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = _load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def build_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source (same flags as ``build``) to ``out_path``."""
    d = os.path.dirname(out_path)
    src = os.path.join(d, "oracle_variant.c")
    with open(src, "w") as fh:
        fh.write(src_text)
    import shutil
    shutil.copy(os.path.join(_HERE, "oracle.h"), os.path.join(d, "oracle.h"))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fno-fast-math", "-o", out_path, src, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(os.path.join(_HERE, "oracle.c")) as fh:
        return fh.read()


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_I64)


def _c3(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(-1, 3) if a.size else np.zeros((0, 3))


def make_params(system=None, potential=None, **over) -> Params:
    """Build oracle parameters from a ``workloads.System`` and ``workloads.Potential``."""
    d = dict(Lx=10.0, Ly=10.0, Lz=10.0, eps=1.0, sigma=1.0, mass=1.0, rc=2.5, eps_w=1.5,
             sigma_w=1.0, rc_w=2.5, shift_energy=1, thermostat_every=0, dt=0.005, T0=1.0,
             tau_B=0.0, slab_half=0.0, r_ads=1.5, bin_width=0.5, dims=3, hard_walls=0)
    if potential is not None:
        for k in ("eps", "sigma", "mass", "rc", "eps_w", "sigma_w", "rc_w", "shift_energy",
                  "r_ads", "bin_width"):
            d[k] = getattr(potential, k)
    if system is not None:
        for k in ("Lx", "Ly", "Lz", "dt", "T0", "tau_B", "thermostat_every", "slab_half"):
            d[k] = getattr(system, k)
        d["dims"] = getattr(system, "dims", 3) or 3
        d["hard_walls"] = 1 if getattr(system, "wall_model", 0) == 1 else 0
    d.update(over)
    return Params(**d)


def lj(r2: float, eps: float = 1.0, sigma: float = 1.0):
    fr, u = ctypes.c_double(), ctypes.c_double()
    lib().orc_lj(r2, eps, sigma, ctypes.byref(fr), ctypes.byref(u))
    return fr.value, u.value


def forces(p: Params, x, wall=None, method: int = 1, nthreads: int = 1):
    """Return (f (n,3), d2wall (n,), stats dict)."""
    x = _c3(x)
    w = _c3(wall if wall is not None else np.zeros((0, 3)))
    n, nw = len(x), len(w)
    f = np.zeros((n, 3))
    d2 = np.zeros(n)
    st = Stats()
    rc = lib().orc_forces(ctypes.byref(p), n, _dp(x), nw, _dp(w), _dp(f), _dp(d2),
                          ctypes.byref(st), method, nthreads)
    if rc != 0:
        raise ValueError("oracle: cutoff must be below half the periodic box")
    return f, d2, st.as_dict()


def kinetic(p: Params, v) -> float:
    v = _c3(v)
    return lib().orc_kinetic(ctypes.byref(p), len(v), _dp(v))


class State:
    """An oracle trajectory: positions, velocities, forces and the step counter."""

    def __init__(self, p: Params, x, v, wall=None, method: int = 1, nthreads: int = 1,
                 pores: Sequence = ()):
        self.p = p
        self.pores = list(pores)
        self._pc = _pores_c(self.pores)
        self.x = _c3(x).copy()
        self.v = _c3(v).copy()
        self.wall = _c3(wall if wall is not None else np.zeros((0, 3)))
        self.method, self.nthreads = method, nthreads
        self.f, self.d2wall, self.stats = forces(p, self.x, self.wall, method, nthreads)
        self.step = 0

    def run(self, nsteps: int):
        """Advance nsteps; returns (ke_log, pe_log)."""
        n = len(self.x)
        ke = np.zeros(max(nsteps, 1))
        pe = np.zeros(max(nsteps, 1))
        step = ctypes.c_int64(self.step)
        st = Stats()
        rc = lib().orc_run_geom(ctypes.byref(self.p), self._pc, len(self.pores), n, _dp(self.x),
                                _dp(self.v), _dp(self.f), len(self.wall), _dp(self.wall),
                                ctypes.byref(step), nsteps, self.method, self.nthreads, _dp(ke),
                                _dp(pe), _dp(self.d2wall), ctypes.byref(st))
        if rc != 0:
            raise ValueError("oracle run failed")
        self.step = step.value
        if nsteps > 0:
            self.stats = st.as_dict()
        return ke[:nsteps], pe[:nsteps]


def _pores_c(pores):
    arr = (PoreC * max(len(pores), 1))()
    for k, q in enumerate(pores):
        arr[k] = PoreC(q.kind, q.cx, q.cy, q.r0, q.r1, q.r_cavity, q.width)
    return arr


def in_solid(p: Params, pores: Sequence, x) -> np.ndarray:
    """Per point: 1 if it lies in the solid of a hard-wall system."""
    x = _c3(x)
    pc = _pores_c(pores)
    return np.array([lib().orc_in_solid(ctypes.byref(p), pc, len(pores), _dp(np.ascontiguousarray(r)))
                     for r in x], dtype=np.int64)


def nbins(p: Params) -> int:
    return lib().orc_nbins(ctypes.byref(p))


def observables(p: Params, pores: Sequence, x, d2wall):
    """Return (occupancy[npores], adsorbed[ngroups], profile[ngroups, nbins])."""
    x = _c3(x)
    npores = len(pores)
    arr = (PoreC * max(npores, 1))()
    for k, q in enumerate(pores):
        arr[k] = PoreC(q.kind, q.cx, q.cy, q.r0, q.r1, q.r_cavity, q.width)
    ng = max(npores, 1)
    nb = nbins(p)
    occ = np.zeros(max(npores, 1), dtype=np.int64)
    ads = np.zeros(ng, dtype=np.int64)
    prof = np.zeros((ng, nb), dtype=np.int64)
    d2 = np.ascontiguousarray(np.asarray(d2wall, dtype=np.float64))
    rc = lib().orc_observables(ctypes.byref(p), arr, npores, len(x), _dp(x), _dp(d2), _ip(occ),
                               _ip(ads), _ip(prof), nb)
    if rc != 0:
        raise ValueError("oracle observables failed")
    return occ[:npores], ads, prof


def molecule_virials(p: Params, x, wall=None, method: int = 1, nthreads: int = 1):
    """Per-molecule virials W_i (half of each vapour pair's r.F plus each wall pair's r.F)."""
    x = _c3(x)
    w = _c3(wall if wall is not None else np.zeros((0, 3)))
    n = len(x)
    f = np.zeros((n, 3))
    d2 = np.zeros(n)
    wv = np.zeros(n)
    st = Stats()
    if lib().orc_forces_w(ctypes.byref(p), n, _dp(x), len(w), _dp(w), _dp(f), _dp(d2), _dp(wv),
                          ctypes.byref(st), method, nthreads) != 0:
        raise ValueError("oracle: cutoff must be below half the periodic box")
    return wv


def pore_volume(p: Params, pore) -> float:
    arr = _pores_c([pore])
    return lib().orc_pore_volume(ctypes.byref(p), arr)


def pore_pressure(p: Params, pores, x, v, wvir):
    """Virial pressure per pore (Sec. 2) from positions, velocities and molecule virials."""
    x, v = _c3(x), _c3(v)
    wv = np.ascontiguousarray(np.asarray(wvir, dtype=np.float64))
    out = np.zeros(max(len(pores), 1))
    lib().orc_pore_pressure(ctypes.byref(p), _pores_c(pores), len(pores), len(x), _dp(x), _dp(v),
                            _dp(wv), _dp(out))
    return out[:len(pores)]
