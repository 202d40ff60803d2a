"""md_forces_noalloc: forces for callers that cannot allocate device memory (for example an
application whose own pool allocator holds nearly all of it, or a latency-critical thread that must
not meet cudaFree's implicit device synchronisation). The entry point takes caller-owned device
arrays and keeps its cell list in a fixed scratch array inside the library.

Checked through the C ABI
- against the context path (md_create + md_get_forces) within the FP64 force tolerance of the
  parity tests, on two calls in a row whose sizes differ, so the second call must not see the
  first call's cell counts;
- directly against the FP64 oracle's forces on the same arrays (max deviation over the RMS force
  <= 1e-10), including molecules on cell faces and on the periodic edge, a system with no wall
  atoms, a box exactly three cells across, and x/y coordinates outside the box, which the entry
  point wraps periodically.
Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-10


def _noalloc(lib, torch, pot, s, x, wall):
    """One md_forces_noalloc call on device copies of x and wall; returns the forces on the host."""
    cpot = md.md_potential_from(pot)
    dx = torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    dw = torch.tensor(np.ascontiguousarray(wall).reshape(-1, 3), dtype=torch.float64,
                      device="cuda")
    df = torch.full_like(dx, float("nan"))
    torch.cuda.synchronize()
    err = ctypes.create_string_buffer(256)
    st = lib.md_forces_noalloc(ctypes.byref(cpot), s.Lx, s.Ly, s.Lz, dx.data_ptr(), len(x),
                               dw.data_ptr() if len(wall) else None, len(wall), df.data_ptr(),
                               None, err, len(err))
    assert st == md.MD_OK, err.value
    torch.cuda.synchronize()
    return df.cpu().numpy()


def _oracle(pot, s, x, wall):
    p = oracle.make_params(s, pot)
    g, _, _ = oracle.forces(p, x, wall, method=0, nthreads=0)   # every pair: the plain definition
    return g


def _check(got, ref):
    rms = np.sqrt((ref ** 2).sum(1).mean())
    assert rms > 0
    assert np.abs(got - ref).max() <= FORCE_TOL * rms


def _move_onto(x, i, axis, value, L):
    """Put molecule i at x[axis] = value if no other molecule comes closer than 0.9 (periodic x, y);
    returns whether it moved."""
    c = x[i].copy()
    c[axis] = value
    d = x - c
    d[:, 0] -= L[0] * np.round(d[:, 0] / L[0])
    d[:, 1] -= L[1] * np.round(d[:, 1] / L[1])
    r = np.sqrt((d ** 2).sum(1))
    r[i] = np.inf
    if r.min() <= 0.9:
        return False
    x[i] = c
    return True


def test_forces_noalloc_matches_context_path_on_two_calls():
    torch = pytest.importorskip("torch")
    mdbuild.build()
    lib = md.load_library()
    pot = W.Potential()
    cpot = md.md_potential_from(pot)
    systems = [W.pore_shape_systems_20k()[3], W.cylinder_pore_1k()]
    refs = []
    for s in systems:
        with md.Simulation(s) as sim:
            refs.append(sim.forces())
    bufs = []
    for s in systems:
        x = torch.tensor(s.x0, dtype=torch.float64, device="cuda")
        w = torch.tensor(s.wall, dtype=torch.float64, device="cuda")
        f = torch.full_like(x, float("nan"))
        bufs.append((x, w, f))
    torch.cuda.synchronize()
    err = ctypes.create_string_buffer(256)
    for s, (x, w, f) in zip(systems, bufs):        # two calls in a row
        st = lib.md_forces_noalloc(ctypes.byref(cpot), s.Lx, s.Ly, s.Lz, x.data_ptr(), s.n_vapor,
                                   w.data_ptr(), s.n_wall, f.data_ptr(), None, err, len(err))
        assert st == md.MD_OK, err.value
    torch.cuda.synchronize()
    for ref, (_, _, f) in zip(refs, bufs):
        got = f.cpu().numpy()
        rms = np.sqrt((ref ** 2).sum(1).mean())
        assert np.abs(got - ref).max() <= FORCE_TOL * rms


def test_forces_noalloc_matches_oracle_with_walls():
    """The small cylindrical pore (wall atoms, pore, reflecting ends) against the oracle's sum over
    every pair, on the same arrays."""
    torch = pytest.importorskip("torch")
    mdbuild.build()
    lib = md.load_library()
    pot = W.Potential()
    s = W.cylinder_pore_1k()
    _check(_noalloc(lib, torch, pot, s, s.x0, s.wall), _oracle(pot, s, s.x0, s.wall))


def test_forces_noalloc_matches_oracle_on_cell_faces_periodic_edge_three_cells_no_wall():
    """A wall-free box exactly three cells of max(rc, rc_w) across in x and y (7.5 = 3 x 2.5),
    with molecules moved onto cell faces (x or y = -L/2 + k * 2.5, z on the z-cell faces) and onto
    the periodic edge -L/2: every pair the oracle finds must be found once, from the right image."""
    torch = pytest.importorskip("torch")
    mdbuild.build()
    lib = md.load_library()
    pot = W.Potential()
    s = W.vapor_only_box(120, 7.5, 10.0, 1.0, seed=31)
    x = s.x0.copy()
    L = (s.Lx, s.Ly)
    targets = [(0, -3.75), (1, -3.75), (0, -1.25), (1, 1.25), (0, 1.25), (1, -1.25), (2, 0.0),
               (2, -2.5), (2, 2.5), (0, 3.75 - 1e-12), (1, 3.75 - 1e-12), (0, 0.0)]
    free = list(range(len(x)))
    for axis, value in targets:   # each target face taken by the first molecule that fits there
        for k, i in enumerate(free):
            if _move_onto(x, i, axis, value, L):
                del free[k]
                break
        else:
            raise AssertionError(f"no molecule fits on {axis} = {value}")
    empty = np.zeros((0, 3))
    _check(_noalloc(lib, torch, pot, s, x, empty), _oracle(pot, s, x, empty))


def test_forces_noalloc_wraps_x_and_y_outside_the_box():
    """Molecules and wall atoms shifted by whole box lengths in x or y (one, two or minus one)
    give the forces of the wrapped configuration."""
    torch = pytest.importorskip("torch")
    mdbuild.build()
    lib = md.load_library()
    pot = W.Potential()
    s = W.cylinder_pore_1k()
    x = s.x0.copy()
    w = s.wall.copy()
    rng = np.random.default_rng(5)
    for arr, k in ((x, 200), (w, 300)):
        rows = rng.choice(len(arr), size=k, replace=False)
        arr[rows, 0] += s.Lx * rng.choice([-1.0, 1.0, 2.0], size=k)
        arr[rows[: k // 2], 1] += s.Ly * rng.choice([-1.0, 1.0], size=k // 2)
    _check(_noalloc(lib, torch, pot, s, x, w), _oracle(pot, s, s.x0, s.wall))


def test_forces_noalloc_rejects_sizes_beyond_its_limit():
    mdbuild.build()
    lib = md.load_library()
    cpot = md.md_potential_from(W.Potential())
    err = ctypes.create_string_buffer(256)
    st = lib.md_forces_noalloc(ctypes.byref(cpot), 100.0, 100.0, 100.0, 1, 200000, 1, 100000, 1,
                               None, err, len(err))
    assert st == md.MD_EINVAL and b"limit" in err.value
    st = lib.md_forces_noalloc(ctypes.byref(cpot), 400.0, 400.0, 400.0, 1, 10, 1, 0, 1, None, err,
                               len(err))
    assert st == md.MD_EINVAL and b"cells" in err.value
    bad = md.md_potential_from(W.Potential(eps=float("nan")))
    st = lib.md_forces_noalloc(ctypes.byref(bad), 10.0, 10.0, 10.0, 1, 10, 1, 0, 1, None, err,
                               len(err))
    assert st == md.MD_EINVAL and b"not finite" in err.value
    st = lib.md_forces_noalloc(ctypes.byref(cpot), 10.0, float("inf"), 10.0, 1, 10, 1, 0, 1, None,
                               err, len(err))
    assert st == md.MD_EINVAL and b"not finite" in err.value
