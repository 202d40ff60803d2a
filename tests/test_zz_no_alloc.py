"""md_forces_noalloc: forces for callers that cannot allocate device memory (for example an
application whose own pool allocator holds nearly all of it, or a latency-critical thread that must
not meet cudaFree's implicit device synchronisation). The entry point takes caller-owned device
arrays and keeps its cell list in a fixed scratch array inside the library.

Checked through the C ABI against the context path (md_create + md_get_forces) within the FP64
force tolerance of the parity tests, on two calls in a row whose sizes differ, so the second call
must not see the first call's cell counts. Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-10


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
