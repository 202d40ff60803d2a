"""The checked build (libmd_checked.so, compiled with -DMD_CHECKED) against the oracle.

In that build every index a kernel reads from device data -- a list entry, the processing order, a
pair slot, a cell or sort index, a staged candidate -- is checked before its access; one outside
its array would be replaced by an in-bounds index and set the sticky status MD_EBOUNDS. The small
cylinder, the four 20k pore shapes and a 12-replica uneven batch run 60 steps (list rebuilds
included) in every pair form -- FP64 deterministic, atomic and packed, all pairs, mixed and
double-float in both accumulations, the cell method in all three precisions, the flat stream, the
small-system method and the thread-per-molecule list build -- in a separate
process that loads the checked library: no check may fire (the synchronising calls would raise
MD_EBOUNDS), and forces and pair counts must match the oracle as in the normal build.
"""
import os
import subprocess
import sys

import pytest

from paper_1812_07993_gb300 import build as mdbuild

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import workloads as W

assert md.library_path().endswith("libmd_checked.so"), md.library_path()
POT = W.Potential()
FP64, MIXED, DF64 = md.MD_PREC_FP64, md.MD_PREC_MIXED, md.MD_PREC_DF64
FORMS = [  # precision, force_accumulate, pair_method, force_tpp (0: keep; 64 the flat stream),
    # small systems only, list build (1 the device's choice, 3 a thread per molecule)
    (FP64, 1, 1, 2, False, 1), (FP64, 2, 1, 2, False, 1), (FP64, 2, 1, 32, False, 1),
    (FP64, 1, 1, 32, False, 1), (FP64, 1, 2, 0, True, 1), (MIXED, 1, 1, 4, False, 1),
    (MIXED, 2, 1, 4, False, 1), (DF64, 2, 1, 4, False, 1), (DF64, 1, 1, 4, False, 1),
    (FP64, 2, 3, 0, False, 1), (MIXED, 2, 3, 0, False, 1), (DF64, 2, 3, 0, False, 1),
    (FP64, 2, 1, 64, False, 3), (MIXED, 2, 1, 64, False, 3), (DF64, 2, 1, 64, False, 1),
    (FP64, 1, 1, 2, False, 3), (FP64, 0, 4, 0, True, 1),
]
workloads = [[W.cylinder_pore_1k()], W.pore_shape_systems_20k(),
             W.replica_batch(n_replicas=12, n_max=20000)]
for k, systems in enumerate(workloads):
    for prec, acc, method, tpp, small_only, build in FORMS:
        if small_only and k > 0:
            continue
        with md.Simulation(systems, precision=prec) as sim:
            sim.set_tuning(force_accumulate=acc, pair_method=method, force_tpp=tpp,
                           list_build=build)
            sim.step(60)
            sim.sync()
            for r, s in enumerate(systems):
                x, _ = sim.state(r)
                g, _, stats = oracle.forces(oracle.make_params(s, POT), x, s.wall, method=1,
                                            nthreads=0)
                f = sim.forces(r)
                if prec == MIXED:
                    err = np.sqrt(((f - g) ** 2).sum() / (g ** 2).sum())
                    assert err <= 1e-5, (k, prec, acc, method, r, err)
                else:
                    err = np.abs(f - g).max() / np.sqrt((g ** 2).sum(1).mean())
                    assert err <= 1e-10, (k, prec, acc, method, r, err)
                o = sim.observables(r)[0]
                assert (o["pairs_vv"], o["pairs_vw"]) == (stats["pairs_vv"], stats["pairs_vw"])
print("checked ok")
'''


def test_checked_build_runs_every_form_without_a_bounds_report():
    path = mdbuild.build(checked=True)
    env = dict(os.environ, MD_LIBRARY=path)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0 and "checked ok" in r.stdout, (r.stdout + r.stderr)[-3000:]
