"""The small-system method (pair_method 4): whole MD steps in one cooperative launch, against the
FP64 oracle.

No lists and no sorting: per step the kernel advances every molecule, meets the other blocks at a
bounded grid barrier, and a warp per molecule screens every vapour molecule of its replica and the
wall atoms of its 27 static cells in FP32, evaluating the candidates in FP64 (the cutoff decided in
FP64) and summing them in a fixed order, with the second half-kick applied; a thermostat step's
scaling is paid at the next step's start. Checked: forces (1e-10 of the RMS force), 25-step
trajectories across two thermostat steps (1e-8), observables, the paper's hard-wall prism pore and
planar pore, the drying pore under Berendsen coupling, bit-for-bit reproducibility, the same run
split by a state read, and the refusals (mixed or double-float contexts, too many molecules).
"""
import dataclasses

import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.Potential()


@pytest.fixture(scope="module", autouse=True)
def built():
    mdbuild.build()
    md.load_library()


def force_err(f, g):
    return np.abs(f - g).max() / np.sqrt((g ** 2).sum(1).mean())


def wrapped_diff(a, b, s):
    d = a - b
    d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
    d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
    return d


def small_sim(systems):
    sim = md.Simulation(systems)
    sim.set_tuning(pair_method=4)
    assert sim.tuning()["pair_method"] == 4
    return sim


SYSTEMS = {
    "cylinder_pore_1k": W.cylinder_pore_1k,
    "paper_prism_pore": W.paper_prism_pore,
    "paper_pore_2d": W.paper_pore_2d,
    "drying_cylinder_pore": W.drying_cylinder_pore,
}


@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_forces_and_25_step_trajectory(name):
    s = SYSTEMS[name]()
    p = oracle.make_params(s, POT)
    st = oracle.State(p, s.x0, s.v0, s.wall, nthreads=0, pores=s.pores)
    with small_sim([s]) as sim:
        g, _, _ = oracle.forces(p, s.x0, s.wall, method=1, nthreads=0)
        if np.any(g):
            assert force_err(sim.forces(0), g) <= 1e-10
        sim.step(25)
        st.run(25)
        x, v = sim.state(0)
        assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-8
        assert np.abs(v - st.v).max() <= 1e-8
        o = sim.observables(0)[0]
        f, d2, stats = oracle.forces(p, st.x, s.wall, method=1, nthreads=0)
        assert (o["pairs_vv"], o["pairs_vw"]) == (stats["pairs_vv"], stats["pairs_vw"])
        assert o["pe"] == pytest.approx(stats["pe_vv"] + stats["pe_vw"], rel=1e-10, abs=1e-10)
        assert o["step"] == 25
        g = sim.forces(0)
        assert force_err(g, f) <= 1e-10


def test_runs_are_bitwise_reproducible_and_a_read_changes_nothing():
    s = W.cylinder_pore_1k()
    out = []
    for split in (None, 10, 7):  # (an odd launch leaves the positions in the second buffer)
        with small_sim([s]) as sim:
            if split:
                sim.step(split)
                sim.state(0)                       # settles the owed thermostat
                sim.observables(0)
                sim.step(30 - split)
            else:
                sim.step(30)
            out.append(sim.state(0))
    for x, v in out[1:]:
        np.testing.assert_array_equal(out[0][0], x)
        np.testing.assert_array_equal(out[0][1], v)


def test_batch_of_small_replicas_matches_alone():
    batch = W.replica_batch(n_replicas=4, n_min=1000, n_max=3000)
    with small_sim(batch) as sim:
        sim.step(15)
        xb = [sim.state(r) for r in range(len(batch))]
    for r, s in enumerate(batch):
        st = oracle.State(oracle.make_params(s, POT), s.x0, s.v0, s.wall, nthreads=0)
        st.run(15)
        assert np.abs(wrapped_diff(xb[r][0], st.x, s)).max() <= 1e-8
        assert np.abs(xb[r][1] - st.v).max() <= 1e-8


def test_refusals():
    s = W.cylinder_pore_1k()
    for prec in (md.MD_PREC_MIXED, md.MD_PREC_DF64):
        with md.Simulation(s, precision=prec) as sim:
            with pytest.raises(md.MDError, match="FP64"):
                sim.set_tuning(pair_method=4)
    with md.Simulation(W.pore_shape_systems_20k()) as sim:
        with pytest.raises(md.MDError, match="16384"):
            sim.set_tuning(pair_method=4)
    with small_sim([s]) as sim:
        with pytest.raises(md.MDError):
            sim.rebuild_lists()
