"""The two Verlet-list builds -- a warp per cell, and a thread per molecule for dilute vapour --
must give the same lists entry for entry. In the deterministic FP64 form (every molecule sums its
own row in list order) equal lists give bit-identical forces, and bit-identical trajectories over
steps with rebuilds; the default lets the device choose by occupancy and matches both. Also the
oracle's forces and pair counts with the thread build, on dense and dilute workloads."""
import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.Potential()
WARP, MOLECULE, AUTO = 2, 3, 1


@pytest.fixture(scope="module", autouse=True)
def built():
    mdbuild.build()
    md.load_library()


def force_err(f, g):
    return np.abs(f - g).max() / np.sqrt((g ** 2).sum(1).mean())


def workloads():
    return {"small_cylinder": [W.cylinder_pore_1k()],
            "shapes_20k": W.pore_shape_systems_20k(),
            "uneven_batch": W.replica_batch(n_replicas=12, n_max=20000),
            "dense_liquid": [W.vapor_only_box(1000, 12.0, 12.0, 1.0, seed=41)]}


@pytest.mark.parametrize("name", ["small_cylinder", "shapes_20k", "uneven_batch", "dense_liquid"])
@pytest.mark.parametrize("precision", [md.MD_PREC_FP64, md.MD_PREC_MIXED])
def test_both_builds_give_the_same_lists(name, precision):
    systems = workloads()[name]
    sims = []
    try:
        for mode in (WARP, MOLECULE, AUTO):
            sim = md.Simulation(systems, precision=precision)
            sims.append(sim)
            sim.set_tuning(force_accumulate=1, list_build=mode)
            assert sim.tuning()["list_build"] == mode
            sim.rebuild_lists()
            sim.compute_forces()
        ref = [sims[0].forces(r) for r in range(len(systems))]
        for sim in sims[1:]:
            for r in range(len(systems)):
                np.testing.assert_array_equal(sim.forces(r), ref[r])
        for sim in sims:
            sim.step(40)
        assert sims[0].observables(0)[0]["n_rebuilds"] >= 3
        for r in range(len(systems)):
            x0, v0 = sims[0].state(r)
            for sim in sims[1:]:
                x, v = sim.state(r)
                np.testing.assert_array_equal(x, x0)
                np.testing.assert_array_equal(v, v0)
    finally:
        for sim in sims:
            sim.close()


@pytest.mark.parametrize("name", ["small_cylinder", "shapes_20k", "uneven_batch"])
def test_thread_build_matches_oracle(name):
    systems = workloads()[name]
    with md.Simulation(systems) as sim:
        sim.set_tuning(force_accumulate=2, list_build=MOLECULE)
        sim.step(30)
        for r, s in enumerate(systems):
            x, _ = sim.state(r)
            g, _, stats = oracle.forces(oracle.make_params(s, POT), x, s.wall, method=1, nthreads=0)
            assert force_err(sim.forces(r), g) <= 1e-10, s.name
            o = sim.observables(r)[0]
            assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]


def test_list_build_option_is_checked():
    with md.Simulation(W.cylinder_pore_1k()) as sim:
        with pytest.raises(md.MDError):
            sim.set_tuning(list_build=4)
        assert sim.tuning()["list_build"] == AUTO
