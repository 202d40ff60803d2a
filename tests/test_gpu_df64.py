"""Double-float pair terms (MD_PREC_DF64) against the FP64 CPU oracle and the FP64 GPU form.

The context is an FP64 one (positions, integration, cutoff decisions near rc, accumulation,
observables); only the pair terms run in double-word FP32 arithmetic (~2^-44 relative per term),
in a half-list form with atomic reaction forces or a full-list form with no atomics.
The bar is the FP64 path's: per-step forces max_i |F - F_oracle| / RMS(F) <= 1e-10, 10-step
trajectories |dr|, |dv| <= 1e-8, integer observables exactly equal -- and, closer, the FP64 GPU
form's forces to 1e-11 of the RMS force.
"""
import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

from test_gpu_parity import (FORCE_TOL, TRAJ_TOL, check_observables, force_err, oracle_params,
                             wrapped_diff)

pytestmark = pytest.mark.gpu

DF = md.MD_PREC_DF64


@pytest.fixture(scope="module", autouse=True)
def built():
    mdbuild.build()
    md.load_library()


@pytest.fixture(scope="module")
def shapes():
    return W.pore_shape_systems_20k()


@pytest.fixture(scope="module")
def shapes_after_ten(shapes):
    states = [oracle.State(oracle_params(s), s.x0, s.v0, s.wall) for s in shapes]
    for st in states:
        st.run(10)
    return states


def test_small_cylinder_forces_trajectory_and_observables():
    s = W.cylinder_pore_1k()
    st = oracle.State(oracle_params(s), s.x0, s.v0, s.wall)
    with md.Simulation(s, precision=DF) as sim, md.Simulation(s) as ref:
        assert sim.tuning()["force_accumulate"] == 2
        g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
        assert force_err(sim.forces(), g) <= FORCE_TOL
        assert force_err(sim.forces(), ref.forces()) <= 1e-11
        sim.step(10)
        st.run(10)
        x, v = sim.state()
        assert np.abs(wrapped_diff(x, st.x, s)).max() <= TRAJ_TOL
        assert np.abs(v - st.v).max() <= TRAJ_TOL
        check_observables(sim, 0, s, st)


@pytest.mark.parametrize("tpp,block,bps,lpt,acc", [
    (1, 256, 4, 1, 2), (2, 128, 2, 1, 2), (4, 256, 4, 1, 2), (4, 128, 1, 2, 2), (8, 256, 4, 1, 2),
    (1, 128, 4, 1, 1), (2, 256, 2, 2, 1), (4, 256, 4, 1, 1), (8, 128, 8, 1, 1), (16, 256, 4, 1, 2),
    (16, 128, 2, 1, 1)])
def test_every_launch_shape_matches_oracle(shapes, shapes_after_ten, tpp, block, bps, lpt, acc):
    """Lanes per molecule, block size, blocks per SM, processing order, and the atomic (half
    list) or full-list form: the oracle's forces, 10-step trajectories (with a thermostat step)
    and integer observables of four pore shapes."""
    with md.Simulation(shapes, precision=DF) as sim:
        sim.set_tuning(force_tpp=tpp, force_block=block, force_blocks_per_sm=bps,
                       order_by_length=lpt, force_accumulate=acc)
        assert sim.tuning()["force_accumulate"] == acc
        sim.compute_forces()
        for r, s in enumerate(shapes):
            g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
            assert force_err(sim.forces(r), g) <= FORCE_TOL, s.name
        sim.step(10)
        for r, (s, st) in enumerate(zip(shapes, shapes_after_ten)):
            x, v = sim.state(r)
            assert np.abs(wrapped_diff(x, st.x, s)).max() <= TRAJ_TOL, s.name
            assert np.abs(v - st.v).max() <= TRAJ_TOL, s.name
            check_observables(sim, r, s, st)


def test_agrees_with_fp64_on_a_filled_pore_over_fifty_steps():
    """A liquid-filled pore (rows of 60-100 entries, many pairs near the LJ minimum where the
    force factor cancels): the FP64 form's forces to 1e-11 of the RMS force, and its trajectory to
    round-off growth over 50 steps (rebuilds and thermostat steps included)."""
    s = W.drying_cylinder_pore()
    with md.Simulation(s, precision=DF) as a, md.Simulation(s) as b:
        b.set_tuning(force_accumulate=2)
        assert force_err(a.forces(), b.forces()) <= 1e-11
        a.step(50)
        b.step(50)
        xa, va = a.state()
        xb, vb = b.state()
        assert np.abs(wrapped_diff(xa, xb, s)).max() <= 1e-8
        assert np.abs(va - vb).max() <= 1e-8
        oa, *_ = a.observables()
        ob, *_ = b.observables()
        assert oa["pairs_vv"] == ob["pairs_vv"] and oa["pairs_vw"] == ob["pairs_vw"]
        assert oa["pe"] == pytest.approx(ob["pe"], rel=1e-10)


def test_full_list_form_is_bitwise_reproducible(shapes):
    """The full-list form sums each molecule's own row in a fixed order with no atomics: two runs,
    and graph replays against plain launches, agree bit for bit; the atomic form agrees with it to
    rounding."""
    runs = []
    for graph in (1, 2, 1):
        with md.Simulation(shapes, precision=DF) as sim:
            sim.set_tuning(force_accumulate=1, use_graph=graph, steps_per_graph=5)
            sim.step(25)
            runs.append([sim.state(r) + (sim.forces(r),) for r in range(len(shapes))])
    for r in range(len(shapes)):
        for k in range(3):
            np.testing.assert_array_equal(runs[0][r][k], runs[1][r][k])
            np.testing.assert_array_equal(runs[0][r][k], runs[2][r][k])
    with md.Simulation(shapes, precision=DF) as sim:
        sim.step(25)
        for r, s in enumerate(shapes):
            x, v = sim.state(r)
            assert np.abs(wrapped_diff(x, runs[0][r][0], s)).max() <= 1e-9
            assert np.abs(v - runs[0][r][1]).max() <= 1e-9


def test_graph_and_plain_launches_agree(shapes):
    with md.Simulation(shapes, precision=DF) as a, md.Simulation(shapes, precision=DF) as b:
        a.set_tuning(use_graph=2)
        b.set_tuning(use_graph=1, steps_per_graph=7)
        a.step(35)
        b.step(35)
        for r, s in enumerate(shapes):
            xa, va = a.state(r)
            xb, vb = b.state(r)
            assert np.abs(wrapped_diff(xa, xb, s)).max() <= 1e-9
            assert np.abs(va - vb).max() <= 1e-9


def test_options_outside_the_mode_are_rejected():
    s = W.cylinder_pore_1k()
    with md.Simulation(s, precision=DF) as sim:
        for bad in (dict(force_tpp=32), dict(pair_method=2)):
            with pytest.raises(md.MDError):
                sim.set_tuning(**bad)
        t, us = sim.autotune(3)
        assert t["force_tpp"] in (1, 2, 4, 8, 16, 64) and us > 0
        g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
        assert force_err(sim.forces(), g) <= FORCE_TOL
