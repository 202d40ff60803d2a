"""The flat stream (force_tpp 64, atomic form) against the FP64 oracle.

A warp reads the rows of its 32 molecules as one stream of list entries, 32 at a time whoever owns
them, screens every entry in FP32 on the cell-local offsets and -- in the FP64 and double-float
forms -- queues the survivors in its registers (the queue runs over chunk boundaries), evaluating 32
queued pairs at a time with the cutoff decided in FP64; both ends of each pair receive its force by
FP64 atomic adds. The pair set must be the oracle's exactly and the forces within the bars of the
other list forms: FP64 and double-float 1e-10 of the RMS force per step and 1e-8 over ten-step
trajectories, mixed 1e-5 RMS. Workloads: the four 20k pore shapes (one context) in both chunk walks
and both processing orders, the 200k cylinder at full size, an uneven batch through rebuilds, a
dense liquid whose rows overflow the queue many times per chunk, an empty replica and a single
molecule, and a wall-free box (Newton's third law).
"""
import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.Potential()
FLAT = 64
PRECS = [(md.MD_PREC_FP64, 1e-10), (md.MD_PREC_DF64, 1e-10), (md.MD_PREC_MIXED, 1e-5)]


@pytest.fixture(scope="module", autouse=True)
def built():
    mdbuild.build()
    md.load_library()


def force_err(f, g):
    return np.abs(f - g).max() / np.sqrt((g ** 2).sum(1).mean())


def rms_rel_err(f, g):
    return np.sqrt(((f - g) ** 2).sum() / (g ** 2).sum())


def wrapped_diff(a, b, s):
    d = a - b
    d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
    d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
    return d


def flat_sim(systems, precision, **shape):
    sim = md.Simulation(systems, precision=precision)
    sim.set_tuning(force_accumulate=2, force_tpp=FLAT, **shape)
    t = sim.tuning()
    assert t["force_tpp"] == FLAT and t["force_accumulate"] == 2
    return sim


def check_forces(sim, systems, precision, tol):
    for r, s in enumerate(systems):
        x, _ = sim.state(r)
        g, _, stats = oracle.forces(oracle.make_params(s, POT), x, s.wall, method=1, nthreads=0)
        f = sim.forces(r)
        if s.n_vapor == 0:
            continue
        if precision == md.MD_PREC_MIXED:
            assert rms_rel_err(f, g) <= tol, s.name
        else:
            assert force_err(f, g) <= tol, s.name
        o = sim.observables(r)[0]
        assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"], s.name


@pytest.fixture(scope="module")
def shapes():
    return W.pore_shape_systems_20k()


@pytest.fixture(scope="module")
def shapes_after_ten(shapes):
    states = []
    for s in shapes:
        st = oracle.State(oracle.make_params(s, POT), s.x0, s.v0, s.wall, nthreads=0)
        st.run(10)
        states.append(st)
    return states


@pytest.mark.parametrize("precision,tol", PRECS)
@pytest.mark.parametrize("walk,lpt,block", [(1, 1, 256), (2, 1, 128), (1, 2, 128), (2, 2, 256)])
def test_flat_stream_forces_and_trajectories_four_shapes(shapes, shapes_after_ten, precision, tol,
                                                         walk, lpt, block):
    """Forces and exact pair counts at the start; after ten steps the FP64 and double-float
    trajectories within 1e-8 of the oracle's, the mixed forces within 1e-5 RMS at its own
    positions."""
    with flat_sim(shapes, precision, chunk_walk=walk, order_by_length=lpt, force_block=block,
                  force_blocks_per_sm=2) as sim:
        check_forces(sim, shapes, precision, tol)
        sim.step(10)
        if precision == md.MD_PREC_MIXED:
            check_forces(sim, shapes, precision, tol)
            return
        for r, (s, st) in enumerate(zip(shapes, shapes_after_ten)):
            x, v = sim.state(r)
            assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-8, s.name
            assert np.abs(v - st.v).max() <= 1e-8, s.name


@pytest.mark.parametrize("precision,tol", PRECS)
def test_flat_stream_large_cylinder(precision, tol):
    """200,000 molecules and ~1.33 M wall atoms (about 2.4 list entries a molecule): every force
    against the oracle, pair counts exact."""
    s = W.cylinder_pore_200k()
    with flat_sim([s], precision) as sim:
        check_forces(sim, [s], precision, tol)


@pytest.mark.parametrize("precision,tol", PRECS)
def test_flat_stream_uneven_batch_after_rebuilds(precision, tol):
    """Twelve uneven replicas (a chunk's molecules may belong to two replicas, each queued pair
    carries its owner's replica) through 120 steps with several rebuilds."""
    batch = W.replica_batch(n_replicas=12, n_max=20000)
    with flat_sim(batch, precision) as sim:
        sim.step(120)
        assert sim.observables(0)[0]["n_rebuilds"] >= 3
        check_forces(sim, batch, precision, tol)


@pytest.mark.parametrize("precision,tol", PRECS)
def test_flat_stream_dense_liquid(precision, tol):
    """A wall-free box at density ~0.58: rows of dozens of entries, so a chunk's stream fills the
    queue many times over and queued pairs of one chunk are evaluated with the next chunk's."""
    s = W.vapor_only_box(1000, 12.0, 12.0, 1.0, seed=41)
    with flat_sim([s], precision) as sim:
        check_forces(sim, [s], precision, tol)
        sim.step(20)
        check_forces(sim, [s], precision, tol)


def test_flat_stream_empty_replica_single_molecule_and_small_cylinder():
    s_empty = W.make_system("b", 9.0, 9.0, 12.0, 2.0, [W.Pore(W.PORE_CYLINDER, r0=2.0)], 0, 1.0, 6)
    s_one = W.make_system("c", 9.0, 9.0, 12.0, 2.0, [W.Pore(W.PORE_INKBOTTLE, r0=1.5, r_cavity=1.9)],
                          1, 1.0, 7)
    systems = [W.cylinder_pore_1k(), s_empty, s_one]
    for precision, tol in PRECS:
        with flat_sim(systems, precision) as sim:
            for r, s in enumerate(systems):
                if s.n_vapor == 0:
                    continue
                x, _ = sim.state(r)
                g, _, _ = oracle.forces(oracle.make_params(s, POT), x, s.wall, method=1)
                f = sim.forces(r)
                if not np.any(g):
                    assert not np.any(f)
                elif precision == md.MD_PREC_MIXED:
                    assert rms_rel_err(f, g) <= tol
                else:
                    assert force_err(f, g) <= tol
            sim.step(5)


def test_flat_stream_net_force_vanishes_without_walls():
    """Newton's third law: every pair adds +p to its owner and -p to its partner, so in a
    wall-free box the net force vanishes to rounding."""
    s = W.vapor_only_box(6000, 36.0, 36.0, 1.0, seed=9)
    for precision in (md.MD_PREC_FP64, md.MD_PREC_DF64):
        with flat_sim([s], precision) as sim:
            f = sim.forces(0)
            assert np.abs(f.sum(0)).max() <= 1e-13 * np.abs(f).sum()


def test_flat_stream_needs_the_atomic_form(shapes):
    with md.Simulation(shapes) as sim:
        sim.set_tuning(force_accumulate=1)
        with pytest.raises(md.MDError):
            sim.set_tuning(force_tpp=FLAT)
        sim.set_tuning(force_accumulate=2, force_tpp=FLAT)
        with pytest.raises(md.MDError):
            sim.set_tuning(force_accumulate=1)
        assert sim.tuning()["force_accumulate"] == 2


def test_flat_stream_agrees_with_the_per_molecule_atomic_kernel(shapes):
    """The same FP64 pair terms summed in another order: within a few ulps of the force scale."""
    with md.Simulation(shapes) as a, flat_sim(shapes, md.MD_PREC_FP64) as b:
        a.set_tuning(force_accumulate=2, force_tpp=2)
        for r in range(len(shapes)):
            assert force_err(b.forces(r), a.forces(r)) <= 1e-13


@pytest.mark.parametrize("precision,tol", PRECS)
def test_switching_from_the_flat_stream_to_a_per_molecule_kernel(shapes, precision, tol):
    """The flat stream's rebuilds keep no processing order: switching to a kernel that walks the
    length-ordered molecules rebuilds the lists (and the order) first."""
    with flat_sim(shapes, precision) as sim:
        sim.step(40)
        assert sim.observables(0)[0]["n_rebuilds"] >= 2
        sim.set_tuning(force_tpp=4, order_by_length=1)
        check_forces(sim, shapes, precision, tol)
        sim.step(5)
        check_forces(sim, shapes, precision, tol)
