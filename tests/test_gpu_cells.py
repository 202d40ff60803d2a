"""The cell-tiled pair kernel (pair_method 3: no Verlet lists) against the FP64 oracle.

Each warp stages the FP32 offsets of a chunk's neighbour cells in shared memory, screens every
staged candidate in FP32, queues the pairs that may lie within the cutoff and evaluates them with
every lane busy, deciding the cutoff in FP64 near rc. The pair set must be the oracle's exactly
(pair counts equal) and the forces within the parity bars of the list forms: FP64 and
double-float 1e-10 of the RMS force per step and 1e-8 over ten-step trajectories, mixed 1e-5 RMS.
Workloads: the small cylinder, the four 20k pore shapes (one context), an uneven batch, a dense
liquid box whose chunks must shrink to fit the staging, the paper's hard-wall pores (3D and planar),
an empty replica and a single molecule.
"""
import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.Potential()
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


def cells_sim(systems, precision, **kw):
    sim = md.Simulation(systems, precision=precision, **kw)
    sim.set_tuning(pair_method=3)
    assert sim.tuning()["pair_method"] == 3
    return sim


def check_forces(sim, systems, precision, tol):
    for r, s in enumerate(systems):
        x, _ = sim.state(r)
        g, _, stats = oracle.forces(oracle.make_params(s, POT), x, s.wall, method=1, nthreads=0)
        f = sim.forces(r)
        if precision == md.MD_PREC_MIXED:
            assert rms_rel_err(f, g) <= tol, s.name
        else:
            assert force_err(f, g) <= tol, s.name
        o = sim.observables(r)[0]
        assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"], s.name


@pytest.fixture(scope="module")
def shapes():
    return W.pore_shape_systems_20k()


@pytest.mark.parametrize("precision,tol", PRECS)
def test_initial_forces_and_pairs_small_cylinder_and_shapes(shapes, precision, tol):
    for systems in ([W.cylinder_pore_1k()], shapes):
        with cells_sim(systems, precision) as sim:
            check_forces(sim, systems, precision, tol)


@pytest.mark.parametrize("precision", [md.MD_PREC_FP64, md.MD_PREC_DF64])
def test_ten_step_trajectories_and_observables(shapes, precision):
    systems = [W.cylinder_pore_1k()] + shapes
    states = [oracle.State(oracle.make_params(s, POT), s.x0, s.v0, s.wall, nthreads=0)
              for s in systems]
    with cells_sim(systems, precision) as sim:
        sim.step(10)
        for r, (s, st) in enumerate(zip(systems, states)):
            st.run(10)
            x, v = sim.state(r)
            assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-8, s.name
            assert np.abs(v - st.v).max() <= 1e-8, s.name
            p = oracle.make_params(s, POT)
            o, occ, ads, prof = sim.observables(r)
            g, d2, stats = oracle.forces(p, st.x, s.wall, method=1, nthreads=0)
            occ_o, ads_o, prof_o = oracle.observables(p, s.pores, st.x, d2)
            assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]
            np.testing.assert_array_equal(occ, occ_o)
            np.testing.assert_array_equal(ads, ads_o)
            np.testing.assert_array_equal(prof, prof_o)
            assert o["pe"] == pytest.approx(stats["pe_vv"] + stats["pe_vw"], rel=1e-10, abs=1e-10)
            assert o["virial_vv"] == pytest.approx(stats["vir_vv"], rel=1e-10, abs=1e-10)
            assert o["virial_vw"] == pytest.approx(stats["vir_vw"], rel=1e-10, abs=1e-10)


def test_mixed_ten_steps_and_observables(shapes):
    """Mixed precision: forces within 1e-5 RMS along the trajectory; the observable pass runs in
    FP64 at the mixed trajectory's positions, so its integer observables equal the oracle's at
    those positions."""
    with cells_sim(shapes, md.MD_PREC_MIXED) as sim:
        sim.step(10)
        for r, s in enumerate(shapes):
            x, _ = sim.state(r)
            p = oracle.make_params(s, POT)
            g, d2, stats = oracle.forces(p, x, s.wall, method=1, nthreads=0)
            assert rms_rel_err(sim.forces(r), g) <= 1e-5
            o, occ, ads, prof = sim.observables(r)
            occ_o, ads_o, prof_o = oracle.observables(p, s.pores, x, d2)
            assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]
            np.testing.assert_array_equal(ads, ads_o)
            np.testing.assert_array_equal(prof, prof_o)


@pytest.mark.parametrize("precision,tol", PRECS)
def test_uneven_batch_after_rebuilds(precision, tol):
    """Twelve uneven replicas through 120 steps (several per-replica cell rebuilds): forces at the
    final positions against the oracle and exact pair counts."""
    batch = W.replica_batch(n_replicas=12, n_max=20000)
    with cells_sim(batch, precision) as sim:
        sim.step(120)
        assert sim.observables(0)[0]["n_rebuilds"] >= 3
        check_forces(sim, batch, precision, tol)


@pytest.mark.parametrize("precision,tol", PRECS)
def test_dense_liquid_chunks_shrink_to_the_staging(precision, tol):
    """A wall-free box at density ~0.58 (about 16 molecules per cell): chunks of 32 molecules do
    not fit the per-warp staging and must be cut; every pair is still found once."""
    s = W.vapor_only_box(1000, 12.0, 12.0, 1.0, seed=41)
    with cells_sim([s], precision) as sim:
        check_forces(sim, [s], precision, tol)
        sim.step(20)
        check_forces(sim, [s], precision, tol)


@pytest.mark.parametrize("name", ["paper_prism_pore", "paper_pore_2d"])
def test_hard_wall_pores(name):
    s = getattr(W, name)()
    st = oracle.State(oracle.make_params(s, POT), s.x0, s.v0, s.wall, nthreads=0, pores=s.pores)
    with cells_sim([s], md.MD_PREC_FP64) as sim:
        sim.step(10)
        st.run(10)
        x, v = sim.state(0)
        assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-8
        assert np.abs(v - st.v).max() <= 1e-8


def test_empty_replica_single_molecule_and_faces():
    s_norm = W.make_system("a", 12.0, 12.0, 20.0, 3.0, [W.Pore(W.PORE_SLIT, width=3.0)], 300, 1.0, 5)
    s_empty = W.make_system("b", 9.0, 9.0, 12.0, 2.0, [W.Pore(W.PORE_CYLINDER, r0=2.0)], 0, 1.0, 6)
    s_one = W.make_system("c", 9.0, 9.0, 12.0, 2.0, [W.Pore(W.PORE_INKBOTTLE, r0=1.5, r_cavity=1.9)],
                          1, 1.0, 7)
    # molecules on the periodic edge and on cell faces of the 12 x 12 box (cells of 3.0)
    for i, (axis, value) in zip(range(0, 300, 37), [(0, -6.0), (1, -6.0), (0, 0.0), (1, 3.0),
                                                      (0, -3.0), (1, 0.0), (0, 3.0), (1, -3.0)]):
        c = s_norm.x0[i].copy()
        c[axis] = value
        d = wrapped_diff(s_norm.x0 - c, np.zeros(3), s_norm)
        r = np.sqrt((d ** 2).sum(1))
        r[i] = np.inf
        if r.min() > 0.9:
            s_norm.x0[i] = c
    systems = [s_norm, s_empty, s_one]
    for precision, tol in PRECS:
        with cells_sim(systems, precision) as sim:
            for r, s in enumerate(systems):
                if s.n_vapor == 0:
                    continue
                x, _ = sim.state(r)
                g, _, stats = oracle.forces(oracle.make_params(s, POT), x, s.wall, method=1)
                f = sim.forces(r)
                if s.n_vapor == 1 and not np.any(g):
                    assert not np.any(f)
                elif precision == md.MD_PREC_MIXED:
                    assert rms_rel_err(f, g) <= tol
                else:
                    assert force_err(f, g) <= tol
            sim.step(5)


def test_net_force_vanishes_without_walls():
    """Newton's third law: in a wall-free box every reaction is the pair force's negative, so
    the net force vanishes to rounding, and x/y momentum holds over steps with rebuilds."""
    s = W.vapor_only_box(6000, 36.0, 36.0, 1.0, seed=9)
    with cells_sim([s], md.MD_PREC_FP64) as sim:
        f = sim.forces(0)
        assert np.abs(f.sum(0)).max() <= 1e-13 * np.abs(f).sum()
        _, v0 = sim.state(0)
        sim.set_tuning(steps_per_graph=10)
        sim.step(200)
        _, v1 = sim.state(0)
        p0, p1 = v0.sum(0), v1.sum(0)
        # the thermostat scales velocities (and momentum) by lambda: compare directions of x/y
        assert np.abs(p1[:2]).max() <= 1e-8 * np.abs(v1).sum() + 10 * np.abs(p0[:2]).max()


def test_switching_methods_keeps_the_state_and_forces(shapes):
    with md.Simulation(shapes) as sim:
        sim.step(15)
        x0, v0 = sim.state(-1)
        f_list = sim.forces(-1)
        sim.set_tuning(pair_method=3)
        x1, v1 = sim.state(-1)
        np.testing.assert_array_equal(x0, x1)
        np.testing.assert_array_equal(v0, v1)
        f_cells = sim.forces(-1)
        assert force_err(f_cells, f_list) <= 1e-12
        sim.set_tuning(pair_method=1)
        assert force_err(sim.forces(-1), f_list) <= 1e-12
        with pytest.raises(md.MDError):
            sim.set_tuning(pair_method=3, force_accumulate=1)


def test_autotune_may_choose_the_cell_method(shapes, tmp_path):
    with md.Simulation(shapes) as sim:
        sim.set_tuning(force_accumulate=2)
        x0, _ = sim.state(-1)
        t, us = sim.autotune(5)
        assert t["pair_method"] in (1, 3) and us > 0
        x1, _ = sim.state(-1)
        np.testing.assert_array_equal(x0, x1)
        for r, s in enumerate(shapes):
            g, _, _ = oracle.forces(oracle.make_params(s, POT), x1[r * 20000:(r + 1) * 20000],
                                    s.wall, method=1, nthreads=0)
            assert force_err(sim.forces(r), g) <= 1e-10
