"""CUDA path (through the C ABI) against the FP64 CPU oracle on identical seeded inputs.

Tolerances (FP64 path): per-step forces max_i |F_gpu - F_oracle| / RMS(F) <= 1e-10; 10-step
trajectories |dr|, |dv| <= 1e-8; energies relative 1e-10; integer observables (pair counts,
occupancy, adsorbed counts, density profiles) exactly equal. Mixed path: RMS force error
sqrt(sum |dF|^2 / sum |F|^2) <= 1e-5.
"""
import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.Potential()
FORCE_TOL = 1e-10
TRAJ_TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def built():
    mdbuild.build()
    md.load_library()


def oracle_params(s, pot=POT, **over):
    return oracle.make_params(s, pot, **over)


def force_err(f, g):
    rms = np.sqrt((g ** 2).sum(1).mean())
    return np.abs(f - g).max() / rms


def rms_rel_err(f, g):
    return np.sqrt(((f - g) ** 2).sum() / (g ** 2).sum())


def wrapped_diff(a, b, s):
    d = a - b
    d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
    d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
    return d


def check_observables(sim, r, s, st, pot=POT):
    o, occ, ads, prof = sim.observables(r)
    p = oracle_params(s, pot)
    f, d2, stats = oracle.forces(p, st.x, st.wall, method=1)
    occ_o, ads_o, prof_o = oracle.observables(p, s.pores, st.x, d2)
    assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]
    np.testing.assert_array_equal(occ, occ_o)
    np.testing.assert_array_equal(ads, ads_o)
    np.testing.assert_array_equal(prof, prof_o)
    pe_o = stats["pe_vv"] + stats["pe_vw"]
    assert o["pe"] == pytest.approx(pe_o, rel=1e-10, abs=1e-10)
    assert o["pe_vw"] == pytest.approx(stats["pe_vw"], rel=1e-10, abs=1e-10)
    assert o["virial_vv"] == pytest.approx(stats["vir_vv"], rel=1e-10, abs=1e-10)
    assert o["virial_vw"] == pytest.approx(stats["vir_vw"], rel=1e-10, abs=1e-10)
    assert o["ke"] == pytest.approx(oracle.kinetic(p, st.v), rel=1e-12)
    wv = oracle.molecule_virials(p, st.x, st.wall, nthreads=0)
    np.testing.assert_allclose(o["pore_pressure"], oracle.pore_pressure(p, s.pores, st.x, st.v, wv),
                               rtol=1e-9, atol=1e-12)
    return o


# ------------------------------------------------------------------------------------------ FP64


def test_initial_forces_small_cylinder():
    s = W.cylinder_pore_1k()
    with md.Simulation(s) as sim:
        f = sim.forces()
    g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
    assert force_err(f, g) <= FORCE_TOL


def test_ten_step_trajectory_small_cylinder_with_thermostat():
    s = W.cylinder_pore_1k()
    st = oracle.State(oracle_params(s), s.x0, s.v0, s.wall)
    with md.Simulation(s) as sim:
        sim.step(10)                     # the thermostat acts on step 10
        x, v = sim.state()
        f = sim.forces()
        st.run(10)
        assert np.abs(wrapped_diff(x, st.x, s)).max() <= TRAJ_TOL
        assert np.abs(v - st.v).max() <= TRAJ_TOL
        assert force_err(f, st.f) <= 1e-8
        o = check_observables(sim, 0, s, st)
        assert o["step"] == 10


def test_per_step_energy_record_small_cylinder():
    s = W.cylinder_pore_1k()
    st = oracle.State(oracle_params(s), s.x0, s.v0, s.wall)
    with md.Simulation(s) as sim:
        for k in range(12):
            sim.step(1)
            ke, pe = st.run(1)
            o, *_ = sim.observables()
            assert o["pe"] == pytest.approx(pe[0], rel=1e-9)
            # the library reports after the thermostat, the oracle log before it
            if (k + 1) % 10:
                assert o["ke"] == pytest.approx(ke[0], rel=1e-9)


@pytest.fixture(scope="module")
def shapes():
    return W.pore_shape_systems_20k()


def test_four_pore_shapes_batched_forces(shapes):
    with md.Simulation(shapes) as sim:
        for r, s in enumerate(shapes):
            g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
            assert force_err(sim.forces(r), g) <= FORCE_TOL, s.name


def test_four_pore_shapes_batched_trajectory_and_observables(shapes):
    states = [oracle.State(oracle_params(s), s.x0, s.v0, s.wall) for s in shapes]
    with md.Simulation(shapes) as sim:
        sim.step(10)
        for r, (s, st) in enumerate(zip(shapes, states)):
            st.run(10)
            x, v = sim.state(r)
            assert np.abs(wrapped_diff(x, st.x, s)).max() <= TRAJ_TOL, s.name
            assert np.abs(v - st.v).max() <= TRAJ_TOL, s.name
            check_observables(sim, r, s, st)


@pytest.fixture(scope="module")
def shapes_after_ten(shapes):
    states = [oracle.State(oracle_params(s), s.x0, s.v0, s.wall) for s in shapes]
    for st in states:
        st.run(10)
    return states


@pytest.mark.parametrize("tpp,block,lpt,acc", [
    (1, 128, 1, 1), (2, 256, 1, 1), (4, 128, 2, 1), (8, 256, 1, 1), (32, 128, 1, 1),
    (32, 256, 1, 1), (32, 128, 2, 1), (1, 256, 1, 2), (2, 128, 1, 2), (4, 256, 2, 2),
    (8, 128, 1, 2), (32, 256, 1, 2), (32, 128, 2, 2), (16, 256, 1, 1), (16, 128, 1, 2)])
def test_every_fp64_launch_shape_matches_oracle(shapes, shapes_after_ten, tpp, block, lpt, acc):
    """Every pair-kernel variant (lanes per molecule, the packed kernel, block size, processing
    order, deterministic or atomic accumulation) gives the oracle's forces and 10-step
    trajectories, pair counts and observables."""
    with md.Simulation(shapes) as sim:
        sim.set_tuning(force_tpp=tpp, force_block=block, force_blocks_per_sm=2, order_by_length=lpt,
                       force_accumulate=acc)
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


@pytest.mark.parametrize("precision,tol", [(md.MD_PREC_FP64, FORCE_TOL), (md.MD_PREC_DF64, FORCE_TOL),
                                           (md.MD_PREC_MIXED, 1e-5)])
@pytest.mark.parametrize("tpp,lpt", [(1, 1), (2, 1), (4, 2), (16, 1)])
def test_static_chunk_walk_matches_oracle(shapes, shapes_after_ten, precision, tol, tpp, lpt):
    """The static round-robin chunk walk of the atomic list kernels (the next chunk's molecule
    prefetched) covers every molecule once: the oracle's forces and pair counts, and in FP64 and
    double-float the 10-step trajectories."""
    with md.Simulation(shapes, precision=precision) as sim:
        sim.set_tuning(force_accumulate=2, force_tpp=tpp, order_by_length=lpt, chunk_walk=2,
                       force_blocks_per_sm=2)
        assert sim.tuning()["chunk_walk"] == 2
        sim.compute_forces()
        for r, s in enumerate(shapes):
            g, _, stats = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
            f = sim.forces(r)
            if precision == md.MD_PREC_MIXED:
                assert rms_rel_err(f, g) <= tol, s.name
            else:
                assert force_err(f, g) <= tol, s.name
            o = sim.observables(r)[0]
            assert (o["pairs_vv"], o["pairs_vw"]) == (stats["pairs_vv"], stats["pairs_vw"])
        sim.step(10)
        if precision != md.MD_PREC_MIXED:
            for r, (s, st) in enumerate(zip(shapes, shapes_after_ten)):
                x, v = sim.state(r)
                assert np.abs(wrapped_diff(x, st.x, s)).max() <= TRAJ_TOL, s.name


def test_atomic_accumulation_agrees_with_deterministic_to_rounding(shapes):
    """The atomic form sums the same FP64 pair forces in another order: forces agree to a few
    ulps of the force scale, trajectories over 20 steps to round-off growth."""
    with md.Simulation(shapes) as a, md.Simulation(shapes) as b:
        b.set_tuning(force_accumulate=2)
        for r in range(len(shapes)):
            assert force_err(b.forces(r), a.forces(r)) <= 1e-13
        a.step(20)
        b.step(20)
        for r, s in enumerate(shapes):
            xa, va = a.state(r)
            xb, vb = b.state(r)
            assert np.abs(wrapped_diff(xa, xb, s)).max() <= 1e-10
            assert np.abs(va - vb).max() <= 1e-10


@pytest.mark.parametrize("tpp", [2, 32])
def test_atomic_forms_agree_with_deterministic_on_a_filled_pore(tpp):
    """A liquid-filled pore (rows of 60-100 entries, the compacted kernel's queue flushing several
    times per warp): the atomic forms give the deterministic form's forces to rounding and keep the
    trajectory to round-off growth over 30 steps, with the same pair counts at the end."""
    s = W.drying_cylinder_pore()
    with md.Simulation(s) as a, md.Simulation(s) as b:
        b.set_tuning(force_accumulate=2, force_tpp=tpp)
        assert force_err(b.forces(), a.forces()) <= 1e-13
        g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
        assert force_err(b.forces(), g) <= FORCE_TOL
        a.step(30)
        b.step(30)
        xa, va = a.state()
        xb, vb = b.state()
        assert np.abs(wrapped_diff(xa, xb, s)).max() <= 1e-9
        assert np.abs(va - vb).max() <= 1e-9
        oa, *_ = a.observables()
        ob, *_ = b.observables()
        assert oa["pairs_vv"] == ob["pairs_vv"] and oa["pairs_vw"] == ob["pairs_vw"]


@pytest.mark.parametrize("tpp", [1, 2, 4, 8, 16])
def test_mixed_atomic_half_list_matches_oracle(shapes, shapes_after_ten, tpp):
    """The mixed form with atomic reaction forces (each vapour pair once): RMS force error <= 1e-5
    against the oracle and close to the full-list mixed form; 10-step trajectories and the
    integer observables as the other mixed tests."""
    with md.Simulation(shapes, precision=md.MD_PREC_MIXED) as a, \
            md.Simulation(shapes, precision=md.MD_PREC_MIXED) as b:
        b.set_tuning(force_accumulate=2, force_tpp=tpp)
        assert b.tuning()["force_accumulate"] == 2
        for r, s in enumerate(shapes):
            g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
            fb = b.forces(r)
            assert rms_rel_err(fb, g) <= 1e-5
            assert rms_rel_err(fb, a.forces(r)) <= 2e-6
        b.step(10)
        for r, (s, st) in enumerate(zip(shapes, shapes_after_ten)):
            x, v = b.state(r)
            assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-5
            assert np.abs(v - st.v).max() <= 1e-4
            o, occ, ads, prof = b.observables(r)
            assert o["step"] == 10
            # half rows: the observable pass meets each vapour pair once and hands the partner its
            # halves -- the pair counts are exact, energies and virial within FP32 pair terms
            g, d2, stats = oracle.forces(oracle_params(s), x, s.wall, method=1)
            assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]
            assert o["pe"] == pytest.approx(stats["pe_vv"] + stats["pe_vw"], rel=1e-5)
            assert o["virial_vv"] == pytest.approx(stats["vir_vv"], rel=1e-4)


def test_all_pairs_method_small_cylinder():
    """The paper's F1 form (every pair each step, no lists): forces, 10-step trajectory with the
    thermostat, pair counts and observables equal the oracle's; switching back to lists gives the
    same forces."""
    s = W.cylinder_pore_1k()
    st = oracle.State(oracle_params(s), s.x0, s.v0, s.wall)
    with md.Simulation(s) as sim:
        sim.set_tuning(pair_method=2)
        assert sim.tuning()["pair_method"] == 2
        g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=0)
        assert force_err(sim.forces(), g) <= FORCE_TOL
        sim.step(10)
        st.run(10)
        x, v = sim.state()
        assert np.abs(wrapped_diff(x, st.x, s)).max() <= TRAJ_TOL
        assert np.abs(v - st.v).max() <= TRAJ_TOL
        check_observables(sim, 0, s, st)
        f_all = sim.forces()
        sim.set_tuning(pair_method=1)
        assert force_err(sim.forces(), f_all) <= 1e-13
    with md.Simulation(s, precision=md.MD_PREC_MIXED) as m, pytest.raises(md.MDError):
        m.set_tuning(pair_method=2)


def test_all_pairs_method_four_shapes(shapes):
    with md.Simulation(shapes) as sim:
        sim.set_tuning(pair_method=2, use_graph=2)
        for r, s in enumerate(shapes):
            g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
            assert force_err(sim.forces(r), g) <= FORCE_TOL, s.name
        sim.step(3)
        o, *_ = sim.observables(0)
        assert o["step"] == 3


def test_whole_context_transfers_match_per_replica(shapes):
    """replica -1 reads and writes every replica at once, concatenated in replica order."""
    with md.Simulation(shapes) as sim:
        sim.step(7)
        x, v = sim.state(-1)
        f = sim.forces(-1)
        per = [sim.state(r) for r in range(len(shapes))]
        np.testing.assert_array_equal(x, np.concatenate([p[0] for p in per]))
        np.testing.assert_array_equal(v, np.concatenate([p[1] for p in per]))
        np.testing.assert_array_equal(f, np.concatenate([sim.forces(r) for r in range(len(shapes))]))
        h0, d0 = sim.transfer_bytes()
        sim.set_state(-1, x, v)
        h1, _ = sim.transfer_bytes()
        assert h1 - h0 >= 48 * len(x)
        x2, v2 = sim.state(-1)
        np.testing.assert_array_equal(x2, x)
        np.testing.assert_array_equal(v2, v)
        # forces re-evaluated at the same positions (the lists kept): equal to rounding
        assert force_err(sim.forces(-1), f) <= 1e-13
        bad = x.copy()
        bad[len(shapes[0].x0) + 5, 2] = 1e3
        with pytest.raises(md.MDError):
            sim.set_state(-1, bad, v)
        np.testing.assert_array_equal(sim.state(-1)[0], x)  # untouched by the rejected call
        with pytest.raises(ValueError):
            sim.set_state(-1, x[:-1], v[:-1])


def test_generated_wall_matches_generator(shapes):
    with md.Simulation(shapes, generate_wall=True) as sim:
        for r, s in enumerate(shapes):
            w = sim.wall(r)
            a = w[np.lexsort(w.T[::-1])]
            b = s.wall[np.lexsort(s.wall.T[::-1])]
            np.testing.assert_array_equal(a, b)


def test_graph_replay_is_bitwise_identical_to_plain_launches():
    s = W.cylinder_pore_1k()
    with md.Simulation(s) as a, md.Simulation(s) as b:
        a.set_tuning(use_graph=2)
        b.set_tuning(use_graph=1, steps_per_graph=5)
        a.step(23)
        b.step(23)
        xa, va = a.state()
        xb, vb = b.state()
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)


def test_runs_are_deterministic():
    s = W.cylinder_pore_1k()
    out = []
    for _ in range(2):
        with md.Simulation(s) as sim:
            sim.step(60)
            out.append(sim.state())
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_set_state_round_trip_and_restart_parity():
    s = W.cylinder_pore_1k()
    with md.Simulation(s) as sim:
        sim.step(7)
        x, v = sim.state()
        sim.set_state(0, x, v)
        x2, v2 = sim.state()
        np.testing.assert_array_equal(x, x2)
        np.testing.assert_array_equal(v, v2)
        st = oracle.State(oracle_params(s), x, v, s.wall)
        st.step = 7
        sim.step(6)
        st.run(6)
        x3, v3 = sim.state()
        assert np.abs(wrapped_diff(x3, st.x, s)).max() <= TRAJ_TOL


def test_rejected_state_names_the_row_and_leaves_the_context_unchanged(shapes):
    """md_set_state checks the rows on the device before loading: a position outside the box (or
    NaN), or a velocity component that is not finite, anywhere in a whole-context load is reported
    with its replica and molecule, nothing is loaded, and the context steps on from where it
    was."""
    with md.Simulation(shapes) as sim, md.Simulation(shapes) as ref:
        sim.step(5)
        ref.step(5)
        x, v = sim.state(-1)
        n0 = shapes[0].n_vapor
        for bad_value, row in ((shapes[2].Lz, n0 + shapes[1].n_vapor + 17), (np.nan, 3)):
            xb = x.copy()
            xb[row, 2] = bad_value
            with pytest.raises(md.MDError, match="outside the box") as err:
                sim.set_state(-1, xb, v)
            rr = 0 if row < n0 else 2
            first = 0 if rr == 0 else n0 + shapes[1].n_vapor
            assert f"replica {rr}: molecule {row - first} " in str(err.value)
        for bad_value in (np.inf, np.nan):   # a velocity component that is not finite
            vb = v.copy()
            vb[n0 + 5, 1] = bad_value
            with pytest.raises(md.MDError, match="non-finite velocity") as err:
                sim.set_state(-1, x, vb)
            assert "replica 1: molecule 5 " in str(err.value)
        x2, v2 = sim.state(-1)
        np.testing.assert_array_equal(x2, x)
        np.testing.assert_array_equal(v2, v)
        sim.step(5)
        ref.step(5)
        for r, s in enumerate(shapes):
            xa, va = sim.state(r)
            xb_, vb = ref.state(r)
            assert np.abs(wrapped_diff(xa, xb_, s)).max() <= 1e-10
            assert np.abs(va - vb).max() <= 1e-10


def place_on(s, axis, value):
    """Move some molecule onto the plane x[axis] = value without creating a close pair."""
    for i in range(s.n_vapor):
        c = s.x0[i].copy()
        c[axis] = value
        d = s.x0 - c
        d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
        d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
        r = np.sqrt((d ** 2).sum(1))
        r[i] = np.inf
        if r.min() > 0.9:
            s.x0[i] = c
            return i
    raise AssertionError("no molecule could be placed")


def test_edge_cases_batch_empty_single_and_wall_free():
    s_norm = W.make_system("a", 12.0, 12.0, 20.0, 3.0, [W.Pore(W.PORE_SLIT, width=3.0)], 300, 1.0, 5)
    s_empty = W.make_system("b", 9.0, 9.0, 12.0, 2.0, [W.Pore(W.PORE_CYLINDER, r0=2.0)], 0, 1.0, 6)
    s_one = W.make_system("c", 9.0, 9.0, 12.0, 2.0, [W.Pore(W.PORE_INKBOTTLE, r0=1.5, r_cavity=1.9)],
                          1, 1.0, 7)
    s_free = W.vapor_only_box(400, 10.0, 14.0, 1.2, seed=8)
    # molecules exactly on cell faces and on the periodic edge of the wall-free box
    place_on(s_free, 0, -5.0)
    place_on(s_free, 1, -5.0 + 10.0 / 3.0)
    systems = [s_norm, s_empty, s_one, s_free]
    states = [oracle.State(oracle_params(s), s.x0, s.v0, s.wall) for s in systems]
    with md.Simulation(systems) as sim:
        for r, (s, st) in enumerate(zip(systems, states)):
            if s.n_vapor:
                f = sim.forces(r)
                if np.abs(st.f).max() == 0:      # an isolated molecule: exactly no force
                    assert np.abs(f).max() == 0, s.name
                else:
                    assert force_err(f, st.f) <= FORCE_TOL, s.name
        sim.step(15)
        for r, (s, st) in enumerate(zip(systems, states)):
            st.run(15)
            x, v = sim.state(r)
            assert x.shape == (s.n_vapor, 3)
            if s.n_vapor:
                assert np.abs(wrapped_diff(x, st.x, s)).max() <= TRAJ_TOL, s.name
                assert np.abs(v - st.v).max() <= TRAJ_TOL, s.name
            o, occ, ads, prof = sim.observables(r)
            assert prof.sum() == s.n_vapor


@pytest.mark.parametrize("precision", [md.MD_PREC_FP64, md.MD_PREC_MIXED])
def test_list_overflow_is_reported(precision):
    s = W.cylinder_pore_1k()
    with pytest.raises(md.MDError) as ei:
        md.Simulation(s, precision=precision, max_neighbors=2, max_wall_neighbors=2)
    assert ei.value.status == md.MD_EOVERFLOW


def test_unstable_motion_is_reported_and_sticky():
    s = W.make_system("u", 12.0, 12.0, 20.0, 3.0, [W.Pore(W.PORE_CYLINDER, r0=3.0)], 10, 1.0, 1)
    s.x0[0] = [0.0, 0.0, 8.0]
    s.x0[1] = [0.3, 0.0, 8.0]                            # nearly overlapping pair
    with md.Simulation(s) as sim:
        sim.step(2)
        with pytest.raises(md.MDError) as ei:
            sim.sync()
        assert ei.value.status == md.MD_EUNSTABLE
        with pytest.raises(md.MDError):
            sim.step(1)


def test_rebuilds_happen_and_lists_stay_complete():
    """A long run: the device-decided rebuilds keep forces exact against a fresh oracle evaluation."""
    s = W.cylinder_pore_1k()
    with md.Simulation(s) as sim:
        sim.step(400)
        x, _ = sim.state()
        f = sim.forces()
        o, *_ = sim.observables()
    assert o["n_rebuilds"] > 3
    g, _, stats = oracle.forces(oracle_params(s), x, s.wall, method=1)
    assert force_err(f, g) <= FORCE_TOL
    assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]


@pytest.mark.parametrize("precision,acc", [(md.MD_PREC_FP64, 1), (md.MD_PREC_FP64, 2),
                                           (md.MD_PREC_MIXED, 2), (md.MD_PREC_DF64, 2)])
def test_rebuild_lists_alone_keeps_the_state_and_the_run_goes_on(shapes, precision, acc):
    """md_rebuild_lists (the chain the bench times) moves records, not values: state and forces
    read back bit for bit; the next force evaluation on the new lists matches the oracle, the
    rebuild is counted, and stepping goes on with forces exact against the oracle."""
    s = shapes[:2]
    tol = FORCE_TOL if precision != md.MD_PREC_MIXED else None
    with md.Simulation(s, precision=precision) as sim:
        sim.set_tuning(force_accumulate=acc)
        sim.step(30)
        x0, v0 = sim.state(-1)
        f0 = sim.forces(-1)
        n0 = sim.observables(0)[0]["n_rebuilds"]
        sim.rebuild_lists()
        x1, v1 = sim.state(-1)
        np.testing.assert_array_equal(x1, x0)
        np.testing.assert_array_equal(v1, v0)
        np.testing.assert_array_equal(sim.forces(-1), f0)
        assert sim.observables(0)[0]["n_rebuilds"] == n0 + 1
        sim.compute_forces()
        f2 = sim.forces(-1)
        sim.step(20)
        x3, _ = sim.state(-1)
        f3 = sim.forces(-1)
    k = 0
    for r, sr in enumerate(s):
        n = sr.n_vapor
        for xs, fs in ((x0, f2), (x3, f3)):
            g, _, _ = oracle.forces(oracle_params(sr), xs[k:k + n], sr.wall, method=1)
            if tol is None:
                assert rms_rel_err(fs[k:k + n], g) <= 1e-5
            else:
                assert force_err(fs[k:k + n], g) <= tol
        k += n


def test_rebuild_lists_is_refused_in_the_all_pairs_mode():
    with md.Simulation(W.cylinder_pore_1k()) as sim:
        sim.set_tuning(pair_method=2)
        with pytest.raises(md.MDError) as ei:
            sim.rebuild_lists()
        assert ei.value.status == md.MD_EINVAL


# ------------------------------------------------------------------------------------------ mixed


def test_mixed_precision_force_error_small_cylinder():
    s = W.cylinder_pore_1k()
    with md.Simulation(s, precision=md.MD_PREC_MIXED) as sim:
        f = sim.forces()
        g, d2, stats = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
        assert rms_rel_err(f, g) <= 1e-5
        # borderline cutoffs and wall distances are decided in FP64: integer results are exact
        o, occ, ads, prof = sim.observables()
        assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]
        _, ads_o, _ = oracle.observables(oracle_params(s), s.pores, s.x0, d2)
        np.testing.assert_array_equal(ads, ads_o)
        st = oracle.State(oracle_params(s), s.x0, s.v0, s.wall)
        errs = []
        for _ in range(10):
            sim.step(1)
            st.run(1)
            x, _ = sim.state()
            g2, _, _ = oracle.forces(oracle_params(s), x, s.wall, method=1)
            errs.append(rms_rel_err(sim.forces(), g2))
        assert max(errs) <= 1e-5


def test_mixed_precision_four_shapes(shapes):
    with md.Simulation(shapes, precision=md.MD_PREC_MIXED) as sim:
        for r, s in enumerate(shapes):
            g, _, _ = oracle.forces(oracle_params(s), s.x0, s.wall, method=1)
            assert rms_rel_err(sim.forces(r), g) <= 1e-5, s.name


def test_mixed_precision_error_after_equilibration(shapes):
    """Hundreds of steps in (condensed, adsorbed layers): the mixed RMS force error against the
    oracle at the mixed run's own positions stays below 1e-5."""
    with md.Simulation(shapes, precision=md.MD_PREC_MIXED) as sim:
        sim.set_tuning(use_graph=1, steps_per_graph=10)
        sim.step(300)
        for r, s in enumerate(shapes):
            x, _ = sim.state(r)
            g, _, stats = oracle.forces(oracle_params(s), x, s.wall, method=1)
            assert rms_rel_err(sim.forces(r), g) <= 1e-5, s.name
            o, *_ = sim.observables(r)
            assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]


@pytest.mark.parametrize("precision", [md.MD_PREC_FP64, md.MD_PREC_MIXED])
def test_atomic_forms_graph_and_plain_launches_agree(shapes, precision):
    """The atomic forms defer each step's second half-kick into the next first half-kick and pay
    it before thermostat steps and reads; graph replays (conditional nodes) and plain launches
    take the same steps, so they agree to rounding over 70 steps with 7 thermostat steps."""
    with md.Simulation(shapes, precision=precision) as a, \
            md.Simulation(shapes, precision=precision) as b:
        a.set_tuning(force_accumulate=2, use_graph=2)
        b.set_tuning(force_accumulate=2, use_graph=1, steps_per_graph=7)
        a.step(70)
        b.step(70)
        for r, s in enumerate(shapes):
            xa, va = a.state(r)
            xb, vb = b.state(r)
            assert np.abs(wrapped_diff(xa, xb, s)).max() <= 1e-9
            assert np.abs(va - vb).max() <= 1e-9
            oa, *_ = a.observables(r)
            ob, *_ = b.observables(r)
            assert oa["ke"] == pytest.approx(ob["ke"], rel=1e-10)


def test_graph_with_conditional_rebuilds_matches_plain_launches_fp64_long():
    shapes4 = W.pore_shape_systems_20k()
    with md.Simulation(shapes4) as a, md.Simulation(shapes4) as b:
        a.set_tuning(use_graph=2)
        b.set_tuning(use_graph=1, steps_per_graph=7)
        a.step(70)
        b.step(70)
        oa, *_ = a.observables(0)
        ob, *_ = b.observables(0)
        assert oa["n_rebuilds"] == ob["n_rebuilds"] > 1
        for r in range(4):
            xa, va = a.state(r)
            xb, vb = b.state(r)
            np.testing.assert_array_equal(xa, xb)
            np.testing.assert_array_equal(va, vb)
        # skipped conditional branches launch nothing
        assert b.kernel_launches() < a.kernel_launches()


# ------------------------------------------------------------------------------------------ large


@pytest.mark.parametrize("precision,tol", [(md.MD_PREC_FP64, FORCE_TOL), (md.MD_PREC_MIXED, 1e-5)])
def test_large_cylinder_forces(precision, tol):
    """200,000 molecules and ~1.33 M wall atoms: every force against the oracle."""
    s = W.cylinder_pore_200k()
    g, _, stats = oracle.forces(oracle_params(s), s.x0, s.wall, method=1, nthreads=0)
    with md.Simulation(s, precision=precision) as sim:
        f = sim.forces()
        o, *_ = sim.observables()
    err = force_err(f, g) if precision == md.MD_PREC_FP64 else rms_rel_err(f, g)
    assert err <= tol
    assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]
