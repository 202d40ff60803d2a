"""GPU parity on the batched and large workloads, and the autotuner.

* an uneven batch of pore systems (the four shapes, radii 2-10, 1,000-20,000 molecules, T* in
  [0.8, 1.2]) in one context: forces per replica (FP64 <= 1e-10 max/RMS, mixed RMS <= 1e-5),
  trajectories and observables;
* the 400 x 400 x 200 array of 16 pores with 2,000,000 molecules and ~6.2 M wall atoms: every
  force against the oracle, pair counts and the per-pore observables;
* the autotuner leaves positions unchanged and forces within tolerance;
* the drying of an initially filled pore with general Berendsen coupling: 10-step parity and the
  occupancy decay over 2,000 steps against the oracle's, over four seeds.
"""
import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import autotune
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


def rms_rel_err(f, g):
    return np.sqrt(((f - g) ** 2).sum() / (g ** 2).sum())


def wrapped_diff(a, b, s):
    d = a - b
    d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
    d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
    return d


@pytest.fixture(scope="module")
def batch():
    return W.replica_batch(n_replicas=12, n_max=20000)


def test_uneven_batch_forces_and_trajectories(batch):
    params = [oracle.make_params(s, POT) for s in batch]
    states = [oracle.State(p, s.x0, s.v0, s.wall, nthreads=0) for p, s in zip(params, batch)]
    with md.Simulation(batch) as sim:
        for r, (s, st) in enumerate(zip(batch, states)):
            assert force_err(sim.forces(r), st.f) <= 1e-10, s.name
        sim.step(10)
        for r, (s, st, p) in enumerate(zip(batch, states, params)):
            st.run(10)
            x, v = sim.state(r)
            assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-8, s.name
            assert np.abs(v - st.v).max() <= 1e-8, s.name
            o, occ, ads, prof = sim.observables(r)
            g, d2, stats = oracle.forces(p, st.x, s.wall, method=1, nthreads=0)
            occ_o, ads_o, prof_o = oracle.observables(p, s.pores, st.x, d2)
            assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]
            np.testing.assert_array_equal(occ, occ_o)
            np.testing.assert_array_equal(ads, ads_o)
            np.testing.assert_array_equal(prof, prof_o)


def test_uneven_batch_double_float(batch):
    """Double-float pair terms on twelve uneven replicas: the FP64 bars (forces 1e-10 of the RMS
    force, 10-step trajectories 1e-8, pair counts exact)."""
    params = [oracle.make_params(s, POT) for s in batch]
    states = [oracle.State(p, s.x0, s.v0, s.wall, nthreads=0) for p, s in zip(params, batch)]
    with md.Simulation(batch, precision=md.MD_PREC_DF64) as sim:
        for r, (s, st) in enumerate(zip(batch, states)):
            assert force_err(sim.forces(r), st.f) <= 1e-10, s.name
        sim.step(10)
        for r, (s, st, p) in enumerate(zip(batch, states, params)):
            st.run(10)
            x, v = sim.state(r)
            assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-8, s.name
            assert np.abs(v - st.v).max() <= 1e-8, s.name
            o, *_ = sim.observables(r)
            _, _, stats = oracle.forces(p, st.x, s.wall, method=1, nthreads=0)
            assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]


def test_uneven_batch_mixed_precision(batch):
    with md.Simulation(batch, precision=md.MD_PREC_MIXED) as sim:
        sim.step(20)
        for r, s in enumerate(batch):
            x, _ = sim.state(r)
            g, _, _ = oracle.forces(oracle.make_params(s, POT), x, s.wall, method=1, nthreads=0)
            assert rms_rel_err(sim.forces(r), g) <= 1e-5, s.name


def test_replica_batch_256_sampled_replicas_at_full_size():
    """The bench's batch workload at full size (256 replicas, 3.1 M vapour molecules, 16.8 M wall
    atoms) in its launch configuration (atomic reaction forces, autotuned launch shape): six
    replicas spread over the size range -- the smallest, the largest and four between -- against
    the oracle one by one, forces per step to the FP64 bar and pair counts exact after 10 steps;
    the double-float form alike, and the mixed form within its RMS bar."""
    batch = W.replica_batch()
    order = sorted(range(len(batch)), key=lambda r: batch[r].n_vapor)
    sample = [order[k] for k in (0, 51, 102, 153, 204, 255)]
    for precision in (md.MD_PREC_FP64, md.MD_PREC_DF64, md.MD_PREC_MIXED):
        with md.Simulation(batch, precision=precision) as sim:
            sim.set_tuning(force_accumulate=2)
            sim.autotune(3)
            sim.step(10)
            for r in sample:
                s = batch[r]
                x, _ = sim.state(r)
                p = oracle.make_params(s, POT)
                g, _, stats = oracle.forces(p, x, s.wall, method=1, nthreads=0)
                f = sim.forces(r)
                if precision == md.MD_PREC_MIXED:
                    assert rms_rel_err(f, g) <= 1e-5, (precision, s.name)
                else:
                    assert force_err(f, g) <= 1e-10, (precision, s.name)
                    o, *_ = sim.observables(r)
                    assert o["pairs_vv"] == stats["pairs_vv"], (precision, s.name)
                    assert o["pairs_vw"] == stats["pairs_vw"], (precision, s.name)


@pytest.mark.parametrize("precision,tol", [(md.MD_PREC_FP64, 1e-10), (md.MD_PREC_MIXED, 1e-5),
                                           (md.MD_PREC_DF64, 1e-10)])
def test_pore_array_2m_every_force_and_per_pore_observables(precision, tol):
    s = W.pore_array_2m()
    p = oracle.make_params(s, POT)
    g, d2, stats = oracle.forces(p, s.x0, s.wall, method=1, nthreads=0)
    with md.Simulation(s, precision=precision) as sim:
        f = sim.forces()
        o, occ, ads, prof = sim.observables()
    fp64_bar = precision != md.MD_PREC_MIXED   # the double-float form meets the FP64 bars
    err = force_err(f, g) if fp64_bar else rms_rel_err(f, g)
    assert err <= tol
    assert o["pairs_vv"] == stats["pairs_vv"] and o["pairs_vw"] == stats["pairs_vw"]
    occ_o, ads_o, prof_o = oracle.observables(p, s.pores, s.x0, d2)
    assert len(occ) == 16
    wv = oracle.molecule_virials(p, s.x0, s.wall, nthreads=0)
    P_o = oracle.pore_pressure(p, s.pores, s.x0, s.v0, wv)
    np.testing.assert_allclose(o["pore_pressure"], P_o,
                               rtol=1e-9 if fp64_bar else 1e-4, atol=1e-12)
    np.testing.assert_array_equal(occ, occ_o)
    np.testing.assert_array_equal(ads, ads_o)
    np.testing.assert_array_equal(prof, prof_o)


@pytest.mark.parametrize("precision", [md.MD_PREC_FP64, md.MD_PREC_MIXED, md.MD_PREC_DF64])
def test_autotune_keeps_state_and_forces(precision, tmp_path):
    shapes = W.pore_shape_systems_20k()
    with md.Simulation(shapes, precision=precision) as sim:
        sim.step(30)
        x0, v0 = sim.state(1)
        res = autotune.tune(sim, trials=3, cache_path=str(tmp_path / "t.json"))
        t = res["tuning"]
        packed = (32,) if precision == md.MD_PREC_FP64 else ()
        flat = (64,) if t["force_accumulate"] == 2 else ()  # the flat stream: atomic form only
        assert t["force_tpp"] in (1, 2, 4, 8, 16) + packed + flat
        assert 1 <= t["force_blocks_per_sm"] <= 8
        assert t["force_block"] in (128, 256) and t["order_by_length"] in (1, 2)
        assert res["us"] > 0 and not res["cached"]
        x1, v1 = sim.state(1)
        np.testing.assert_array_equal(x0, x1)
        np.testing.assert_array_equal(v0, v1)
        g, _, _ = oracle.forces(oracle.make_params(shapes[1], POT), x1, shapes[1].wall, method=1)
        f = sim.forces(1)
        if precision != md.MD_PREC_MIXED:
            assert force_err(f, g) <= 1e-10
        else:
            assert rms_rel_err(f, g) <= 1e-5
        again = autotune.tune(sim, cache_path=str(tmp_path / "t.json"))
        assert again["cached"] and again["tuning"] == t
        sim.step(5)


# ------------------------------------------------------------------ drying of a filled pore


def test_drying_run_ten_steps_general_berendsen():
    """A filled pore with Berendsen coupling tau_B = 0.5 (not plain rescaling): 10 steps, exact
    occupancy and adsorbed counts, trajectories within 1e-8 of the oracle."""
    s = W.drying_cylinder_pore()
    p = oracle.make_params(s, POT)
    st = oracle.State(p, s.x0, s.v0, s.wall)
    with md.Simulation(s) as sim:
        sim.step(10)
        st.run(10)
        x, v = sim.state()
        d = x - st.x
        d[:, :2] -= 40.0 * np.round(d[:, :2] / 40.0)
        assert np.abs(d).max() <= 1e-8
        assert np.abs(v - st.v).max() <= 1e-8
        o, occ, ads, prof = sim.observables()
        occ_o, ads_o, prof_o = oracle.observables(p, s.pores, st.x, st.d2wall)
        np.testing.assert_array_equal(occ, occ_o)
        np.testing.assert_array_equal(ads, ads_o)
        np.testing.assert_array_equal(prof, prof_o)


def test_drying_run_occupancy_decay_matches_oracle():
    """Pore occupancy over 2,000 steps of drying, four seeds: the GPU and oracle means at every
    checkpoint agree within the seed-to-seed standard error, and the pore empties."""
    seeds = [7, 17, 27, 37]
    systems = [W.drying_cylinder_pore(seed=sd) for sd in seeds]
    every, nck = 250, 8
    gpu = np.zeros((len(seeds), nck))
    with md.Simulation(systems) as sim:
        for c in range(nck):
            sim.step(every)
            for r in range(len(seeds)):
                gpu[r, c] = sim.observables(r)[1].sum()
    ora = np.zeros_like(gpu)
    for r, s in enumerate(systems):
        p = oracle.make_params(s, POT)
        st = oracle.State(p, s.x0, s.v0, s.wall, nthreads=0)
        for c in range(nck):
            st.run(every)
            ora[r, c] = oracle.observables(p, s.pores, st.x, st.d2wall)[0].sum()
    k = len(seeds)
    se = np.sqrt(gpu.var(0, ddof=1) / k + ora.var(0, ddof=1) / k) + 1.0
    z = (gpu.mean(0) - ora.mean(0)) / se
    print("occupancy GPU", gpu.mean(0), "oracle", ora.mean(0), "z", z)
    assert np.abs(z).max() <= 4.0
    assert gpu.mean(0)[-1] < 0.9 * 1000 and ora.mean(0)[-1] < 0.9 * 1000


def test_batched_replicas_evolve_as_they_would_alone():
    """Each replica rebuilds its lists on its own schedule (grouped with others near their skin
    limit): a batch of six uneven systems run together gives every replica the trajectory it has
    when run alone, to rounding (the rebuild moments differ, the pair sets do not)."""
    batch = W.replica_batch(6, seed=11, n_min=1000, n_max=8000)
    with md.Simulation(batch) as sim:
        sim.step(60)
        together = [sim.state(r) for r in range(len(batch))]
        nreb = sim.observables(0)[0]["n_rebuilds"]
    assert nreb > 3
    for r, s in enumerate(batch):
        with md.Simulation(s) as solo:
            solo.step(60)
            x, v = solo.state()
        d = x - together[r][0]
        d[:, :2] -= np.array([s.Lx, s.Ly]) * np.round(d[:, :2] / np.array([s.Lx, s.Ly]))
        assert np.abs(d).max() <= 1e-9, s.name
        assert np.abs(v - together[r][1]).max() <= 1e-9, s.name


def test_skin_choice_changes_speed_not_physics(batch):
    """The skin is the autotuner's to pick: forces and pair counts do not depend on it (every
    pair within the cutoff is listed at any skin), a larger skin rebuilds no more often, and
    choose_skin returns one of the candidates with a timing for each."""
    import dataclasses
    systems = batch[:3]
    forces, pairs = [], []
    for skin in (0.2, 0.8):
        pot = dataclasses.replace(W.Potential(), skin=skin)
        with md.Simulation(systems, pot) as sim:
            forces.append(sim.forces(-1))
            o = [sim.observables(r)[0] for r in range(len(systems))]
            pairs.append([(x["pairs_vv"], x["pairs_vw"]) for x in o])
    rms = np.sqrt((forces[0] ** 2).sum(1).mean())
    assert np.abs(forces[0] - forces[1]).max() <= 1e-12 * rms
    assert pairs[0] == pairs[1]
    got = autotune.choose_skin(systems, skins=(0.2, 0.8), steps=60, warmup=5)
    assert got["skin"] in (0.2, 0.8)
    rows = {r["skin"]: r for r in got["table"]}
    assert all("steps_per_s" in rows[k] and rows[k]["steps_per_s"] > 0 for k in (0.2, 0.8))
    assert rows[0.8]["rebuilds"] <= rows[0.2]["rebuilds"]


def test_cell_side_changes_speed_not_physics(batch, tmp_path):
    """Cells larger than the list radius hold more molecules each: the forces, the pair counts and
    a 20-step trajectory are those of the smallest cells (every pair within the list radius still
    lies in neighbouring cells); choose_geometry times the candidates and caches its choice."""
    import dataclasses
    systems = batch[:3]
    out = []
    for cell in (0.0, 4.5):
        pot = dataclasses.replace(W.Potential(), skin=0.3, cell_size=cell)
        with md.Simulation(systems, pot) as sim:
            sim.set_tuning(force_accumulate=1)   # deterministic: runs comparable step by step
            f0 = sim.forces(-1)
            o = [sim.observables(r)[0] for r in range(len(systems))]
            sim.step(20)
            out.append((f0, [(x["pairs_vv"], x["pairs_vw"]) for x in o], sim.state(-1)))
    rms = np.sqrt((out[0][0] ** 2).sum(1).mean())
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-12 * rms
    assert out[0][1] == out[1][1]
    assert np.abs(out[0][2][1] - out[1][2][1]).max() <= 1e-9
    with pytest.raises(md.MDError, match="cell_size"):
        md.Simulation(systems, dataclasses.replace(W.Potential(), cell_size=2.0))
    got = autotune.choose_geometry(systems, skins=(0.3, 0.6), cell_scales=(1.0, 1.5), steps=40,
                                   warmup=5, cache_path=str(tmp_path / "t.json"))
    assert got["skin"] in (0.3, 0.6) and got["cell_size"] in (0.0, 1.5 * (2.5 + got["skin"]))
    assert autotune.choose_geometry(systems, cache_path=str(tmp_path / "t.json"))["cached"]
