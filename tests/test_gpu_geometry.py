"""The paper's own geometry on the GPU (Sec. 4 and Sec. 5): hard reflecting pore walls, a
rectangular prism pore closed on five faces, and the planar (2D) system, against the FP64 oracle.

* free flight (no pair forces) for 4,000 steps: every reflection off the slab faces, the prism's
  side walls and its floor, in 3D and in the plane, equals the oracle's to rounding;
* interacting systems: forces, 10-step trajectories and integer observables as in the other parity
  tests (max|dF|/RMS(F) <= 1e-10, |dr|, |dv| <= 1e-8, counts exact), the planar invariants
  (y = vy = fy = 0) and the planar thermostat's 2N degrees of freedom;
* the drying of the paper's pore over 2,000 steps: pore occupancy against the oracle's over seeds.
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
    rms = np.sqrt((g ** 2).sum(1).mean())
    return np.abs(f - g).max() / rms


def wrapped(d, s):
    d = d.copy()
    d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
    d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
    return d


SYSTEMS = {"prism3d": lambda **k: W.paper_prism_pore(**k), "plane2d": lambda **k: W.paper_pore_2d(**k)}


@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_free_flight_reflections_match_oracle(name):
    """No pair forces (eps = 0): 4,000 steps of reflections off every face; the paths are not
    chaotic, so GPU and oracle agree to rounding over the whole run."""
    s = SYSTEMS[name]()
    s = dataclasses.replace(s, thermostat_every=0)
    pot = dataclasses.replace(POT, eps=0.0)
    p = oracle.make_params(s, pot)
    st = oracle.State(p, s.x0, s.v0, None, pores=s.pores)
    with md.Simulation(s, pot) as sim:
        for _ in range(4):
            sim.step(1000)
            st.run(1000)
            x, v = sim.state()
            assert np.abs(wrapped(x - st.x, s)).max() <= 1e-9
            assert np.abs(v - st.v).max() <= 1e-12
            assert oracle.in_solid(p, s.pores, x).sum() == 0
        # every molecule has been reflected many times: speeds unchanged, directions not
        np.testing.assert_allclose((v ** 2).sum(1), (s.v0 ** 2).sum(1), rtol=1e-12)
        assert (np.sign(v) != np.sign(s.v0)).any(axis=1).mean() > 0.25
        if name == "plane2d":
            assert (x[:, 1] == 0.0).all() and (v[:, 1] == 0.0).all()


@pytest.mark.parametrize("name", sorted(SYSTEMS))
@pytest.mark.parametrize("precision", [md.MD_PREC_FP64, md.MD_PREC_MIXED, md.MD_PREC_DF64])
def test_interacting_ten_steps_and_observables(name, precision):
    s = SYSTEMS[name]()
    p = oracle.make_params(s, POT)
    st = oracle.State(p, s.x0, s.v0, None, pores=s.pores)
    with md.Simulation(s, precision=precision) as sim:
        g, _, _ = oracle.forces(p, s.x0, None)
        f0 = sim.forces()
        fp64_bar = precision != md.MD_PREC_MIXED   # the double-float form meets the FP64 bars
        if fp64_bar:
            assert force_err(f0, g) <= 1e-10
        else:
            assert np.sqrt(((f0 - g) ** 2).sum() / (g ** 2).sum()) <= 1e-5
        sim.step(10)                                   # thermostat on step 10
        st.run(10)
        x, v = sim.state()
        tol = 1e-8 if fp64_bar else 1e-5
        assert np.abs(wrapped(x - st.x, s)).max() <= tol
        assert np.abs(v - st.v).max() <= tol
        o, occ, ads, prof = sim.observables()
        occ_o, ads_o, prof_o = oracle.observables(p, s.pores, st.x, st.d2wall)
        if fp64_bar:
            np.testing.assert_array_equal(occ, occ_o)
            np.testing.assert_array_equal(prof, prof_o)
            wv = oracle.molecule_virials(p, st.x, None)
            np.testing.assert_allclose(o["pore_pressure"],
                                       oracle.pore_pressure(p, s.pores, st.x, st.v, wv),
                                       rtol=1e-9, atol=1e-12)
        assert ads.sum() == 0                          # no wall atoms
        if name == "plane2d":
            f = sim.forces()
            assert (x[:, 1] == 0.0).all() and (v[:, 1] == 0.0).all() and (f[:, 1] == 0.0).all()
            # the planar thermostat: T over 2N degrees of freedom (rescaling, tau_B = n_th dt)
            s2 = dataclasses.replace(s, tau_B=0.0, T0=0.6)
            with md.Simulation(s2, precision=precision) as sim2:
                sim2.step(10)
                _, v2 = sim2.state()
                assert (v2 ** 2).sum() / (2 * len(v2)) == pytest.approx(0.6, rel=1e-12)
                assert sim2.observables()[0]["T"] == pytest.approx(0.6, rel=1e-12)


def test_invalid_geometry_is_rejected():
    s = W.paper_pore_2d()
    bad = s.x0.copy()
    bad[3, 1] = 0.5
    with pytest.raises(md.MDError):
        md.Simulation(dataclasses.replace(s, x0=bad))
    with pytest.raises(md.MDError):
        md.Simulation(dataclasses.replace(s, wall_model=0))
    c = W.paper_prism_pore()
    with pytest.raises(md.MDError):
        md.Simulation(dataclasses.replace(c, pores=[W.Pore(W.PORE_CYLINDER, r0=2.0)]))
    with md.Simulation(s) as sim:
        x, v = sim.state()
        x[0, 1] = 0.25
        with pytest.raises(md.MDError):
            sim.set_state(0, x, v)


@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_drying_of_the_papers_pore_matches_oracle(name):
    """Occupancy of the paper's pore over 2,000 steps, four seeds each side: GPU and oracle means
    agree within the seed-to-seed standard error at every checkpoint, and the pore empties."""
    seeds = [41, 51, 61, 71]
    systems = [SYSTEMS[name](seed=sd) for sd in seeds]
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
        st = oracle.State(p, s.x0, s.v0, None, nthreads=0, pores=s.pores)
        for c in range(nck):
            st.run(every)
            ora[r, c] = oracle.observables(p, s.pores, st.x, st.d2wall)[0].sum()
    k = len(seeds)
    se = np.sqrt(gpu.var(0, ddof=1) / k + ora.var(0, ddof=1) / k) + 1.0
    z = (gpu.mean(0) - ora.mean(0)) / se
    n0 = float(np.sum([W.carve_mask(s.x0, s.pores[0], s.Lx, s.Ly, s.slab_half).sum()
                       for s in systems])) / k
    print(name, "occupancy GPU", gpu.mean(0), "oracle", ora.mean(0), "z", z, "start", n0)
    assert np.abs(z).max() <= 4.0
    assert gpu.mean(0)[-1] < n0 and ora.mean(0)[-1] < n0
