"""Long-run agreement with the FP64 oracle, where trajectories have long since decorrelated:

* NVE energy drift (thermostat off) of the FP64 and the mixed-precision GPU forms against the
  oracle's own drift on the same equilibrated state: linear fits of E_total / N against time.
* time-averaged axial density profiles and adsorbed counts over several independent seeds: GPU and
  oracle means agree within the seed-to-seed standard error (|z| per bin, chi^2 over bins).
"""
import dataclasses
import math

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


def drift(times, energies):
    """|slope| of a least-squares line through E/N(t), in eps per molecule per tau."""
    return abs(np.polyfit(times, energies, 1)[0])


@pytest.fixture(scope="module")
def equilibrated():
    s = W.cylinder_pore_1k()
    with md.Simulation(s) as sim:
        sim.step(600)
        x, v = sim.state()
    nve = dataclasses.replace(s, x0=x, v0=v, thermostat_every=0)
    return nve


def test_nve_energy_drift_fp64_mixed_and_oracle(equilibrated):
    s = equilibrated
    nsteps, every = 2000, 20
    t = np.arange(every, nsteps + 1, every) * s.dt
    series = {}
    for name, prec in (("fp64", md.MD_PREC_FP64), ("mixed", md.MD_PREC_MIXED)):
        e = []
        with md.Simulation(s, precision=prec) as sim:
            for _ in range(nsteps // every):
                sim.step(every)
                o, *_ = sim.observables()
                e.append((o["ke"] + o["pe"]) / s.n_vapor)
        series[name] = np.array(e)
    st = oracle.State(oracle.make_params(s, POT), s.x0, s.v0, s.wall, nthreads=0)
    e = []
    for _ in range(nsteps // every):
        ke, pe = st.run(every)
        e.append((ke[-1] + pe[-1]) / s.n_vapor)
    series["oracle"] = np.array(e)
    d = {k: drift(t, v) for k, v in series.items()}
    fluct = {k: np.std(v - np.polyval(np.polyfit(t, v, 1), t)) for k, v in series.items()}
    print("NVE drift (eps/molecule/tau):", d, "fluctuation:", fluct)
    scale = max(d["oracle"], 1e-5)
    assert d["fp64"] <= 5 * scale + 1e-5
    assert d["mixed"] <= 5 * scale + 1e-5
    assert fluct["mixed"] <= 3 * fluct["oracle"] + 1e-6


def test_long_run_profiles_and_adsorption_match_oracle():
    seeds = [101, 102, 103, 104, 105, 106]
    systems = [W.cylinder_pore_1k(seed=sd) for sd in seeds]
    nsteps, every, burn = 3000, 25, 1000
    # GPU: all seeds as replicas of one context
    gpu_prof, gpu_ads = [], []
    with md.Simulation(systems) as sim:
        sim.step(burn)
        acc_p = [0.0] * len(systems)
        acc_a = [0.0] * len(systems)
        nsamp = 0
        for _ in range((nsteps - burn) // every):
            sim.step(every)
            for r in range(len(systems)):
                o, occ, ads, prof = sim.observables(r)
                acc_p[r] = acc_p[r] + prof[0].astype(float)
                acc_a[r] += ads.sum()
            nsamp += 1
        gpu_prof = np.array([a / nsamp for a in acc_p])
        gpu_ads = np.array(acc_a) / nsamp
    ora_prof, ora_ads = [], []
    for s in systems:
        p = oracle.make_params(s, POT)
        st = oracle.State(p, s.x0, s.v0, s.wall, nthreads=0)
        st.run(burn)
        ap, aa, n = 0.0, 0.0, 0
        for _ in range((nsteps - burn) // every):
            st.run(every)
            _, ads, prof = oracle.observables(p, s.pores, st.x, st.d2wall)
            ap = ap + prof[0].astype(float)
            aa += ads.sum()
            n += 1
        ora_prof.append(ap / n)
        ora_ads.append(aa / n)
    ora_prof, ora_ads = np.array(ora_prof), np.array(ora_ads)
    # coarse bins (4 profile bins -> 1) to keep the per-bin counts well above zero
    def coarse(a):
        return a.reshape(a.shape[0], -1, 4).sum(-1)
    g, o = coarse(gpu_prof), coarse(ora_prof)
    k = len(seeds)
    se = np.sqrt(g.var(0, ddof=1) / k + o.var(0, ddof=1) / k) + 1e-9
    z = (g.mean(0) - o.mean(0)) / se
    used = (g.mean(0) + o.mean(0)) > 1.0
    chi2 = float((z[used] ** 2).sum())
    dof = int(used.sum())
    print("profile |z| max", np.abs(z[used]).max(), "chi2/dof", chi2 / dof)
    assert np.abs(z[used]).max() <= 5.0
    assert chi2 <= dof + 6 * math.sqrt(2 * dof)
    se_a = math.sqrt(gpu_ads.var(ddof=1) / k + ora_ads.var(ddof=1) / k) + 1e-9
    za = (gpu_ads.mean() - ora_ads.mean()) / se_a
    print("adsorbed GPU", gpu_ads.mean(), "oracle", ora_ads.mean(), "z", za)
    assert abs(za) <= 4.0
