"""Checks against the numbers the paper prints (tests/golden/paper_parameters.txt).

The paper prints no physical results, only parameters and timings. These tests pin the two
readings that rest on those numbers: the reduced-unit range of the Berendsen rise time that the
thermostat accepts (Sec. 2), and the total molecule counts behind the Table 4 per-particle times.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1812_07993_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def load():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, *v = line.split()
            out[k] = [float(t) for t in v]
    return out


def reduced_time_ps(g):
    """LJ time unit sigma sqrt(m / eps) for water (m = 18 u), in ps."""
    sigma = g["sigma_angstrom"][0] * 1e-10
    eps = g["epsilon_ev"][0] * 1.602176634e-19
    m = 18.0 * 1.66053906660e-27
    return sigma * math.sqrt(m / eps) * 1e12


def test_reduced_units():
    g = load()
    tau = reduced_time_ps(g)
    assert tau == pytest.approx(1.668, abs=2e-3)
    assert g["dt_ps"][0] / tau == pytest.approx(0.0096, abs=1e-4)
    lo, hi = (t / tau for t in g["tau_B_ps"])
    assert lo == pytest.approx(0.060, abs=1e-3) and hi == pytest.approx(1.199, abs=2e-3)


def test_table4_per_particle_times_use_the_total_counts():
    g = load()
    for dim in ("2d", "3d"):
        n = g[f"n_total_{dim}"][0]
        for step, per in zip(g[f"one_step_{dim}_ms"], g[f"per_particle_{dim}_ms"]):
            assert step / n == pytest.approx(per, abs=6e-6)


@pytest.mark.parametrize("end", [0, 1])
def test_thermostat_over_the_papers_rise_time_range(end):
    """At both ends of the paper's tau_B range (in reduced units) the Berendsen factor is real and
    moves T toward T0 by the fraction n_th dt / tau_B."""
    g = load()
    tau_B = g["tau_B_ps"][end] / reduced_time_ps(g)
    s = W.make_system("tb", 12.0, 12.0, 20.0, 3.0, [W.Pore(W.PORE_CYLINDER, r0=3.0)], 150, 1.3, 2)
    p = oracle.make_params(s, W.Potential(), thermostat_every=10, T0=0.9, tau_B=tau_B)
    st = oracle.State(p, s.x0, s.v0, s.wall)
    ke, _ = st.run(10)
    T_before = 2 * ke[-1] / (3 * len(st.v))
    T_after = (st.v ** 2).sum() / (3 * len(st.v))
    assert np.isfinite(T_after)
    assert T_after == pytest.approx(T_before + (10 * 0.005 / tau_B) * (0.9 - T_before), rel=1e-12)
