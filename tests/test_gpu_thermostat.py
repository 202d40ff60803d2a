"""Berendsen scaling (Fig. 4) paid inside the next step's first kernel, against the oracle.

A thermostat step (every n_th) leaves its scaling owed; the next step's k_integrate_first pays it
(partial sums of v(t+dt)^2, a bounded grid barrier whose last block computes lambda, then the
scaling before this step's half-kick), or, when the state is read in between, the settle kernels
pay it first. Both routes must give the oracle's trajectory: 25 steps in one go (scalings paid at
steps 11 and 21 inside the step kernel) and the same 25 steps with a state read after step 20 (the
settle route), for replicas with different n_th in one context, in every accumulation form.
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


def wrapped_diff(a, b, s):
    d = a - b
    d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
    d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
    return d


@pytest.fixture(scope="module")
def systems():
    base = W.replica_batch(n_replicas=6, n_max=8000)
    # different thermostat periods and couplings per replica, one without thermostat
    every = [10, 7, 10, 0, 5, 10]
    tau = [0.0, 0.0, 0.5, 0.0, 0.0, 0.25]
    return [dataclasses.replace(s, thermostat_every=n, tau_B=t) for s, n, t in zip(base, every, tau)]


FORMS = [  # precision, force_accumulate, pair_method, trajectory tolerance
    (md.MD_PREC_FP64, 2, 1, 1e-8), (md.MD_PREC_FP64, 1, 1, 1e-8), (md.MD_PREC_FP64, 2, 3, 1e-8),
    (md.MD_PREC_DF64, 2, 1, 1e-8), (md.MD_PREC_DF64, 1, 1, 1e-8),
]


@pytest.mark.parametrize("prec,acc,method,tol", FORMS)
@pytest.mark.parametrize("read_at", [None, 20])
def test_thermostat_paid_in_the_step_kernel_or_settled_before_a_read(systems, prec, acc, method,
                                                                      tol, read_at):
    states = [oracle.State(oracle.make_params(s, POT), s.x0, s.v0, s.wall, nthreads=0)
              for s in systems]
    with md.Simulation(systems, precision=prec) as sim:
        sim.set_tuning(force_accumulate=acc, pair_method=method)
        if read_at is None:
            sim.step(25)
        else:
            sim.step(read_at)
            sim.state(-1)                       # settles the owed kick and scaling
            sim.step(25 - read_at)
        for r, (s, st) in enumerate(zip(systems, states)):
            st.run(25)
            x, v = sim.state(r)
            assert np.abs(wrapped_diff(x, st.x, s)).max() <= tol, (s.name, r)
            assert np.abs(v - st.v).max() <= tol, (s.name, r)


def test_graph_replays_and_plain_launches_agree(systems):
    """The step kernel with its barrier inside CUDA-graph replays of 10 steps and in plain
    launches: the same trajectory bit for bit in the deterministic form."""
    out = []
    for use_graph in (1, 2):
        with md.Simulation(systems) as sim:
            sim.set_tuning(force_accumulate=1, use_graph=use_graph, steps_per_graph=10)
            sim.step(30)
            out.append(sim.state(-1))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
