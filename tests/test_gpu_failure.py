"""Failure detection on the GPU without a fault: the step kernels' grid barrier (the thermostat's
sums; every step of the small-system method) bounds its waits. md_check_barrier_timeout runs a
kernel in which one block never arrives: the other's wait must run out (about a second), the
device must report MD_ETIMEOUT, and the context must go on afterwards -- its later steps, with
thermostat steps and barriers, still matching the oracle. Also: a context that switches between
the small-system method and the Verlet lists (different grid sizes at the same barrier) keeps
its barrier aligned."""
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


@pytest.mark.parametrize("method", [1, 4])
def test_a_wait_that_runs_out_reports_and_the_context_goes_on(method):
    s = W.cylinder_pore_1k()
    st = oracle.State(oracle.make_params(s, POT), s.x0, s.v0, s.wall, nthreads=0)
    with md.Simulation([s]) as sim:
        sim.set_tuning(force_accumulate=2, pair_method=method)
        sim.step(13)                     # a thermostat step (every 10) is owed across the check
        seconds = sim.check_barrier_timeout()
        assert 0.01 < seconds < 30.0
        sim.step(17)
        st.run(30)
        x, v = sim.state(0)
        assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-8
        assert np.abs(v - st.v).max() <= 1e-8
        sim.sync()


def test_switching_between_small_and_list_methods_keeps_the_barrier():
    s = W.cylinder_pore_1k()
    st = oracle.State(oracle.make_params(s, POT), s.x0, s.v0, s.wall, nthreads=0)
    with md.Simulation([s]) as sim:
        sim.set_tuning(force_accumulate=2)
        done = 0
        for method, n in ((4, 7), (1, 11), (4, 13), (1, 9)):   # thermostat steps in every leg
            sim.set_tuning(pair_method=method)
            sim.step(n)
            done += n
        st.run(done)
        x, v = sim.state(0)
        assert np.abs(wrapped_diff(x, st.x, s)).max() <= 1e-8
        assert np.abs(v - st.v).max() <= 1e-8
