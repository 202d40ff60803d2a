"""md_set_state on the list methods keeps the stored order and rebuilds only where the skin test
asks for it, against the FP64 oracle.

A state read back and loaded again rebuilds nothing. Every molecule moved by less than skin/2
(random directions) still rebuilds nothing, and the lists must still hold every pair within the
cutoff: the pair counts equal the oracle's and the forces match it at the moved positions. One
molecule moved by more than skin/2 has its replica's lists rebuilt (the rebuild is counted), with
the same checks. Stepping on from a load follows the oracle's trajectory. Every list form is
covered (FP64 per-molecule lists, the flat stream, mixed, double-float, the cell method), and a
batch where one replica is loaded alone.
"""
import numpy as np
import pytest

import oracle
import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.Potential()
HALF_SKIN = 0.5 * POT.skin


@pytest.fixture(scope="module", autouse=True)
def built():
    mdbuild.build()
    md.load_library()


FORMS = {  # name: (precision, tuning)
    "fp64_lists": (md.MD_PREC_FP64, dict(force_tpp=4, force_accumulate=2, pair_method=1)),
    "fp64_gather": (md.MD_PREC_FP64, dict(force_tpp=4, force_accumulate=1, pair_method=1)),
    "flat_stream": (md.MD_PREC_FP64, dict(force_tpp=64, force_accumulate=2, pair_method=1)),
    "mixed": (md.MD_PREC_MIXED, dict(force_accumulate=2, pair_method=1)),
    "double_float": (md.MD_PREC_DF64, dict(force_accumulate=2, pair_method=1)),
    "cells": (md.MD_PREC_FP64, dict(force_accumulate=2, pair_method=3)),
}


def wrap(x, s):
    y = x.copy()
    y[:, 0] = (y[:, 0] + 0.5 * s.Lx) % s.Lx - 0.5 * s.Lx
    y[:, 1] = (y[:, 1] + 0.5 * s.Ly) % s.Ly - 0.5 * s.Ly
    return y


def jiggle(x, s, rng, scale):
    """Every molecule moved by scale * skin/2 at most, in a random direction (z kept inside)."""
    d = rng.normal(size=x.shape)
    d *= (scale * HALF_SKIN * rng.uniform(0.5, 1.0, len(x)) / np.linalg.norm(d, axis=1))[:, None]
    y = wrap(x + d, s)
    y[:, 2] = np.clip(y[:, 2], -0.5 * s.Lz + 1e-9, 0.5 * s.Lz - 1e-9)
    return y


def loneliest(x, s):
    """The molecule furthest from every other molecule and wall atom (a safe one to move)."""
    best, k = -1.0, 0
    for i in range(len(x)):
        d = x - x[i]
        d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
        d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
        r2 = (d ** 2).sum(1)
        r2[i] = np.inf
        m = r2.min()
        if len(s.wall):
            dw = s.wall - x[i]
            dw[:, 0] -= s.Lx * np.round(dw[:, 0] / s.Lx)
            dw[:, 1] -= s.Ly * np.round(dw[:, 1] / s.Ly)
            m = min(m, (dw ** 2).sum(1).min())
        if m > best:
            best, k = m, i
    return k


def check_forces(sim, r, s, x, precision):
    p = oracle.make_params(s, POT)
    g, _, stats = oracle.forces(p, x, s.wall, method=1)
    f = sim.forces(r)
    if precision == md.MD_PREC_MIXED:
        assert np.sqrt(((f - g) ** 2).sum() / (g ** 2).sum()) <= 1e-5
    else:
        assert np.abs(f - g).max() / np.sqrt((g ** 2).sum(1).mean()) <= 1e-10
    o = sim.observables(r)[0]
    assert (o["pairs_vv"], o["pairs_vw"]) == (stats["pairs_vv"], stats["pairs_vw"])


def rebuilds(sim):
    return sim.observables(0)[0]["n_rebuilds"]


@pytest.mark.parametrize("form", sorted(FORMS))
def test_load_rebuilds_only_past_half_the_skin(form):
    precision, tuning = FORMS[form]
    s = W.cylinder_pore_1k()
    rng = np.random.default_rng(7)
    with md.Simulation(s, precision=precision) as sim:
        sim.set_tuning(**tuning)
        sim.step(7)
        sim.rebuild_lists()              # every molecule's reference is now where it stands
        x, v = sim.state()
        n0 = rebuilds(sim)
        sim.set_state(0, x, v)                       # the same state: nothing to rebuild
        assert rebuilds(sim) == n0
        x2, v2 = sim.state()
        np.testing.assert_array_equal(x2, x)
        np.testing.assert_array_equal(v2, v)
        check_forces(sim, 0, s, x, precision)
        xj = jiggle(x, s, rng, 0.9)                  # all within skin/2 of the last build
        sim.set_state(0, xj, v)
        assert rebuilds(sim) == n0
        np.testing.assert_array_equal(sim.state()[0], xj)
        check_forces(sim, 0, s, xj, precision)
        k = loneliest(x, s)
        xf = xj.copy()
        xf[k] = x[k]
        xf[k, 0] += 1.6 * HALF_SKIN                  # one molecule past skin/2
        xf = wrap(xf, s)
        sim.set_state(0, xf, v)
        assert rebuilds(sim) == n0 + 1
        check_forces(sim, 0, s, xf, precision)
        if precision == md.MD_PREC_FP64:
            st = oracle.State(oracle.make_params(s, POT), xf, v, s.wall)
            st.step = 7
            sim.step(12)
            st.run(12)
            xs, vs = sim.state()
            d = xs - st.x
            d[:, 0] -= s.Lx * np.round(d[:, 0] / s.Lx)
            d[:, 1] -= s.Ly * np.round(d[:, 1] / s.Ly)
            assert np.abs(d).max() <= 1e-8
            assert np.abs(vs - st.v).max() <= 1e-8


def test_one_replica_of_a_batch_loaded_alone():
    batch = W.replica_batch(n_replicas=3, n_min=1000, n_max=2500)
    rng = np.random.default_rng(11)
    with md.Simulation(batch) as sim:
        sim.set_tuning(force_tpp=64, force_accumulate=2)
        sim.step(5)
        sim.rebuild_lists()
        xs = [sim.state(r) for r in range(3)]
        n0 = rebuilds(sim)
        x1 = jiggle(xs[1][0], batch[1], rng, 0.9)
        sim.set_state(1, x1, xs[1][1])
        assert rebuilds(sim) == n0
        for r, x in ((0, xs[0][0]), (1, x1), (2, xs[2][0])):
            check_forces(sim, r, batch[r], x, md.MD_PREC_FP64)
        k = loneliest(xs[1][0], batch[1])
        x1[k] = xs[1][0][k]
        x1[k, 1] += 1.6 * HALF_SKIN
        x1 = wrap(x1, batch[1])
        sim.set_state(1, x1, xs[1][1])
        assert rebuilds(sim) == n0 + 1
        for r, x in ((0, xs[0][0]), (1, x1), (2, xs[2][0])):
            check_forces(sim, r, batch[r], x, md.MD_PREC_FP64)
        np.testing.assert_array_equal(sim.state(0)[0], xs[0][0])
        np.testing.assert_array_equal(sim.state(2)[0], xs[2][0])
