"""Symmetries of the GPU path itself, in every pair form (Sec. 2, Eq. 1 and Eq. 2).

Newton's third law. In a wall-free box (periodic x, y; reflecting z; no wall atoms, no thermostat) the pair forces are
the only forces, and each pair's force acts on both molecules with opposite signs:

* the net force over all molecules vanishes, up to the rounding of the per-molecule sums;
* x and y momentum are conserved step after step (z reflections change only z momentum).

The half-list forms apply each pair's force to both ends once (exactly antisymmetric); the full
list forms compute it from both rows on exactly antisymmetric cell-local offsets. A list that
lost a pair on one side only, a reaction force with the wrong sign or index, or a deferred kick
applied to one side only would show up here.

Invariances of the forces, which depend only on the pair separations (minimum image in x, y):

* translating vapour and wall together in x and y (periodic) leaves every molecule's force as
  it was, though cells, lists and summation orders all change;
* rotating a square box with a cylinder pore on its axis by 90 degrees about z (the wall lattice
  maps onto itself) rotates every force the same way, which would catch an x/y mix-up;
* permuting the caller's molecule order permutes the forces.
"""
import dataclasses

import numpy as np
import pytest

import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (precision, force_accumulate, pair_method, relative bound on |sum f| / sum |f|, relative bound on
# the x/y momentum change / sum |v| over the run). FP64 and double-float pair terms sum in FP64;
# the mixed form sums FP32 pair forces with compensation, then in FP64.
FORMS = [
    ("fp64-deterministic", md.MD_PREC_FP64, 1, 1, 1e-13, 1e-12),
    ("fp64-atomic", md.MD_PREC_FP64, 2, 1, 1e-13, 1e-12),
    ("fp64-all-pairs", md.MD_PREC_FP64, 1, 2, 1e-13, 1e-12),
    ("mixed-deterministic", md.MD_PREC_MIXED, 1, 1, 1e-7, 1e-8),
    ("mixed-atomic", md.MD_PREC_MIXED, 2, 1, 1e-7, 1e-8),
    ("df64-deterministic", md.MD_PREC_DF64, 1, 1, 1e-12, 1e-11),
    ("df64-atomic", md.MD_PREC_DF64, 2, 1, 1e-12, 1e-11),
    ("fp64-cells", md.MD_PREC_FP64, 2, 3, 1e-13, 1e-12),
    ("mixed-cells", md.MD_PREC_MIXED, 2, 3, 1e-7, 1e-8),
    ("df64-cells", md.MD_PREC_DF64, 2, 3, 1e-12, 1e-11),
    ("fp64-small", md.MD_PREC_FP64, 1, 4, 1e-13, 1e-12),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    mdbuild.build()
    md.load_library()


@pytest.fixture(scope="module")
def box():
    # density ~0.22 sigma^-3, like the vapour of the pore workloads; 7 x 7 x 7 cells
    s = W.vapor_only_box(6000, 30.0, 30.0, 1.0, seed=31)
    return dataclasses.replace(s, thermostat_every=0)


@pytest.mark.parametrize("name,prec,acc,method,ftol,ptol", FORMS, ids=[f[0] for f in FORMS])
def test_net_force_vanishes_and_xy_momentum_is_conserved(box, name, prec, acc, method, ftol, ptol):
    with md.Simulation(box, precision=prec) as sim:
        sim.set_tuning(force_accumulate=acc, pair_method=method)
        f = sim.forces(-1)
        total = np.abs(f).sum()
        assert total > 0
        assert np.abs(f.sum(0)).max() <= ftol * total, (name, f.sum(0), total)
        _, v0 = sim.state(-1)
        p0 = v0.sum(0)
        sim.step(400)
        x1, v1 = sim.state(-1)
        f1 = sim.forces(-1)
        o, *_ = sim.observables(0)
    assert np.isfinite(x1).all() and np.isfinite(v1).all()
    assert o["n_rebuilds"] > 1 or method == 2  # the lists were rebuilt during the run
    assert np.abs(f1.sum(0)).max() <= ftol * np.abs(f1).sum(), name
    scale = np.abs(v1).sum()
    dp = v1.sum(0) - p0
    assert abs(dp[0]) <= ptol * scale and abs(dp[1]) <= ptol * scale, (name, dp, scale)
    # the z reflections do act: z momentum is not conserved in general, and it is not checked


# (precision, force_accumulate, relative bound on max |F_a - F_b| / max |F|): FP64 and
# double-float forces agree to rounding; the mixed form's FP32 pair terms on different cell
# offsets differ at its own error level
INV_FORMS = [
    ("fp64-deterministic", md.MD_PREC_FP64, 1, 1e-10),
    ("fp64-atomic", md.MD_PREC_FP64, 2, 1e-10),
    ("mixed-deterministic", md.MD_PREC_MIXED, 1, 1e-4),
    ("mixed-atomic", md.MD_PREC_MIXED, 2, 1e-4),
    ("df64-atomic", md.MD_PREC_DF64, 2, 1e-10),
]


def forces_of(s, prec, acc):
    with md.Simulation(s, precision=prec) as sim:
        sim.set_tuning(force_accumulate=acc)
        return sim.forces(-1)


def wrap_xy(p, s):
    q = p.copy()
    for k, L in ((0, s.Lx), (1, s.Ly)):
        q[:, k] = np.mod(q[:, k] + 0.5 * L, L) - 0.5 * L
        q[:, k] = np.where(q[:, k] >= 0.5 * L, q[:, k] - L, q[:, k])  # rounding at the edge
    return q


def close(fa, fb, tol):
    return np.abs(fa - fb).max() <= tol * np.abs(fa).max()


@pytest.fixture(scope="module")
def pore():
    return W.cylinder_pore_1k()


@pytest.mark.parametrize("name,prec,acc,tol", INV_FORMS, ids=[f[0] for f in INV_FORMS])
def test_forces_invariant_under_xy_translation(pore, name, prec, acc, tol):
    s = pore
    t = np.array([3.7, -5.3, 0.0])
    moved = dataclasses.replace(s, x0=wrap_xy(s.x0 + t, s), wall=wrap_xy(s.wall + t, s))
    fa, fb = forces_of(s, prec, acc), forces_of(moved, prec, acc)
    assert np.abs(fa).max() > 1.0
    assert close(fa, fb, tol), (name, np.abs(fa - fb).max(), np.abs(fa).max())


@pytest.mark.parametrize("name,prec,acc,tol", INV_FORMS, ids=[f[0] for f in INV_FORMS])
def test_forces_rotate_with_the_system(pore, name, prec, acc, tol):
    s = pore
    assert s.Lx == s.Ly and s.pores[0].cx == 0.0 and s.pores[0].cy == 0.0

    def rot(p):  # (x, y, z) -> (-y, x, z)
        return np.stack([-p[:, 1], p[:, 0], p[:, 2]], axis=1)

    turned = dataclasses.replace(s, x0=wrap_xy(rot(s.x0), s), v0=rot(s.v0),
                                 wall=wrap_xy(rot(s.wall), s))
    fa, fb = forces_of(s, prec, acc), forces_of(turned, prec, acc)
    assert close(rot(fa), fb, tol), (name, np.abs(rot(fa) - fb).max(), np.abs(fa).max())


@pytest.mark.parametrize("name,prec,acc,tol", INV_FORMS, ids=[f[0] for f in INV_FORMS])
def test_forces_follow_a_permutation_of_the_molecules(pore, name, prec, acc, tol):
    s = pore
    perm = np.random.default_rng(5).permutation(s.n_vapor)
    shuffled = dataclasses.replace(s, x0=s.x0[perm].copy(), v0=s.v0[perm].copy())
    fa, fb = forces_of(s, prec, acc), forces_of(shuffled, prec, acc)
    assert close(fa[perm], fb, tol), (name, np.abs(fa[perm] - fb).max(), np.abs(fa).max())
