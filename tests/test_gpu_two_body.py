"""Every pair-force form against Eq. 2 evaluated exactly, one pair at a time.

A batch of 288 replicas, each holding one vapour pair or one molecule beside one wall atom
(separations 0.8-2.499 sigma, random directions, some across the periodic edge; coordinates on a
2^-20 grid so that their differences are exact), is evaluated by every launch shape and form, and
each force is compared with the exact rational force on the same doubles (``two_body_cases``). The
FP64 forms must land within a few ulps of the error scale S (the sum of the repulsive and
attractive magnitudes): 1e-15 at most, 3e-16 in the RMS -- the level of a correctly rounded
evaluation, which pins the reciprocal 1/r^2 (seeded through an FP32 reciprocal, refined by one
third-order Newton step) to IEEE accuracy, not merely to the 1e-10 parity bar. The double-float
form is held to its ~2^-44 arithmetic and the mixed form to FP32.
"""
import numpy as np
import pytest

import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

import two_body_cases as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mdbuild.build()
    md.load_library()


@pytest.fixture(scope="module")
def systems():
    return T.cases()


FP64_FORMS = [  # (force_tpp (0: keep; 64 the flat stream), force_accumulate, pair_method: 1
    # lists, 2 all, 3 cells, 4 small systems)
    (1, 2, 1), (2, 2, 1), (4, 2, 1), (8, 2, 1), (16, 2, 1), (32, 2, 1), (64, 2, 1),
    (2, 1, 1), (32, 1, 1), (2, 2, 2), (0, 2, 3), (0, 0, 4),
]


def _errors(systems, precision, tpp, acc, method):
    with md.Simulation(systems, precision=precision) as sim:
        sim.set_tuning(force_tpp=tpp, force_accumulate=acc, pair_method=method)
        sim.compute_forces()
        f = sim.forces(-1)
    off = np.cumsum([0] + [s.n_vapor for s in systems])
    return T.errors(systems, [f[off[k]:off[k + 1]] for k in range(len(systems))])


@pytest.mark.parametrize("tpp,acc,method", FP64_FORMS)
def test_fp64_pair_forms_within_a_few_ulps_of_exact(systems, tpp, acc, method):
    e = _errors(systems, md.MD_PREC_FP64, tpp, acc, method)
    assert len(e) == 480
    assert e.max() <= 1e-15, e.max()
    assert np.sqrt((e ** 2).mean()) <= 3e-16


@pytest.mark.parametrize("tpp,acc,method", [(4, 2, 1), (64, 2, 1), (2, 1, 1), (0, 2, 3)])
def test_double_float_pair_terms_near_their_precision(systems, tpp, acc, method):
    e = _errors(systems, md.MD_PREC_DF64, tpp, acc, method)
    assert e.max() <= 5e-13, e.max()


@pytest.mark.parametrize("tpp,acc,method", [(4, 2, 1), (64, 2, 1), (4, 1, 1), (0, 2, 3)])
def test_mixed_pair_terms_near_fp32(systems, tpp, acc, method):
    e = _errors(systems, md.MD_PREC_MIXED, tpp, acc, method)
    assert e.max() <= 1e-5, e.max()
