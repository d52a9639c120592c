"""Host logic of the batched form, no GPU: lane assignment (mm_assign_lanes)
and the argument checks of mm_step_batch.

Lane assignment is Graham's longest-processing-time rule; it is pinned by what
that rule guarantees rather than by a second copy of it: every pair gets a
lane in range, the makespan is within Graham's bound (4/3 - 1/(3m)) of the
optimum found by brute force on small inputs, equal costs spread round robin,
and a pair that costs more than all others together sits alone.
"""

import ctypes as C
import itertools

import numpy as np
import pytest

from paper_1801_04181_gb300 import _native, assign_lanes


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1801_04181_gb300.build import build

    build()
    return _native.load()


def _makespan(costs, lanes, m):
    load = np.zeros(m)
    for c, l in zip(costs, lanes):
        load[l] += c
    return load.max()


def _optimum(costs, m):
    best = np.inf
    for lanes in itertools.product(range(m), repeat=len(costs)):
        best = min(best, _makespan(costs, lanes, m))
    return best


@pytest.mark.parametrize("seed,n,m", [(0, 7, 2), (1, 8, 3), (2, 6, 4), (3, 9, 3)])
def test_lpt_within_graham_bound_of_brute_force(seed, n, m):
    rng = np.random.default_rng(seed)
    costs = rng.uniform(1.0, 10.0, n).tolist()
    lanes = assign_lanes(costs, m)
    assert all(0 <= l < m for l in lanes)
    opt = _optimum(costs, m)
    assert _makespan(costs, lanes, m) <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-12


def test_equal_costs_round_robin_and_dominant_pair_alone():
    assert assign_lanes([1.0] * 7, 3) == [0, 1, 2, 0, 1, 2, 0]
    lanes = assign_lanes([1.0, 100.0, 2.0, 3.0], 2)
    assert lanes[1] == 0 and lanes[0] == lanes[2] == lanes[3] == 1
    assert assign_lanes([], 4) == []
    assert assign_lanes([5.0, 3.0], 1) == [0, 0]


def test_lane_assignment_rejects_bad_input():
    L = _native.load()
    out = (C.c_int * 2)()
    assert L.mm_assign_lanes((C.c_double * 2)(1.0, 2.0), 2, 0, out) == _native.MM_EINVAL
    assert L.mm_assign_lanes((C.c_double * 2)(1.0, -2.0), 2, 2, out) == _native.MM_EINVAL
    assert L.mm_assign_lanes((C.c_double * 2)(1.0, float("nan")), 2, 2, out) == _native.MM_EINVAL
    assert L.mm_assign_lanes(None, 2, 2, out) == _native.MM_EINVAL


def test_step_batch_rejects_bad_arguments_without_gpu():
    L = _native.load()
    bad = C.c_int(7)
    dt = (C.c_double * 2)(1e-13, 1e-13)
    # no contexts, nothing to do
    assert L.mm_step_batch(None, 0, 3, None, None, C.byref(bad)) == 0 and bad.value == -1
    assert L.mm_step_batch(None, 2, 3, None, dt, C.byref(bad)) == _native.MM_EINVAL
    ctxs = (C.c_void_p * 2)(None, None)
    assert L.mm_step_batch(ctxs, 2, 3, None, dt, C.byref(bad)) == _native.MM_EINVAL and bad.value == 0
    assert L.mm_step_batch(ctxs, -1, 3, None, dt, None) == _native.MM_EINVAL

