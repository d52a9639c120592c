"""The shared-memory FFT planner (mm_fft_plan), no GPU: every 2-3-5 length gets
a plan of supported radices that multiplies out to it with the fewest stages
(checked against a dynamic-programming count), the lengths whose orders were
measured on GB300 get those orders, and other lengths are rejected."""

import numpy as np
import pytest

from paper_1801_04181_gb300 import _native


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1801_04181_gb300.build import build

    build()
    return _native.load()


RADICES = (2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16)


def _fewest_stages(L):
    """Fewest factors from RADICES whose product is L (dynamic programming)."""
    best = {1: 0}
    for n in range(2, L + 1):
        if L % n:
            continue
        best[n] = min((best[n // r] + 1 for r in RADICES if n % r == 0 and (n // r) in best), default=10 ** 9)
    return best[L]


def test_fft_plans_multiply_out_with_fewest_stages():
    from paper_1801_04181_gb300 import fft_plan

    for L in range(2, 2400, 2):
        m = L
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m != 1:
            continue
        plan = fft_plan(L)
        assert int(np.prod(plan)) == L and all(r in RADICES for r in plan)
        assert len(plan) == _fewest_stages(L)


def test_fft_plans_of_the_measured_lengths():
    """The orders measured fastest on the stick-slip grid (2160 x 540) and the cubes (144)."""
    from paper_1801_04181_gb300 import fft_plan

    assert fft_plan(540) == [4, 9, 15]
    assert fft_plan(2160) == [16, 9, 15]
    assert fft_plan(144) == [16, 9]


def test_fft_plan_rejects_lengths_outside_2_3_5():
    from paper_1801_04181_gb300 import MMError, fft_plan

    for L in (0, 7, 14, 22):
        with pytest.raises(MMError):
            fft_plan(L)
