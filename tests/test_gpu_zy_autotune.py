"""The FFT-plan autotuner on the GPU: it picks one of the candidate radix
orders for every transform length of a pair, and the fields computed with the
tuned plans still match the oracle (any order computes the same DFT).

Collected late (after the other GPU tests, before the no-allocation file):
tuned plans are process-wide, and the tests before it run on the model's plans.
"""

import numpy as np
import pytest

import workloads
from oracle import fields as OF
from oracle.interaction import stray_interaction
from tests.pair_setup import force_scale, gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_autotune_keeps_parity():
    from paper_1801_04181_gb300 import fft_plan, tuned_plan

    fp, _, _ = workloads.film_pair_plain(n=(45, 30, 2), gap=2, seed=4)
    fp.u0 = (0.3, 0.6, 0.0)
    m0, m1 = workloads.random_unit(fp.n_base, 4), workloads.random_unit(fp.n_slider, 9)
    mm = gpu_pair(fp, m0, m1, mech=False)
    info = mm.plan_info(0)
    ntuned = mm.autotune(candidates=4, reps=2)
    assert ntuned >= 1
    for L in set(info["fft"]):
        plan = tuned_plan(L)
        assert plan is not None and int(np.prod(plan)) == L
        assert len(plan) == len(fft_plan(L))  # a fewest-stage order
    H = mm.compute_stray_field(0).double().cpu().numpy()
    F, E = mm.get_force(1)
    Hd = mm.compute_demag(0).double().cpu().numpy()
    mm.close()
    M0, M1 = fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1
    ref = stray_interaction(M0, M1, fp.cell, fp.offsets[0], fp.offsets[1], fp.u0, True, return_box=True)
    assert rel_l2(H, ref["H"]) < TOL
    assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * force_scale(ref["hess_n"], M1, fp.cell)
    assert rel_l2(Hd, OF.demag_conv(M0, fp.cell)) < TOL
