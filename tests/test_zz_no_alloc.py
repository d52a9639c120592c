"""The no-allocation entry point agrees with the allocating one (GPU).

mm_spline_field_noalloc serves callers that cannot allocate device memory
while they drive the library (their memory belongs to their own pool
allocator, or cudaMalloc's implicit synchronisation would stall their stepping
loop).  It evaluates the stray field, force and energy of a target from a
coefficient box the caller holds, using only a fixed scratch array inside the
library.  Here it is fed the prefiltered box of mm_compute_potential and must
reproduce mm_compute_stray_field / mm_get_force within the parity tolerance,
on two calls in a row (the shared scratch keeps the previous call's contents).
This file is collected last so that a failure here leaves every other test run.
"""

import numpy as np
import pytest

import workloads
from oracle.interaction import stray_interaction
from tests.pair_setup import force_scale, gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    from paper_1801_04181_gb300 import spline_field_noalloc

    fp, _, _ = workloads.film_pair_plain(n=(40, 24, 2), gap=2, seed=13)
    fp.n_slider = (36, 20, 2)
    fp.u0 = (0.3, 0.45, 0.0)
    fp.lateral = (3, -2)
    m0 = workloads.random_unit(fp.n_base, 13)
    m1 = workloads.random_unit(fp.n_slider, 14)
    mm = gpu_pair(fp, m0, m1, mech=False)

    H_ref = mm.compute_stray_field(0)
    F_ref, E_ref = mm.get_force(1)
    coef, lo = mm.compute_potential(0, prefiltered=True)
    pos0 = [fp.offsets[1][a] - fp.offsets[0][a] + fp.u0[a] for a in range(3)]
    m_t = torch.as_tensor(np.ascontiguousarray(m1), dtype=torch.float32, device="cuda")
    ref = stray_interaction(fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1, fp.cell, fp.offsets[0],
                            fp.offsets[1], fp.u0, True, return_box=True)
    scale = force_scale(ref["hess_n"], fp.mat_slider.Ms * m1, fp.cell)

    for _ in range(2):
        H = torch.full_like(m_t, float("nan"))
        FE = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        spline_field_noalloc(coef, lo, pos0, m_t, fp.cell, fp.mat_slider.Ms, H, FE)
        torch.cuda.synchronize()
        assert rel_l2(H.double().cpu().numpy(), H_ref.double().cpu().numpy()) < TOL
        fe = FE.cpu().numpy()
        assert np.max(np.abs(fe[:3] - np.array(F_ref))) < TOL * scale
        assert abs(fe[3] - E_ref) < TOL * abs(E_ref)
    mm.close()


def test_noalloc_rejects_out_of_box_targets_and_bad_shapes():
    """A target whose spline support leaves the box is refused with MM_ERANGE;
    the Python side refuses arrays of the wrong shape before the C call (the
    kernel reads m at 0, N and 2N, so a (2, ...) array would be read past its
    end).  Oversized targets are covered by the CPU test of the C ABI."""
    import torch
    from paper_1801_04181_gb300 import MMError, spline_field_noalloc

    coef = torch.zeros((8, 20, 20), dtype=torch.float32, device="cuda")
    m_t = torch.zeros((3, 2, 8, 8), dtype=torch.float32, device="cuda")
    FE = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(MMError) as e:
        spline_field_noalloc(coef, (0, 0, 0), (15.0, 2.0, 2.0), m_t, (1e-9,) * 3, 1e6, None, FE)
    assert e.value.status == -4  # MM_ERANGE: support leaves the box
    with pytest.raises(ValueError):
        spline_field_noalloc(coef, (0, 0, 0), (2.0, 2.0, 2.0), m_t[:2], (1e-9,) * 3, 1e6, None, FE)
    with pytest.raises(ValueError):
        spline_field_noalloc(coef[0], (0, 0, 0), (2.0, 2.0, 2.0), m_t, (1e-9,) * 3, 1e6, None, FE)
    with pytest.raises(ValueError):
        spline_field_noalloc(coef, (0, 0, 0), (2.0, 2.0, 2.0), m_t, (1e-9,) * 3, 1e6, None, None)
