"""Energy gradients (mm_backward_energy, the transposed path) against the FP64
oracle's (oracle/adjoint.py, itself pinned by finite differences), through the
C ABI; and the torch.autograd wrapper on top of it.

Bar: relative L2 <= 1e-5 for dE/dm of either magnet, dE/du against the size
of the terms that cancel in Eq. (EQForce), as for the force.
"""

import numpy as np
import pytest

import workloads
from oracle.adjoint import energy_gradients
from oracle.interaction import stray_interaction
from tests.pair_setup import force_scale, gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _pair(n0, n1, gap, u, seed, axis=2, lateral=(0, 0), Ms=(8e5, 1.1e6)):
    fp, _, _ = workloads.film_pair_plain(n0, gap, seed)
    fp.n_slider = n1
    fp.stack_axis = axis
    fp.lateral = lateral
    fp.u0 = u
    fp.mat_base.Ms = Ms[0]
    fp.mat_slider = workloads.Material(Ms=Ms[1], Aex=1.3e-11, alpha=0.5)
    return fp, workloads.random_unit(n0, seed), workloads.random_unit(n1, seed + 5)


CASES = [
    ((40, 24, 2), (33, 17, 1), 2, (0.31, 0.2, 0.0), 2, (3, -2)),     # thin films
    ((12, 10, 7), (9, 11, 6), 3, (0.37, 0.2, 0.15), 0, (1, 0)),      # direct z sum
    ((11, 9, 10), (10, 8, 9), 2, (0.55, -0.3, 0.2), 0, (0, 1)),      # z by FFT
]


@pytest.mark.parametrize("n0,n1,gap,u,axis,lateral", CASES)
def test_energy_gradients_match_oracle(n0, n1, gap, u, axis, lateral):
    fp, m0, m1 = _pair(n0, n1, gap, u, 3, axis, lateral)
    offs = fp.offsets
    mm = gpu_pair(fp, m0, m1, mech=False)
    Ms = (fp.mat_base.Ms, fp.mat_slider.Ms)
    ms = (m0, m1)
    for src in (0, 1):
        t = 1 - src
        du, gs, gt = mm.backward_energy(src)
        ref = energy_gradients(Ms[src] * ms[src], Ms[t] * ms[t], fp.cell, offs[src], offs[t], u, t == 1)
        assert rel_l2(gs.double().cpu().numpy(), Ms[src] * ref["dE_dMs"]) < TOL
        assert rel_l2(gt.double().cpu().numpy(), Ms[t] * ref["dE_dMt"]) < TOL
        box = stray_interaction(Ms[src] * ms[src], Ms[t] * ms[t], fp.cell, offs[src], offs[t], u, t == 1,
                                return_box=True)
        scale = force_scale(box["hess_n"], Ms[t] * ms[t], fp.cell)
        assert np.max(np.abs(np.array(du) - ref["dE_du"])) < TOL * scale
    mm.close()


def test_energy_gradients_repeat_and_autograd():
    import torch
    from paper_1801_04181_gb300 import InteractionEnergy

    fp, m0, m1 = _pair((24, 18, 2), (20, 16, 2), 2, (0.4, 0.1, 0.0), 7)
    mm = gpu_pair(fp, m0, m1, mech=False)
    du_a, gs_a, gt_a = mm.backward_energy(0)
    du_b, gs_b, gt_b = mm.backward_energy(0)
    assert torch.equal(gs_a, gs_b) and torch.equal(gt_a, gt_b) and du_a == du_b
    ms = torch.tensor(m0, dtype=torch.float32, device="cuda", requires_grad=True)
    mt = torch.tensor(m1, dtype=torch.float32, device="cuda", requires_grad=True)
    u = torch.tensor([c * d for c, d in zip(fp.u0, fp.cell)], dtype=torch.float64, requires_grad=True)
    E = InteractionEnergy.apply(mm, 0, ms, mt, u)
    E.backward()
    assert torch.allclose(ms.grad, gs_a) and torch.allclose(mt.grad, gt_a)
    assert np.allclose(u.grad.numpy(), du_a)
    # E is linear in m of either magnet: a finite step along the gradient's
    # own direction changes it by <g, step> (FP32 fields, so a loose bar)
    step = 0.05 * gs_a / gs_a.norm()
    _, E0 = mm.get_force(1)
    mm.set_magnetization(0, ms.detach() + step)
    mm.compute_stray_field(0)
    _, E1 = mm.get_force(1)
    assert abs((E1 - E0) - float((gs_a * step).sum())) <= 1e-3 * abs(float((gs_a * step).sum()))
    mm.close()
