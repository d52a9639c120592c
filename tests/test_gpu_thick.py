"""Thick magnets (nz > 4) against the FP64 CPU oracle, through the C ABI.

Sources of up to 8 layers take z by a direct sum over planes between the
y-forward and y-inverse passes; thicker ones take z by FFT.  Both are covered.

Same bar as the thin-film parity tests: relative L2 <= 1e-5 per field, forces
against the size of the terms that cancel in Eq. (EQForce).  Sizes are odd
and ragged so that every pass sees partial tiles: several z-pass tiles of
eight y positions, gather chunks of four layers with a short last chunk, and
z grids of several FFT stages.
"""

import numpy as np
import pytest

import workloads
from oracle import fields as OF
from oracle.interaction import stray_interaction
from tests.pair_setup import force_scale, gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _cubes(n0, n1, gap, u, seed, lateral=(0, 0), axis=0):
    fp, _, _ = workloads.cube_pair(n0, gap, seed)
    fp.n_slider = n1
    fp.stack_axis = axis
    fp.lateral = lateral
    fp.u0 = u
    m0 = workloads.random_unit(n0, seed)
    m1 = workloads.random_unit(n1, seed + 3)
    return fp, m0, m1


@pytest.mark.parametrize("n", [(13, 11, 9), (10, 12, 7), (9, 8, 16)])
def test_thick_demag_matches_oracle(n):
    fp, m0, m1 = _cubes(n, n, 3, (0.0, 0.0, 0.0), 2)
    mm = gpu_pair(fp, m0, m1, mech=False)
    for g, m in ((0, m0), (1, m1)):
        H = mm.compute_demag(g).double().cpu().numpy()
        ref = OF.demag_conv(fp.mat_base.Ms * m, fp.cell)
        assert rel_l2(H, ref) < TOL
    assert (mm.plan_info(0)["Qz"] > 0) == (n[2] > 8)
    mm.close()


@pytest.mark.parametrize("n0,n1,gap,u,axis", [
    ((12, 10, 8), (9, 11, 6), 3, (0.37, 0.2, 0.0), 0),
    ((12, 10, 10), (9, 11, 9), 3, (0.37, 0.2, 0.1), 0),
    ((11, 9, 7), (11, 9, 7), 2, (1.6, -0.3, 0.45), 0),
    ((10, 9, 6), (8, 7, 5), 2, (0.25, 0.5, 0.7), 2),
])
def test_thick_potential_box_matches_oracle(n0, n1, gap, u, axis):
    from oracle.spline import prefilter_3d

    fp, m0, m1 = _cubes(n0, n1, gap, u, 7, axis=axis)
    offs = fp.offsets
    mm = gpu_pair(fp, m0, m1, mech=False)
    for src in (0, 1):
        t = 1 - src
        phi, lo = mm.compute_potential(src, prefiltered=False)
        coef, _ = mm.compute_potential(src, prefiltered=True)
        n_t = fp.n_slider if t == 1 else fp.n_base
        box_lo, box_dims = OF.box_for_target(n_t, offs[t], offs[src], u, t == 1)
        assert tuple(lo) == tuple(box_lo)
        m_s = m0 if src == 0 else m1
        ref = OF.potential_conv(fp.mat_base.Ms * m_s, fp.cell, box_lo, box_dims)
        assert rel_l2(phi.double().cpu().numpy(), ref) < TOL
        assert rel_l2(coef.double().cpu().numpy(), prefilter_3d(ref)) < TOL
    mm.close()


@pytest.mark.parametrize("n0,n1,gap,u,axis,lateral", [
    ((12, 10, 8), (9, 11, 6), 3, (0.37, 0.2, 0.0), 0, (0, 0)),
    ((12, 10, 10), (9, 11, 9), 3, (0.37, 0.2, 0.1), 0, (1, 0)),
    ((13, 9, 12), (10, 8, 4), 2, (0.55, 0.3, 0.2), 2, (1, 2)),    # z-FFT source over a thin target
    ((11, 9, 7), (11, 9, 7), 2, (1.6, -0.3, 0.45), 0, (2, -1)),
    ((10, 9, 6), (8, 7, 5), 2, (0.25, 0.5, 0.7), 2, (0, 0)),
    ((20, 14, 2), (9, 7, 6), 2, (0.6, 0.1, 0.3), 2, (3, 2)),   # thin source under a thick target
])
def test_thick_stray_field_force_energy_match_oracle(n0, n1, gap, u, axis, lateral):
    fp, m0, m1 = _cubes(n0, n1, gap, u, 5, lateral=lateral, axis=axis)
    offs = fp.offsets
    mm = gpu_pair(fp, m0, m1, mech=False)
    Ms = fp.mat_base.Ms
    for src in (0, 1):
        t = 1 - src
        Hg = mm.compute_stray_field(src).double().cpu().numpy()
        F, E = mm.get_force(t)
        M_s = Ms * (m0 if src == 0 else m1)
        M_t = Ms * (m1 if t == 1 else m0)
        ref = stray_interaction(M_s, M_t, fp.cell, offs[src], offs[t], u, t == 1, return_box=True)
        assert rel_l2(Hg, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M_t, fp.cell)
        assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
        assert abs(E - ref["E"]) < TOL * abs(ref["E"]) + 1e-6 * scale * fp.cell[0]
    mm.close()


def test_thick_whole_cell_displacement_is_index_shift_bitwise():
    fp, m0, m1 = _cubes((12, 10, 7), (12, 10, 7), 3, (1.0, 0.0, 0.0), 9)
    mm = gpu_pair(fp, m0, m1, mech=False)
    H_a = mm.compute_stray_field(0).cpu().numpy()
    F_a, _ = mm.get_force(1)
    mm.close()
    fp.gap = 4
    fp.u0 = (0.0, 0.0, 0.0)
    mm = gpu_pair(fp, m0, m1, mech=False)
    H_b = mm.compute_stray_field(0).cpu().numpy()
    F_b, _ = mm.get_force(1)
    mm.close()
    assert np.array_equal(H_a, H_b)
    assert F_a == F_b


def test_thick_fixed_dt_steps_match_oracle():
    """Three fixed-dt Dormand-Prince steps of two vortex cubes, slider pulled along x."""
    fp, m0, m1 = workloads.cube_pair((10, 9, 8), 3, 4)
    fp.u0 = (0.3, 0.0, 0.0)
    fp.mech.x0_spring = 2e-9
    fp.mech.v_drive = 50.0
    mm = gpu_pair(fp, m0, m1)
    from oracle import dynamics as D
    from tests.pair_setup import oracle_system

    sysm = oracle_system(fp)
    dt = 5e-14
    t_ref, y = D.run_fixed(sysm, [m0, m1, 0.0, 0.0], dt, 3)
    mm.step(3, dt)
    x, v, tt = mm.get_slider_state()
    for g in (0, 1):
        got = mm.get_magnetization(g).double().cpu().numpy()
        assert rel_l2(got, y[g]) < TOL
        init = m0 if g == 0 else m1
        assert rel_l2(got - init, y[g] - init) < 1e-3
    assert abs(tt - t_ref) < 1e-20
    assert abs(x - y[2]) <= 1e-5 * abs(y[2])
    assert abs(v - y[3]) <= 1e-5 * abs(y[3])
    mm.close()
