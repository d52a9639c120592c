"""Periodic in-plane boundaries on the GPU against the periodic oracle.

Both films span one period in x and y; kernels summed over periodic images,
circular convolutions, periodic spline and wrapped interpolation and exchange
(oracle/periodic.py states the reading).  Tolerances as for the open path:
rel L2 <= 1e-5 per field, forces against the cancelling-term scale.
"""

import numpy as np
import pytest

import workloads
from oracle import periodic as OP
from tests.pair_setup import force_scale, gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _pair(n, gap, seed, u, lateral=(0, 0), R=1, kind="random"):
    if kind == "random":
        fp, _, _ = workloads.film_pair_plain(n=n, gap=gap, seed=seed)
        m0, m1 = workloads.random_unit(n, seed), workloads.random_unit(n, seed + 5)
    else:
        fp, m0, m1 = workloads.film_pair_stick_slip(n=n, gap=gap, seed=seed)
    fp.u0 = u
    fp.lateral = lateral
    fp.periodic = 3
    fp.pbc_images = R
    return fp, m0, m1


def _system(fp):
    return OP.PeriodicSystem([fp.n_base, fp.n_slider], fp.cell, fp.offsets,
                             [fp.mat_base.as_dict(), fp.mat_slider.as_dict()], fp.mech.as_dict(), fp.pbc_images,
                             u0=fp.u0, H_ext=fp.H_ext)


@pytest.mark.parametrize("n,gap,u,lateral", [
    ((24, 20, 2), 3, (0.37, 0.6, 0.0), (3, -2)),
    ((30, 16, 1), 2, (1.8, -0.25, 0.0), (0, 0)),
    ((20, 18, 5), 2, (0.5, 0.2, 0.0), (1, 1)),   # 5 layers: z summed in a pass of its own
])
def test_periodic_stray_field_force_energy_and_demag(n, gap, u, lateral):
    fp, m0, m1 = _pair(n, gap, 3, u, lateral)
    mm = gpu_pair(fp, m0, m1, mech=False)
    kern = {}
    for src in (0, 1):
        t = 1 - src
        H = mm.compute_stray_field(src).double().cpu().numpy()
        F, E = mm.get_force(t)
        Ms = fp.mat_base.Ms
        M_s, M_t = Ms * (m0 if src == 0 else m1), Ms * (m1 if t == 1 else m0)
        ref = OP.stray_interaction_periodic(M_s, M_t, fp.cell, fp.offsets[src], fp.offsets[t], u, t == 1,
                                            fp.pbc_images, kernels=kern, return_box=True)
        assert rel_l2(H, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M_t, fp.cell)
        assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
        assert abs(E - ref["E"]) < TOL * abs(ref["E"]) + 1e-6 * scale * fp.cell[0]
        Hd = mm.compute_demag(src).double().cpu().numpy()
        assert rel_l2(Hd, OP.demag_periodic(M_s, fp.cell, fp.pbc_images, kern)) < TOL
    mm.close()


def test_periodic_potential_box():
    fp, m0, m1 = _pair((24, 20, 2), 3, 7, (0.3, 0.45, 0.0), (5, 2))
    mm = gpu_pair(fp, m0, m1, mech=False)
    for src in (0, 1):
        t = 1 - src
        phi, lo = mm.compute_potential(src, prefiltered=False)
        coef, _ = mm.compute_potential(src, prefiltered=True)
        z_lo, bz = OP.box_z(fp.n_base[2], fp.offsets[t][2], fp.offsets[src][2], 0.0, t == 1, 4)
        assert tuple(lo) == (0, 0, z_lo) and tuple(phi.shape) == (bz, 20, 24)
        ref = OP.potential_periodic(fp.mat_base.Ms * (m0 if src == 0 else m1), fp.cell, z_lo, bz, fp.pbc_images)
        assert rel_l2(phi.double().cpu().numpy(), ref) < TOL
        assert rel_l2(coef.double().cpu().numpy(), OP.prefilter_periodic(ref)) < TOL
    mm.close()


def test_periodic_whole_period_move():
    """Moving the slider by whole periods changes nothing beyond rounding."""
    fp, m0, m1 = _pair((24, 20, 2), 3, 9, (0.37, 0.6, 0.0))
    mm = gpu_pair(fp, m0, m1, mech=False)
    Ha = mm.compute_stray_field(0).double().cpu().numpy()
    Fa, _ = mm.get_force(1)
    mm.set_displacement(((0.37 + 24) * fp.cell[0], (0.6 - 40) * fp.cell[1], 0.0))
    Hb = mm.compute_stray_field(0).double().cpu().numpy()
    Fb, _ = mm.get_force(1)
    mm.close()
    assert rel_l2(Hb, Ha) < 1e-6
    assert np.max(np.abs(np.array(Fa) - np.array(Fb))) <= 1e-5 * np.max(np.abs(Fa))


def test_periodic_torque_and_fixed_dt_steps():
    """Effective field with wrapped exchange, and three fixed-dt Dormand-Prince
    steps of spring-pulled periodic PMA films."""
    from oracle import dynamics as D
    from oracle.dynamics import llg_rhs

    fp, m0, m1 = _pair((32, 24, 2), 5, 4, (0.25, 0.1, 0.0), kind="pma")
    fp.mech.x0_spring = 2e-9
    fp.mech.v_drive = 50.0
    sysm = _system(fp)
    mm = gpu_pair(fp, m0, m1)
    H_ref, _, _ = sysm.fields(m0, m1, 0.0)
    for g, m in ((0, m0), (1, m1)):
        dm, H = mm.compute_torque(g)
        assert rel_l2(H.double().cpu().numpy(), H_ref[g]) < TOL
        assert rel_l2(dm.double().cpu().numpy(), llg_rhs(m, H_ref[g], fp.mat_base.alpha)) < TOL
    dt = 5e-14
    t_ref, y = D.run_fixed(sysm, [m0, m1, 0.0, 0.0], dt, 3)
    mm.step(3, dt)
    x, v, _ = mm.get_slider_state()
    for g, init in ((0, m0), (1, m1)):
        got = mm.get_magnetization(g).double().cpu().numpy()
        assert rel_l2(got, y[g]) < TOL
        assert rel_l2(got - init, y[g] - init) < 1e-3
    assert abs(x - y[2]) <= 1e-5 * abs(y[2])
    assert abs(v - y[3]) <= 1e-5 * abs(y[3])
    mm.close()


def test_periodic_rejects_unequal_periods_and_unsupported_calls():
    from paper_1801_04181_gb300 import MMError

    fp, m0, m1 = _pair((24, 20, 2), 3, 1, (0.3, 0.0, 0.0))
    fp.n_slider = (24, 18, 2)
    m1 = workloads.random_unit(fp.n_slider, 2)
    with pytest.raises(MMError) as e:
        mm = gpu_pair(fp, m0, m1, mech=False)
        mm.compute_stray_field(0)
    assert e.value.status == -1
    fp, m0, m1 = _pair((24, 20, 2), 3, 1, (0.3, 0.0, 0.0))
    mm = gpu_pair(fp, m0, m1, mech=False)
    with pytest.raises(MMError) as e:
        mm.backward_energy(0)
    assert e.value.status == -7
    mm.close()
