"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance: relative L2 error <= 1e-5 per field for the FP32 path; forces are
compared against the size of the terms that cancel in Eq. (EQForce)
(|F - F_ref| <= 1e-5 mu0 V sum |M| ||Hess||), energies relative.  Sizes span
several CTA tiles and ragged edges (odd extents, nz = 1..4, partial 32 x 8
gather tiles).
"""

import numpy as np
import pytest

import workloads
from oracle import fields as OF
from oracle import kernels as OK
from oracle.interaction import stray_interaction
from tests.pair_setup import force_scale, gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _pair(n0, n1, gap, seed, u_cells, Ms=8e5, lateral=(0, 0)):
    fp, _, _ = workloads.film_pair_plain(n=n0, gap=gap, seed=seed)
    fp.n_slider = n1
    fp.u0 = u_cells
    fp.lateral = lateral
    m0 = workloads.random_unit(n0, seed)
    m1 = workloads.random_unit(n1, seed + 7)
    fp.mat_base.Ms = Ms
    return fp, m0, m1, fp.offsets


def _gpu(fp, m0, m1, offsets, **kw):
    assert list(offsets) == list(fp.offsets)
    return gpu_pair(fp, m0, m1, mech=False, **kw)


def test_kernel_values_fp64_match_oracle():
    from paper_1801_04181_gb300 import eval_kernel_fp64

    cell = (4e-9, 3e-9, 2e-9)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.integers(-6, 7, size=(40, 3)), rng.integers(-60, 61, size=(40, 3)),
                          [[0, 0, 0], [1, 0, 0], [16, 3, 1], [17, 3, 1], [0, 0, 16], [0, 0, 17]]])
    off = idx * np.array(cell)
    S = eval_kernel_fp64(0, off, cell).cpu().numpy()
    N = eval_kernel_fp64(1, off, cell).cpu().numpy()
    S_ref = OK.S_kernel(off[:, 0], off[:, 1], off[:, 2], *cell)
    N_ref = OK.N_kernel(off[:, 0], off[:, 1], off[:, 2], *cell)
    for got, ref in ((S, S_ref), (N, N_ref)):
        scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
        # the closed forms cancel ~1e6 at 16 cells: FP64 rounding order differs
        assert np.max(np.abs(got - ref) / scale) < 1e-8


@pytest.mark.parametrize("n0,n1,gap,u", [
    ((40, 24, 1), (40, 24, 1), 1, (0.3125, 0.0, 0.0)),
    ((37, 21, 2), (29, 26, 3), 2, (0.71, 0.45, 0.0)),
    ((33, 17, 4), (33, 17, 1), 3, (1.6, -0.2, 0.3)),
])
def test_potential_box_matches_oracle(n0, n1, gap, u):
    fp, m0, m1, offs = _pair(n0, n1, gap, 11, u)
    mm = _gpu(fp, m0, m1, offs)
    for src in (0, 1):
        t = 1 - src
        phi, lo = mm.compute_potential(src, prefiltered=False)
        coef, lo2 = mm.compute_potential(src, prefiltered=True)
        n_t = (fp.n_slider if t == 1 else fp.n_base)
        box_lo, box_dims = OF.box_for_target(n_t, offs[t], offs[src], u, t == 1)
        assert tuple(lo) == tuple(box_lo) and tuple(lo2) == tuple(box_lo)
        assert tuple(phi.shape) == tuple(reversed(box_dims))
        Ms = fp.mat_base.Ms if src == 0 else fp.mat_slider.Ms
        m_s = m0 if src == 0 else m1
        ref = OF.potential_conv(Ms * m_s, fp.cell, box_lo, box_dims)
        assert rel_l2(phi.double().cpu().numpy(), ref) < TOL
        from oracle.spline import prefilter_3d
        assert rel_l2(coef.double().cpu().numpy(), prefilter_3d(ref)) < TOL
    mm.close()


@pytest.mark.parametrize("n0,n1,gap,u", [
    ((40, 24, 1), (40, 24, 1), 1, (0.3125, 0.0, 0.0)),
    ((37, 21, 2), (29, 26, 3), 2, (0.71, 0.45, 0.0)),
    ((70, 19, 4), (45, 33, 2), 3, (2.6, -1.2, 0.3)),
    ((64, 64, 1), (64, 64, 1), 1, (0.0, 0.0, 0.0)),
])
@pytest.mark.parametrize("lateral", [(0, 0), (9, -5)])
def test_stray_field_force_energy_match_oracle(n0, n1, gap, u, lateral):
    fp, m0, m1, offs = _pair(n0, n1, gap, 5, u, lateral=lateral)
    mm = _gpu(fp, m0, m1, offs)
    for src in (0, 1):
        t = 1 - src
        Hg = mm.compute_stray_field(src).double().cpu().numpy()
        F, E = mm.get_force(t)
        Ms_s = fp.mat_base.Ms if src == 0 else fp.mat_slider.Ms
        Ms_t = fp.mat_slider.Ms if t == 1 else fp.mat_base.Ms
        M_s = Ms_s * (m0 if src == 0 else m1)
        M_t = Ms_t * (m1 if t == 1 else m0)
        ref = stray_interaction(M_s, M_t, fp.cell, offs[src], offs[t], u, t == 1, return_box=True)
        assert rel_l2(Hg, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M_t, fp.cell)
        assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
        assert abs(E - ref["E"]) < TOL * abs(ref["E"]) + 1e-6 * scale * fp.cell[0]
    mm.close()


@pytest.mark.parametrize("n,axis,Q,plan", [((12, 256, 2), 1, 540, [4, 9, 15]),
                                           ((1024, 12, 2), 0, 2160, [16, 9, 15])])
def test_stick_slip_transform_lengths_match_oracle(n, axis, Q, plan):
    """Films 256 cells wide in y (1024 long in x) take the 540-point y (2160-point
    x) transform of the stick-slip pair, whose plans run with their lengths as
    compile-time constants: the stray field, force and energy both ways and the
    demag field against the oracle on a strip of that width (length)."""
    from paper_1801_04181_gb300 import fft_plan, tuned_plan

    fp, m0, m1, offs = _pair(n, n, 5, 9, (0.43, 0.0, 0.0))
    mm = _gpu(fp, m0, m1, offs)
    for src in (0, 1):
        assert mm.plan_info(src)["fft"][axis] == Q
        assert (tuned_plan(Q) or fft_plan(Q)) == plan
    for src in (0, 1):
        t = 1 - src
        Hg = mm.compute_stray_field(src).double().cpu().numpy()
        F, E = mm.get_force(t)
        Ms_s = fp.mat_base.Ms if src == 0 else fp.mat_slider.Ms
        Ms_t = fp.mat_slider.Ms if t == 1 else fp.mat_base.Ms
        M_s = Ms_s * (m0 if src == 0 else m1)
        M_t = Ms_t * (m1 if t == 1 else m0)
        ref = stray_interaction(M_s, M_t, fp.cell, offs[src], offs[t], (0.43, 0.0, 0.0), t == 1, return_box=True)
        assert rel_l2(Hg, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M_t, fp.cell)
        assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
        assert abs(E - ref["E"]) < TOL * abs(ref["E"]) + 1e-6 * scale * fp.cell[0]
    for g in (0, 1):
        Hd = mm.compute_demag(g).double().cpu().numpy()
        Ms = fp.mat_base.Ms if g == 0 else fp.mat_slider.Ms
        ref = OF.demag_conv(Ms * (m0 if g == 0 else m1), fp.cell)
        assert rel_l2(Hd, ref) < TOL
    mm.close()


@pytest.mark.parametrize("n", [(40, 24, 1), (37, 21, 2), (33, 17, 3), (19, 31, 4)])
def test_demag_matches_oracle(n):
    fp, m0, m1, offs = _pair(n, n, 2, 21, (0.0, 0.0, 0.0))
    mm = _gpu(fp, m0, m1, offs)
    for g, m in ((0, m0), (1, m1)):
        H = mm.compute_demag(g).double().cpu().numpy()
        ref = OF.demag_conv(fp.mat_base.Ms * m, fp.cell)
        assert rel_l2(H, ref) < TOL
    mm.close()


def test_whole_cell_displacement_is_index_shift_bitwise():
    fp, m0, m1, offs = _pair((36, 20, 2), (36, 20, 2), 2, 31, (1.0, 0.0, 0.0))
    mm = _gpu(fp, m0, m1, offs)
    H_a = mm.compute_stray_field(0).cpu().numpy()
    F_a, _ = mm.get_force(1)
    mm.close()
    fp.lateral = (1, 0)
    fp.u0 = (0.0, 0.0, 0.0)
    mm = _gpu(fp, m0, m1, fp.offsets)
    H_b = mm.compute_stray_field(0).cpu().numpy()
    F_b, _ = mm.get_force(1)
    mm.close()
    assert np.array_equal(H_a, H_b)
    assert F_a == F_b


def test_offset_sweep_plain_films():
    """64x64x1 films, gap 1 cell, 16 offsets in [0, 1): field and x-force per offset."""
    fp, m0, m1 = workloads.film_pair_plain(n=(64, 64, 1), gap=1, seed=0)
    mm = gpu_pair(fp, m0, m1, mech=False)
    M0 = fp.mat_base.Ms * m0
    M1 = fp.mat_slider.Ms * m1
    cache = {}
    for k in range(16):
        u = (k / 16.0, 0.0, 0.0)
        mm.set_displacement(tuple(v * c for v, c in zip(u, fp.cell)))
        mm.compute_fields()
        F, E = mm.get_force(1)
        Hg = mm.compute_stray_field(0).double().cpu().numpy()
        ref = stray_interaction(M0, M1, fp.cell, fp.offsets[0], fp.offsets[1], u, True,
                                kernel_cache=cache, return_box=True)
        assert rel_l2(Hg, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M1, fp.cell)
        assert abs(F[0] - ref["F"][0]) < TOL * scale
    mm.close()


def test_torque_matches_oracle():
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(48, 20, 2), gap=5, seed=2)
    fp.u0 = (0.4, 0.0, 0.0)
    fp.H_ext = (1e4, -2e4, 5e4)
    mm = gpu_pair(fp, m0, m1)
    from tests.pair_setup import oracle_system
    from oracle.dynamics import llg_rhs

    sysm = oracle_system(fp)
    H_ref, _, _ = sysm.fields(m0, m1, 0.0)
    for g, m in ((0, m0), (1, m1)):
        dm, H = mm.compute_torque(g)
        assert rel_l2(H.double().cpu().numpy(), H_ref[g]) < TOL
        ref = llg_rhs(m, H_ref[g], fp.mat_base.alpha)
        assert rel_l2(dm.double().cpu().numpy(), ref) < TOL
    mm.close()


def test_fixed_dt_steps_match_oracle():
    """Five fixed-dt Dormand-Prince steps of spring-pulled PMA films (shrunk)."""
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(40, 24, 2), gap=5, seed=4)
    fp.u0 = (0.25, 0.0, 0.0)
    fp.mech.x0_spring = 2e-9
    fp.mech.v_drive = 50.0
    mm = gpu_pair(fp, m0, m1)
    from tests.pair_setup import oracle_system
    from oracle import dynamics as D

    sysm = oracle_system(fp)
    dt = 5e-14
    t_ref, y = D.run_fixed(sysm, [m0, m1, 0.0, 0.0], dt, 5)
    t, _ = mm.step(5, dt)
    x, v, tt = mm.get_slider_state()
    for g in (0, 1):
        got = mm.get_magnetization(g).double().cpu().numpy()
        assert rel_l2(got, y[g]) < TOL
        # the per-step change is what the stepper computes: compare it too
        init = m0 if g == 0 else m1
        assert rel_l2(got - init, y[g] - init) < 1e-3
    assert abs(tt - t_ref) < 1e-20
    assert abs(x - y[2]) <= 1e-5 * abs(y[2])
    assert abs(v - y[3]) <= 1e-5 * abs(y[3])
    mm.close()


def test_euler_steps_match_oracle():
    """Five fixed-dt explicit Euler steps of the same spring-pulled films: one
    field evaluation per step, the slider advanced by the same step (Sec. III)."""
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(40, 24, 2), gap=5, seed=4)
    fp.u0 = (0.25, 0.0, 0.0)
    fp.mech.x0_spring = 2e-9
    fp.mech.v_drive = 50.0
    mm = gpu_pair(fp, m0, m1, integrator="euler")
    from tests.pair_setup import oracle_system
    from oracle import dynamics as D

    dt = 5e-14
    t_ref, y = D.run_euler(oracle_system(fp), [m0, m1, 0.0, 0.0], dt, 5)
    t, _ = mm.step(5, dt)
    x, v, tt = mm.get_slider_state()
    for g in (0, 1):
        got = mm.get_magnetization(g).double().cpu().numpy()
        init = m0 if g == 0 else m1
        assert rel_l2(got, y[g]) < TOL
        assert rel_l2(got - init, y[g] - init) < 1e-3
    assert abs(tt - t_ref) < 1e-20
    assert abs(x - y[2]) <= 1e-5 * abs(y[2])
    assert abs(v - y[3]) <= 1e-5 * abs(y[3])
    # the Euler and RK45 results differ by the Euler step's O(dt^2) error:
    # the test would not tell them apart if the two paths were the same
    _, y45 = D.run_fixed(oracle_system(fp), [m0, m1, 0.0, 0.0], dt, 5)
    assert rel_l2(y[0] - m0, y45[0] - m0) > 1e-2
    mm.close()


def test_euler_rejects_adaptive_and_conduction():
    """The Euler integrator steps with a fixed dt (no error estimate), and the
    eddy coupling is defined on the RK45 step: both requests are refused."""
    from paper_1801_04181_gb300 import MMError, MovingMagnets

    with pytest.raises(MMError):
        MovingMagnets(adaptive=True, integrator="euler")
    with pytest.raises(ValueError):
        MovingMagnets(integrator="midpoint")
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(16, 8, 1), gap=5, seed=4)
    mm = gpu_pair(fp, m0, m1, integrator="euler")
    with pytest.raises(MMError):
        mm.set_conductivity(0, 1e6)
    mm.close()


def test_checkpoint_resume_is_bitwise():
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(32, 16, 2), gap=5, seed=8)
    fp.mech.x0_spring = 1e-9
    mm = gpu_pair(fp, m0, m1)
    mm.step(2, 5e-14)
    blob = mm.get_state()
    mm.step(3, 5e-14)
    a = [mm.get_magnetization(g).cpu().numpy() for g in (0, 1)]
    sa = mm.get_slider_state()
    mm.set_state(blob)
    mm.step(3, 5e-14)
    b = [mm.get_magnetization(g).cpu().numpy() for g in (0, 1)]
    sb = mm.get_slider_state()
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    assert sa == sb
    mm.close()


@pytest.mark.parametrize("n0,n1,gap,u,lateral", [
    ((20, 17, 2), (18, 15, 2), 2, (0.3, 0.45, 0.0), (1, -2)),
    ((37, 9, 1), (33, 11, 3), 3, (1.7, -0.25, 0.0), (0, 0)),
    ((12, 13, 6), (11, 10, 2), 2, (0.6, 0.2, 0.0), (2, 1)),   # a 6-layer source: z summed in its own pass
])
def test_componentwise_variant_matches_oracle(n0, n1, gap, u, lateral):
    """The direct componentwise interpolation of the tensor field (Sec. II.A's
    second method) against the oracle's, both directions, element by element
    within the field bar."""
    from oracle.variants import stray_field_componentwise

    fp, m0, m1, offs = _pair(n0, n1, gap, 17, u, lateral=lateral)
    mm = _gpu(fp, m0, m1, offs)
    for src in (0, 1):
        t = 1 - src
        H = mm.compute_stray_field_componentwise(src).double().cpu().numpy()
        Ms = fp.mat_base.Ms if src == 0 else fp.mat_slider.Ms
        m_s = m0 if src == 0 else m1
        n_t = fp.n_slider if t == 1 else fp.n_base
        ref = stray_field_componentwise(Ms * m_s, fp.cell, offs[src], offs[t], n_t, u, t == 1)
        assert rel_l2(H, ref) < TOL
    mm.close()


def test_adaptive_steps_accept_and_stay_normalised():
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(48, 24, 2), gap=5, seed=9)
    mm = gpu_pair(fp, m0, m1, adaptive=True, rtol=1e-5)
    t, dt = mm.step(10, 1e-14)
    acc, rej = mm.step_stats()
    assert acc == 10 and t > 0 and dt > 0
    for g in (0, 1):
        m = mm.get_magnetization(g).double().cpu().numpy()
        assert np.max(np.abs(np.sqrt((m ** 2).sum(axis=0)) - 1)) < 1e-6
    mm.close()


def test_adaptive_attempts_match_oracle():
    """Adaptive Dormand-Prince steps of shrunk stick-slip films, attempt by
    attempt, with a first step far too large (so the controller rejects and
    shrinks it):
      * replay: the oracle steps from the same state with the GPU's dt of each
        attempt; the error norms agree within TOL times the size of the terms
        that cancel in them (dt sum_j |b5_j - b4_j| max |k_j|, the reading of
        the force tolerance applied to the error estimate) and the accept /
        reject decisions are identical wherever err is not within that
        tolerance of rtol;
      * run_adaptive from the same start: the same decisions, and step sizes
        within 1e-3 relative (dt is 0.9 (rtol/err)^(1/5) times the last one,
        so a relative error e of err moves the next dt by e/5 and nothing
        accumulates);
      * the accepted state (m of both films, x, v) against run_adaptive's."""
    from oracle import dynamics as D
    from tests.pair_setup import oracle_system

    fp, m0, m1 = workloads.film_pair_stick_slip(n=(40, 24, 2), gap=5, seed=21)
    fp.u0 = (0.3, 0.0, 0.0)
    fp.mech.x0_spring = 2e-9
    fp.mech.v_drive = 50.0
    # about three times the step the controller settles to on these films
    # (~2.5e-13 s, held by the stiffest exchange modes): the oracle's err is
    # ~3e-3, so the attempt is rejected while its stage values stay bounded
    # (from ~2e-12 s on, the stages blow up: err 63 at 2e-12 s, 2e61 at 4e-12 s)
    rtol, dt0, nacc = 1e-5, 8e-13, 6
    mm = gpu_pair(fp, m0, m1, adaptive=True, rtol=rtol)
    mm.clear_attempt_log()
    t_gpu, dt_gpu = mm.step(nacc, dt0)
    log = mm.attempt_log()
    assert sum(a["accepted"] for a in log) == nacc
    assert not log[0]["accepted"], "the first attempt should be rejected"
    x_gpu, v_gpu, _ = mm.get_slider_state()
    got = [mm.get_magnetization(g).double().cpu().numpy() for g in (0, 1)]
    mm.close()

    sysm = oracle_system(fp)
    sum_db = sum(abs(b5 - b4) for b5, b4 in zip(D.DP_B5, D.DP_B4))
    # replay at the GPU's step sizes
    t, y, k1 = 0.0, [m0, m1, 0.0, 0.0], None
    for a in log:
        assert abs(a["t"] - t) <= 1e-12 * max(t, 1e-30)
        y5, y4, ks = D.dp45_embedded(sysm, t, y, a["dt"], k1)
        err = max(float(np.max(np.abs(y5[i] - y4[i]))) for i in (0, 1))
        kmax = max(float(np.max(np.abs(k[i]))) for k in ks for i in (0, 1))
        tol = TOL * a["dt"] * sum_db * kmax
        assert abs(a["err"] - err) <= tol, (a, err, tol)
        if abs(err - rtol) > tol:
            assert a["accepted"] == (err <= rtol), (a, err)
        if a["accepted"]:
            y = [D.normalise(y5[0]), D.normalise(y5[1]), y5[2], y5[3]]
            t += a["dt"]
            k1 = ks[6]
    # the oracle's own adaptive run from the same start
    trace = []
    t_ref, y_ref, dt_ref, acc, rej = D.run_adaptive(sysm, [m0, m1, 0.0, 0.0], dt0, nacc, rtol, trace=trace)
    assert len(trace) == len(log)
    for a, b in zip(log, trace):
        assert a["accepted"] == b["accepted"]
        assert abs(a["dt"] - b["dt"]) <= 1e-3 * b["dt"]
    assert abs(dt_gpu - dt_ref) <= 1e-3 * dt_ref
    assert abs(t_gpu - t_ref) <= 1e-3 * t_ref
    for g in (0, 1):
        assert rel_l2(got[g], y_ref[g]) < 1e-4
    assert abs(x_gpu - y_ref[2]) <= 1e-3 * abs(y_ref[2])
    assert abs(v_gpu - y_ref[3]) <= 1e-3 * abs(y_ref[3])


def test_bad_arguments_are_rejected():
    from paper_1801_04181_gb300 import MMError, MovingMagnets

    mm = MovingMagnets()
    with pytest.raises(MMError):
        mm.set_grid(0, (8, 8, 0), (1e-9, 1e-9, 1e-9))   # empty grid
    with pytest.raises(MMError):
        mm.set_grid(2, (8, 8, 1), (1e-9, 1e-9, 1e-9))   # no magnet 2
    mm.set_grid(0, (8, 8, 1), (1e-9, 1e-9, 1e-9))
    with pytest.raises(MMError):
        mm.set_grid(1, (8, 8, 1), (2e-9, 1e-9, 1e-9))   # different cell
    with pytest.raises(MMError):
        mm.compute_fields()                             # nothing else set
    mm.close()


def test_power_bookkeeping_matches_oracle():
    """P_in = -F . v_s, the Gilbert dissipation of each magnet and the drive's
    viscous loss at a state with the slider moving (Sec. III, after Eq. (EQForce))."""
    from oracle.dynamics import power_balance
    from tests.pair_setup import oracle_system

    fp, m0, m1 = workloads.film_pair_stick_slip(n=(44, 22, 2), gap=5, seed=6)
    fp.u0 = (0.35, 0.0, 0.0)
    fp.H_ext = (2e4, 0.0, -1e4)
    mm = gpu_pair(fp, m0, m1)
    x, v = 3e-10, 4.0
    mm.set_slider_state(x, v, 0.0)
    P = mm.power()
    ref = power_balance(oracle_system(fp), m0, m1, x, v)
    for g in (0, 1):
        assert abs(P["P_diss"][g] - ref["P_diss"][g]) <= TOL * ref["P_diss"][g]
    box = stray_interaction(fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1, fp.cell, fp.offsets[0], fp.offsets[1],
                            oracle_system(fp).displacement(x), True, return_box=True)
    scale = force_scale(box["hess_n"], fp.mat_slider.Ms * m1, fp.cell)
    assert abs(P["P_in"] - ref["P_in"]) <= TOL * scale * v
    assert abs(P["P_visc"] - ref["P_visc"]) <= 1e-12 * ref["P_visc"]
    # the call leaves the state alone: stepping still works and repeats it
    mm.step(1, 5e-14)
    mm.close()


def _dc_bound(H_ref, cell, rel):
    """Bound on |D - D_ref| (and |C - C_ref|) from a field error of `rel` times the
    rms field: each central difference moves by at most twice the field error
    over 2 d_a, and a divergence or curl component sums two or three of them."""
    rms = float(np.sqrt(np.mean(np.sum(np.asarray(H_ref, float) ** 2, axis=0))))
    return rel * 3.0 * rms * sum(1.0 / d for d in cell)


def test_div_curl_of_interpolated_stray_field_matches_oracle():
    """Sec. IV.A: a frozen random base film (four layers, so z derivatives
    exist), its stray field sampled inside the slider at partial moves x; the
    CUDA diagnostic on the CUDA field against the oracle's diagnostic on the
    same FP32 field and on the oracle's own FP64 field."""
    from oracle.diagnostics import div_curl_means

    fp, m0, m1 = workloads.film_pair_plain((26, 21, 4), 1, 5)
    fp.n_slider = (23, 19, 4)
    M0, M1 = fp.mat_base.Ms * m0, fp.mat_slider.Ms * workloads.random_unit(fp.n_slider, 6)
    for u in (0.0, 0.3125, 0.75):
        fp.u0 = (u, 0.0, 0.0)
        mm = gpu_pair(fp, m0, M1 / fp.mat_slider.Ms, mech=False)
        H = mm.compute_stray_field(0)
        D, C = mm.div_curl(H, fp.cell)
        Hn = H.double().cpu().numpy()
        Dg, Cg = div_curl_means(Hn, fp.cell)
        b32 = _dc_bound(Hn, fp.cell, 1e-6)
        assert abs(D - Dg) <= b32 and abs(C - Cg) <= b32
        ref = stray_interaction(M0, M1, fp.cell, fp.offsets[0], fp.offsets[1], fp.u0, True)
        Dr, Cr = div_curl_means(ref["H"], fp.cell)
        assert rel_l2(Hn, ref["H"]) < TOL
        b = _dc_bound(ref["H"], fp.cell, TOL)
        assert abs(D - Dr) <= b and abs(C - Cr) <= b
        assert D > 0 and C > 0
        mm.close()


@pytest.mark.parametrize("n0,n1,gap,u", [
    ((30, 22, 2), (27, 19, 3), 2, (0.41, 0.17, 0.0)),
    ((25, 24, 1), (25, 24, 1), 1, (1.75, -0.3, 0.0)),
])
def test_fd4_variant_matches_oracle(n0, n1, gap, u):
    """The four-point difference variant of the stray field against the oracle's.
    Differencing FP32 values of phi costs up to (1 + 8 + 8 + 1)/12 of their
    rounding per cell over d: the bar is the larger of the field bar and three
    FP32 roundings of the rms interpolant value propagated that way."""
    from oracle.variants import stray_field_fd4

    fp, m0, m1, offs = _pair(n0, n1, gap, 12, u)
    mm = _gpu(fp, m0, m1, offs)
    for src in (0, 1):
        t = 1 - src
        H = mm.compute_stray_field_fd4(src).double().cpu().numpy()
        Ms = fp.mat_base.Ms if src == 0 else fp.mat_slider.Ms
        m_s = m0 if src == 0 else m1
        n_t = fp.n_slider if t == 1 else fp.n_base
        ref, val = stray_field_fd4(Ms * m_s, fp.cell, offs[src], offs[t], n_t, u, t == 1)
        err = np.linalg.norm((H - ref).ravel())
        rms_v = float(np.sqrt(np.mean(val ** 2)))
        bound = 3 * 2.0 ** -23 * rms_v * 1.5 * np.sqrt(sum(1.0 / d ** 2 for d in fp.cell)) * np.sqrt(H[0].size)
        assert err <= max(TOL * np.linalg.norm(ref.ravel()), bound)
        # a sanity check only: the variant and the analytic gradient of the same
        # interpolant differ by the difference's truncation error
        Ha = mm.compute_stray_field(src).double().cpu().numpy()
        assert 0.0 < rel_l2(H, Ha) < 1.0
    mm.close()
