"""Parity at the benchmark size: 1024 x 256 x 2 stick-slip film pair (GPU).

The CUDA path runs the grids and launch configuration bench.py times; the FP64
oracle evaluates the same stray field (linear convolution, banded prefilter,
64-term evaluation), force, energy and self-demag field at full size.  Its
kernel windows are filled by a spawn process pool (one z plane per task).
Both directions (base -> slider and slider -> base), one fixed-dt
Dormand-Prince step of the whole pair with the slider, and the index-shift
property at full size, bit for bit on the GPU.
"""

import multiprocessing as mp
import os

import numpy as np
import pytest

import workloads
from oracle import fields as OF
from oracle.interaction import stray_interaction
from tests.pair_setup import force_scale, gpu_pair, oracle_kernel_windows, oracle_system, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def pool():
    p = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    yield p
    p.close()
    p.join()


def test_full_size_stray_field_force_and_demag(pool):
    fp, m0, m1 = workloads.film_pair_stick_slip(seed=0)
    fp.u0 = (0.37, 0.0, 0.0)
    mm = gpu_pair(fp, m0, m1)
    H = mm.compute_stray_field(0).double().cpu().numpy()
    F, E = mm.get_force(1)
    Hd = mm.compute_demag(0).double().cpu().numpy()
    info = mm.plan_info(0)
    mm.close()

    box_lo, box_dims = OF.box_for_target(fp.n_slider, fp.offsets[1], fp.offsets[0], fp.u0, True)
    assert tuple(info["box_lo"]) == tuple(box_lo) and tuple(info["box"]) == tuple(box_dims)
    S, N = oracle_kernel_windows(fp.n_base, fp.cell, box_lo, box_dims, pool)
    key = ("S", (3,) + tuple(reversed(fp.n_base)), tuple(fp.cell), tuple(box_lo), tuple(box_dims))
    M0, M1 = fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1
    ref = stray_interaction(M0, M1, fp.cell, fp.offsets[0], fp.offsets[1], fp.u0, True,
                            kernel_cache={key: S}, return_box=True)
    assert rel_l2(H, ref["H"]) < TOL
    scale = force_scale(ref["hess_n"], M1, fp.cell)
    assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
    assert abs(E - ref["E"]) < TOL * abs(ref["E"])
    Hd_ref = OF.demag_conv(M0, fp.cell, kernel=N)
    assert rel_l2(Hd, Hd_ref) < TOL


def test_full_size_slider_to_base_stray_field_and_force(pool):
    fp, m0, m1 = workloads.film_pair_stick_slip(seed=0)
    fp.u0 = (0.37, 0.0, 0.0)
    mm = gpu_pair(fp, m0, m1)
    H = mm.compute_stray_field(1).double().cpu().numpy()
    F, E = mm.get_force(0)
    Hd = mm.compute_demag(1).double().cpu().numpy()
    info = mm.plan_info(1)
    mm.close()

    box_lo, box_dims = OF.box_for_target(fp.n_base, fp.offsets[0], fp.offsets[1], fp.u0, False)
    assert tuple(info["box_lo"]) == tuple(box_lo) and tuple(info["box"]) == tuple(box_dims)
    S, N = oracle_kernel_windows(fp.n_slider, fp.cell, box_lo, box_dims, pool)
    key = ("S", (3,) + tuple(reversed(fp.n_slider)), tuple(fp.cell), tuple(box_lo), tuple(box_dims))
    M0, M1 = fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1
    ref = stray_interaction(M1, M0, fp.cell, fp.offsets[1], fp.offsets[0], fp.u0, False,
                            kernel_cache={key: S}, return_box=True)
    assert rel_l2(H, ref["H"]) < TOL
    scale = force_scale(ref["hess_n"], M0, fp.cell)
    assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
    assert abs(E - ref["E"]) < TOL * abs(ref["E"])
    assert rel_l2(Hd, OF.demag_conv(M1, fp.cell, kernel=N)) < TOL


def test_full_size_fixed_dt_step_of_the_pair(pool):
    """One Dormand-Prince step (seven field evaluations: both stray fields,
    both demag fields, exchange, anisotropy, LLG, slider) of the whole
    1024 x 256 x 2 pair against the oracle's run_fixed, at a step size of the
    order the adaptive bench run settles to.  m of both films within TOL
    (rel L2), and their per-step change within 1e-3; the slider's x and v
    within TOL relative plus the share of a force error of TOL times the
    cancelling-term scale (integrated over the step)."""
    from oracle import dynamics as D

    fp, m0, m1 = workloads.film_pair_stick_slip(seed=0)
    fp.u0 = (0.37, 0.0, 0.0)
    fp.mech.x0_spring = 2e-9
    dt = 3e-13
    mm = gpu_pair(fp, m0, m1, adaptive=False)
    mm.step(1, dt)
    got = [mm.get_magnetization(g).double().cpu().numpy() for g in (0, 1)]
    x, v, t = mm.get_slider_state()
    mm.close()

    sysm = oracle_system(fp)
    M0, M1 = fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1
    for src, tgt, o_s, o_t, slider in ((fp.n_base, fp.n_slider, 0, 1, True), (fp.n_slider, fp.n_base, 1, 0, False)):
        box_lo, box_dims = OF.box_for_target(tgt, fp.offsets[o_t], fp.offsets[o_s], fp.u0, slider)
        S, N = oracle_kernel_windows(src, fp.cell, box_lo, box_dims, pool)
        sysm.cache[("S", (3,) + tuple(reversed(src)), tuple(fp.cell), tuple(box_lo), tuple(box_dims))] = S
        sysm.cache[("N", (3,) + tuple(reversed(src)))] = N
    ref0 = stray_interaction(M0, M1, fp.cell, fp.offsets[0], fp.offsets[1], fp.u0, True,
                             kernel_cache=sysm.cache, return_box=True)
    fscale = force_scale(ref0["hess_n"], M1, fp.cell)
    t_ref, y = D.run_fixed(sysm, [m0, m1, 0.0, 0.0], dt, 1)
    assert abs(t - t_ref) <= 1e-12 * t_ref
    for g, init in ((0, m0), (1, m1)):
        assert rel_l2(got[g], y[g]) < TOL
        assert rel_l2(got[g] - init, y[g] - init) < 1e-3
    me = fp.mech
    dv = TOL * fscale / me.mass * dt
    assert abs(v - y[3]) <= TOL * abs(y[3]) + dv
    assert abs(x - y[2]) <= TOL * abs(y[2]) + dv * dt


def test_full_size_index_shift_bitwise():
    fp, m0, m1 = workloads.film_pair_stick_slip(seed=1)
    fp.u0 = (1.0, 0.0, 0.0)
    mm = gpu_pair(fp, m0, m1, mech=False)
    Ha = mm.compute_stray_field(0).cpu().numpy()
    Fa, _ = mm.get_force(1)
    mm.close()
    fp.u0 = (0.0, 0.0, 0.0)
    fp.lateral = (1, 0)
    mm = gpu_pair(fp, m0, m1, mech=False)
    Hb = mm.compute_stray_field(0).cpu().numpy()
    Fb, _ = mm.get_force(1)
    mm.close()
    assert np.array_equal(Ha, Hb) and Fa == Fb
