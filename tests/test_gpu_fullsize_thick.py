"""Parity at the full sizes of the thick workloads (GPU): two 64^3 vortex cubes
of 2 nm cells side by side along x, and a pair of 512 x 512 x 8 films.

The CUDA path plans these as any caller gets them (the cubes with z by FFT,
the 8-layer films with a direct z sum between the y passes); the
FP64 oracle evaluates the same stray field, force, energy and self-demag field
at full size, its kernel windows filled by a spawn process pool.
"""

import multiprocessing as mp
import os

import numpy as np
import pytest

import workloads
from oracle import fields as OF
from oracle.interaction import stray_interaction
from tests.pair_setup import force_scale, gpu_pair, oracle_kernel_windows, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def pool():
    p = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    yield p
    p.close()
    p.join()


def _check(fp, m0, m1, pool):
    mm = gpu_pair(fp, m0, m1, mech=False)
    H = mm.compute_stray_field(0).double().cpu().numpy()
    F, E = mm.get_force(1)
    Hd = mm.compute_demag(0).double().cpu().numpy()
    info = mm.plan_info(0)
    mm.close()
    assert (info["Qz"] > 0) == (fp.n_base[2] > 8)
    box_lo, box_dims = OF.box_for_target(fp.n_slider, fp.offsets[1], fp.offsets[0], fp.u0, True)
    S, N = oracle_kernel_windows(fp.n_base, fp.cell, box_lo, box_dims, pool)
    key = ("S", (3,) + tuple(reversed(fp.n_base)), tuple(fp.cell), tuple(box_lo), tuple(box_dims))
    M0, M1 = fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1
    ref = stray_interaction(M0, M1, fp.cell, fp.offsets[0], fp.offsets[1], fp.u0, True,
                            kernel_cache={key: S}, return_box=True)
    assert rel_l2(H, ref["H"]) < TOL
    scale = force_scale(ref["hess_n"], M1, fp.cell)
    assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
    assert abs(E - ref["E"]) < TOL * abs(ref["E"]) + 1e-6 * scale * fp.cell[0]
    assert rel_l2(Hd, OF.demag_conv(M0, fp.cell, kernel=N)) < TOL


def test_full_size_cubes_64(pool):
    fp, m0, m1 = workloads.cube_pair((64, 64, 64), 3, 0)
    fp.u0 = (0.4, 0.0, 0.0)
    _check(fp, m0, m1, pool)


def test_full_size_films_512x512x8(pool):
    fp, m0, m1 = workloads.film_pair_plain((512, 512, 8), 1, 3)
    fp.u0 = (0.3, 0.2, 0.0)
    _check(fp, m0, m1, pool)


def test_full_size_cubes_index_shift_bitwise():
    fp, m0, m1 = workloads.cube_pair((64, 64, 64), 3, 1)
    fp.u0 = (1.0, 0.0, 0.0)
    mm = gpu_pair(fp, m0, m1, mech=False)
    H_a = mm.compute_stray_field(0).cpu().numpy()
    F_a, _ = mm.get_force(1)
    mm.close()
    fp.gap, fp.u0 = 4, (0.0, 0.0, 0.0)
    mm = gpu_pair(fp, m0, m1, mech=False)
    H_b = mm.compute_stray_field(0).cpu().numpy()
    F_b, _ = mm.get_force(1)
    mm.close()
    assert np.array_equal(H_a, H_b)
    assert F_a == F_b


def test_full_size_cubes_64_energy_gradients():
    """The adjoint at the differentiation workload's size: dE/dm of both cubes
    and dE/du against the oracle's FP64 gradients."""
    from oracle.adjoint import energy_gradients

    fp, m0, m1 = workloads.cube_pair((64, 64, 64), 3, 2)
    fp.u0 = (1.7, 0.0, 0.0)
    mm = gpu_pair(fp, m0, m1, mech=False)
    du, gs, gt = mm.backward_energy(0)
    mm.close()
    Ms = fp.mat_base.Ms
    ref = energy_gradients(Ms * m0, Ms * m1, fp.cell, fp.offsets[0], fp.offsets[1], fp.u0, True)
    assert rel_l2(gs.double().cpu().numpy(), Ms * ref["dE_dMs"]) < TOL
    assert rel_l2(gt.double().cpu().numpy(), Ms * ref["dE_dMt"]) < TOL
    assert np.max(np.abs(np.array(du) - ref["dE_du"])) < 1e-4 * np.max(np.abs(ref["dE_du"]))

