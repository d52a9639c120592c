"""Parity at the benchmark size: 1024 x 256 x 2 stick-slip film pair (GPU).

The CUDA path runs the grids and launch configuration bench.py times; the FP64
oracle evaluates the same stray field (linear convolution, banded prefilter,
64-term evaluation), force, energy and self-demag field at full size.  Its
kernel windows are filled by a spawn process pool (one z plane per task).
Also the index-shift property at full size, bit for bit on the GPU.
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
