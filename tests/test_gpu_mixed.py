"""Parity of the reduced-precision form (MM_MIXED) with the FP64 oracle (GPU).

The y transforms run as split-BF16 DFT products on the tensor cores (FP32
accumulation, the y prefilter folded into the inverse matrix); everything
else is the FP32 path.  Bar: relative L2 error <= 1e-4 per field (the
potential box and its coefficients, the stray field, the self-demag field,
m after fixed-dt steps); forces against 1e-4 of the size of the terms that
cancel in Eq. (EQForce), energies relative.  Sizes: small films with ragged
extents (odd sizes, nz = 1..4, u past a cell, lateral offsets), the 64 x 64 x 1
offset sweep, and at full size the 1024 x 256 x 2 stick-slip pair and the
512 x 512 x 8 films, against the oracle evaluated at full size.
"""

import multiprocessing as mp
import os

import numpy as np
import pytest

import workloads
from oracle import fields as OF
from oracle.interaction import stray_interaction
from oracle.spline import prefilter_3d
from tests.pair_setup import force_scale, gpu_pair, oracle_kernel_windows, oracle_system, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def pool():
    p = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    yield p
    p.close()
    p.join()


def _pair(n0, n1, gap, seed, u_cells, Ms=8e5, lateral=(0, 0)):
    fp, _, _ = workloads.film_pair_plain(n=n0, gap=gap, seed=seed)
    fp.n_slider = n1
    fp.u0 = u_cells
    fp.lateral = lateral
    m0 = workloads.random_unit(n0, seed)
    m1 = workloads.random_unit(n1, seed + 7)
    fp.mat_base.Ms = Ms
    return fp, m0, m1


def _mixed(fp, m0, m1, **kw):
    kw.setdefault("mech", False)
    return gpu_pair(fp, m0, m1, precision="mixed", **kw)


@pytest.mark.parametrize("n0,n1,gap,u", [
    ((40, 24, 1), (40, 24, 1), 1, (0.3125, 0.0, 0.0)),
    ((37, 21, 2), (29, 26, 3), 2, (0.71, 0.45, 0.0)),
    ((33, 17, 4), (33, 17, 1), 3, (1.6, -0.2, 0.3)),
])
def test_mixed_potential_box_matches_oracle(n0, n1, gap, u):
    fp, m0, m1 = _pair(n0, n1, gap, 11, u)
    mm = _mixed(fp, m0, m1)
    offs = fp.offsets
    for src in (0, 1):
        t = 1 - src
        phi, lo = mm.compute_potential(src, prefiltered=False)
        coef, _ = mm.compute_potential(src, prefiltered=True)
        n_t = fp.n_slider if t == 1 else fp.n_base
        box_lo, box_dims = OF.box_for_target(n_t, offs[t], offs[src], u, t == 1)
        assert tuple(lo) == tuple(box_lo)
        Ms = fp.mat_base.Ms if src == 0 else fp.mat_slider.Ms
        ref = OF.potential_conv(Ms * (m0 if src == 0 else m1), fp.cell, box_lo, box_dims)
        e_phi = rel_l2(phi.double().cpu().numpy(), ref)
        e_coef = rel_l2(coef.double().cpu().numpy(), prefilter_3d(ref))
        assert e_phi < TOL and e_coef < TOL
        # the tensor-core products really are in reduced precision: the error
        # is well above the FP32 path's (~1e-7) -- the path under test ran
        assert e_phi > 1e-7
    mm.close()


@pytest.mark.parametrize("n0,n1,gap,u,lateral", [
    ((40, 24, 1), (40, 24, 1), 1, (0.3125, 0.0, 0.0), (0, 0)),
    ((37, 21, 2), (29, 26, 3), 2, (0.71, 0.45, 0.0), (9, -5)),
    ((70, 19, 4), (45, 33, 2), 3, (2.6, -1.2, 0.3), (0, 0)),
    ((64, 64, 1), (64, 64, 1), 1, (0.0, 0.0, 0.0), (0, 0)),
])
def test_mixed_stray_field_force_energy_demag_match_oracle(n0, n1, gap, u, lateral):
    fp, m0, m1 = _pair(n0, n1, gap, 5, u, lateral=lateral)
    mm = _mixed(fp, m0, m1)
    offs = fp.offsets
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
        assert abs(E - ref["E"]) < TOL * abs(ref["E"]) + 1e-5 * scale * fp.cell[0]
        Hd = mm.compute_demag(src).double().cpu().numpy()
        assert rel_l2(Hd, OF.demag_conv(M_s, fp.cell)) < TOL
    mm.close()


def test_mixed_offset_sweep_plain_films():
    """The 64 x 64 x 1 films, gap 1 cell, 16 offsets in [0, 1): field and x-force per offset."""
    fp, m0, m1 = workloads.film_pair_plain(n=(64, 64, 1), gap=1, seed=0)
    mm = _mixed(fp, m0, m1)
    M0, M1 = fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1
    cache = {}
    for k in range(16):
        u = (k / 16.0, 0.0, 0.0)
        mm.set_displacement(tuple(v * c for v, c in zip(u, fp.cell)))
        mm.compute_fields()
        F, _ = mm.get_force(1)
        Hg = mm.compute_stray_field(0).double().cpu().numpy()
        ref = stray_interaction(M0, M1, fp.cell, fp.offsets[0], fp.offsets[1], u, True,
                                kernel_cache=cache, return_box=True)
        assert rel_l2(Hg, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M1, fp.cell)
        assert abs(F[0] - ref["F"][0]) < TOL * scale
    mm.close()


def test_mixed_fixed_dt_steps_match_oracle():
    """Five fixed-dt Dormand-Prince steps of spring-pulled PMA films (shrunk
    stick-slip pair) in reduced precision: m of both films within the bar."""
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(40, 24, 2), gap=5, seed=4)
    fp.u0 = (0.25, 0.0, 0.0)
    fp.mech.x0_spring = 2e-9
    fp.mech.v_drive = 50.0
    mm = _mixed(fp, m0, m1, mech=True)
    from oracle import dynamics as D

    dt = 5e-14
    _, y = D.run_fixed(oracle_system(fp), [m0, m1, 0.0, 0.0], dt, 5)
    mm.step(5, dt)
    x, v, _ = mm.get_slider_state()
    for g in (0, 1):
        got = mm.get_magnetization(g).double().cpu().numpy()
        init = m0 if g == 0 else m1
        assert rel_l2(got, y[g]) < TOL
        assert rel_l2(got - init, y[g] - init) < 1e-2
    assert abs(x - y[2]) <= 1e-4 * abs(y[2])
    assert abs(v - y[3]) <= 1e-4 * abs(y[3])
    mm.close()


def test_mixed_periodic_films_match_oracle():
    """Periodic in-plane boundaries in reduced precision: the wrapped prefilter
    folded into the inverse DFT matrix; stray field, force, demag and the
    coefficient box against the periodic oracle."""
    from oracle import periodic as OP

    fp, m0, m1 = workloads.film_pair_stick_slip(n=(24, 20, 2), gap=3, seed=3)
    fp.u0 = (0.37, 0.6, 0.0)
    fp.lateral = (3, -2)
    fp.periodic = 3
    fp.pbc_images = 2
    mm = _mixed(fp, m0, m1)
    kern = {}
    for src in (0, 1):
        t = 1 - src
        H = mm.compute_stray_field(src).double().cpu().numpy()
        F, _ = mm.get_force(t)
        Ms = fp.mat_base.Ms
        M_s, M_t = Ms * (m0 if src == 0 else m1), Ms * (m1 if t == 1 else m0)
        ref = OP.stray_interaction_periodic(M_s, M_t, fp.cell, fp.offsets[src], fp.offsets[t], fp.u0, t == 1,
                                            fp.pbc_images, kernels=kern, return_box=True)
        assert rel_l2(H, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M_t, fp.cell)
        assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
        Hd = mm.compute_demag(src).double().cpu().numpy()
        assert rel_l2(Hd, OP.demag_periodic(M_s, fp.cell, fp.pbc_images, kern)) < TOL
        coef, lo = mm.compute_potential(src, prefiltered=True)
        z_lo, bz = OP.box_z(fp.n_base[2], fp.offsets[t][2], fp.offsets[src][2], 0.0, t == 1, 4)
        phi = OP.potential_periodic(M_s, fp.cell, z_lo, bz, fp.pbc_images)
        assert rel_l2(coef.double().cpu().numpy(), OP.prefilter_periodic(phi)) < TOL
    mm.close()


def test_mixed_rejects_sources_thicker_than_eight_layers():
    from paper_1801_04181_gb300 import MMError

    fp, m0, m1 = _pair((12, 10, 9), (12, 10, 2), 2, 1, (0.2, 0.0, 0.0))
    mm = _mixed(fp, m0, m1)
    # the plan is made with the first field evaluation
    with pytest.raises(MMError, match="8 layers"):
        mm.compute_stray_field(0)
    mm.close()


def _full_check(fp, m0, m1, pool):
    mm = _mixed(fp, m0, m1)
    H = mm.compute_stray_field(0).double().cpu().numpy()
    F, E = mm.get_force(1)
    Hd = mm.compute_demag(0).double().cpu().numpy()
    mm.close()
    box_lo, box_dims = OF.box_for_target(fp.n_slider, fp.offsets[1], fp.offsets[0], fp.u0, True)
    S, N = oracle_kernel_windows(fp.n_base, fp.cell, box_lo, box_dims, pool)
    key = ("S", (3,) + tuple(reversed(fp.n_base)), tuple(fp.cell), tuple(box_lo), tuple(box_dims))
    M0, M1 = fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1
    ref = stray_interaction(M0, M1, fp.cell, fp.offsets[0], fp.offsets[1], fp.u0, True,
                            kernel_cache={key: S}, return_box=True)
    e_H = rel_l2(H, ref["H"])
    assert e_H < TOL
    scale = force_scale(ref["hess_n"], M1, fp.cell)
    assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
    assert abs(E - ref["E"]) < TOL * abs(ref["E"]) + 1e-5 * scale * fp.cell[0]
    e_Hd = rel_l2(Hd, OF.demag_conv(M0, fp.cell, kernel=N))
    assert e_Hd < TOL
    return e_H, e_Hd


def test_mixed_full_size_stick_slip(pool):
    fp, m0, m1 = workloads.film_pair_stick_slip(seed=0)
    fp.u0 = (0.37, 0.0, 0.0)
    _full_check(fp, m0, m1, pool)


def test_mixed_full_size_films_512x512x8(pool):
    fp, m0, m1 = workloads.film_pair_plain((512, 512, 8), 1, 3)
    fp.u0 = (0.3, 0.2, 0.0)
    _full_check(fp, m0, m1, pool)


@pytest.mark.parametrize("n0,n1,gap,u,lateral", [
    ((21, 13, 1), (19, 17, 3), 2, (0.45, 0.3, 0.0), (1, -1)),   # odd extents: unpaired x-forward rows
    ((16, 1, 1), (16, 1, 1), 1, (0.7, 0.0, 0.0), (0, 0)),       # one y row: one K chunk, mostly padding
    ((20, 14, 8), (18, 12, 2), 2, (0.35, 0.2, 0.0), (0, 0)),    # 8 layers: the thickest source offered
])
def test_mixed_ragged_geometries_match_oracle(n0, n1, gap, u, lateral):
    fp, m0, m1 = _pair(n0, n1, gap, 23, u, lateral=lateral)
    mm = _mixed(fp, m0, m1)
    offs = fp.offsets
    for src in (0, 1):
        t = 1 - src
        Hg = mm.compute_stray_field(src).double().cpu().numpy()
        F, _ = mm.get_force(t)
        Ms = fp.mat_base.Ms if src == 0 else fp.mat_slider.Ms
        M_s = Ms * (m0 if src == 0 else m1)
        M_t = (fp.mat_slider.Ms if t == 1 else fp.mat_base.Ms) * (m1 if t == 1 else m0)
        ref = stray_interaction(M_s, M_t, fp.cell, offs[src], offs[t], u, t == 1, return_box=True)
        assert rel_l2(Hg, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M_t, fp.cell)
        assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
        Hd = mm.compute_demag(src).double().cpu().numpy()
        assert rel_l2(Hd, OF.demag_conv(M_s, fp.cell)) < TOL
    mm.close()


def test_mixed_batch_equals_pairs_stepped_alone():
    """Pairs of uneven sizes stepped together in reduced precision on two lane
    streams take, bit for bit, the steps they take alone."""
    import torch

    from paper_1801_04181_gb300 import assign_lanes, step_batch

    pairs = []
    for n, u, v, seed in [((40, 24, 1), (0.25, 0.0, 0.0), 3.0, 11), ((33, 20, 2), (7.6, 0.0, 0.0), 0.4, 12),
                          ((48, 16, 3), (1.9, 0.0, 0.0), 9.0, 13)]:
        fp, m0, m1 = workloads.film_pair_stick_slip(n=n, gap=5, seed=seed)
        fp.u0, fp.mech.v_drive, fp.mech.x0_spring = u, v, 1e-9
        pairs.append((fp, m0, m1))
    lanes = assign_lanes([fp.cells() for fp, _, _ in pairs], 2)
    streams = [torch.cuda.Stream() for _ in range(max(lanes) + 1)]
    batch = [gpu_pair(fp, m0, m1, adaptive=True, rtol=1e-5, stream=streams[l], precision="mixed")
             for (fp, m0, m1), l in zip(pairs, lanes)]
    step_batch(batch, 3, [1e-14] * len(batch))
    torch.cuda.synchronize()
    got = [([mm.get_magnetization(g).cpu().numpy() for g in (0, 1)], mm.get_slider_state()) for mm in batch]
    for mm in batch:
        mm.close()
    for (fp, m0, m1), (m_b, s_b) in zip(pairs, got):
        mm = _mixed(fp, m0, m1, adaptive=True, mech=True)
        mm.step(3, 1e-14)
        for g in (0, 1):
            assert np.array_equal(mm.get_magnetization(g).cpu().numpy(), m_b[g])
        assert mm.get_slider_state() == s_b
        mm.close()


def test_mixed_adaptive_steps_accept_and_stay_normalised():
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(48, 24, 2), gap=5, seed=9)
    mm = _mixed(fp, m0, m1, adaptive=True, mech=True)
    t, dt = mm.step(10, 1e-14)
    acc, _ = mm.step_stats()
    assert acc == 10 and t > 0 and dt > 0
    for g in (0, 1):
        m = mm.get_magnetization(g).double().cpu().numpy()
        assert np.max(np.abs(np.sqrt((m ** 2).sum(axis=0)) - 1)) < 1e-6
    mm.close()


def test_mixed_componentwise_variant_stays_fp32():
    """The comparison variant runs its own FP32 passes in a reduced-precision
    context: it meets the FP32 bar (1e-5) against the oracle."""
    from oracle.variants import stray_field_componentwise

    fp, m0, m1 = _pair((20, 17, 2), (18, 15, 2), 2, 17, (0.3, 0.45, 0.0), lateral=(1, -2))
    mm = _mixed(fp, m0, m1)
    offs = fp.offsets
    for src in (0, 1):
        t = 1 - src
        H = mm.compute_stray_field_componentwise(src).double().cpu().numpy()
        Ms = fp.mat_base.Ms if src == 0 else fp.mat_slider.Ms
        n_t = fp.n_slider if t == 1 else fp.n_base
        ref = stray_field_componentwise(Ms * (m0 if src == 0 else m1), fp.cell, offs[src], offs[t], n_t,
                                        (0.3, 0.45, 0.0), t == 1)
        assert rel_l2(H, ref) < 1e-5
    mm.close()


def test_mixed_eddy_coupled_steps_match_oracle():
    """Three coupled steps of conducting films (as the FP32 test in
    test_gpu_eddy.py) in reduced precision: m within the 1e-4 bar while the
    coupling moves the per-step change by ~4e-3; the next eddy field within
    2 EPS_B |B| / |B_n - B_{n-1}| with EPS_B = 2e-5 (the reduced-precision
    field error, ~1e-5 measured, times 2)."""
    from oracle import dynamics as D
    from oracle import eddy as OE

    fp, _, _ = workloads.film_pair_stick_slip(n=(16, 12, 2), gap=3, seed=5)
    m0, m1 = workloads.random_unit(fp.n_base, 5), workloads.random_unit(fp.n_slider, 6)
    fp.mech.x0_spring = 2e-9
    sigma, dt, n = 1e11, 2e-14, 3
    mm = _mixed(fp, m0, m1, mech=True)
    mm.set_conductivity(0, sigma)
    mm.set_conductivity(1, sigma)
    mm.step(n, dt)
    got = [mm.get_magnetization(g).double().cpu().numpy() for g in (0, 1)]
    He = [mm.get_eddy_field(g).double().cpu().numpy() for g in (0, 1)]
    mm.close()
    y0 = [m0, m1, 0.0, 0.0]
    cs = OE.EddyCoupledSystem(oracle_system(fp), (sigma, sigma))
    B_hist, t, y, k1 = [], 0.0, list(y0), None
    for _ in range(n):
        y5, _, k7 = D.dp45_step(cs, t, y, dt, k1)
        B_hist.append([b.copy() for b in cs.last_B])
        cs.accept(dt)
        y = [D.normalise(y5[0]), D.normalise(y5[1]), y5[2], y5[3]]
        t += dt
        k1 = k7
    for g in (0, 1):
        assert rel_l2(got[g], y[g]) < TOL
        assert rel_l2(got[g] - y0[g], y[g] - y0[g]) < 1e-2
        dB = np.linalg.norm((B_hist[-1][g] - B_hist[-2][g]).ravel())
        tol = max(TOL, 2 * 2e-5 * np.linalg.norm(B_hist[-1][g].ravel()) / dB)
        assert rel_l2(He[g], cs.Heddy[g]) < tol
