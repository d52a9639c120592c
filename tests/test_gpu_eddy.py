"""Eddy currents on the GPU against the oracle (oracle/eddy.py): the current
density J and the field H_eddy of a conducting magnet for a given dB/dt.

E_sol and H_eddy come from the FP32 potential path (the usual 1e-5 bar); the
electric potential is solved in FP64 to a residual of 1e-9 of its source, so
J and H_eddy carry the FP32 bar too.
"""

import numpy as np
import pytest
import torch

import workloads
from oracle import eddy as OE
from tests.pair_setup import gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5
EPS_B = 2e-7


def _ctx(n, cell=(2e-9, 2e-9, 2e-9), gap=3, seed=0):
    fp, _, _ = workloads.film_pair_plain(n=n, gap=gap, seed=seed)
    fp.cell = cell
    m0, m1 = workloads.random_unit(n, seed), workloads.random_unit(n, seed + 1)
    return fp, gpu_pair(fp, m0, m1, mech=False)


@pytest.mark.parametrize("n,kind", [((12, 10, 7), "random"), ((12, 10, 7), "uniform"), ((20, 16, 2), "random"),
                                    ((9, 9, 9), "uniform")])
def test_eddy_field_matches_oracle(n, kind):
    fp, mm = _ctx(n)
    rng = np.random.default_rng(7)
    nx, ny, nz = n
    if kind == "random":
        B = rng.standard_normal((3, nz, ny, nx)) * 1e9
    else:
        B = np.zeros((3, nz, ny, nx))
        B[0], B[2] = 4e8, 1e9
    sigma = 1e6
    Bt = torch.as_tensor(B, dtype=torch.float32, device="cuda")
    for mag in (0, 1):
        H, J, sweeps = mm.eddy_field(mag, Bt, sigma)
        ref = OE.eddy_field(B.astype(np.float32).astype(np.float64), fp.cell, sigma, return_all=True)
        assert rel_l2(J.double().cpu().numpy(), ref["J"]) < TOL, sweeps
        assert rel_l2(H.double().cpu().numpy(), ref["H"]) < TOL
        assert sweeps > 0
    mm.close()


def test_eddy_field_of_no_change_is_zero():
    fp, mm = _ctx((8, 7, 3))
    B = torch.zeros((3, 3, 7, 8), dtype=torch.float32, device="cuda")
    H, J, sweeps = mm.eddy_field(0, B, 1e6)
    assert sweeps == 0 and float(H.abs().max()) == 0.0 and float(J.abs().max()) == 0.0
    mm.close()


def test_eddy_coupled_steps_match_oracle():
    """Three fixed-dt Dormand-Prince steps of conducting films with the eddy
    fields coupled in (lagged by one step) against the oracle's coupled run.
    Random unit m (strong exchange, fast motion) and a conductivity far above
    any metal's (1e11 S/m), so that the coupling moves the per-step change of
    m by ~4e-3. Checked: m of both films within the field bar and their change
    within 1e-3 (as for the other step tests), while the change without eddy
    fields differs by more than twice that bar (the test is not vacuous); the
    eddy field the next step would add within the bar widened by the
    cancellation in B_n - B_{n-1}: each B carries the FP32 field path's error
    (5e-8 of |B| measured on this pair; EPS_B = 2e-7 allows 4 times that), so
    the difference is good to 2 EPS_B |B| / |B_n - B_{n-1}| (|B| is ~100
    times the difference here)."""
    from oracle import dynamics as D
    from tests.pair_setup import oracle_system

    fp, _, _ = workloads.film_pair_stick_slip(n=(16, 12, 2), gap=3, seed=5)
    m0, m1 = workloads.random_unit(fp.n_base, 5), workloads.random_unit(fp.n_slider, 6)
    fp.mech.x0_spring = 2e-9
    sigma, dt, n = 1e11, 2e-14, 3
    mm = gpu_pair(fp, m0, m1)
    mm.set_conductivity(0, sigma)
    mm.set_conductivity(1, sigma)
    mm.step(n, dt)
    got = [mm.get_magnetization(g).double().cpu().numpy() for g in (0, 1)]
    He = [mm.get_eddy_field(g).double().cpu().numpy() for g in (0, 1)]
    x, v, _ = mm.get_slider_state()
    mm.close()

    y0 = [m0, m1, 0.0, 0.0]
    cs = OE.EddyCoupledSystem(oracle_system(fp), (sigma, sigma))
    B_hist = []
    t, y, k1 = 0.0, list(y0), None
    for _ in range(n):
        y5, _, k7 = D.dp45_step(cs, t, y, dt, k1)
        B_hist.append([b.copy() for b in cs.last_B])
        cs.accept(dt)
        y = [D.normalise(y5[0]), D.normalise(y5[1]), y5[2], y5[3]]
        t += dt
        k1 = k7
    _, yp = D.run_fixed(oracle_system(fp), y0, dt, n)
    for g in (0, 1):
        assert rel_l2(got[g], y[g]) < TOL
        assert rel_l2(got[g] - y0[g], y[g] - y0[g]) < 1e-3
        assert rel_l2(yp[g] - y0[g], y[g] - y0[g]) > 2e-3
        dB = np.linalg.norm((B_hist[-1][g] - B_hist[-2][g]).ravel())
        tol = max(TOL, 2 * EPS_B * np.linalg.norm(B_hist[-1][g].ravel()) / dB)
        assert rel_l2(He[g], cs.Heddy[g]) < tol
    assert abs(x - y[2]) <= 1e-5 * abs(y[2])


@pytest.mark.parametrize("n0,n1,gap,u,lateral", [
    ((12, 10, 2), (12, 10, 2), 2, (0.37, 0.0, 0.0), (0, 0)),
    ((14, 9, 3), (10, 11, 2), 3, (1.6, -0.45, 0.0), (2, -1)),
])
def test_eddy_field_on_other_matches_oracle(n0, n1, gap, u, lateral):
    """The field of one magnet's currents inside the other (interpolated on the
    potential box), both directions, against the oracle."""
    fp, _, _ = workloads.film_pair_plain(n=n0, gap=gap, seed=4)
    fp.n_slider = n1
    fp.u0 = u
    fp.lateral = lateral
    fp.cell = (2e-9, 2e-9, 2e-9)
    m0, m1 = workloads.random_unit(n0, 1), workloads.random_unit(n1, 2)
    mm = gpu_pair(fp, m0, m1, mech=False)
    rng = np.random.default_rng(9)
    for src in (0, 1):
        t = 1 - src
        n_s = n0 if src == 0 else n1
        J = rng.standard_normal((3, n_s[2], n_s[1], n_s[0])) * 1e10
        H = mm.eddy_field_on_other(src, torch.as_tensor(J, dtype=torch.float32, device="cuda"))
        n_t = n1 if t == 1 else n0
        ref = OE.current_field_on_other(J.astype(np.float32).astype(np.float64), fp.cell, fp.offsets[src],
                                        fp.offsets[t], n_t, u, t == 1)
        assert rel_l2(H.double().cpu().numpy(), ref) < TOL
    mm.close()


def test_eddy_of_a_conducting_base_reaches_an_insulating_slider():
    """Only the base conducts: after three coupled steps the slider's eddy
    field is the field of the base's currents, against the oracle's coupled
    run (bar widened by the flux-difference cancellation as above)."""
    from oracle import dynamics as D
    from tests.pair_setup import oracle_system

    fp, _, _ = workloads.film_pair_stick_slip(n=(16, 12, 2), gap=3, seed=5)
    m0, m1 = workloads.random_unit(fp.n_base, 5), workloads.random_unit(fp.n_slider, 6)
    fp.mech.x0_spring = 2e-9
    sigma, dt, n = 1e11, 2e-14, 3
    mm = gpu_pair(fp, m0, m1)
    mm.set_conductivity(0, sigma)
    mm.step(n, dt)
    got = [mm.get_magnetization(g).double().cpu().numpy() for g in (0, 1)]
    He = [mm.get_eddy_field(g).double().cpu().numpy() for g in (0, 1)]
    mm.close()
    y0 = [m0, m1, 0.0, 0.0]
    cs = OE.EddyCoupledSystem(oracle_system(fp), (sigma, 0.0))
    B_hist, t, y, k1 = [], 0.0, list(y0), None
    for _ in range(n):
        y5, _, k7 = D.dp45_step(cs, t, y, dt, k1)
        B_hist.append([b.copy() for b in cs.last_B])
        cs.accept(dt)
        y = [D.normalise(y5[0]), D.normalise(y5[1]), y5[2], y5[3]]
        t += dt
        k1 = k7
    assert np.linalg.norm(He[1]) > 0.0
    dB = np.linalg.norm((B_hist[-1][0] - B_hist[-2][0]).ravel())
    tol = max(TOL, 2 * EPS_B * np.linalg.norm(B_hist[-1][0].ravel()) / dB)
    for g in (0, 1):
        assert rel_l2(got[g], y[g]) < TOL
        assert rel_l2(He[g], cs.Heddy[g]) < tol
