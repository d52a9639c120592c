"""Pins of the oracle's local fields, LLG torque and DP45 stepping (Sec. II, III, IV.B).

* damped precession of one spin in a uniform field: closed form
  tan(theta/2) = tan(theta0/2) exp(-alpha gamma0 H t/(1+alpha^2)), azimuth rate
  gamma0 H/(1+alpha^2);
* the DP45 pair is 5th order on a linear ODE (global error ~ dt^5);
* the tableau satisfies the Runge-Kutta order conditions (b5: order 5, b4:
  order 4 and not 5); the embedded solution converges at rate 4; the error
  estimate scales as dt^5 and equals the 4th-order local error against an
  independent integrator (scipy DOP853);
* the adaptive controller on a single spin: rejection of an oversized first
  step with the 0.2 clamp, err held near 0.9^5 rtol, the 5x growth clamp and
  dt_max when nothing moves, tolerance proportionality of the global error;
* exchange field of a spin wave: eigenvalue (2A/mu0 Ms)(2 cos(k d) - 2)/d^2;
* anisotropy field along the axis, 2 Ku/(mu0 Ms) (m.k);
* slider without magnetic force: critically damped spring, closed form;
* the explicit Euler integrator: first order on the single spin (the error
  against the closed form halves with dt), and on the slider alone, a linear
  ODE, it is the explicit recurrence x += dt v, v += dt a(t, x, v) exactly.
"""

import numpy as np
import pytest

from oracle import GAMMA_LL, MU0
from oracle import dynamics as D


class SingleSpin:
    """One spin in a uniform field; x, v carried along unchanged."""

    def __init__(self, H, alpha):
        self.H = np.asarray(H, float)[:, None, None, None]
        self.alpha = alpha

    def rhs(self, t, y):
        m = y[0]
        dm = D.llg_rhs(m, np.broadcast_to(self.H, m.shape), self.alpha)
        return [dm, np.zeros_like(y[1]), 0.0, 0.0]


def test_single_spin_damped_precession():
    H0, alpha = 1e5, 0.1
    th0, ph0 = 0.8, 0.3
    m0 = np.array([np.sin(th0) * np.cos(ph0), np.sin(th0) * np.sin(ph0), np.cos(th0)])
    sys = SingleSpin((0, 0, H0), alpha)
    y = [m0[:, None, None, None].copy(), np.zeros((3, 1, 1, 1)), 0.0, 0.0]
    gamma0 = MU0 * GAMMA_LL
    dt = 1e-13
    n = 400
    t, k1 = 0.0, None
    for _ in range(n):
        y5, _, k1 = D.dp45_step(sys, t, y, dt, k1)
        y = [D.normalise(y5[0]), y5[1], y5[2], y5[3]]
        t += dt
    m = y[0][:, 0, 0, 0]
    theta = np.arccos(m[2])
    phi = np.arctan2(m[1], m[0])
    th_ref = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-alpha * gamma0 * H0 * t / (1 + alpha ** 2)))
    # precession is counter-clockwise about +H for the -gamma0 m x H torque
    ph_ref = ph0 + gamma0 * H0 * t / (1 + alpha ** 2)
    assert abs(theta - th_ref) < 1e-9
    assert abs(np.angle(np.exp(1j * (phi - ph_ref)))) < 1e-9


class Linear:
    def __init__(self, lam):
        self.lam = lam

    def rhs(self, t, y):
        return [self.lam * y[0], self.lam * y[1], 0.0, 0.0]


def test_dp45_is_fifth_order():
    lam = -1.0 + 2.0j
    errs = []
    for n in (10, 20, 40):
        dt = 1.0 / n
        y = [np.ones(1, complex), np.ones(1, complex), 0.0, 0.0]
        t, k1 = 0.0, None
        for _ in range(n):
            y, _, k1 = D.dp45_step(Linear(lam), t, y, dt, k1)
            t += dt
        errs.append(abs(y[0][0] - np.exp(lam)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 4.7), rates


def test_exchange_spin_wave_eigenvalue():
    nx = 40
    d = 4e-9
    k = 2 * np.pi * 3 / nx
    x = np.arange(nx)
    m = np.zeros((3, 1, 1, nx))
    m[0, 0, 0] = 0.01 * np.cos(k * x)
    m[2] = 1.0
    A, Ms = 1.3e-11, 8e5
    H = D.exchange_field(m, Ms, A, (d, d, d))
    lam = 2 * A / (MU0 * Ms) * (2 * np.cos(k * d / d) - 2) / d ** 2
    np.testing.assert_allclose(H[0, 0, 0, 1:-1], lam * m[0, 0, 0, 1:-1], rtol=1e-9,
                               atol=1e-12 * abs(lam) * 0.01)
    # free ends: the end cell sees only its one neighbour
    assert abs(H[0, 0, 0, 0] - 2 * A / (MU0 * Ms) * (m[0, 0, 0, 1] - m[0, 0, 0, 0]) / d ** 2) < 1e-9
    np.testing.assert_allclose(H[2], 0.0, atol=1e-20)


def test_anisotropy_field():
    m = np.array([0.6, 0.0, 0.8])[:, None, None, None]
    H = D.anisotropy_field(m, 1e6, 1e6, (0, 0, 2.0))
    np.testing.assert_allclose(H[:, 0, 0, 0], [0, 0, 2e6 / (MU0 * 1e6) * 0.8])


def test_slider_critically_damped_spring():
    """With the magnets far apart, x(t) follows m x'' = k (v t - x) - g m x'."""
    from oracle.dynamics import System
    cell = (4e-9, 4e-9, 4e-9)
    mat = dict(Ms=1.0, Aex=0.0, Ku=0.0, ku_axis=(0, 0, 1), alpha=0.5)
    k, mass, v = 1e-3, 2.5e-18, 1.0
    w = np.sqrt(k / mass)
    mech = dict(mass=mass, k=k, v_drive=v, gamma_v=2 * w, dir=(1, 0, 0))
    sys = System([(2, 2, 1), (2, 2, 1)], cell, [(0, 0, 0), (0, 0, 40)], [mat, mat], mech)
    m = np.zeros((3, 1, 2, 2))
    m[2] = 1.0
    y = [m.copy(), m.copy(), 0.0, 0.0]
    dt = 2e-9
    t, yy = D.run_fixed(sys, y, dt, 30)
    # x'' + 2w x' + w^2 x = w^2 v t:  x = v t - 2v/w + (2v/w + v t) e^{-wt} ... (x(0)=x'(0)=0)
    x_ref = v * t - 2 * v / w + (2 * v / w + v * t) * np.exp(-w * t)
    assert abs(yy[2] - x_ref) < 1e-6 * abs(x_ref)


def test_dissipation_power_is_the_llg_energy_rate():
    """For the Landau-Lifshitz right-hand side, mu0 Ms V sum H . dm/dt (the rate
    at which the field's energy -mu0 Ms V m . H changes for a frozen H, with
    the sign of a loss) equals P_diss: a pin of the formula against the
    independently pinned LLG right-hand side."""
    rng = np.random.default_rng(11)
    m = rng.standard_normal((3, 2, 3, 4))
    m /= np.sqrt((m * m).sum(axis=0))
    H = 1e5 * rng.standard_normal((3, 2, 3, 4))
    Ms, alpha, cell = 1.1e6, 0.37, (4e-9, 3e-9, 2e-9)
    V = np.prod(cell)
    rate = MU0 * Ms * V * float(np.sum(H * D.llg_rhs(m, H, alpha)))
    P = D.dissipation_power(m, H, Ms, alpha, cell)
    assert P > 0
    assert abs(P - rate) <= 1e-12 * abs(rate)


def test_dissipation_power_single_spin_closed_form():
    """One spin at angle theta to a uniform field H: |M x H|^2 = Ms^2 H^2 sin^2(theta)."""
    from oracle import GAMMA_LL
    th, Hz, Ms, alpha, cell = 0.7, 2e5, 8e5, 0.1, (2e-9, 2e-9, 2e-9)
    m = np.array([np.sin(th), 0.0, np.cos(th)])[:, None, None, None]
    H = np.array([0.0, 0.0, Hz])[:, None, None, None]
    ref = MU0 * GAMMA_LL * alpha * MU0 * np.prod(cell) * Ms * Hz ** 2 * np.sin(th) ** 2 / (1 + alpha ** 2)
    assert abs(D.dissipation_power(m, H, Ms, alpha, cell) - ref) <= 1e-13 * ref
    # parallel to the field: nothing to relax
    m_par = np.array([0.0, 0.0, 1.0])[:, None, None, None]
    assert D.dissipation_power(m_par, H, Ms, alpha, cell) == 0.0


def test_power_input_is_minus_force_dot_velocity():
    """P_in = -F . v_s with the force of the base on the slider (the
    System's own Eq. (EQForce) evaluation) and v_s along the drive direction."""
    from oracle.dynamics import System
    cell = (4e-9, 4e-9, 4e-9)
    mat = dict(Ms=8e5, Aex=1.3e-11, Ku=0.0, ku_axis=(0, 0, 1), alpha=0.5)
    mech = dict(mass=2.5e-18, k=1e-3, v_drive=1.0, gamma_v=4e7, dir=(1, 1, 0))
    sys = System([(6, 5, 1), (5, 4, 1)], cell, [(0, 0, 0), (1, 0, 2)], [mat, mat], mech, u0=(0.3, 0.1, 0))
    rng = np.random.default_rng(3)
    m0 = rng.standard_normal((3, 1, 5, 6)); m0 /= np.sqrt((m0 * m0).sum(axis=0))
    m1 = rng.standard_normal((3, 1, 4, 5)); m1 /= np.sqrt((m1 * m1).sum(axis=0))
    v = 2.5
    P = D.power_balance(sys, m0, m1, 1e-10, v)
    e = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    assert abs(P["P_in"] + float(np.dot(P["F"], v * e))) <= 1e-15 * np.linalg.norm(P["F"]) * v
    assert abs(P["P_visc"] - 4e7 * 2.5e-18 * v * v) <= 1e-15 * P["P_visc"]
    assert all(p > 0 for p in P["P_diss"])
    # reversing the velocity reverses the input power
    assert abs(D.power_balance(sys, m0, m1, 1e-10, -v)["P_in"] + P["P_in"]) <= 1e-12 * abs(P["P_in"])


# ---------------------------------------------------------------- adaptive stepping
# Order conditions of explicit Runge-Kutta methods (Butcher rooted trees): a
# weight vector b is of order p when sum_i b_i Phi_i(tree) = 1/gamma(tree) for
# every tree of up to p nodes.  With c = A 1, the elementary weights are
# products of c and A as written in each entry.
def _order_conditions(A, b, c):
    A = np.array([list(r) + [0.0] * (7 - len(r)) for r in A])
    b = np.asarray(b)
    c = np.asarray(c)
    Ac, Ac2, Ac3 = A @ c, A @ c ** 2, A @ c ** 3
    AAc = A @ Ac
    return {
        # order 1..4 (8 trees)
        "b": (b.sum(), 1.0), "bc": (b @ c, 1 / 2), "bc2": (b @ c ** 2, 1 / 3), "bAc": (b @ Ac, 1 / 6),
        "bc3": (b @ c ** 3, 1 / 4), "bcAc": (b @ (c * Ac), 1 / 8), "bAc2": (b @ Ac2, 1 / 12),
        "bAAc": (b @ AAc, 1 / 24),
        # order 5 (9 trees)
        "bc4": (b @ c ** 4, 1 / 5), "bc2Ac": (b @ (c ** 2 * Ac), 1 / 10), "bcAc2": (b @ (c * Ac2), 1 / 15),
        "bcAAc": (b @ (c * AAc), 1 / 30), "b(Ac)2": (b @ Ac ** 2, 1 / 20), "bAc3": (b @ Ac3, 1 / 20),
        "bAcAc": (b @ (A @ (c * Ac)), 1 / 40), "bAAc2": (b @ (A @ Ac2), 1 / 60),
        "bAAAc": (b @ (A @ AAc), 1 / 120),
    }


def test_dp45_tableau_satisfies_the_order_conditions():
    """b5 is of order 5, the embedded b4 of order 4 but not 5 (so y5 - y4 is a
    nonzero estimate of the 4th-order local error), and c_i = sum_j a_ij."""
    A, c = D.DP_A, np.asarray(D.DP_C)
    for i, row in enumerate(A):
        assert abs(sum(row) - c[i]) < 1e-14
    cond5 = _order_conditions(A, D.DP_B5, c)
    for name, (got, want) in cond5.items():
        assert abs(got - want) < 1e-14, name
    cond4 = _order_conditions(A, D.DP_B4, c)
    names4 = ["b", "bc", "bc2", "bAc", "bc3", "bcAc", "bAc2", "bAAc"]
    for name in names4:
        got, want = cond4[name]
        assert abs(got - want) < 1e-14, name
    assert max(abs(g - w) for n, (g, w) in cond4.items() if n not in names4) > 1e-4


def test_dp45_embedded_solution_is_fourth_order():
    """Propagating the embedded solution y4 alone converges at rate 4 on
    y' = lambda y (global error against exp(lambda t))."""
    lam = -1.0 + 2.0j
    errs = []
    for n in (10, 20, 40, 80):
        dt = 1.0 / n
        y = [np.ones(1, complex), np.ones(1, complex), 0.0, 0.0]
        t = 0.0
        for _ in range(n):
            _, y, _ = D.dp45_embedded(Linear(lam), t, y, dt)
            t += dt
        errs.append(abs(y[0][0] - np.exp(lam)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 3.7) & (rates < 4.5)), rates


class SmoothNonlinear:
    """A smooth non-autonomous system in the two 'magnet' slots:
    a' = -a b + sin(t),  b' = a^2 - b/2  (elementwise on arrays of 2)."""

    def rhs(self, t, y):
        a, b = y[0], y[1]
        return [-a * b + np.sin(t), a * a - 0.5 * b, 0.0, 0.0]


def _reference_step(t0, y0, dt):
    from scipy.integrate import solve_ivp

    def f(t, z):
        a, b = z[:2], z[2:]
        return np.concatenate([-a * b + np.sin(t), a * a - 0.5 * b])

    sol = solve_ivp(f, (t0, t0 + dt), np.concatenate([y0[0], y0[1]]), method="DOP853", rtol=1e-13,
                    atol=1e-15)
    z = sol.y[:, -1]
    return z[:2], z[2:]


def test_dp45_error_estimate_is_the_fourth_order_local_error():
    """err = max |y5 - y4| scales as dt^5 on a smooth nonlinear problem and
    equals, to leading order, the true local error of y4 against an
    independent high-accuracy integrator (scipy's DOP853)."""
    sysm = SmoothNonlinear()
    y0 = [np.array([0.7, -0.4]), np.array([0.2, 1.1]), 0.0, 0.0]
    t0 = 0.3
    errs = []
    for dt in (0.2, 0.1, 0.05, 0.025):
        _, err, _ = D.dp45_step(sysm, t0, y0, dt)
        errs.append(err)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 4.6) & (rates < 5.4)), rates
    dt = 0.025
    y5, y4, _ = D.dp45_embedded(sysm, t0, y0, dt)
    a_ref, b_ref = _reference_step(t0, y0, dt)
    true4 = max(np.max(np.abs(y4[0] - a_ref)), np.max(np.abs(y4[1] - b_ref)))
    true5 = max(np.max(np.abs(y5[0] - a_ref)), np.max(np.abs(y5[1] - b_ref)))
    assert true5 < 0.05 * true4
    assert abs(errs[-1] - true4) < 0.05 * true4


def _spin_y0(th0=0.8, ph0=0.3):
    m0 = np.array([np.sin(th0) * np.cos(ph0), np.sin(th0) * np.sin(ph0), np.cos(th0)])
    # the second slot holds a frozen unit vector (SingleSpin gives it no motion)
    return [m0[:, None, None, None].copy(), m0[:, None, None, None].copy(), 0.0, 0.0]


def test_run_adaptive_controller_sequence_on_a_single_spin():
    """Damped precession with a first step far too large: the attempt is
    rejected and dt shrinks by the clamped controller factor; every attempt
    after that is accepted with err near 0.9^5 rtol; the accepted trajectory
    matches the closed form within the summed per-step tolerance."""
    H0, alpha, rtol = 1e5, 0.1, 1e-8
    gamma0 = MU0 * GAMMA_LL
    sysm = SingleSpin((0, 0, H0), alpha)
    trace = []
    t, y, dt_next, acc, rej = D.run_adaptive(sysm, _spin_y0(), 5e-11, 40, rtol, trace=trace)
    assert acc == 40 and rej == len(trace) - 40 and rej >= 1
    assert not trace[0]["accepted"] and trace[0]["err"] > 1e3 * rtol
    # hand-applied controller: factor 0.9 (rtol/err)^(1/5), clamped to [0.2, 5]
    for a, b in zip(trace[:-1], trace[1:]):
        fac = min(5.0, max(0.2, 0.9 * (rtol / a["err"]) ** 0.2))
        assert b["dt"] == a["dt"] * fac
        assert b["t"] == (a["t"] + a["dt"] if a["accepted"] else a["t"])
        assert a["accepted"] == (a["err"] <= rtol)
    # the first attempt is so far off that its factor is the 0.2 clamp
    assert trace[1]["dt"] == 0.2 * trace[0]["dt"]
    # once converged the controller holds err at 0.9^5 rtol ~ 0.59 rtol
    tail = [a["err"] / rtol for a in trace[-20:]]
    assert all(a["accepted"] for a in trace[-20:])
    assert 0.4 < np.median(tail) < 0.8, tail
    m = y[0][:, 0, 0, 0]
    th_ref = 2 * np.arctan(np.tan(0.4) * np.exp(-alpha * gamma0 * H0 * t / (1 + alpha ** 2)))
    assert abs(np.arccos(m[2]) - th_ref) < 40 * rtol


def test_run_adaptive_zero_error_grows_dt_by_five_to_dt_max():
    """With no field nothing moves, err = 0, every attempt is accepted and dt
    grows by the upper clamp 5 per step until dt_max holds it."""
    sysm = SingleSpin((0, 0, 0.0), 0.1)
    trace = []
    D.run_adaptive(sysm, _spin_y0(), 1e-15, 6, 1e-6, dt_max=1e-12, trace=trace)
    np.testing.assert_allclose([a["dt"] for a in trace], [1e-15, 5e-15, 2.5e-14, 1.25e-13, 6.25e-13, 1e-12],
                               rtol=1e-14)
    assert all(a["accepted"] and a["err"] == 0.0 for a in trace)


def test_run_adaptive_tolerance_proportionality():
    """Tightening rtol by 1e3 tightens the global error of the accepted
    trajectory (against the closed form) by at least 1e2."""
    H0, alpha = 1e5, 0.1
    gamma0 = MU0 * GAMMA_LL
    sysm = SingleSpin((0, 0, H0), alpha)
    errs = []
    T = 2e-10
    for rtol in (1e-5, 1e-8):
        t, y, dt = 0.0, _spin_y0(), 1e-13
        # stop exactly at T: accepted steps until the last one, then one fixed step to T
        k = 0
        while True:
            t1, y1, dt1, _, _ = D.run_adaptive(sysm, y, dt, 1, rtol, t0=t)
            if t1 >= T:
                break
            t, y, dt = t1, y1, dt1
            k += 1
        t, y = D.run_fixed(sysm, y, T - t, 1, t0=t)
        th_ref = 2 * np.arctan(np.tan(0.4) * np.exp(-alpha * gamma0 * H0 * t / (1 + alpha ** 2)))
        errs.append(abs(np.arccos(y[0][2, 0, 0, 0]) - th_ref))
    assert errs[1] < 1e-2 * errs[0], errs


def test_euler_is_first_order_on_the_single_spin():
    H0, alpha = 1e5, 0.1
    th0 = 0.8
    m0 = np.array([np.sin(th0), 0.0, np.cos(th0)])
    sys = SingleSpin((0, 0, H0), alpha)
    gamma0 = MU0 * GAMMA_LL
    T = 2e-11
    errs = []
    for n in (200, 400, 800):
        y = [m0[:, None, None, None].copy(), m0[:, None, None, None].copy(), 0.0, 0.0]
        t, y = D.run_euler(sys, y, T / n, n)
        th = np.arccos(y[0][2, 0, 0, 0])
        th_ref = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-alpha * gamma0 * H0 * t / (1 + alpha ** 2)))
        errs.append(abs(th - th_ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2


def test_euler_steps_the_slider_explicitly():
    from oracle.dynamics import System
    cell = (4e-9, 4e-9, 4e-9)
    mat = dict(Ms=1.0, Aex=0.0, Ku=0.0, ku_axis=(0, 0, 1), alpha=0.5)
    k, mass, v_d = 1e-3, 2.5e-18, 1.0
    w = np.sqrt(k / mass)
    mech = dict(mass=mass, k=k, v_drive=v_d, gamma_v=2 * w, dir=(1, 0, 0), x0_spring=3e-10)
    sys = System([(2, 2, 1), (2, 2, 1)], cell, [(0, 0, 0), (0, 0, 40)], [mat, mat], mech)
    m = np.zeros((3, 1, 2, 2))
    m[2] = 1.0
    dt, n = 1e-10, 60
    _, y = D.run_euler(sys, [m.copy(), m.copy(), 0.0, 0.0], dt, n)
    x = v = t = 0.0
    for _ in range(n):
        a = k / mass * (v_d * t + 3e-10 - x) - 2 * w * v  # the magnets' force is ~1e-19 of this
        x, v, t = x + dt * v, v + dt * a, t + dt
    assert abs(y[2] - x) <= 1e-9 * abs(x) and abs(y[3] - v) <= 1e-9 * abs(v)
