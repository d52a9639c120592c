"""Pins of the oracle's local fields, LLG torque and DP45 stepping (Sec. II, III, IV.B).

* damped precession of one spin in a uniform field: closed form
  tan(theta/2) = tan(theta0/2) exp(-alpha gamma0 H t/(1+alpha^2)), azimuth rate
  gamma0 H/(1+alpha^2);
* the DP45 pair is 5th order on a linear ODE (global error ~ dt^5);
* exchange field of a spin wave: eigenvalue (2A/mu0 Ms)(2 cos(k d) - 2)/d^2;
* anisotropy field along the axis, 2 Ku/(mu0 Ms) (m.k);
* slider without magnetic force: critically damped spring, closed form.
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
