"""Local fields, LLG torque and the Dormand-Prince step with slider motion, FP64.

Test infrastructure only.

Sec. II eq. (1) with the standard sign (the printed -gamma H x m conflicts with
its own damping term): Gilbert form dm/dt = -gamma0 m x H + alpha m x dm/dt,
integrated in its explicit Landau-Lifshitz form
    dm/dt = -gamma0/(1 + alpha^2) [ m x H + alpha m x (m x H) ],
gamma0 = mu0 * 1.7595e11 rad/(s T).
Effective field (Sec. II): exchange (6 neighbours, free ends), uniaxial
anisotropy, uniform Zeeman, own demag (Sec. III.A) and the interpolated stray
field of the other magnet (Sec. II.A).
Slider (Sec. III, IV.B): m_s x'' = k (v_d t + x_0 - x) - gamma_v m_s x' + F_m . e,
with F_m the Eq. (EQForce) force of the base on the slider; x is integrated
with the magnetisation by the Dormand-Prince 5(4) pair (Sec. III).
Power bookkeeping (Sec. III, after Eq. (EQForce)): the input -F_m . v_s and the
Gilbert dissipation of each magnet (dissipation_power, power_balance).
"""

import numpy as np

from . import GAMMA_LL, MU0
from .fields import demag_conv, demag_kernel_window
from .interaction import stray_interaction

# Dormand-Prince 5(4) tableau (Dormand & Prince 1980)
DP_C = [0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0]
DP_A = [
    [],
    [1 / 5],
    [3 / 40, 9 / 40],
    [44 / 45, -56 / 15, 32 / 9],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
    [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84],
]
DP_B5 = [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0]
DP_B4 = [5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40]


def exchange_field(m, Ms, Aex, cell):
    """H_ex = 2A/(mu0 Ms) sum over present neighbours (m_nb - m)/d_a^2 (free ends)."""
    H = np.zeros_like(m)
    pref = 2.0 * Aex / (MU0 * Ms)
    for axis, d in zip((3, 2, 1), cell):  # array axes of x, y, z
        n = m.shape[axis]
        if n < 2:
            continue
        diff = np.diff(m, axis=axis) / (d * d)  # m[i+1] - m[i]
        lo = [slice(None)] * 4
        hi = [slice(None)] * 4
        lo[axis] = slice(0, n - 1)
        hi[axis] = slice(1, n)
        H[tuple(lo)] += diff   # cell i gains (m[i+1] - m[i])
        H[tuple(hi)] -= diff   # cell i+1 gains (m[i] - m[i+1])
    return pref * H


def anisotropy_field(m, Ms, Ku, axis):
    """H_an = 2 Ku/(mu0 Ms) (m . k) k for a unit easy axis k."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    proj = np.einsum("c...,c->...", m, k)
    return (2.0 * Ku / (MU0 * Ms)) * proj[None] * k[:, None, None, None]


def llg_rhs(m, H, alpha):
    """Landau-Lifshitz right-hand side; m (3, ...) unit, H (3, ...) in A/m."""
    gamma0 = MU0 * GAMMA_LL
    mxH = np.cross(m, H, axis=0)
    mxmxH = np.cross(m, mxH, axis=0)
    return -gamma0 / (1.0 + alpha * alpha) * (mxH + alpha * mxmxH)


class System:
    """Two magnets (0 = base, 1 = slider) plus the slider's (x, v) along e."""

    def __init__(self, shapes, cell, offsets, materials, mechanics, u0=(0.0, 0.0, 0.0),
                 H_ext=(0.0, 0.0, 0.0)):
        self.cell = tuple(float(c) for c in cell)
        self.offsets = [tuple(int(v) for v in o) for o in offsets]
        self.mat = materials          # list of dicts: Ms, Aex, Ku, ku_axis, alpha
        self.mech = mechanics         # dict: mass, k, v_drive, gamma_v, dir, x0_spring
        self.u0 = np.asarray(u0, dtype=np.float64)
        self.H_ext = np.asarray(H_ext, dtype=np.float64)
        self.shapes = shapes
        self.cache = {}
        e = np.asarray(mechanics["dir"], dtype=np.float64)
        self.e = e / np.linalg.norm(e)

    def displacement(self, x):
        """u (cells) of the slider for mechanical position x (m) along e."""
        return self.u0 + x * self.e / np.asarray(self.cell)

    def demag(self, g, m):
        key = ("N", m.shape)
        if key not in self.cache:
            n = (m.shape[3], m.shape[2], m.shape[1])
            self.cache[key] = demag_kernel_window(n, self.cell)
        return demag_conv(self.mat[g]["Ms"] * m, self.cell, kernel=self.cache[key])

    def fields(self, m0, m1, x):
        """Effective fields of both magnets and the force of the base on the slider."""
        u = self.displacement(x)
        M0 = self.mat[0]["Ms"] * m0
        M1 = self.mat[1]["Ms"] * m1
        on1 = stray_interaction(M0, M1, self.cell, self.offsets[0], self.offsets[1], u, True,
                                kernel_cache=self.cache)
        on0 = stray_interaction(M1, M0, self.cell, self.offsets[1], self.offsets[0], u, False,
                                kernel_cache=self.cache)
        H = []
        for g, (m, stray) in enumerate(((m0, on0["H"]), (m1, on1["H"]))):
            p = self.mat[g]
            h = self.demag(g, m) + stray
            h = h + exchange_field(m, p["Ms"], p["Aex"], self.cell)
            h = h + anisotropy_field(m, p["Ms"], p["Ku"], p["ku_axis"])
            h = h + self.H_ext[:, None, None, None]
            H.append(h)
        return H, on1, on0

    def rhs(self, t, y):
        m0, m1, x, v = y
        H, on1, _ = self.fields(m0, m1, x)
        me = self.mech
        F = float(np.dot(on1["F"], self.e))
        acc = (me["k"] * (me["v_drive"] * t + me.get("x0_spring", 0.0) - x)
               - me["gamma_v"] * me["mass"] * v + F) / me["mass"]
        return [llg_rhs(m0, H[0], self.mat[0]["alpha"]), llg_rhs(m1, H[1], self.mat[1]["alpha"]),
                v, acc]


def _axpy_state(y, ks, coefs, dt):
    out = []
    for idx in range(len(y)):
        acc = y[idx]
        for k, a in zip(ks, coefs):
            if a != 0.0:
                acc = acc + dt * a * k[idx]
        out.append(acc)
    return out


def dp45_stages(system, t, y, dt, k1=None):
    """The seven stage derivatives k_1..k_7 of one Dormand-Prince step of size
    dt from (t, y) and the 5th-order solution y5 (the stage-7 input, since
    a_7j = b5_j); k1 may be passed in (first-same-as-last)."""
    ks = [system.rhs(t, y) if k1 is None else k1]
    for i in range(1, 7):
        yi = _axpy_state(y, ks, DP_A[i], dt)
        ks.append(system.rhs(t + DP_C[i] * dt, yi))
    return ks, yi


def dp45_embedded(system, t, y, dt, k1=None):
    """The 5th- and embedded 4th-order solutions of one step: (y5, y4, ks)."""
    ks, y5 = dp45_stages(system, t, y, dt, k1)
    return y5, _axpy_state(y, ks, DP_B4, dt), ks


def dp45_step(system, t, y, dt, k1=None):
    """One Dormand-Prince 5(4) step of size dt (no rejection).

    Returns (y5, err, k7): y5 the 5th-order solution (not renormalised), err the
    max-norm over both magnets' m of dt * sum (b5 - b4) k (= y5 - y4, the
    local error estimate of the embedded 4th-order solution), k7 = f(t + dt, y5)
    for first-same-as-last reuse.
    """
    ks, y5 = dp45_stages(system, t, y, dt, k1)
    err = 0.0
    for idx in (0, 1):
        e = sum((DP_B5[j] - DP_B4[j]) * ks[j][idx] for j in range(7))
        err = max(err, float(np.max(np.abs(dt * e))))
    return y5, err, ks[6]


def normalise(m):
    return m / np.sqrt(np.sum(m * m, axis=0, keepdims=True))


def run_fixed(system, y0, dt, nsteps, t0=0.0):
    """nsteps fixed DP45 steps with renormalisation and FSAL reuse of k7."""
    t, y, k1 = t0, list(y0), None
    for _ in range(nsteps):
        y5, _, k7 = dp45_step(system, t, y, dt, k1)
        y = [normalise(y5[0]), normalise(y5[1]), y5[2], y5[3]]
        t += dt
        k1 = k7
    return t, y


def euler_step(system, t, y, dt):
    """One explicit Euler step of the LLG equation and the slider's Newton
    equation together (Sec. III: the equations of motion are solved in the
    Euler solver as in the RK45 one): y + dt f(t, y), then m renormalised."""
    y1 = _axpy_state(y, [system.rhs(t, y)], [1.0], dt)
    return [normalise(y1[0]), normalise(y1[1]), y1[2], y1[3]]


def run_euler(system, y0, dt, nsteps, t0=0.0):
    """nsteps explicit Euler steps of size dt."""
    t, y = t0, list(y0)
    for _ in range(nsteps):
        y = euler_step(system, t, y, dt)
        t += dt
    return t, y


def run_adaptive(system, y0, dt, nsteps, rtol, t0=0.0, dt_min=0.0, dt_max=np.inf, trace=None):
    """nsteps accepted adaptive DP45 steps; controller dt *= clamp(0.9 (rtol/err)^(1/5), 0.2, 5).

    An attempt is accepted when err <= rtol (or dt <= dt_min).  trace: a list
    that receives one dict per attempt (t, dt, err, accepted) in order."""
    t, y, k1 = t0, list(y0), None
    accepted = rejected = 0
    while accepted < nsteps:
        y5, err, k7 = dp45_step(system, t, y, dt, k1)
        fac = 5.0 if err == 0.0 else min(5.0, max(0.2, 0.9 * (rtol / err) ** 0.2))
        ok = err <= rtol or dt <= dt_min
        if trace is not None:
            trace.append(dict(t=t, dt=dt, err=err, accepted=ok))
        if ok:
            y = [normalise(y5[0]), normalise(y5[1]), y5[2], y5[3]]
            t += dt
            k1 = k7
            accepted += 1
        else:
            rejected += 1
        dt = min(max(dt * fac, dt_min), dt_max)
    return t, y, dt, accepted, rejected


def dissipation_power(m, H, Ms, alpha, cell):
    """Gilbert dissipation of one magnet (Sec. III, after Eq. (EQForce)), W:

        P_diss = gamma0 alpha mu0 V / ((1 + alpha^2) Ms) sum_i |M_i x H_eff,i|^2

    with M = Ms m and gamma0 = mu0 * 1.7595e11 the prefactor of the LLG
    equation of Sec. II eq. (1) (its H is in A/m, so its gamma is gamma0).
    m (3, ...) unit vectors, H (3, ...) the effective field in A/m."""
    gamma0 = MU0 * GAMMA_LL
    V = float(np.prod(np.asarray(cell, dtype=np.float64)))
    M = Ms * np.asarray(m, dtype=np.float64)
    MxH = np.cross(M, np.asarray(H, dtype=np.float64), axis=0)
    return gamma0 * alpha * MU0 * V / ((1.0 + alpha * alpha) * Ms) * float(np.sum(MxH * MxH))


def power_balance(system, m0, m1, x, v):
    """Power bookkeeping of the moving slider (Sec. III, after Eq. (EQForce)):
    P_in = -F_m^s . v_s, pumped into the magnets by the slider moving at
    v_s = v e against the force F_m^s of the base on it; P_diss of each magnet
    at its effective field; P_visc = gamma_v m v^2, the viscous damping of the
    drive.  In the steady state P_in balances the two dissipations."""
    H, on1, _ = system.fields(m0, m1, x)
    P_diss = [dissipation_power(m, H[g], system.mat[g]["Ms"], system.mat[g]["alpha"], system.cell)
              for g, m in enumerate((m0, m1))]
    P_in = -float(np.dot(on1["F"], v * system.e))
    me = system.mech
    return dict(P_in=P_in, P_diss=P_diss, P_visc=me["gamma_v"] * me["mass"] * v * v, F=on1["F"], H=H)
