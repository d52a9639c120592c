"""Periodic in-plane boundary conditions, FP64 (test infrastructure only).

Sec. III says the moving-magnet extension supports periodic boundary
conditions, Sec. III.A that with periodic boundaries the potential's extra
values beyond the domain are copied from its other side, and Sec. IV.B runs
the friction films periodic in the film plane.  The reading taken here (the
paper gives no formulas for it):

  * both films span one lateral period, Px = nx cells along x and Py = ny
    along y (the same for both magnets); z stays open;
  * every kernel (the potential kernel S and the demag tensor N) is summed
    over (2R + 1)^2 periodic images, offsets d + (i Px, j Py) for |i|, |j| <= R,
    each image evaluated exactly as a single kernel value (closed forms near,
    quadrature far); at the Nyquist offset d = P/2 of an even period the two
    truncations (images of +P/2 and of -P/2) are averaged, so the periodic
    kernel keeps the evenness or oddness of the kernel in every axis;
  * fields are circular convolutions over the period in x and y;
  * the potential lives on every node of the period in x and y (and on the
    usual box in z); its cubic B-spline is periodic in x and y (the exact
    circulant inverse of (1, 4, 1)/6) and has mirror ends in z; evaluation
    wraps the 64 taps around the period -- the copied margin of Sec. III.A;
  * the exchange field wraps around the period in x and y.

Steps follow the non-periodic oracle (fields.py, interaction.py, dynamics.py)
in the paper's order.
"""

import math

import numpy as np

from . import MU0
from .dynamics import anisotropy_field, llg_rhs
from .kernels import N_kernel, S_kernel
from .spline import evaluate, prefilter_1d

NCOMP = {"S": 3, "N": 6}


def _kernel(kind, X, Y, Z, cell):
    f = S_kernel if kind == "S" else N_kernel
    return f(X, Y, Z, *cell)


def periodic_kernel_plane(kind, P, cell, dz, R):
    """K_per on the circular grid (Py, Px, ncomp) for z offset dz (cells):
    circular index x holds the signed offset sx in (-Px/2, Px/2]."""
    Px, Py = P
    sx = np.arange(Px)
    sx = np.where(2 * sx > Px, sx - Px, sx)
    sy = np.arange(Py)
    sy = np.where(2 * sy > Py, sy - Py, sy)

    def image_sum(SX, SY):
        acc = 0.0
        for i in range(-R, R + 1):
            for j in range(-R, R + 1):
                acc = acc + _kernel(kind, (SX + i * Px) * cell[0], (SY + j * Py) * cell[1],
                                    np.full_like(SX, dz, dtype=np.float64) * cell[2], cell)
        return acc

    SY, SX = np.meshgrid(sy.astype(np.float64), sx.astype(np.float64), indexing="ij")
    K = image_sum(SX, SY)
    # Nyquist offsets of even periods: average the truncations of +P/2 and -P/2
    nyx = (Px % 2 == 0) & (2 * SX == Px)
    nyy = (Py % 2 == 0) & (2 * SY == Py)
    if nyx.any():
        K = np.where(nyx[..., None], 0.5 * (K + image_sum(np.where(nyx, -SX, SX), SY)), K)
    if nyy.any():
        # for the corner (both Nyquist) this averages all four sign pairs
        K = np.where(nyy[..., None], 0.5 * (K + _ny_flip(kind, SX, SY, nyx, nyy, image_sum)), K)
    return K


def _ny_flip(kind, SX, SY, nyx, nyy, image_sum):
    """The y-Nyquist partner of K: -Py/2 in y, with the x average where x is Nyquist too."""
    A = image_sum(SX, np.where(nyy, -SY, SY))
    if nyx.any():
        B = image_sum(np.where(nyx, -SX, SX), np.where(nyy, -SY, SY))
        A = np.where(nyx[..., None], 0.5 * (A + B), A)
    return A


def circ_conv2(K, m):
    """Circular convolution over the last two axes: out(n) = sum_j K(n - j) m(j)."""
    return np.real(np.fft.ifft2(np.fft.fft2(K) * np.fft.fft2(m)))


def demag_periodic(M, cell, R, kernels=None):
    """H = -sum_j N_per(i - j) M_j over the magnet's own layers, circular in x, y."""
    _, nz, ny, nx = M.shape
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
    if kernels is None:
        kernels = {}
    H = np.zeros_like(M)
    for iz in range(nz):
        for jz in range(nz):
            dz = iz - jz
            if ("N", dz) not in kernels:
                kernels[("N", dz)] = periodic_kernel_plane("N", (nx, ny), cell, dz, R)
            K = kernels[("N", dz)]
            for a in range(3):
                for b in range(3):
                    H[a, iz] -= circ_conv2(K[..., comp[(a, b)]], M[b, jz])
    return H


def box_z(n_t_z, o_t_z, o_s_z, u_z, target_is_slider, margin):
    """z extent of the potential box (the non-periodic axis), as in fields.box_for_target."""
    sigma = 1.0 if target_is_slider else -1.0
    p_min = (o_t_z - o_s_z) + sigma * u_z
    lo = math.floor(p_min) - 1 - margin
    hi = math.floor(p_min + n_t_z - 1) + 2 + margin
    return lo, hi - lo + 1


def potential_periodic(M, cell, z_lo, bz, R, kernels=None):
    """phi on every node of the period (x, y) and on box planes z_lo .. z_lo + bz - 1
    (source lattice nodes): (bz, Py, Px), phi(n) = sum_j S_per(n - j) . M_j."""
    _, nz, ny, nx = M.shape
    if kernels is None:
        kernels = {}
    phi = np.zeros((bz, ny, nx))
    for zb in range(bz):
        for jz in range(nz):
            dz = z_lo + zb - jz
            if ("S", dz) not in kernels:
                kernels[("S", dz)] = periodic_kernel_plane("S", (nx, ny), cell, dz, R)
            K = kernels[("S", dz)]
            for c in range(3):
                phi[zb] += circ_conv2(K[..., c], M[c, jz])
    return phi


def prefilter_periodic_1d(phi, axis):
    """B-spline coefficients along a periodic axis: the circulant inverse of
    (c[k-1] + 4 c[k] + c[k+1]) / 6 = phi[k], by FFT."""
    phi = np.asarray(phi, dtype=np.float64)
    n = phi.shape[axis]
    k = np.arange(n)
    sym = (4.0 + 2.0 * np.cos(2.0 * np.pi * k / n)) / 6.0
    shape = [1] * phi.ndim
    shape[axis] = n
    return np.real(np.fft.ifft(np.fft.fft(phi, axis=axis) / sym.reshape(shape), axis=axis))


def prefilter_periodic(phi):
    """(bz, Py, Px): periodic in x and y, mirror ends in z."""
    c = prefilter_periodic_1d(phi, 2)
    c = prefilter_periodic_1d(c, 1)
    return prefilter_1d(c, 0)


def evaluate_periodic(coef, pos, z_lo):
    """Interpolant, gradient and Hessian at source-lattice positions pos (..., 3):
    x and y wrap around the period (the coefficients are extended by two nodes
    copied from the other side), z is box-local from plane z_lo."""
    bz, Py, Px = coef.shape
    ext = np.pad(coef, ((0, 0), (2, 2), (2, 2)), mode="wrap")
    p = np.array(pos, dtype=np.float64)
    p[..., 0] = np.mod(p[..., 0], Px) + 2.0
    p[..., 1] = np.mod(p[..., 1], Py) + 2.0
    p[..., 2] = p[..., 2] - z_lo
    return evaluate(ext, p)


def target_positions(n_t, o_t, o_s, u, target_is_slider):
    sigma = 1.0 if target_is_slider else -1.0
    iz, iy, ix = np.meshgrid(np.arange(n_t[2]), np.arange(n_t[1]), np.arange(n_t[0]), indexing="ij")
    return np.stack([ix + (o_t[0] - o_s[0]) + sigma * u[0], iy + (o_t[1] - o_s[1]) + sigma * u[1],
                     iz + (o_t[2] - o_s[2]) + sigma * u[2]], axis=-1).astype(np.float64)


def stray_interaction_periodic(M_s, M_t, cell, o_s, o_t, u, target_is_slider, R, margin=4, kernels=None,
                               return_box=False):
    """Stray field, Eq. (EQForce) force and interaction energy of the source on
    the target with periodic x, y: the steps of interaction.stray_interaction
    (potential, prefilter, 64-term evaluation, H = -grad phi, F, E)."""
    n_t = (M_t.shape[3], M_t.shape[2], M_t.shape[1])
    z_lo, bz = box_z(n_t[2], o_t[2], o_s[2], u[2], target_is_slider, margin)
    phi = potential_periodic(M_s, cell, z_lo, bz, R, kernels)
    coef = prefilter_periodic(phi)
    pos = target_positions(n_t, o_t, o_s, u, target_is_slider)
    _, grad_n, hess_n = evaluate_periodic(coef, pos, z_lo)
    d = np.asarray(cell, dtype=np.float64)
    grad = grad_n / d
    hess = hess_n / d[:, None] / d[None, :]
    Mt = np.moveaxis(M_t, 0, -1)
    V = d.prod()
    out = dict(H=-np.moveaxis(grad, -1, 0), E=MU0 * V * np.sum(Mt * grad),
               F=-MU0 * V * np.einsum("zyxab,zyxa->b", hess, Mt))
    if return_box:
        out.update(phi=phi, coef=coef, z_lo=z_lo, hess_n=hess_n)
    return out


def exchange_field_periodic(m, Ms, Aex, cell):
    """H_ex = 2A/(mu0 Ms) sum_nb (m_nb - m)/d_a^2: x and y neighbours wrap, z ends are free."""
    pref = 2.0 * Aex / (MU0 * Ms)
    H = np.zeros_like(m)
    for axis, d in ((3, cell[0]), (2, cell[1])):
        if m.shape[axis] > 1:
            H += (np.roll(m, 1, axis=axis) + np.roll(m, -1, axis=axis) - 2.0 * m) / (d * d)
    nz = m.shape[1]
    if nz > 1:
        diff = np.diff(m, axis=1) / (cell[2] ** 2)
        H[:, :-1] += diff
        H[:, 1:] -= diff
    return pref * H


class PeriodicSystem:
    """Two films periodic in x and y (0 = base, 1 = slider) plus the slider's
    (x, v) along e; the same right-hand side as dynamics.System with the
    periodic fields above."""

    def __init__(self, shapes, cell, offsets, materials, mechanics, R, u0=(0.0, 0.0, 0.0),
                 H_ext=(0.0, 0.0, 0.0), margin=4):
        self.cell = tuple(float(c) for c in cell)
        self.offsets = [tuple(int(v) for v in o) for o in offsets]
        self.mat = materials
        self.mech = mechanics
        self.R = R
        self.margin = margin
        self.u0 = np.asarray(u0, dtype=np.float64)
        self.H_ext = np.asarray(H_ext, dtype=np.float64)
        self.kernels = {}
        e = np.asarray(mechanics["dir"], dtype=np.float64)
        self.e = e / np.linalg.norm(e)

    def displacement(self, x):
        return self.u0 + x * self.e / np.asarray(self.cell)

    def fields(self, m0, m1, x):
        u = self.displacement(x)
        M0 = self.mat[0]["Ms"] * m0
        M1 = self.mat[1]["Ms"] * m1
        on1 = stray_interaction_periodic(M0, M1, self.cell, self.offsets[0], self.offsets[1], u, True, self.R,
                                         self.margin, self.kernels)
        on0 = stray_interaction_periodic(M1, M0, self.cell, self.offsets[1], self.offsets[0], u, False, self.R,
                                         self.margin, self.kernels)
        H = []
        for g, (m, stray) in enumerate(((m0, on0["H"]), (m1, on1["H"]))):
            p = self.mat[g]
            h = demag_periodic(p["Ms"] * m, self.cell, self.R, self.kernels) + stray
            h = h + exchange_field_periodic(m, p["Ms"], p["Aex"], self.cell)
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
        return [llg_rhs(m0, H[0], self.mat[0]["alpha"]), llg_rhs(m1, H[1], self.mat[1]["alpha"]), v, acc]
