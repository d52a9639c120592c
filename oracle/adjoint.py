"""Gradients of the interaction energy, FP64 (test infrastructure only).

The energy of target t in the field of source s (Sec. II.A, with Eq. (EQForce))

    E = mu0 V sum_i M_t(i) . grad phi_s(x_i),   phi_s = spline of (S * M_s) on the box

is linear in M_s and in M_t.  Its gradients, each written out from that form:

  * dE/dM_t(i) = mu0 V grad phi_s(x_i)                        (the evaluation itself)
  * dE/du      = sigma mu0 V sum_i Hess phi_s(x_i) M_t(i) = -sigma F_t
                 (x_i = o_t - o_s + i + sigma u; sigma = +1 when t is the slider)
  * dE/dM_s    = K^T P^T G^T (mu0 V M_t / d):
      G^T  the transposed evaluation: every target spreads mu0 V M_t,a / d_a over
           its 64 coefficients with the derivative weights of axis a;
      P^T  the transposed prefilter: per axis, a solve with the transposed mirror
           band matrix (the oracle's own banded solve, transposed);
      K^T  the transposed potential sum: Mbar_c(j) = sum_b S_c(b - j) phibar(b),
           a valid-mode correlation of the kernel window with phibar.
Derivatives in node units are divided by the cell size of their axis, as in
interaction.py.
"""

import numpy as np
from scipy.linalg import solve_banded
from scipy.signal import correlate

from . import MU0
from .fields import (MARGIN, box_for_target, potential_conv, potential_kernel_window,
                     target_positions)
from .spline import evaluate, prefilter_3d, weights


def prefilter_T_1d(y, axis):
    """Transpose of spline.prefilter_1d along one axis: solve with the transposed band."""
    y = np.moveaxis(np.asarray(y, dtype=np.float64), axis, 0)
    b = y.shape[0]
    if b == 1:
        return np.moveaxis(y.copy(), 0, axis)
    # the forward band: super 1/6 (row 0: 2/6), diagonal 4/6, sub 1/6 (row b-1: 2/6);
    # transposed, the 2/6 entries move to (1, 0) and (b - 2, b - 1)
    ab = np.zeros((3, b))
    ab[0, 1:] = 1.0 / 6.0
    ab[1, :] = 4.0 / 6.0
    ab[2, :-1] = 1.0 / 6.0
    ab[0, b - 1] = 2.0 / 6.0   # (B^T)[b-2, b-1] = B[b-1, b-2]
    ab[2, 0] = 2.0 / 6.0       # (B^T)[1, 0] = B[0, 1]
    x = solve_banded((1, 1), ab, y.reshape(b, -1))
    return np.moveaxis(x.reshape(y.shape), 0, axis)


def prefilter_T_3d(y):
    """Transpose of spline.prefilter_3d on a (bz, by, bx) box."""
    x = prefilter_T_1d(y, 0)
    x = prefilter_T_1d(x, 1)
    return prefilter_T_1d(x, 2)


def evaluate_T(g_n, pos, box_shape):
    """Transpose of the gradient part of spline.evaluate.

    g_n: (..., 3) weights on the node-unit gradient at each point; pos as in
    spline.evaluate.  Returns the (bz, by, bx) coefficient array c such that
    sum(c * coef) = sum_i g_n(i) . grad_n(coef)(pos_i) for every coef.
    """
    P = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    G = np.asarray(g_n, dtype=np.float64).reshape(-1, 3)
    base = np.floor(P).astype(np.int64)
    frac = P - base
    wx, wy, wz = weights(frac[:, 0]), weights(frac[:, 1]), weights(frac[:, 2])
    lo = base - 1
    c = np.zeros(box_shape)
    for kz in range(4):
        for ky in range(4):
            for kx in range(4):
                v = (G[:, 0] * wx[1, kx] * wy[0, ky] * wz[0, kz] +
                     G[:, 1] * wx[0, kx] * wy[1, ky] * wz[0, kz] +
                     G[:, 2] * wx[0, kx] * wy[0, ky] * wz[1, kz])
                np.add.at(c, (lo[:, 2] + kz, lo[:, 1] + ky, lo[:, 0] + kx), v)
    return c


def potential_T(phibar, n_s, cell, box_lo, box_dims, kernel=None):
    """Transpose of fields.potential_conv: Mbar_c(j) = sum_b S_c(b - j) phibar(b), (3, nz, ny, nx)."""
    S = potential_kernel_window(n_s, cell, box_lo, box_dims) if kernel is None else kernel
    out = np.zeros((3, n_s[2], n_s[1], n_s[0]))
    for c in range(3):
        # window index of offset b - j is b' - j + n_s - 1: a valid correlation, reversed
        out[c] = correlate(S[..., c], phibar, mode="valid", method="fft")[::-1, ::-1, ::-1]
    return out


def energy_gradients(M_s, M_t, cell, o_s, o_t, u, target_is_slider, kernel=None, margin=MARGIN):
    """E and its gradients dE/dM_s (3, n_s), dE/dM_t (3, n_t) in J/(A/m) and dE/du (3,) in J/m."""
    n_s = (M_s.shape[3], M_s.shape[2], M_s.shape[1])
    n_t = (M_t.shape[3], M_t.shape[2], M_t.shape[1])
    box_lo, box_dims = box_for_target(n_t, o_t, o_s, u, target_is_slider, margin=margin)
    S = potential_kernel_window(n_s, cell, box_lo, box_dims) if kernel is None else kernel
    phi = potential_conv(M_s, cell, box_lo, box_dims, kernel=S)
    coef = prefilter_3d(phi)
    pos = target_positions(n_t, o_t, o_s, u, target_is_slider) - np.asarray(box_lo, float)
    _, grad_n, hess_n = evaluate(coef, pos)
    d = np.asarray(cell, dtype=np.float64)
    V = d.prod()
    grad = grad_n / d
    hess = hess_n / d[:, None] / d[None, :]
    Mt = np.moveaxis(M_t, 0, -1)
    E = MU0 * V * np.sum(Mt * grad)
    F = -MU0 * V * np.einsum("zyxab,zyxa->b", hess, Mt)
    sigma = 1.0 if target_is_slider else -1.0
    dE_du = -sigma * F
    dE_dMt = MU0 * V * np.moveaxis(grad, -1, 0)
    cbar = evaluate_T(MU0 * V * Mt / d, pos, coef.shape)
    phibar = prefilter_T_3d(cbar)
    dE_dMs = potential_T(phibar, n_s, cell, box_lo, box_dims, kernel=S)
    return dict(E=E, F=F, dE_du=dE_du, dE_dMt=dE_dMt, dE_dMs=dE_dMs, box_lo=box_lo, box_dims=box_dims)
