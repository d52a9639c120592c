"""Cubic B-spline prefilter and 64-term tricubic evaluation, FP64 (test infrastructure only).

Sec. III.A: B-splines do not interpolate, so the samples phi are first turned
into coefficients c (the prefilter of Unser / Ruijters-Thevenaz), then the
interpolant and its gradient are evaluated from the 4 x 4 x 4 = 64 nearest
coefficients at the full floating-point position (Sec. IV.D: 64 lookups, no
texture-position rounding).

Prefilter, per axis: solve (c[k-1] + 4 c[k] + c[k+1]) / 6 = phi[k] on the box
with mirror (whole-sample symmetric) ends, c[-1] = c[1], c[b] = c[b-2] -- a
banded linear solve, not the recursive filter, so this side shares no
algorithm with the CUDA path.

Evaluation at x = floor(x) + t, nodes floor(x) - 1 ... floor(x) + 2 with
weights  w0 = (1-t)^3/6,  w1 = (3t^3 - 6t^2 + 4)/6,  w2 = (-3t^3 + 3t^2 + 3t + 1)/6,
w3 = t^3/6  and their first and second derivatives in t.
"""

import numpy as np
from scipy.linalg import solve_banded


def prefilter_1d(phi, axis):
    """B-spline coefficients along one axis (mirror ends), by banded solve."""
    phi = np.moveaxis(np.asarray(phi, dtype=np.float64), axis, 0)
    b = phi.shape[0]
    if b == 1:
        return np.moveaxis(phi.copy(), 0, axis)
    ab = np.zeros((3, b))
    ab[0, 1:] = 1.0 / 6.0   # super-diagonal
    ab[1, :] = 4.0 / 6.0    # diagonal
    ab[2, :-1] = 1.0 / 6.0  # sub-diagonal
    # mirror ends fold c[-1] = c[1] into row 0 and c[b] = c[b-2] into row b-1
    ab[0, 1] = 2.0 / 6.0
    ab[2, b - 2] = 2.0 / 6.0
    flat = phi.reshape(b, -1)
    c = solve_banded((1, 1), ab, flat)
    return np.moveaxis(c.reshape(phi.shape), 0, axis)


def prefilter_3d(phi):
    """Coefficients of the tensor-product spline on a (bz, by, bx) box."""
    c = prefilter_1d(phi, 2)
    c = prefilter_1d(c, 1)
    return prefilter_1d(c, 0)


def weights(t):
    """Cubic B-spline weights and t-derivatives at fraction t: (3, 4, ...) = (w, w', w'')."""
    t = np.asarray(t, dtype=np.float64)
    w = np.stack([(1 - t) ** 3 / 6,
                  (3 * t ** 3 - 6 * t ** 2 + 4) / 6,
                  (-3 * t ** 3 + 3 * t ** 2 + 3 * t + 1) / 6,
                  t ** 3 / 6])
    d1 = np.stack([-(1 - t) ** 2 / 2,
                   (9 * t ** 2 - 12 * t) / 6,
                   (-9 * t ** 2 + 6 * t + 3) / 6,
                   t ** 2 / 2])
    d2 = np.stack([1 - t,
                   3 * t - 2,
                   -3 * t + 1,
                   t])
    return np.stack([w, d1, d2])


def evaluate(c, pos):
    """Interpolant, gradient and Hessian at box-local node coordinates.

    c: (bz, by, bx) coefficients; pos: (..., 3) positions (x, y, z) in nodes,
    measured from box node 0.  Returns (value, grad(...,3), hess(...,3,3)) in
    node units.  Every point reads its own 64 coefficients.
    """
    pos = np.asarray(pos, dtype=np.float64)
    shape = pos.shape[:-1]
    P = pos.reshape(-1, 3)
    base = np.floor(P).astype(np.int64)
    frac = P - base
    wx, wy, wz = weights(frac[:, 0]), weights(frac[:, 1]), weights(frac[:, 2])
    bz, by, bx = c.shape
    lo = base - 1
    if (lo < 0).any() or (lo[:, 0] + 3 >= bx).any() or (lo[:, 1] + 3 >= by).any() \
            or (lo[:, 2] + 3 >= bz).any():
        raise ValueError("evaluation point outside the coefficient box")
    val = np.zeros(len(P))
    grad = np.zeros((len(P), 3))
    hess = np.zeros((len(P), 3, 3))
    for kz in range(4):
        for ky in range(4):
            for kx in range(4):
                cc = c[lo[:, 2] + kz, lo[:, 1] + ky, lo[:, 0] + kx]
                # derivative orders (dx, dy, dz) of the separable weight product
                def W(ox, oy, oz):
                    return wx[ox, kx] * wy[oy, ky] * wz[oz, kz]
                val += W(0, 0, 0) * cc
                grad[:, 0] += W(1, 0, 0) * cc
                grad[:, 1] += W(0, 1, 0) * cc
                grad[:, 2] += W(0, 0, 1) * cc
                hess[:, 0, 0] += W(2, 0, 0) * cc
                hess[:, 1, 1] += W(0, 2, 0) * cc
                hess[:, 2, 2] += W(0, 0, 2) * cc
                hess[:, 0, 1] += W(1, 1, 0) * cc
                hess[:, 0, 2] += W(1, 0, 1) * cc
                hess[:, 1, 2] += W(0, 1, 1) * cc
    hess[:, 1, 0] = hess[:, 0, 1]
    hess[:, 2, 0] = hess[:, 0, 2]
    hess[:, 2, 1] = hess[:, 1, 2]
    return val.reshape(shape), grad.reshape(shape + (3,)), hess.reshape(shape + (3, 3))
