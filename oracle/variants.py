"""Comparison variant of the stray field, FP64 (test infrastructure only).

Sec. III.A mentions a four-point central finite difference for the gradient
of the potential.  Here it is applied to the same B-spline interpolant the
main path differentiates analytically: phi is evaluated at every displaced
target centre and at the centres one and two cells away along each axis, and

    H_a(i) = -(-phi(i + 2 e_a) + 8 phi(i + e_a) - 8 phi(i - e_a) + phi(i - 2 e_a)) / (12 d_a).
"""

import numpy as np

from .fields import box_for_target, potential_conv, target_positions
from .spline import evaluate, prefilter_3d


def fd4_gradient(values, cell):
    """-FD4 gradient on the interior of a (nz + 4, ny + 4, nx + 4) array of values
    (two extra centres on each side); returns (3, nz, ny, nx)."""
    V = np.asarray(values, dtype=np.float64)
    nz, ny, nx = V.shape[0] - 4, V.shape[1] - 4, V.shape[2] - 4
    c = (slice(2, 2 + nz), slice(2, 2 + ny), slice(2, 2 + nx))
    H = np.empty((3, nz, ny, nx))
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        def sh(k):
            s = list(c)
            s[ax] = slice(2 + k, 2 + k + (nz, ny, nx)[ax])
            return V[tuple(s)]
        H[a] = -(-sh(2) + 8.0 * sh(1) - 8.0 * sh(-1) + sh(-2)) / (12.0 * cell[a])
    return H


def stray_field_fd4(M_s, cell, o_s, o_t, n_t, u, target_is_slider, kernel=None):
    """H (3, nz_t, ny_t, nx_t) of source M_s at the target centres by the
    four-point difference of the interpolated potential (margin 4 box), and the
    interpolant's values at the extended centres (nz_t + 4, ny_t + 4, nx_t + 4)."""
    box_lo, box_dims = box_for_target(n_t, o_t, o_s, u, target_is_slider)
    phi = potential_conv(M_s, cell, box_lo, box_dims, kernel=kernel)
    coef = prefilter_3d(phi)
    ext = (n_t[0] + 4, n_t[1] + 4, n_t[2] + 4)
    o_ext = (o_t[0] - 2, o_t[1] - 2, o_t[2] - 2)
    pos = target_positions(ext, o_ext, o_s, u, target_is_slider) - np.asarray(box_lo, float)
    val, _, _ = evaluate(coef, pos)
    return fd4_gradient(val, cell), val
