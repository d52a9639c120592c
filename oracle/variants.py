"""Comparison variants of the stray field, FP64 (test infrastructure only).

Four-point difference.  Sec. III.A mentions a four-point central finite
difference for the gradient of the potential.  Here it is applied to the same
B-spline interpolant the main path differentiates analytically: phi is
evaluated at every displaced target centre and at the centres one and two
cells away along each axis, and

    H_a(i) = -(-phi(i + 2 e_a) + 8 phi(i + e_a) - 8 phi(i - e_a) + phi(i - 2 e_a)) / (12 d_a).

Direct componentwise interpolation.  Sec. II.A names two ways to interpolate
the demagnetising field between cells: through the scalar potential (the main
path), or directly, component by component, from the field vectors of the
tensor method; Sec. IV.A compares their divergence and curl.  Here the field
of the source on the nodes of the box around the displaced target,

    H_a(n) = -sum_j sum_b N_ab(n - j) M_b(j)    (N the cell-averaged demag tensor),

is computed on the same box as the potential (Sec. III.A, four-cell margin),
each component is prefiltered to cubic B-spline coefficients (mirror ends)
and evaluated, 64 taps, at the displaced target centres.
"""

import numpy as np

from scipy.signal import fftconvolve

from .fields import MARGIN, box_for_target, potential_conv, target_positions
from .kernels import N_kernel
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


# components of the symmetric tensor N stored as xx yy zz xy xz yz
_NCOMP = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}


def field_kernel_window(n_s, cell, box_lo, box_dims):
    """N over the offsets d = n - j of box nodes n from source cells j, per axis
    [box_lo - (n_s - 1), box_hi]; shape (..., 6)."""
    dx, dy, dz = cell
    d_lo = [box_lo[a] - (n_s[a] - 1) for a in range(3)]
    d_len = [box_dims[a] + n_s[a] - 1 for a in range(3)]
    Z, Y, X = np.meshgrid(np.arange(d_len[2]) + d_lo[2], np.arange(d_len[1]) + d_lo[1],
                          np.arange(d_len[0]) + d_lo[0], indexing="ij")
    return N_kernel(X * dx, Y * dy, Z * dz, dx, dy, dz)


def field_on_box(M, cell, box_lo, box_dims, kernel=None):
    """H_a(n) = -sum_j sum_b N_ab(n - j) M_b(j) at every box node, (3, bz, by, bx)
    A/m, by linear convolution ('valid' window, like the potential)."""
    _, nz, ny, nx = M.shape
    N = field_kernel_window((nx, ny, nz), cell, box_lo, box_dims) if kernel is None else kernel
    H = np.zeros((3,) + tuple(reversed(box_dims)))
    for a in range(3):
        for b in range(3):
            H[a] -= fftconvolve(N[..., _NCOMP[(a, b)]], M[b], mode="valid")
    return H


def field_on_box_direct(M, cell, box_lo, box_dims):
    """The same sum as field_on_box by an explicit loop over source cells (tiny grids)."""
    dx, dy, dz = cell
    _, nz, ny, nx = M.shape
    bx, by, bz = box_dims
    Z, Y, X = np.meshgrid(np.arange(bz) + box_lo[2], np.arange(by) + box_lo[1], np.arange(bx) + box_lo[0],
                          indexing="ij")
    H = np.zeros((3, bz, by, bx))
    for jz in range(nz):
        for jy in range(ny):
            for jx in range(nx):
                N = N_kernel((X - jx) * dx, (Y - jy) * dy, (Z - jz) * dz, dx, dy, dz)
                for a in range(3):
                    for b in range(3):
                        H[a] -= N[..., _NCOMP[(a, b)]] * M[b, jz, jy, jx]
    return H


def stray_field_componentwise(M_s, cell, o_s, o_t, n_t, u, target_is_slider, kernel=None, margin=MARGIN):
    """H (3, nz_t, ny_t, nx_t) of source M_s at the displaced target centres by
    direct componentwise B-spline interpolation of the tensor field on the box."""
    box_lo, box_dims = box_for_target(n_t, o_t, o_s, u, target_is_slider, margin=margin)
    Hb = field_on_box(M_s, cell, box_lo, box_dims, kernel=kernel)
    pos = target_positions(n_t, o_t, o_s, u, target_is_slider) - np.asarray(box_lo, float)
    return np.stack([evaluate(prefilter_3d(Hb[a]), pos)[0] for a in range(3)])
