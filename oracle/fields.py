"""Potential on a box and self-demag field, FP64 (test infrastructure only).

Geometry convention (shared reading, Sec. II.A and III):
  * magnet g has nx x ny x nz cuboid cells of common size (dx, dy, dz) and an
    integer lattice offset o_g (cells); arrays are indexed [comp, z, y, x];
  * the slider (g = 1) is displaced by u (cells, real) from its lattice place;
  * a target cell i of magnet t sits, in node coordinates of source s (node j
    = centre of source cell j), at  p = o_t - o_s + i + sigma u,  with
    sigma = +1 when t is the slider and -1 when s is the slider;
  * the potential box (Sec. III.A, four-cell margin) spans, per axis,
    [floor(p_min) - 1 - m, floor(p_max) + 2 + m],  m = 4: the cubic-spline
    support of every target centre plus the margin.

Potential: phi(n) = sum_j S((n - j) * cell) . M_j   (Sec. III.A, S at centres)
Demag:     H(i)  = -sum_j N((i - j) * cell) M_j     (Sec. III.A)
Both are written as direct sums (tiny grids) and as the same sums evaluated by
plain linear convolution ('valid' window of scipy.signal.fftconvolve).
"""

import math

import numpy as np
from scipy.signal import fftconvolve

from .kernels import N_kernel, S_kernel

MARGIN = 4


def box_for_target(n_t, o_t, o_s, u, target_is_slider, margin=MARGIN):
    """Box (lo, dims) per axis in source node coordinates, axis order (x, y, z)."""
    sigma = 1.0 if target_is_slider else -1.0
    lo, dims = [], []
    for a in range(3):
        p_min = (o_t[a] - o_s[a]) + sigma * u[a]
        p_max = p_min + (n_t[a] - 1)
        b_lo = math.floor(p_min) - 1 - margin
        b_hi = math.floor(p_max) + 2 + margin
        lo.append(b_lo)
        dims.append(b_hi - b_lo + 1)
    return tuple(lo), tuple(dims)


def target_positions(n_t, o_t, o_s, u, target_is_slider):
    """Node coordinates p (x, y, z) of every target centre, shape (nz, ny, nx, 3)."""
    sigma = 1.0 if target_is_slider else -1.0
    iz, iy, ix = np.meshgrid(np.arange(n_t[2]), np.arange(n_t[1]), np.arange(n_t[0]), indexing="ij")
    p = np.stack([ix + (o_t[0] - o_s[0]) + sigma * u[0],
                  iy + (o_t[1] - o_s[1]) + sigma * u[1],
                  iz + (o_t[2] - o_s[2]) + sigma * u[2]], axis=-1)
    return p.astype(np.float64)


def potential_direct(M, cell, box_lo, box_dims):
    """phi on box nodes by the direct sum over source cells.

    M: (3, nz, ny, nx) magnetisation in A/m; cell = (dx, dy, dz) in metres.
    Returns phi (bz, by, bx) in amperes.
    """
    dx, dy, dz = cell
    _, nz, ny, nx = M.shape
    bx, by, bz = box_dims
    Z, Y, X = np.meshgrid(np.arange(bz) + box_lo[2], np.arange(by) + box_lo[1],
                          np.arange(bx) + box_lo[0], indexing="ij")
    phi = np.zeros((bz, by, bx))
    for jz in range(nz):
        for jy in range(ny):
            for jx in range(nx):
                S = S_kernel((X - jx) * dx, (Y - jy) * dy, (Z - jz) * dz, dx, dy, dz)
                phi += S[..., 0] * M[0, jz, jy, jx] + S[..., 1] * M[1, jz, jy, jx] \
                    + S[..., 2] * M[2, jz, jy, jx]
    return phi


def potential_kernel_window(n_s, cell, box_lo, box_dims):
    """S over the offsets d = n - j, per axis [box_lo - (n_s - 1), box_hi]; (..., 3)."""
    dx, dy, dz = cell
    d_lo = [box_lo[a] - (n_s[a] - 1) for a in range(3)]
    d_len = [box_dims[a] + n_s[a] - 1 for a in range(3)]
    Z, Y, X = np.meshgrid(np.arange(d_len[2]) + d_lo[2], np.arange(d_len[1]) + d_lo[1],
                          np.arange(d_len[0]) + d_lo[0], indexing="ij")
    return S_kernel(X * dx, Y * dy, Z * dz, dx, dy, dz)


def potential_conv(M, cell, box_lo, box_dims, kernel=None):
    """Same sum as potential_direct, by linear convolution over the offset window.

    Offsets d = n - j needed per axis run over [box_lo - (n_s - 1), box_hi];
    the 'valid' part of (kernel * M) is exactly phi on the box.
    """
    _, nz, ny, nx = M.shape
    S = potential_kernel_window((nx, ny, nz), cell, box_lo, box_dims) if kernel is None else kernel
    phi = np.zeros(tuple(reversed(box_dims)))
    for c in range(3):
        phi += fftconvolve(S[..., c], M[c], mode="valid")
    return phi


def demag_direct(M, cell):
    """H(i) = -sum_j N(i - j) M_j over the magnet's own cells, (3, nz, ny, nx) A/m."""
    dx, dy, dz = cell
    _, nz, ny, nx = M.shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    H = np.zeros_like(M)
    for jz in range(nz):
        for jy in range(ny):
            for jx in range(nx):
                N = N_kernel((X - jx) * dx, (Y - jy) * dy, (Z - jz) * dz, dx, dy, dz)
                m = M[:, jz, jy, jx]
                H[0] -= N[..., 0] * m[0] + N[..., 3] * m[1] + N[..., 4] * m[2]
                H[1] -= N[..., 3] * m[0] + N[..., 1] * m[1] + N[..., 5] * m[2]
                H[2] -= N[..., 4] * m[0] + N[..., 5] * m[1] + N[..., 2] * m[2]
    return H


def demag_kernel_window(n_s, cell):
    """N over offsets d in [-(n - 1), n - 1] per axis, shape (2nz-1, 2ny-1, 2nx-1, 6)."""
    dx, dy, dz = cell
    nx, ny, nz = n_s
    Z, Y, X = np.meshgrid(np.arange(-(nz - 1), nz), np.arange(-(ny - 1), ny),
                          np.arange(-(nx - 1), nx), indexing="ij")
    return N_kernel(X * dx, Y * dy, Z * dz, dx, dy, dz)


def demag_conv(M, cell, kernel=None):
    """Same sum as demag_direct, by linear convolution ('valid' window)."""
    _, nz, ny, nx = M.shape
    N = demag_kernel_window((nx, ny, nz), cell) if kernel is None else kernel
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4,
            (1, 2): 5, (2, 1): 5}
    H = np.zeros_like(M)
    for a in range(3):
        for b in range(3):
            H[a] -= fftconvolve(N[..., comp[(a, b)]], M[b], mode="valid")
    return H


def _S_chunk(args):
    X, Y, Z, cell = args
    return S_kernel(X, Y, Z, *cell)


def _N_chunk(args):
    X, Y, Z, cell = args
    return N_kernel(X, Y, Z, *cell)


def _window_pooled(fun, lo, length, cell, pool):
    dx, dy, dz = cell
    jobs = []
    for iz in range(length[2]):
        Y, X = np.meshgrid(np.arange(length[1]) + lo[1], np.arange(length[0]) + lo[0], indexing="ij")
        Z = np.full_like(X, iz + lo[2])
        jobs.append((X * dx, Y * dy, Z * dz, cell))
    return np.stack(pool.map(fun, jobs))


def kernel_windows_pooled(n_s, cell, box_lo, box_dims, pool):
    """The S window of a box and the N window of a source grid, one z plane per
    pool task: the same values as potential_kernel_window / demag_kernel_window,
    computed in parallel (pass a multiprocessing pool made with 'spawn')."""
    d_lo = [box_lo[a] - (n_s[a] - 1) for a in range(3)]
    d_len = [box_dims[a] + n_s[a] - 1 for a in range(3)]
    S = _window_pooled(_S_chunk, d_lo, d_len, cell, pool)
    N = _window_pooled(_N_chunk, [-(n - 1) for n in n_s], [2 * n - 1 for n in n_s], cell, pool)
    return S, N
