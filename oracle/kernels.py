"""Cell-integrated interaction kernels, FP64 (test infrastructure only).

S  -- scalar-potential kernel of Abert et al. as used in Sec. III.A:
      S(r_i - r_j) = (1/4pi) int_{V_j} grad' (1/|r - r'|) d^3r'  at r = r_i,
      evaluated at the target cell CENTRE (Sec. III.A: centres, not corners).
      phi(r_i) = sum_j S(r_i - r_j) . M_j   and   H = -grad phi.
N  -- demagnetisation tensor of Sec. III.A, H_d(r_i) = -sum_j N(r_i - r_j) M_j,
      the target-cell average of the field of a uniformly magnetised source cell
      (Newell, Williams & Dunlop 1993 closed form).

Far field (the paper is silent on how the kernels are integrated at range):
for max(|X/a|, |Y/b|, |Z/c|) > R_FAR cells both kernels switch from the closed
forms, which lose digits to cancellation at range, to tensor-product 3-point
Gauss-Legendre quadrature of the point kernel: over the source cell for S, and
over source and target cells for N.  At 16 cells the Newell closed form is
good to ~5e-8 and the 3-point rule to ~6e-10 (relative, against a 5-point
rule); at 32 cells the closed form is off by up to ~7e-6 for flat cells.

Lengths may be in any unit (metres, or cells); S has the unit of length, N is
dimensionless.  All functions broadcast over numpy arrays of offsets.
"""

import numpy as np

R_FAR = 16  # cells; closed form for max-norm offset <= R_FAR, quadrature beyond

_GL3_NODES = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
_GL3_WEIGHTS = np.array([5.0, 8.0, 5.0]) / 9.0


# ----------------------------------------------------------------------------
# S kernel
# ----------------------------------------------------------------------------

def _asinh_ratio(num, den2):
    """asinh(num / sqrt(den2)) with the 0 * asinh(x/0) limits handled by callers."""
    den = np.sqrt(den2)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.arcsinh(np.where(den2 > 0, num / np.where(den2 > 0, den, 1.0), 0.0))


def _rect_antiderivative(xi, y, z):
    """F(y, z) with d2F/dydz = 1/sqrt(xi^2 + y^2 + z^2).

    Textbook primitive  y ln(z+R) + z ln(y+R) - xi atan(yz/(xi R)),  written
    with asinh:  ln(z+R) = asinh(z/sqrt(xi^2+y^2)) + ln sqrt(xi^2+y^2); the
    dropped logarithm depends on y only (resp. z only) and cancels in the
    four-corner sum, so the asinh form gives the same rectangle integral
    without the ln(z+R) cancellation for z < 0.
    """
    xi = np.asarray(xi, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    R = np.sqrt(xi * xi + y * y + z * z)
    t1 = y * _asinh_ratio(z, xi * xi + y * y)  # y * asinh(z / sqrt(xi^2+y^2)); 0 when y = xi = 0
    t2 = z * _asinh_ratio(y, xi * xi + z * z)
    with np.errstate(divide="ignore", invalid="ignore"):
        den = xi * R
        t3 = np.where(den != 0, xi * np.arctan(y * z / np.where(den != 0, den, 1.0)), 0.0)
    return t1 + t2 - t3


def rect_potential(xi, y1, y2, z1, z2):
    """int_{y1}^{y2} int_{z1}^{z2} dy dz / sqrt(xi^2 + y^2 + z^2)  (4-corner sum)."""
    F = _rect_antiderivative
    return F(xi, y2, z2) - F(xi, y1, z2) - F(xi, y2, z1) + F(xi, y1, z1)


def _S_closed(X, Y, Z, a, b, c):
    """Closed form of S (Sec. III.A).

    d/dx' of 1/|r - r'| integrates in x' to the two faces x' = +-a/2 of the
    source cell:  S_x = (1/4pi) [I(X - a/2) - I(X + a/2)],  where I(xi) is the
    potential of the unit-density rectangle of the face at normal distance xi.
    Same for y and z by permutation.
    """
    inv4pi = 1.0 / (4.0 * np.pi)
    Sx = inv4pi * (rect_potential(X - a / 2, Y - b / 2, Y + b / 2, Z - c / 2, Z + c / 2)
                   - rect_potential(X + a / 2, Y - b / 2, Y + b / 2, Z - c / 2, Z + c / 2))
    Sy = inv4pi * (rect_potential(Y - b / 2, X - a / 2, X + a / 2, Z - c / 2, Z + c / 2)
                   - rect_potential(Y + b / 2, X - a / 2, X + a / 2, Z - c / 2, Z + c / 2))
    Sz = inv4pi * (rect_potential(Z - c / 2, X - a / 2, X + a / 2, Y - b / 2, Y + b / 2)
                   - rect_potential(Z + c / 2, X - a / 2, X + a / 2, Y - b / 2, Y + b / 2))
    return np.stack([Sx, Sy, Sz], axis=-1)


def _S_quadrature(X, Y, Z, a, b, c):
    """S by 3x3x3 Gauss-Legendre over the source cell of (r - r')/(4pi |r - r'|^3)."""
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros(np.broadcast(X, Y, Z).shape + (3,))
    V = a * b * c
    for i, (xi, wi) in enumerate(zip(_GL3_NODES, _GL3_WEIGHTS)):
        for j, (yj, wj) in enumerate(zip(_GL3_NODES, _GL3_WEIGHTS)):
            for k, (zk, wk) in enumerate(zip(_GL3_NODES, _GL3_WEIGHTS)):
                w = wi * wj * wk / 8.0  # weights normalised to mean over the cell
                dx = X - xi * a / 2
                dy = Y - yj * b / 2
                dz = Z - zk * c / 2
                r3 = (dx * dx + dy * dy + dz * dz) ** 1.5
                out[..., 0] += w * dx / r3
                out[..., 1] += w * dy / r3
                out[..., 2] += w * dz / r3
    return out * (V / (4.0 * np.pi))


def S_kernel(X, Y, Z, a, b, c):
    """S(R) for the target-minus-source offset R = (X, Y, Z); returns (..., 3)."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, np.float64), np.asarray(Y, np.float64),
                                  np.asarray(Z, np.float64))
    far = np.maximum(np.maximum(np.abs(X / a), np.abs(Y / b)), np.abs(Z / c)) > R_FAR + 1e-9
    out = np.empty(X.shape + (3,))
    if np.any(~far):
        out[~far] = _S_closed(X[~far], Y[~far], Z[~far], a, b, c)
    if np.any(far):
        out[far] = _S_quadrature(X[far], Y[far], Z[far], a, b, c)
    return out


# ----------------------------------------------------------------------------
# Demag tensor N
# ----------------------------------------------------------------------------

def _newell_f(x, y, z):
    """Newell f(x, y, z): its 27-point second difference gives N_xx."""
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t1 = 0.5 * y * (z2 - x2) * _asinh_ratio(y, x2 + z2)
    t2 = 0.5 * z * (y2 - x2) * _asinh_ratio(z, x2 + y2)
    with np.errstate(divide="ignore", invalid="ignore"):
        den = x * R
        t3 = np.where(den != 0, x * y * z * np.arctan(y * z / np.where(den != 0, den, 1.0)), 0.0)
    t4 = (2.0 * x2 - y2 - z2) * R / 6.0
    return t1 + t2 - t3 + t4


def _newell_g(x, y, z):
    """Newell g(x, y, z): its 27-point second difference gives N_xy."""
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t1 = x * y * z * _asinh_ratio(z, x2 + y2)
    t2 = y * (3.0 * z2 - y2) * _asinh_ratio(x, y2 + z2) / 6.0
    t3 = x * (3.0 * z2 - x2) * _asinh_ratio(y, x2 + z2) / 6.0
    with np.errstate(divide="ignore", invalid="ignore"):
        d4 = z * R
        t4 = np.where(d4 != 0, z2 * z * np.arctan(x * y / np.where(d4 != 0, d4, 1.0)) / 6.0, 0.0)
        d5 = y * R
        t5 = np.where(d5 != 0, z * y2 * np.arctan(x * z / np.where(d5 != 0, d5, 1.0)) / 2.0, 0.0)
        d6 = x * R
        t6 = np.where(d6 != 0, z * x2 * np.arctan(y * z / np.where(d6 != 0, d6, 1.0)) / 2.0, 0.0)
    t7 = x * y * R / 3.0
    return t1 + t2 + t3 - t4 - t5 - t6 - t7


def _second_difference_3d(fun, X, Y, Z, a, b, c):
    """prod over axes of (2 f(s) - f(s - h) - f(s + h)), applied to fun(X, Y, Z)."""
    total = 0.0
    for ex, wx in ((-1, -1.0), (0, 2.0), (1, -1.0)):
        for ey, wy in ((-1, -1.0), (0, 2.0), (1, -1.0)):
            for ez, wz in ((-1, -1.0), (0, 2.0), (1, -1.0)):
                total = total + wx * wy * wz * fun(X + ex * a, Y + ey * b, Z + ez * c)
    return total


def _N_closed(X, Y, Z, a, b, c):
    """Newell closed form, components (xx, yy, zz, xy, xz, yz)."""
    s = 1.0 / (4.0 * np.pi * a * b * c)
    Nxx = _second_difference_3d(lambda x, y, z: _newell_f(x, y, z), X, Y, Z, a, b, c)
    Nyy = _second_difference_3d(lambda x, y, z: _newell_f(y, x, z), X, Y, Z, a, b, c)
    Nzz = _second_difference_3d(lambda x, y, z: _newell_f(z, x, y), X, Y, Z, a, b, c)
    Nxy = _second_difference_3d(lambda x, y, z: _newell_g(x, y, z), X, Y, Z, a, b, c)
    Nxz = _second_difference_3d(lambda x, y, z: _newell_g(x, z, y), X, Y, Z, a, b, c)
    Nyz = _second_difference_3d(lambda x, y, z: _newell_g(y, z, x), X, Y, Z, a, b, c)
    return np.stack([Nxx, Nyy, Nzz, Nxy, Nxz, Nyz], axis=-1) * s


def _pair_difference_rule():
    """Nodes/weights of (t - s) for independent 3-point GL points t and s on [-1, 1].

    Averaging a function of (t - s) over target and source points equals a
    weighted sum over the distinct differences; merging equal differences only
    regroups the 9 terms of the tensor product.
    """
    diffs = {}
    for ti, tw in zip(_GL3_NODES, _GL3_WEIGHTS):
        for si, sw in zip(_GL3_NODES, _GL3_WEIGHTS):
            key = round(ti - si, 12)
            diffs[key] = diffs.get(key, 0.0) + (tw / 2.0) * (sw / 2.0)
    nodes = np.array(sorted(diffs))
    weights = np.array([diffs[k] for k in sorted(diffs)])
    return nodes, weights


def _N_quadrature(X, Y, Z, a, b, c):
    """Cell-averaged point-dipole tensor, N = -(1/4pi) V <(3 d d^T - |d|^2 I)/|d|^5>.

    The average runs over 3-point Gauss-Legendre points of both the target and
    the source cell in every axis (d = R + t - s).
    """
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros(np.broadcast(X, Y, Z).shape + (6,))
    nodes, weights = _pair_difference_rule()
    V = a * b * c
    for u, wu in zip(nodes, weights):
        for v, wv in zip(nodes, weights):
            for t, wt in zip(nodes, weights):
                w = wu * wv * wt
                dx = X + u * a / 2
                dy = Y + v * b / 2
                dz = Z + t * c / 2
                r2 = dx * dx + dy * dy + dz * dz
                r5 = r2 * r2 * np.sqrt(r2)
                out[..., 0] += w * (3 * dx * dx - r2) / r5
                out[..., 1] += w * (3 * dy * dy - r2) / r5
                out[..., 2] += w * (3 * dz * dz - r2) / r5
                out[..., 3] += w * (3 * dx * dy) / r5
                out[..., 4] += w * (3 * dx * dz) / r5
                out[..., 5] += w * (3 * dy * dz) / r5
    return -out * (V / (4.0 * np.pi))


def N_kernel(X, Y, Z, a, b, c):
    """Demag tensor N(R) for R = target - source; returns (..., 6) = xx, yy, zz, xy, xz, yz."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, np.float64), np.asarray(Y, np.float64),
                                  np.asarray(Z, np.float64))
    far = np.maximum(np.maximum(np.abs(X / a), np.abs(Y / b)), np.abs(Z / c)) > R_FAR + 1e-9
    out = np.empty(X.shape + (6,))
    if np.any(~far):
        out[~far] = _N_closed(X[~far], Y[~far], Z[~far], a, b, c)
    if np.any(far):
        out[far] = _N_quadrature(X[far], Y[far], Z[far], a, b, c)
    return out


def N_as_matrix(n6):
    """(..., 6) -> (..., 3, 3) symmetric tensor."""
    xx, yy, zz, xy, xz, yz = (n6[..., k] for k in range(6))
    return np.stack([np.stack([xx, xy, xz], -1), np.stack([xy, yy, yz], -1),
                     np.stack([xz, yz, zz], -1)], -2)
