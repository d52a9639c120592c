"""Pins of the direct componentwise interpolation (oracle/variants.py), CPU only.

* the field on the box by convolution equals the explicit sum over source
  cells (pins the offset window and the component bookkeeping of N);
* far from a small source the box field is the point-dipole field
  V/(4 pi r^3) (3 (M.r) r / r^2 - M), with (d/r)^2 convergence (pins the sign
  H = -N M and the kernel's scale);
* at a whole-cell displacement every target centre is a box node, where the
  interpolant reproduces the box field exactly (prefilter + evaluation);
* a field that is a cubic polynomial on the box is reproduced between nodes
  away from the mirror ends (exact cubic reproduction of the B-spline);
* for a smooth distant source the componentwise and the potential-gradient
  fields agree: both approximate the same continuum field.
"""

import numpy as np

from oracle import variants as V
from oracle.fields import box_for_target, target_positions
from oracle.interaction import stray_interaction
from oracle.spline import evaluate, prefilter_3d

CELL = (4e-9, 3e-9, 2e-9)


def test_field_on_box_convolution_equals_direct_sum():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((3, 2, 3, 4)) * 8e5
    lo, dims = box_for_target((3, 2, 2), (1, 0, 4), (0, 0, 0), (0.3, 0.2, 0.0), True)
    a = V.field_on_box(M, CELL, lo, dims)
    b = V.field_on_box_direct(M, CELL, lo, dims)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_far_box_field_is_dipole_field():
    M0 = np.array([3e5, -2e5, 6e5])
    errs = []
    for dist in (12, 24):
        M = np.zeros((3, 1, 1, 1))
        M[:, 0, 0, 0] = M0
        lo = (dist, -3, 2)
        dims = (1, 1, 1)
        H = V.field_on_box(M, CELL, lo, dims)[:, 0, 0, 0]
        r = np.array([lo[0] * CELL[0], lo[1] * CELL[1], lo[2] * CELL[2]])
        rn = np.linalg.norm(r)
        Vc = np.prod(CELL)
        ref = Vc / (4 * np.pi * rn ** 3) * (3 * np.dot(M0, r) * r / rn ** 2 - M0)
        errs.append(np.linalg.norm(H - ref) / np.linalg.norm(ref))
    assert errs[0] < 2e-2 and errs[1] < errs[0] / 3.0, errs


def test_whole_cell_displacement_reproduces_the_box_field():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((3, 2, 5, 6)) * 8e5
    n_t, o_t, u = (4, 3, 2), (1, 1, 4), (1.0, 0.0, 0.0)
    H = V.stray_field_componentwise(M, CELL, (0, 0, 0), o_t, n_t, u, True)
    lo, dims = box_for_target(n_t, o_t, (0, 0, 0), u, True)
    Hb = V.field_on_box(M, CELL, lo, dims)
    p = target_positions(n_t, o_t, (0, 0, 0), u, True).astype(int) - np.asarray(lo)
    ref = Hb[:, p[..., 2], p[..., 1], p[..., 0]]
    assert np.max(np.abs(H - ref)) <= 1e-10 * np.max(np.abs(Hb))


def test_interpolant_reproduces_cubic_field_between_nodes():
    bz, by, bx = 14, 13, 15
    z, y, x = np.meshgrid(np.arange(bz), np.arange(by), np.arange(bx), indexing="ij")
    f = 0.3 * x ** 3 - 0.2 * x * y * z + 0.7 * y ** 2 - z ** 3 + 2.0 * x - 1.0
    coef = prefilter_3d(f)
    rng = np.random.default_rng(3)
    pos = 5.0 + 3.0 * rng.random((20, 3))   # >= 5 nodes from the ends in every axis
    val, _, _ = evaluate(coef, pos)
    X, Y, Z = pos[:, 0], pos[:, 1], pos[:, 2]
    exact = 0.3 * X ** 3 - 0.2 * X * Y * Z + 0.7 * Y ** 2 - Z ** 3 + 2.0 * X - 1.0
    assert np.max(np.abs(val - exact)) < 1e-2 * np.max(np.abs(exact))


def test_componentwise_and_potential_fields_agree_far_from_the_source():
    # a uniformly magnetised 4 x 4 x 2 block, target 10 cells above: the field
    # is smooth on the cell scale, so both interpolations see the same field
    M = np.zeros((3, 2, 4, 4))
    M[0], M[2] = 4e5, 7e5
    n_t, o_t, u = (4, 4, 1), (0, 0, 12), (0.37, 0.21, 0.0)
    Mt = np.zeros((3, 1, 4, 4))
    Hc = V.stray_field_componentwise(M, CELL, (0, 0, 0), o_t, n_t, u, True)
    Hp = stray_interaction(M, Mt, CELL, (0, 0, 0), o_t, u, True)["H"]
    assert np.linalg.norm(Hc - Hp) < 2e-2 * np.linalg.norm(Hp)
