"""Pins of the oracle's potential and self-demag field (Sec. III.A).

* potential of a uniformly magnetised cuboid: the cell sum telescopes to the
  potential of the two charged end faces, integrated here with scipy dblquad;
* potential far from a small magnet: point dipole of its total moment;
* direct sum == linear convolution (two evaluations of the same sum);
* demag of a uniformly magnetised cube averages to -M/3; a wide thin film
  magnetised out of plane has H_z ~ -M at its centre;
* box convention: sizes and placement of Sec. III.A's four-cell margin.
"""

import numpy as np
import pytest
from scipy import integrate

from oracle import fields as F

CELL = (4e-9, 4e-9, 4e-9)


def face_potential(point, x_face, y1, y2, z1, z2):
    """int over the face x = x_face of dA / |r - r'| by adaptive quadrature."""
    px, py, pz = point
    val, _ = integrate.dblquad(lambda z, y: 1 / np.sqrt((px - x_face) ** 2 + (py - y) ** 2
                                                        + (pz - z) ** 2),
                               y1, y2, z1, z2, epsabs=1e-22, epsrel=1e-12)
    return val


def test_uniform_cuboid_potential_is_end_face_charges():
    nx, ny, nz = 6, 4, 3
    Ms = 8e5
    M = np.zeros((3, nz, ny, nx))
    M[0] = Ms
    dx, dy, dz = CELL
    box_lo, box_dims = (-3, -2, -2), (12, 8, 7)
    phi = F.potential_conv(M, CELL, box_lo, box_dims)
    # cuboid spans [-dx/2, (nx-1/2) dx] etc. around node coordinates
    x0, x1 = -dx / 2, (nx - 0.5) * dx
    y0, y1 = -dy / 2, (ny - 0.5) * dy
    z0, z1 = -dz / 2, (nz - 0.5) * dz
    rng = np.random.default_rng(3)
    for _ in range(6):
        k = [int(rng.integers(0, d)) for d in box_dims]
        p = [(box_lo[a] + k[a]) * CELL[a] for a in range(3)]
        ref = Ms / (4 * np.pi) * (face_potential(p, x1, y0, y1, z0, z1)
                                  - face_potential(p, x0, y0, y1, z0, z1))
        got = phi[k[2], k[1], k[0]]
        assert abs(got - ref) <= 1e-9 * Ms * dx, (k, got, ref)


def test_potential_direct_equals_convolution():
    rng = np.random.default_rng(4)
    M = rng.standard_normal((3, 2, 5, 7)) * 1e5
    box_lo, box_dims = (-6, -5, 4), (15, 11, 9)
    a = F.potential_direct(M, CELL, box_lo, box_dims)
    b = F.potential_conv(M, CELL, box_lo, box_dims)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(a).max())


def test_potential_far_field_is_point_dipole():
    M = np.zeros((3, 2, 2, 2))
    M[:, :, :, :] = np.array([3e5, -2e5, 5e5])[:, None, None, None]
    box_lo, box_dims = (40, -30, 25), (3, 3, 3)
    phi = F.potential_conv(M, CELL, box_lo, box_dims)
    m_tot = np.array([3e5, -2e5, 5e5]) * 8 * np.prod(CELL)
    centre = np.array([0.5, 0.5, 0.5]) * np.array(CELL)
    for k in [(0, 0, 0), (2, 1, 2)]:
        r = np.array([(box_lo[a] + k[a]) * CELL[a] for a in range(3)]) - centre
        ref = m_tot @ r / (4 * np.pi * np.linalg.norm(r) ** 3)
        assert abs(phi[k[2], k[1], k[0]] - ref) < 2e-3 * abs(ref)


def test_demag_direct_equals_convolution():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((3, 2, 3, 4)) * 1e5
    a = F.demag_direct(M, CELL)
    b = F.demag_conv(M, CELL)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(a).max())


def test_demag_uniform_cube_average_is_one_third():
    n = 6
    Ms = 1e6
    for axis in range(3):
        M = np.zeros((3, n, n, n))
        M[axis] = Ms
        H = F.demag_conv(M, CELL)
        avg = H.reshape(3, -1).mean(axis=1)
        expect = np.zeros(3)
        expect[axis] = -Ms / 3
        np.testing.assert_allclose(avg, expect, atol=1e-10 * Ms)


def test_demag_thin_film_out_of_plane():
    n = 64
    M = np.zeros((3, 1, n, n))
    M[2] = 1e6
    H = F.demag_conv(M, CELL)
    hz = H[2, 0, n // 2, n // 2]
    assert -1e6 < hz < -0.95e6


def test_box_convention():
    lo, dims = F.box_for_target((64, 64, 1), (0, 0, 2), (0, 0, 0), (0.25, 0.0, 0.0), True)
    assert lo == (-5, -5, -3) and dims == (75, 75, 12)
    lo, dims = F.box_for_target((64, 64, 1), (0, 0, 0), (0, 0, 2), (0.25, 0.0, 0.0), False)
    assert lo == (-6, -5, -7) and dims == (75, 75, 12)
    lo, dims = F.box_for_target((1024, 256, 2), (0, 0, 7), (0, 0, 0), (0.0, 0.0, 0.0), True)
    assert lo == (-5, -5, 2) and dims == (1035, 267, 13)
