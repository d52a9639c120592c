"""Pins of the oracle's B-spline prefilter and 64-term evaluation (Sec. III.A, IV.D).

* the banded mirror-end solve equals the periodic spline of the whole-sample
  symmetric extension (period 2b - 2), solved independently in Fourier space;
* the interpolant reproduces the samples at the nodes and cubic polynomials in
  the interior (up to the 0.268^d decay of the end effect);
* gradient and Hessian equal finite differences of the evaluated interpolant;
* weights form a partition of unity with zero-sum derivatives.
"""

import numpy as np
import pytest

from oracle import spline as S


def periodic_mirror_coefficients(phi):
    """Coefficients of the symmetric extension by a circulant solve via numpy FFT."""
    b = len(phi)
    ext = np.concatenate([phi, phi[-2:0:-1]])  # length 2b - 2
    L = len(ext)
    k = np.arange(L)
    symbol = (4 + 2 * np.cos(2 * np.pi * k / L)) / 6
    c = np.real(np.fft.ifft(np.fft.fft(ext) / symbol))
    return c[:b]


@pytest.mark.parametrize("b", [2, 3, 5, 12, 40])
def test_prefilter_equals_mirror_periodic_spline(b):
    rng = np.random.default_rng(b)
    phi = rng.standard_normal(b)
    c = S.prefilter_1d(phi, 0)
    np.testing.assert_allclose(c, periodic_mirror_coefficients(phi), atol=1e-12)


def test_interpolates_nodes_3d():
    rng = np.random.default_rng(7)
    phi = rng.standard_normal((9, 10, 12))
    c = S.prefilter_3d(phi)
    # every node whose 4 x 4 x 4 support lies inside the box
    z, y, x = np.meshgrid(np.arange(1, 7), np.arange(1, 8), np.arange(1, 10), indexing="ij")
    pos = np.stack([x, y, z], -1).astype(float)
    val, _, _ = S.evaluate(c, pos)
    np.testing.assert_allclose(val, phi[1:7, 1:8, 1:10], atol=1e-12)


def test_reproduces_cubics_in_interior():
    b = 60
    xs = np.arange(b, dtype=float)
    coef = [0.3, -1.2, 0.05, 0.001]

    def p(x):
        return coef[0] + coef[1] * x + coef[2] * x ** 2 + coef[3] * x ** 3

    phi = np.broadcast_to(p(xs)[None, None, :], (6, 6, b)).copy()
    c = S.prefilter_3d(phi)
    pts = np.array([[x, 2.5, 2.5] for x in np.linspace(25.0, 34.7, 17)])
    val, grad, hess = S.evaluate(c, pts)
    x = pts[:, 0]
    np.testing.assert_allclose(val, p(x), rtol=1e-9)
    np.testing.assert_allclose(grad[:, 0], coef[1] + 2 * coef[2] * x + 3 * coef[3] * x ** 2, rtol=1e-8)
    np.testing.assert_allclose(hess[:, 0, 0], 2 * coef[2] + 6 * coef[3] * x, rtol=1e-7)
    np.testing.assert_allclose(grad[:, 1:], 0, atol=1e-9)


def test_derivatives_match_finite_differences():
    rng = np.random.default_rng(8)
    c = rng.standard_normal((8, 9, 10))
    p0 = np.array([[4.3, 3.7, 3.2], [5.01, 4.99, 4.5]])
    h = 1e-5
    _, g, H = S.evaluate(c, p0)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        vp, gp, _ = S.evaluate(c, p0 + e)
        vm, gm, _ = S.evaluate(c, p0 - e)
        np.testing.assert_allclose((vp - vm) / (2 * h), g[:, a], atol=1e-8)
        np.testing.assert_allclose((gp - gm) / (2 * h), H[:, :, a], atol=1e-7)


def test_weights_partition_of_unity():
    t = np.linspace(0, 1, 11)
    w = S.weights(t)
    np.testing.assert_allclose(w[0].sum(axis=0), 1.0, atol=1e-15)
    np.testing.assert_allclose(w[1].sum(axis=0), 0.0, atol=1e-15)
    np.testing.assert_allclose(w[2].sum(axis=0), 0.0, atol=1e-14)
    # first moment: sum_k w_k (k - 1) = t  (nodes floor-1 .. floor+2)
    np.testing.assert_allclose((w[0] * (np.arange(4) - 1)[:, None]).sum(axis=0), t, atol=1e-15)


def test_fd4_gradient_of_interpolated_cubic_is_exact():
    """The four-point difference is exact for cubics, and the B-spline of a cubic
    reproduces it in the interior: the variant's H equals -grad of the cubic at
    every displaced centre (pins the stencil, its signs and the centre offsets)."""
    from oracle.variants import fd4_gradient

    cell = (4e-9, 3e-9, 2e-9)
    rng = np.random.default_rng(4)
    a = rng.standard_normal(10)

    def phi(x, y, z):  # node coordinates
        return (a[0] * x ** 3 + a[1] * y ** 3 + a[2] * z ** 3 + a[3] * x * y * z + a[4] * x * x * y
                + a[5] * y * y * z + a[6] * x + a[7] * y * z + a[8] * z * z + a[9])

    def grad(x, y, z):
        return np.stack([3 * a[0] * x ** 2 + a[3] * y * z + 2 * a[4] * x * y + a[6],
                         3 * a[1] * y ** 2 + a[3] * x * z + a[4] * x * x + 2 * a[5] * y * z + a[7] * z,
                         3 * a[2] * z ** 2 + a[3] * x * y + a[5] * y * y + a[7] * y + 2 * a[8] * z])

    from oracle.spline import evaluate
    # exact cubic values at the extended centres, then FD4 in node units (cell 1)
    n = (5, 4, 3)
    f = (0.37, 0.61, 0.13)
    zz, yy, xx = np.meshgrid(np.arange(n[2] + 4) - 2 + f[2], np.arange(n[1] + 4) - 2 + f[1],
                             np.arange(n[0] + 4) - 2 + f[0], indexing="ij")
    H = fd4_gradient(phi(xx, yy, zz), (1.0, 1.0, 1.0))
    g = grad(xx[2:-2, 2:-2, 2:-2], yy[2:-2, 2:-2, 2:-2], zz[2:-2, 2:-2, 2:-2])
    np.testing.assert_allclose(H, -g, rtol=1e-11, atol=1e-11 * np.abs(g).max())
    # through the interpolant: samples of the cubic on a box whose ends are far away
    B = 40
    bz, by, bx = np.meshgrid(np.arange(B), np.arange(B), np.arange(B), indexing="ij")
    coef = S.prefilter_3d(phi(bx, by, bz))
    pos = np.stack([xx + 17, yy + 17, zz + 17], axis=-1)
    val, _, _ = evaluate(coef, pos)
    H2 = fd4_gradient(val, cell)
    g2 = grad(xx[2:-2, 2:-2, 2:-2] + 17, yy[2:-2, 2:-2, 2:-2] + 17, zz[2:-2, 2:-2, 2:-2] + 17)
    for c in range(3):
        np.testing.assert_allclose(H2[c], -g2[c] / cell[c], rtol=1e-6, atol=1e-6 * np.abs(g2[c]).max() / cell[c])
