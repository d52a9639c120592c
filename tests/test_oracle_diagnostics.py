"""Pins of the divergence / curl diagnostics (oracle/diagnostics.py), CPU only:
fields whose central differences are exact (linear and quadratic), and a
cell-by-cell loop on a small random field."""

import numpy as np

from oracle.diagnostics import div_curl_means

CELL = (4e-9, 3e-9, 2e-9)


def _grid(n):
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz) * CELL[2], np.arange(ny) * CELL[1], np.arange(nx) * CELL[0],
                          indexing="ij")
    return x, y, z


def test_linear_field_div_is_trace_curl_is_antisymmetric_part():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 3)) * 1e12   # A/m per m
    x, y, z = _grid((7, 6, 5))
    r = np.stack([x, y, z])
    H = np.einsum("ab,b...->a...", A, r) + 1e5
    D, C = div_curl_means(H, CELL)
    assert abs(D - abs(np.trace(A))) <= 1e-9 * abs(np.trace(A))
    w = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    assert abs(C - np.linalg.norm(w)) <= 1e-9 * np.linalg.norm(w)


def test_gradient_of_quadratic_potential_is_curl_free():
    """H = -grad(phi) for a quadratic phi: central differences are exact, so
    curl = 0 and div = -laplacian(phi) everywhere."""
    x, y, z = _grid((8, 7, 6))
    a, b, c, p, q, s = 3e14, -1e14, 5e13, 2e14, -4e13, 7e13
    # phi = a x^2 + b y^2 + c z^2 + p x y + q y z + s x z
    H = -np.stack([2 * a * x + p * y + s * z, 2 * b * y + p * x + q * z, 2 * c * z + q * y + s * x])
    D, C = div_curl_means(H, CELL)
    lap = 2 * (a + b + c)
    assert abs(D - abs(lap)) <= 1e-9 * abs(lap)
    assert C <= 1e-9 * abs(lap)


def test_thin_axis_drops_its_derivatives():
    """An axis of fewer than three cells contributes no derivative; the means run
    over the cells interior along the others."""
    rng = np.random.default_rng(1)
    H = rng.standard_normal((3, 2, 5, 6))
    D, C = div_curl_means(H, CELL)
    Hd = H.copy()
    Hd[2] += 7.0 * np.arange(2)[:, None, None]   # a z gradient of Hz: invisible
    assert div_curl_means(Hd, CELL) == (D, C)


def test_random_field_against_cell_loop():
    rng = np.random.default_rng(2)
    nx, ny, nz = 5, 4, 3
    H = rng.standard_normal((3, nz, ny, nx))
    d = CELL
    sd = sc = 0.0
    cnt = 0
    for k in range(1, nz - 1):
        for j in range(1, ny - 1):
            for i in range(1, nx - 1):
                def g(c, a):
                    e = [0, 0, 0]
                    e[a] = 1
                    return (H[c, k + e[2], j + e[1], i + e[0]] - H[c, k - e[2], j - e[1], i - e[0]]) / (2 * d[a])
                sd += abs(g(0, 0) + g(1, 1) + g(2, 2))
                cx, cy, cz = g(2, 1) - g(1, 2), g(0, 2) - g(2, 0), g(1, 0) - g(0, 1)
                sc += (cx * cx + cy * cy + cz * cz) ** 0.5
                cnt += 1
    D, C = div_curl_means(H, CELL)
    assert abs(D - sd / cnt) <= 1e-12 * D
    assert abs(C - sc / cnt) <= 1e-12 * C
