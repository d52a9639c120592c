"""Pins of the oracle's S and N kernels (Sec. III.A) to facts outside the oracle.

* S: oddness, the point-dipole far field, numerical cubature of its defining
  integral, and Gauss's theorem relating it to N;
* N: the self-term identities of a cube and a flat cell (trace 1), zero trace
  off the self-term (Laplace), the point-dipole far field, and continuity
  across the closed-form / quadrature switch.
"""

import numpy as np
import pytest
from scipy import integrate

from oracle import kernels as K


def dipole_N(R, V):
    r = np.linalg.norm(R)
    T = -(3 * np.outer(R, R) / r ** 5 - np.eye(3) / r ** 3) * V / (4 * np.pi)
    return np.array([T[0, 0], T[1, 1], T[2, 2], T[0, 1], T[0, 2], T[1, 2]])


CELLS = [(1.0, 1.0, 1.0), (1.0, 0.8, 0.5)]


@pytest.mark.parametrize("cell", CELLS)
def test_S_is_odd(cell):
    rng = np.random.default_rng(1)
    R = rng.integers(-6, 7, size=(20, 3)) * np.array(cell)
    S1 = K.S_kernel(R[:, 0], R[:, 1], R[:, 2], *cell)
    S2 = K.S_kernel(-R[:, 0], -R[:, 1], -R[:, 2], *cell)
    np.testing.assert_allclose(S1, -S2, atol=1e-15)
    np.testing.assert_allclose(K.S_kernel(0.0, 0.0, 0.0, *cell), 0.0, atol=1e-15)


@pytest.mark.parametrize("cell", CELLS)
def test_S_far_field_is_point_dipole(cell):
    V = np.prod(cell)
    errs = []
    for r in (8.0, 16.0, 30.0):
        R = np.array([0.6, -0.5, 0.62]) / np.linalg.norm([0.6, -0.5, 0.62]) * r
        S = K.S_kernel(*R, *cell)
        dip = V * R / (4 * np.pi * np.linalg.norm(R) ** 3)
        errs.append(np.linalg.norm(S - dip) / np.linalg.norm(dip))
    # the cell-size correction falls off as (cell / r)^2
    assert errs[0] < 5e-3
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.0


@pytest.mark.parametrize("R", [(1.0, 0.0, 0.0), (1.0, 1.0, 0.0), (0.0, 2.0, 1.0), (2.0, -1.0, 1.0)])
def test_S_matches_cubature_of_definition(R):
    """S = (1/4pi) int_cell (r - r') / |r - r'|^3 d^3r', integrated numerically."""
    a, b, c = 1.0, 1.0, 1.0
    X, Y, Z = R
    got = K.S_kernel(X, Y, Z, a, b, c)
    ref = []
    for comp in range(3):
        def f(z, y, x):
            d = np.array([X - x, Y - y, Z - z])
            return d[comp] / np.linalg.norm(d) ** 3
        val, _ = integrate.tplquad(f, -a / 2, a / 2, -b / 2, b / 2, -c / 2, c / 2,
                                   epsabs=1e-12, epsrel=1e-10)
        ref.append(val / (4 * np.pi))
    np.testing.assert_allclose(got, ref, rtol=1e-7, atol=1e-10)


def test_rect_potential_matches_dblquad():
    for xi, y1, y2, z1, z2 in [(0.5, -0.5, 0.5, -0.5, 0.5), (1.5, -2.5, -1.5, 0.5, 1.5),
                               (0.0, 1.0, 2.0, -1.0, 3.0), (-3.0, -0.5, 0.5, 2.0, 5.0)]:
        ref, _ = integrate.dblquad(lambda z, y: 1 / np.sqrt(xi ** 2 + y ** 2 + z ** 2),
                                   y1, y2, z1, z2, epsabs=1e-13, epsrel=1e-11)
        assert abs(K.rect_potential(xi, y1, y2, z1, z2) - ref) < 1e-9 * max(1, abs(ref))


@pytest.mark.parametrize("cell", CELLS)
def test_S_continuous_across_far_switch(cell):
    for R in [(K.R_FAR, 3, -5), (K.R_FAR, K.R_FAR, 1), (-7, K.R_FAR, 2)]:
        R = np.array(R, float) * np.array(cell)
        c = K._S_closed(*R, *cell)
        q = K._S_quadrature(*R, *cell)
        assert np.linalg.norm(c - q) / np.linalg.norm(c) < 1e-8


def test_N_self_terms():
    np.testing.assert_allclose(K.N_kernel(0.0, 0.0, 0.0, 1, 1, 1), [1 / 3, 1 / 3, 1 / 3, 0, 0, 0],
                               atol=1e-14)
    for cell in [(1.0, 1.0, 0.25), (1.0, 0.8, 0.5), (2.0, 1.0, 1.0)]:
        n = K.N_kernel(0.0, 0.0, 0.0, *cell)
        assert abs(n[:3].sum() - 1.0) < 1e-12
        np.testing.assert_allclose(n[3:], 0.0, atol=1e-14)
    flat = K.N_kernel(0.0, 0.0, 0.0, 1.0, 1.0, 0.25)
    assert flat[2] > flat[0] and abs(flat[0] - flat[1]) < 1e-14


@pytest.mark.parametrize("cell", CELLS)
def test_N_trace_free_off_self_and_even(cell):
    rng = np.random.default_rng(2)
    R = rng.integers(-5, 6, size=(30, 3)).astype(float)
    R = R[np.any(R != 0, axis=1)] * np.array(cell)
    N = K.N_kernel(R[:, 0], R[:, 1], R[:, 2], *cell)
    np.testing.assert_allclose(N[:, :3].sum(axis=1), 0.0, atol=1e-12)
    Nm = K.N_kernel(-R[:, 0], -R[:, 1], -R[:, 2], *cell)
    np.testing.assert_allclose(N, Nm, atol=1e-13)
    Nx = K.N_kernel(-R[:, 0], R[:, 1], R[:, 2], *cell)  # mirror x: xy, xz flip sign
    np.testing.assert_allclose(Nx * np.array([1, 1, 1, -1, -1, 1]), N, atol=1e-13)


@pytest.mark.parametrize("cell", CELLS)
def test_N_far_field_is_point_dipole(cell):
    V = np.prod(cell)
    errs = []
    for r in (8.0, 16.0):
        R = np.array([0.7, 0.45, -0.55]) / np.linalg.norm([0.7, 0.45, -0.55]) * r
        n = K.N_kernel(*R, *cell)
        d = dipole_N(R, V)
        errs.append(np.abs(n - d).max() / np.abs(d).max())
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 3.5


@pytest.mark.parametrize("cell", CELLS)
def test_N_continuous_across_far_switch(cell):
    for R in [(K.R_FAR, 3, -5), (K.R_FAR, K.R_FAR, 1), (-7, K.R_FAR, 2)]:
        R = np.array(R, float) * np.array(cell)
        c = K._N_closed(*R, *cell)
        q = K._N_quadrature(*R, *cell)
        # at the switch the closed form keeps ~5e-8 against cancellation and the
        # 3-point rule ~1e-9 against its truncation
        assert np.abs(c - q).max() / np.abs(c).max() < 2e-7


@pytest.mark.parametrize("R", [(1, 0, 0), (2, 1, 0), (1, 1, 1), (0, 0, 3), (3, -2, 1)])
def test_N_from_S_by_gauss_theorem(R):
    """Cell-averaged H = -(1/V) int grad phi = -(1/V) oint phi n dA, phi = S(r) . M.

    So N[a, b] = (1/V) [int over the +a face of S_b - int over the -a face of S_b],
    with S evaluated at continuous points of the target faces.  Ties the Newell
    closed form to the S closed form through an identity neither side uses.
    """
    cell = np.array([1.0, 0.8, 0.5])
    touching = max(abs(v) for v in R) == 1
    R = np.array(R, float) * cell
    V = cell.prod()
    # a face that touches the source cell has edge singularities in grad S:
    # Gauss-Legendre still converges there, only algebraically
    nodes, weights = np.polynomial.legendre.leggauss(96 if touching else 16)
    s1, s2 = np.meshgrid(nodes, nodes, indexing="ij")
    w = np.outer(weights, weights) / 4
    got = np.zeros((3, 3))
    for a in range(3):
        o1, o2 = [k for k in range(3) if k != a]
        for side in (+1, -1):
            p = np.zeros(s1.shape + (3,)) + R
            p[..., a] += side * cell[a] / 2
            p[..., o1] += s1 * cell[o1] / 2
            p[..., o2] += s2 * cell[o2] / 2
            S = K.S_kernel(p[..., 0], p[..., 1], p[..., 2], *cell)
            got[a] += side * np.einsum("ij,ijc->c", w, S) * cell[o1] * cell[o2] / V
    N = K.N_as_matrix(K.N_kernel(*R, *cell))
    tol = 5e-8 if touching else 1e-11
    np.testing.assert_allclose(got, N, atol=tol * np.abs(N).max())
