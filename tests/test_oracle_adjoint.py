"""Pins of the oracle's energy gradients (oracle/adjoint.py), CPU only.

Each adjoint piece must be the exact transpose of the forward oracle step it
reverses (inner-product identities against the independently pinned forward
functions), and the assembled gradients must match finite differences of the
forward energy: E is linear in M_s and in M_t, so a unit step is exact up to
rounding; in u a central difference with h = 1e-3 cell.
"""

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import fields as OF
from oracle.interaction import stray_interaction
from oracle.spline import evaluate, prefilter_3d

CELL = (4e-9, 3e-9, 2e-9)


def _pair(seed, n_s=(6, 5, 2), n_t=(7, 4, 3)):
    rng = np.random.default_rng(seed)
    M_s = 8e5 * rng.standard_normal((3,) + tuple(reversed(n_s)))
    M_t = 1.1e6 * rng.standard_normal((3,) + tuple(reversed(n_t)))
    return M_s, M_t


def test_prefilter_transpose_identity():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((7, 9, 12))
    y = rng.standard_normal((7, 9, 12))
    lhs = np.sum(A.prefilter_T_3d(y) * x)
    rhs = np.sum(y * prefilter_3d(x))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_evaluate_transpose_identity():
    rng = np.random.default_rng(1)
    c = rng.standard_normal((8, 9, 10))
    pos = np.stack([rng.uniform(1.0, 6.9, 50), rng.uniform(1.0, 5.9, 50), rng.uniform(1.0, 4.9, 50)], axis=-1)
    g = rng.standard_normal((50, 3))
    _, grad_n, _ = evaluate(c, pos)
    lhs = np.sum(A.evaluate_T(g, pos, c.shape) * c)
    rhs = np.sum(g * grad_n)
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(g * grad_n))


def test_potential_transpose_identity():
    M_s, _ = _pair(2)
    n_s = (M_s.shape[3], M_s.shape[2], M_s.shape[1])
    box_lo, box_dims = (-3, 4, 3), (9, 7, 6)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(tuple(reversed(box_dims)))
    lhs = np.sum(A.potential_T(psi, n_s, CELL, box_lo, box_dims) * M_s)
    phi = OF.potential_conv(M_s, CELL, box_lo, box_dims)
    rhs = np.sum(psi * phi)
    assert abs(lhs - rhs) <= 1e-10 * np.sum(np.abs(psi * phi))


@pytest.mark.parametrize("target_is_slider", [True, False])
def test_energy_gradients_match_finite_differences(target_is_slider):
    M_s, M_t = _pair(4)
    o_s, o_t = ((0, 0, 0), (1, -1, 4)) if target_is_slider else ((1, -1, 4), (0, 0, 0))
    u = (0.37, 0.21, 0.11)
    g = A.energy_gradients(M_s, M_t, CELL, o_s, o_t, u, target_is_slider)

    def E(Ms, Mt, uu):
        return stray_interaction(Ms, Mt, CELL, o_s, o_t, uu, target_is_slider)["E"]

    E0 = E(M_s, M_t, u)
    assert abs(g["E"] - E0) <= 1e-12 * abs(E0)
    rng = np.random.default_rng(5)
    for _ in range(3):
        es = 1e5 * rng.standard_normal(M_s.shape)
        et = 1e5 * rng.standard_normal(M_t.shape)
        ds = E(M_s + es, M_t, u) - E0
        dt = E(M_s, M_t + et, u) - E0
        assert abs(ds - np.sum(g["dE_dMs"] * es)) <= 1e-9 * np.sum(np.abs(g["dE_dMs"] * es))
        assert abs(dt - np.sum(g["dE_dMt"] * et)) <= 1e-9 * np.sum(np.abs(g["dE_dMt"] * et))
    # single cells of the source, every component
    for (c, z, y, x) in [(0, 0, 0, 0), (1, 1, 4, 5), (2, 1, 2, 3)]:
        e = np.zeros_like(M_s)
        e[c, z, y, x] = 1e5
        assert np.isclose(E(M_s + e, M_t, u) - E0, 1e5 * g["dE_dMs"][c, z, y, x], rtol=1e-7,
                          atol=1e-9 * abs(E0))
    h = 1e-3
    for a in range(3):
        up = list(u); um = list(u)
        up[a] += h; um[a] -= h
        fd = (E(M_s, M_t, tuple(up)) - E(M_s, M_t, tuple(um))) / (2 * h * CELL[a])
        assert abs(fd - g["dE_du"][a]) <= 1e-5 * np.max(np.abs(g["dE_du"])) + 1e-6 * abs(fd)
