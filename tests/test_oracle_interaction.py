"""Pins of the oracle's stray field, Eq. (EQForce) force and interaction energy.

* F = -dE/du by central differences (h = 1e-3 cell): ties the Hessian to the
  gradient and fixes the force sign;
* a whole-cell displacement equals moving the lattice offset by one cell;
* far apart, the stray field is the point-dipole field of the source moment
  (units, the minus sign of H = -grad phi and the cell-size scaling);
* the direct-sum and convolution potentials give the same field;
* Newton's third law for smooth (uniform) magnets at integer displacement.
"""

import numpy as np
import pytest

from oracle import MU0
from oracle.interaction import stray_interaction
from workloads import random_unit

CELL = (4e-9, 4e-9, 4e-9)


def test_force_is_minus_energy_gradient():
    Ms = 8e5
    Ms_ = Ms * random_unit((8, 7, 1), 11)
    Mt = Ms * random_unit((8, 7, 1), 12)
    o_s, o_t = (0, 0, 0), (0, 0, 2)
    u = np.array([0.37, 0.21, 0.13])
    base = stray_interaction(Ms_, Mt, CELL, o_s, o_t, u, True)
    h = 1e-3
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        Ep = stray_interaction(Ms_, Mt, CELL, o_s, o_t, u + e, True)["E"]
        Em = stray_interaction(Ms_, Mt, CELL, o_s, o_t, u - e, True)["E"]
        dE_du = (Ep - Em) / (2 * h)
        F_fd = -dE_du / CELL[a]
        scale = np.abs(base["F"]).max()
        assert abs(base["F"][a] - F_fd) < 1e-5 * scale, (a, base["F"][a], F_fd)


def test_whole_cell_displacement_is_index_shift():
    Ms = 8e5
    Ms_ = Ms * random_unit((9, 6, 2), 21)
    Mt = Ms * random_unit((9, 6, 2), 22)
    a = stray_interaction(Ms_, Mt, CELL, (0, 0, 0), (0, 0, 3), (1.0, 0.0, 0.0), True)
    b = stray_interaction(Ms_, Mt, CELL, (0, 0, 0), (1, 0, 3), (0.0, 0.0, 0.0), True)
    np.testing.assert_allclose(a["H"], b["H"], rtol=0, atol=1e-12 * np.abs(a["H"]).max())
    np.testing.assert_allclose(a["F"], b["F"], rtol=1e-12)
    # and for the slider as source (sigma = -1)
    c = stray_interaction(Mt, Ms_, CELL, (0, 0, 3), (0, 0, 0), (1.0, 0.0, 0.0), False)
    d = stray_interaction(Mt, Ms_, CELL, (1, 0, 3), (0, 0, 0), (0.0, 0.0, 0.0), False)
    np.testing.assert_allclose(c["H"], d["H"], rtol=0, atol=1e-12 * np.abs(c["H"]).max())


def test_far_stray_field_is_dipole_field():
    Ms = 8e5
    m = np.array([0.3, -0.5, 0.81])
    m = m / np.linalg.norm(m)
    Ms_ = np.zeros((3, 2, 2, 2)) + (Ms * m)[:, None, None, None]
    Mt = np.zeros((3, 1, 1, 1)) + np.array([0.0, 0.0, 1.0])[:, None, None, None] * Ms
    o_t = (30, -20, 25)
    res = stray_interaction(Ms_, Mt, CELL, (0, 0, 0), o_t, (0.0, 0.0, 0.0), True)
    r = np.array(o_t, float) * CELL[0] - 0.5 * CELL[0]
    mom = Ms * m * 8 * CELL[0] ** 3
    rn = np.linalg.norm(r)
    H_dip = (3 * r * (mom @ r) / rn ** 5 - mom / rn ** 3) / (4 * np.pi)
    np.testing.assert_allclose(res["H"][:, 0, 0, 0], H_dip, rtol=3e-3)


def test_direct_and_convolution_agree():
    Ms = 8e5
    Ms_ = Ms * random_unit((5, 4, 1), 31)
    Mt = Ms * random_unit((5, 4, 1), 32)
    u = (0.4, 0.0, 0.0)
    a = stray_interaction(Ms_, Mt, CELL, (0, 0, 0), (0, 0, 2), u, True, direct=True)
    b = stray_interaction(Ms_, Mt, CELL, (0, 0, 0), (0, 0, 2), u, True)
    np.testing.assert_allclose(a["H"], b["H"], atol=1e-11 * np.abs(a["H"]).max())
    np.testing.assert_allclose(a["F"], b["F"], atol=1e-11 * np.abs(a["F"]).max())


def test_newton_third_law_uniform_magnets():
    Ms = 8e5
    Mb = np.zeros((3, 2, 12, 14))
    Mb[2] = Ms
    Ms_ = np.zeros((3, 2, 12, 14))
    Ms_[0] = Ms
    # the pair kernel (cell-integrated source, point target) is symmetric, so
    # without interpolation the two forces cancel exactly; what remains is the
    # spline error, which the mirror ends of a 4-cell margin raise in z
    for margin, tol in ((4, 1e-2), (8, 4e-3)):
        on_slider = stray_interaction(Mb, Ms_, CELL, (0, 0, 0), (5, 3, 8), (2.0, 1.0, 0.0), True,
                                      margin=margin)
        on_base = stray_interaction(Ms_, Mb, CELL, (5, 3, 8), (0, 0, 0), (2.0, 1.0, 0.0), False,
                                    margin=margin)
        F1, F0 = on_slider["F"], on_base["F"]
        assert np.linalg.norm(F1 + F0) < tol * np.linalg.norm(F1) * 2
        assert abs(on_slider["E"] - on_base["E"]) < 1e-3 * abs(on_slider["E"])
