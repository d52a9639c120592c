"""Pins of the periodic in-plane boundary conditions (oracle/periodic.py), CPU only.

* an infinite film magnetised uniformly along z (periodic, so infinite in the
  plane) has H = -Ms z inside, nothing in plane, and no stray field outside;
  magnetised in plane it has no field at all: the image sums converge to
  these limits as the number of images R grows;
* the periodic prefilter solves the circulant system exactly (against a
  dense solve) and the periodic spline interpolates its samples;
* a whole-period displacement changes nothing; a whole-cell displacement
  is an index shift (np.roll) of the source;
* F = -dE/du by central differences of the periodic interpolant's energy;
* with one image (R = 0) and a period long enough that no wrapped offset
  falls inside the source-to-box window, the periodic potential equals the
  open-boundary one on the box (the convolution is the same sum).
"""

import numpy as np

from oracle import fields as OF
from oracle import periodic as P

CELL = (4e-9, 4e-9, 4e-9)


def _uniform(n, m):
    nx, ny, nz = n
    M = np.zeros((3, nz, ny, nx))
    for c in range(3):
        M[c] = m[c]
    return M


def test_uniform_perpendicular_film_limits():
    n, Ms = (8, 8, 2), 8e5
    M = _uniform(n, (0.0, 0.0, Ms))
    errs = []
    for R in (2, 8):
        H = P.demag_periodic(M, CELL, R)
        # inside: H = -Ms z, no in-plane component (by symmetry, exactly)
        assert np.max(np.abs(H[:2])) < 1e-9 * Ms
        errs.append(np.max(np.abs(H[2] + Ms)) / Ms)
    assert errs[1] < errs[0] / 2.5 and errs[1] < 2e-2, errs
    # outside (3 cells above): the stray field of an infinite sheet vanishes
    Mt = _uniform((8, 8, 1), (0.0, 0.0, 0.0))
    out = []
    for R in (2, 8):
        r = P.stray_interaction_periodic(M, Mt, CELL, (0, 0, 0), (0, 0, 5), (0.3, 0.4, 0.0), True, R)
        out.append(np.max(np.abs(r["H"])) / Ms)
    # truncated to (2R + 1)^2 periods the sheet's charges leave a field ~ 1/(2R + 1)
    assert out[1] < out[0] / 2.5 and out[1] < 2e-2, out


def test_uniform_in_plane_film_has_no_field():
    n, Ms = (8, 6, 2), 8e5
    M = _uniform(n, (Ms * 0.6, Ms * 0.8, 0.0))
    errs = [np.max(np.abs(P.demag_periodic(M, CELL, R))) / Ms for R in (2, 8)]
    assert errs[1] < errs[0] / 2.5 and errs[1] < 1e-2, errs


def test_periodic_prefilter_is_the_circulant_inverse():
    rng = np.random.default_rng(0)
    n = 11
    phi = rng.standard_normal((3, n))
    A = np.zeros((n, n))
    for k in range(n):
        A[k, k] = 4 / 6
        A[k, (k - 1) % n] += 1 / 6
        A[k, (k + 1) % n] += 1 / 6
    ref = np.linalg.solve(A, phi.T).T
    got = P.prefilter_periodic_1d(phi, 1)
    assert np.max(np.abs(got - ref)) < 1e-13
    # interpolation: the spline of the coefficients equals phi at every node
    # (every x, y node; the interior z nodes, whose taps stay in the 5-plane box)
    c = rng.standard_normal((5, 7, 9))
    coef = P.prefilter_periodic(c)
    z, y, x = np.meshgrid(np.arange(5), np.arange(7), np.arange(9), indexing="ij")
    pos = np.stack([x, y, z - 3], axis=-1).astype(float)  # source lattice: plane 0 of the box is z = -3
    val, _, _ = P.evaluate_periodic(coef, pos[1:3], -3)
    assert np.max(np.abs(val - c[1:3])) < 1e-12 * np.max(np.abs(c))


def test_whole_period_move_and_index_shift():
    rng = np.random.default_rng(4)
    n0, n1 = (10, 8, 2), (10, 8, 1)
    M0 = rng.standard_normal((3, 2, 8, 10)) * 8e5
    M1 = rng.standard_normal((3, 1, 8, 10)) * 8e5
    kern = {}
    a = P.stray_interaction_periodic(M0, M1, CELL, (0, 0, 0), (0, 0, 4), (0.3, 0.6, 0.0), True, 1, kernels=kern)
    b = P.stray_interaction_periodic(M0, M1, CELL, (0, 0, 0), (0, 0, 4), (10.3, -7.4, 0.0), True, 1, kernels=kern)
    assert np.max(np.abs(a["H"] - b["H"])) <= 1e-9 * np.max(np.abs(a["H"]))
    # u = (1, 0, 0) equals rolling the target's lattice offset by one cell
    c = P.stray_interaction_periodic(M0, M1, CELL, (0, 0, 0), (0, 0, 4), (1.0, 0.0, 0.0), True, 1, kernels=kern)
    d = P.stray_interaction_periodic(M0, M1, CELL, (0, 0, 0), (1, 0, 4), (0.0, 0.0, 0.0), True, 1, kernels=kern)
    assert np.max(np.abs(c["H"] - d["H"])) <= 1e-9 * np.max(np.abs(c["H"]))
    assert np.max(np.abs(c["F"] - d["F"])) <= 1e-9 * np.max(np.abs(c["F"]))


def test_periodic_force_is_minus_energy_gradient():
    rng = np.random.default_rng(5)
    M0 = rng.standard_normal((3, 2, 8, 10)) * 8e5
    M1 = rng.standard_normal((3, 1, 8, 10)) * 8e5
    kern = {}
    u0 = np.array([0.41, 0.27, 0.0])
    r = P.stray_interaction_periodic(M0, M1, CELL, (0, 0, 0), (0, 0, 4), tuple(u0), True, 1, kernels=kern)
    h = 1e-3
    for a in (0, 1):
        du = np.zeros(3)
        du[a] = h
        Ep = P.stray_interaction_periodic(M0, M1, CELL, (0, 0, 0), (0, 0, 4), tuple(u0 + du), True, 1,
                                          kernels=kern)["E"]
        Em = P.stray_interaction_periodic(M0, M1, CELL, (0, 0, 0), (0, 0, 4), tuple(u0 - du), True, 1,
                                          kernels=kern)["E"]
        dE = (Ep - Em) / (2 * h * CELL[a])
        assert abs(r["F"][a] + dE) <= 1e-5 * (abs(dE) + 1e-3 * np.max(np.abs(r["F"])))


def test_single_image_long_period_equals_open_potential():
    # a source of 3 x 3 cells at the start of a period of 24 x 20: every box
    # node of the 3 x 3 target at offset (2, 1) sees the source at offsets
    # |d| < P / 2, so the circular sum with R = 0 is the open sum
    rng = np.random.default_rng(6)
    Ms = rng.standard_normal((3, 1, 3, 3)) * 8e5
    M = np.zeros((3, 1, 20, 24))
    M[:, :, :3, :3] = Ms
    z_lo, bz = P.box_z(1, 3, 0, 0.0, True, 4)
    phi = P.potential_periodic(M, CELL, z_lo, bz, 0)
    lo, dims = OF.box_for_target((3, 3, 1), (2, 1, 3), (0, 0, 0), (0.0, 0.0, 0.0), True)
    ref = OF.potential_conv(Ms, CELL, lo, dims)
    got = phi[:, np.arange(lo[1], lo[1] + dims[1]) % 20][:, :, np.arange(lo[0], lo[0] + dims[0]) % 24]
    assert lo[2] == z_lo and dims[2] == bz
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_periodic_kernels_keep_their_parities():
    """Every component of S and N is even or odd in x and in y; the periodic
    image sums keep that exactly (the Nyquist offset of an even period is the
    average of the two truncations), which is what lets their spectra be real
    or imaginary quarter planes."""
    # parity (x, y) of S_x, S_y, S_z and of N_xx, N_yy, N_zz, N_xy, N_xz, N_yz
    par = {"S": [(-1, 1), (1, -1), (1, 1)], "N": [(1, 1), (1, 1), (1, 1), (-1, -1), (-1, 1), (1, -1)]}
    Px, Py = 8, 6
    fx = (-np.arange(Px)) % Px
    fy = (-np.arange(Py)) % Py
    for kind in ("S", "N"):
        K = P.periodic_kernel_plane(kind, (Px, Py), CELL, 1, 2)
        scale = np.max(np.abs(K))
        for c, (sx, sy) in enumerate(par[kind]):
            k = K[..., c]
            assert np.max(np.abs(k[:, fx] - sx * k)) <= 1e-11 * scale, (kind, c)
            assert np.max(np.abs(k[fy, :] - sy * k)) <= 1e-11 * scale, (kind, c)
