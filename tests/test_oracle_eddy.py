"""Pins of the eddy-current oracle (oracle/eddy.py), CPU only.

* step 1, E_sol = -sum dB/dt x S: far from one cell it is the point form
  -V dB/dt x r / (4 pi r^3) with (d/r)^2 convergence; for a uniform dB/dt in
  a cube it is -dB/dt x g, g = sum S the field of a uniform cube (div g = 1,
  and by cubic symmetry (v . grad) g = v/3 at the centre), so its curl at the
  centre is -dB/dt + dB/dt/3 = -(2/3) dB/dt (the dB/dt of the cells alone is
  cut off at the surface) and its divergence vanishes;
* step 2 reproduces a manufactured solution: phi* = x^2 - y^2 is harmonic
  also for the discrete Laplacian, and with the surface fluxes it implies
  the solver returns phi* - mean(phi*) exactly;
* the current leaves no charge: the source the surface fluxes of E_sol make
  has (nearly) zero sum, by the divergence theorem;
* step 4, H = sum J x S: far from one cell it is the Biot-Savart point form
  V J x r / (4 pi r^3);
* Lenz's law: the field of the eddy currents a uniform dB/dt drives opposes
  dB/dt at the centre of the magnet (this fixes the sign of step 1), and
  it is linear in dB/dt;
* the field of one magnet's currents inside the other (interpolated on the
  potential box): at a whole-cell move the spline reproduces its nodes, so
  it equals the direct sum of J x S at the target centres; ten and twenty
  cells from one current cell it is the Biot-Savart point form within 1e-4,
  also at sub-cell moves;
* with only the base conducting, the coupled system puts the field of the
  base's currents into the slider.
"""

import numpy as np

from oracle import eddy as E

CELL = (2e-9, 2e-9, 2e-9)


def _point_form(vec, r, V):
    rn = np.linalg.norm(r)
    return V * np.cross(vec, r) / (4 * np.pi * rn ** 3)


def test_far_fields_are_the_point_forms():
    """One source cell: E_sol -> -V dB/dt x r/(4 pi r^3), H -> V J x r/(4 pi r^3)."""
    v = np.array([0.3, -0.7, 0.5])
    errs = []
    for dist in (8, 16):
        n = (dist + 1, 1, 1)
        V = np.zeros((3, 1, 1, dist + 1))
        V[:, 0, 0, 0] = v
        S = E.self_S_window(n, CELL)
        out = E.cross_S(V, S)[:, 0, 0, dist]   # at the cell dist away along x
        r = np.array([dist * CELL[0], 0.0, 0.0])
        ref = -_point_form(-v, r, np.prod(CELL))  # cross_S gives + V x S; E_sol takes the minus
        errs.append(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 3, errs


def test_solenoidal_field_curl_and_divergence_in_a_cube():
    n = (14, 14, 14)
    B = np.zeros((3, 14, 14, 14))
    Bdot = np.array([2e9, -1e9, 3e9])
    for c in range(3):
        B[c] = Bdot[c]
    Es = -E.cross_S(B, E.self_S_window(n, CELL))
    d = CELL[0]
    c = slice(5, 9)

    def dd(F, ax):
        return (np.roll(F, -1, axis=ax) - np.roll(F, 1, axis=ax)) / (2 * d)
    curl = np.stack([dd(Es[2], 1) - dd(Es[1], 0), dd(Es[0], 0) - dd(Es[2], 2), dd(Es[1], 2) - dd(Es[0], 1)])
    div = dd(Es[0], 2) + dd(Es[1], 1) + dd(Es[2], 0)
    for a in range(3):
        got = curl[a][c, c, c]
        assert np.max(np.abs(got + (2.0 / 3.0) * Bdot[a])) < 2e-2 * np.max(np.abs(Bdot))
    assert np.max(np.abs(div[c, c, c])) < 2e-2 * np.max(np.abs(Bdot)) * 1.0


def test_neumann_solver_reproduces_a_manufactured_solution():
    cell = (2e-9, 3e-9, 1.5e-9)
    nx, ny, nz = 7, 6, 4
    z, y, x = np.meshgrid(np.arange(nz) * cell[2], np.arange(ny) * cell[1], np.arange(nx) * cell[0], indexing="ij")
    phi_star = x ** 2 - (cell[0] / cell[1]) ** 0 * y ** 2   # discrete Laplacian: 2 - 2 = 0
    Es = np.zeros((3, nz, ny, nx))
    # surface fluxes of phi*: forward differences on + faces, backward on - faces
    for a, ax, coord in ((0, 2, x), (1, 1, y), (2, 0, z)):
        d = cell[a]
        f = lambda q: q ** 2 if a == 0 else (-(q ** 2) if a == 1 else 0.0 * q)
        last = [slice(None)] * 3
        first = [slice(None)] * 3
        n_a = (nx, ny, nz)[a]
        last[ax] = slice(n_a - 1, n_a)
        first[ax] = slice(0, 1)
        q_last, q_first = coord[tuple(last)], coord[tuple(first)]
        Es[a][tuple(last)] = (f(q_last + d) - f(q_last)) / d
        Es[a][tuple(first)] = (f(q_first) - f(q_first - d)) / d
    phi = E.solve_phi((nx, ny, nz), cell, Es)
    ref = phi_star - phi_star.mean()
    assert np.max(np.abs(phi - ref)) <= 1e-9 * np.max(np.abs(ref))
    # and the ghost gradient is the exact gradient of the quadratic at the cell centres
    g = E.grad_with_ghosts(phi, Es, cell)
    assert np.max(np.abs(g[0] - 2 * x)) <= 1e-9 * np.max(np.abs(2 * x))
    assert np.max(np.abs(g[1] + 2 * y)) <= 1e-9 * np.max(np.abs(2 * y))


def test_surface_source_is_compatible():
    rng = np.random.default_rng(3)
    n = (10, 9, 8)
    B = rng.standard_normal((3, 8, 9, 10)) * 1e9
    Es = -E.cross_S(B, E.self_S_window(n, CELL))
    A, b = E.neumann_system(n, CELL, Es)
    # before the mean is removed: the net outward flux of E_sol is small against its terms
    raw = b + 0.0
    nx, ny, nz = n
    flux = 0.0
    scale = 0.0
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        area = np.prod(CELL) / CELL[a]
        n_a = n[a]
        last = [slice(None)] * 3
        first = [slice(None)] * 3
        last[ax] = slice(n_a - 1, n_a)
        first[ax] = slice(0, 1)
        flux += area * (Es[a][tuple(last)].sum() - Es[a][tuple(first)].sum())
        scale += area * (np.abs(Es[a][tuple(last)]).sum() + np.abs(Es[a][tuple(first)]).sum())
    assert abs(flux) < 5e-2 * scale
    assert abs(raw.sum()) < 1e-12 * np.abs(raw).sum()  # the mean is removed


def test_lenz_law_and_linearity():
    n = (10, 10, 10)
    B = np.zeros((3, 10, 10, 10))
    B[2] = 1e9
    S = E.self_S_window(n, CELL)
    H = E.eddy_field(B, CELL, 1e6, S=S)
    c = slice(4, 6)
    assert np.all(H[2][c, c, c] < 0)
    # (the central 2 x 2 x 2 cells sit half a cell off the centre: a small radial part)
    assert np.max(np.abs(H[:2][:, c, c, c])) < 2e-2 * np.max(np.abs(H[2][c, c, c]))
    H2 = E.eddy_field(-2.5 * B, CELL, 1e6, S=S)
    assert np.max(np.abs(H2 + 2.5 * H)) <= 1e-9 * np.max(np.abs(H))


def test_coupled_system_without_conductivity_is_the_plain_system():
    """sigma = 0: the eddy-coupled time step is the plain one (only the order
    of the field sums differs)."""
    import workloads
    from oracle import dynamics as D
    from tests.pair_setup import oracle_system

    fp, m0, m1 = workloads.film_pair_stick_slip(n=(12, 8, 2), gap=3, seed=2)
    fp.mech.x0_spring = 2e-9
    y0 = [m0, m1, 0.0, 0.0]
    t_a, ya = D.run_fixed(oracle_system(fp), y0, 5e-14, 3)
    t_b, yb = E.run_fixed_eddy(E.EddyCoupledSystem(oracle_system(fp), (0.0, 0.0)), y0, 5e-14, 3)
    assert t_a == t_b
    for g in (0, 1):
        assert np.max(np.abs(ya[g] - yb[g])) < 1e-12
    assert abs(ya[2] - yb[2]) <= 1e-12 * abs(ya[2])


def test_coupled_eddy_field_is_lagged_by_one_step():
    """The first step runs without eddy field and only records B; after the
    second, H_eddy is the eddy field of (B_2 - B_1)/dt, linear in sigma; an
    insulating magnet gets only the field of the other magnet's currents."""
    import workloads
    from tests.pair_setup import oracle_system

    fp, m0, m1 = workloads.film_pair_stick_slip(n=(12, 8, 2), gap=3, seed=2)
    y0 = [m0, m1, 0.0, 0.0]
    one = E.EddyCoupledSystem(oracle_system(fp), (2e6, 0.0))
    E.run_fixed_eddy(one, y0, 5e-14, 1)
    assert one.Heddy[0] is None and one.B_prev[0] is not None
    cs = E.EddyCoupledSystem(oracle_system(fp), (2e6, 0.0))
    E.run_fixed_eddy(cs, y0, 5e-14, 2)
    assert cs.Heddy[0] is not None and cs.Heddy[1] is not None
    r = E.eddy_field((cs.B_prev[0] - one.B_prev[0]) / 5e-14, fp.cell, 2e6, return_all=True)
    assert np.max(np.abs(cs.Heddy[0] - r["H"])) <= 1e-9 * np.max(np.abs(r["H"]))
    on1 = E.current_field_on_other(r["J"], fp.cell, fp.offsets[0], fp.offsets[1], fp.n_slider, cs.last_u, True)
    assert np.max(np.abs(cs.Heddy[1] - on1)) <= 1e-9 * np.max(np.abs(on1))
    cs2 = E.EddyCoupledSystem(oracle_system(fp), (4e6, 0.0))
    E.run_fixed_eddy(cs2, y0, 5e-14, 2)
    for g in (0, 1):
        assert np.max(np.abs(cs2.Heddy[g] - 2.0 * cs.Heddy[g])) <= 1e-9 * np.max(np.abs(cs.Heddy[g]))


def _direct_cross(J, cell, pos):
    """sum_j J(r_j) x S(p - r_j) at node positions pos (..., 3), over the source cells."""
    from oracle.kernels import S_kernel
    _, nz, ny, nx = J.shape
    out = np.zeros(pos.shape[:-1] + (3,))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                d = (pos - np.array([i, j, k], float)) * np.asarray(cell)
                out += np.cross(J[:, k, j, i], S_kernel(d[..., 0], d[..., 1], d[..., 2], *cell))
    return np.moveaxis(out, -1, 0)


def test_field_on_other_at_whole_cell_moves_is_the_direct_sum():
    from oracle.fields import target_positions
    rng = np.random.default_rng(3)
    J = rng.standard_normal((3, 2, 3, 4)) * 1e10
    n_s, n_t = (4, 3, 2), (5, 4, 2)
    o_s, o_t = (0, 0, 0), (-1, 1, 4)
    for u, slider in (((1.0, 0.0, 0.0), True), ((0.0, -2.0, 0.0), False)):
        H = E.current_field_on_other(J, CELL, o_s, o_t, n_t, u, slider)
        ref = _direct_cross(J, CELL, target_positions(n_t, o_t, o_s, u, slider))
        assert np.linalg.norm(H - ref) <= 1e-10 * np.linalg.norm(ref)


def test_field_on_other_far_from_one_current_cell_is_biot_savart():
    from oracle.fields import target_positions
    Jv = np.array([0.4, -0.9, 0.2]) * 1e11
    V = float(np.prod(CELL))
    errs = []
    for gap in (10, 20):
        J = np.zeros((3, 1, 1, 1))
        J[:, 0, 0, 0] = Jv
        n_t, o_t, u = (2, 2, 1), (0, 0, gap), (0.37, 0.21, 0.0)
        H = E.current_field_on_other(J, CELL, (0, 0, 0), o_t, n_t, u, True)
        pos = target_positions(n_t, o_t, (0, 0, 0), u, True)
        ref = np.stack([_point_form(Jv, pos[k, j, i] * np.asarray(CELL), V)
                        for k in range(1) for j in range(2) for i in range(2)])
        got = np.moveaxis(H, 0, -1).reshape(-1, 3)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    # a cubic cell has no quadrupole: the point form holds to ~(d/r)^4, so
    # both distances sit at the interpolation and quadrature floor
    assert max(errs) < 1e-4


def test_coupled_field_of_the_base_currents_reaches_the_slider():
    import workloads
    from oracle import dynamics as D
    from tests.pair_setup import oracle_system
    fp, _, _ = workloads.film_pair_stick_slip(n=(8, 6, 2), gap=2, seed=5)
    m0, m1 = workloads.random_unit(fp.n_base, 5), workloads.random_unit(fp.n_slider, 6)
    cs = E.EddyCoupledSystem(oracle_system(fp), (1e11, 0.0))
    E.run_fixed_eddy(cs, [m0, m1, 0.0, 0.0], 2e-14, 2)
    assert cs.Heddy[0] is not None and cs.Heddy[1] is not None
    assert np.linalg.norm(cs.Heddy[1]) > 0.0
    # insulating both: no eddy field anywhere
    cs0 = E.EddyCoupledSystem(oracle_system(fp), (0.0, 0.0))
    E.run_fixed_eddy(cs0, [m0, m1, 0.0, 0.0], 2e-14, 2)
    assert cs0.Heddy == [None, None]
