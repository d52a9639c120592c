"""Eddy currents of a conducting magnet, FP64 (test infrastructure only).

Sec. III.B (the method of Torres et al.): with the rate of change dB/dt of the
flux density in the magnet's cells,

  1. the solenoidal electric field by the cell-integrated kernel S of the
     scalar potential (Sec. III.A),
         E_sol(r_i) = -sum_j dB/dt(r_j) x S(r_i - r_j)
     -- the sign of the section's first formula, -(1/4 pi) dB/dt x the
     integral of (r - r')/|r - r'|^3, which is 4 pi S (Faraday's law; the
     second printed form drops the minus);
  2. the irrotational field E_irrot = -grad phi_E, phi_E solving Laplace's
     equation in the magnet with d phi_E / dn = E_sol . n on its surface, so
     that the current stays tangential to the surface;
  3. J = sigma (E_sol + E_irrot), sigma uniform;
  4. the field of the currents by the same kernel,
         H_eddy(r_i) = sum_j J(r_j) x S(r_i - r_j)
     (Biot-Savart: (1/4 pi) integral of J x (r - r')/|r - r'|^3).

current_field_on_other evaluates the field of one magnet's currents inside
the other magnet.  Sec. II says the eddy field, not being the gradient of a
potential, is interpolated as field vectors inside the moving magnet (as a
non-uniform external field is); the reading: step 4's sum at the nodes of
the potential box around the other magnet (Sec. III.A's box), each component
prefiltered and evaluated by the cubic B-spline at the displaced cell
centres, as the stray field's potential is.

EddyCoupledSystem / run_fixed_eddy put H_eddy into the effective field of
the time step (the coupling, a reading stated there).

Discretisation of step 2 (the paper's is not given; this reading is the
plain cell-centred one): for every cell and axis a of spacing d_a, the face
flux towards a neighbour is (phi_nb - phi)/d_a and, on a surface face,
d phi/dn = E_sol . n taken from the cell; the divergence of the fluxes is
zero in every cell.  The source term is made exactly compatible by removing
its mean, and phi_E has zero mean.  At a surface face the cell-centred
gradient uses the ghost value that the boundary condition gives.
"""

import numpy as np
from scipy.signal import fftconvolve
from scipy.sparse import coo_matrix
from scipy.sparse.linalg import cg

from . import MU0
from .kernels import S_kernel


def self_S_window(n, cell):
    """S over the offsets d = i - j of a magnet's own cells, (2nz-1, 2ny-1, 2nx-1, 3)."""
    nx, ny, nz = n
    dx, dy, dz = cell
    Z, Y, X = np.meshgrid(np.arange(-(nz - 1), nz), np.arange(-(ny - 1), ny), np.arange(-(nx - 1), nx),
                          indexing="ij")
    return S_kernel(X * dx, Y * dy, Z * dz, dx, dy, dz)


def cross_S(V, S):
    """sum_j V(r_j) x S(r_i - r_j) over the own cells: (3, nz, ny, nx)."""
    conv = [[fftconvolve(S[..., c], V[b], mode="valid") for c in range(3)] for b in range(3)]
    out = np.empty_like(V)
    out[0] = conv[1][2] - conv[2][1]
    out[1] = conv[2][0] - conv[0][2]
    out[2] = conv[0][1] - conv[1][0]
    return out


def neumann_system(n, cell, Esol):
    """The cell-centred Neumann problem of step 2: (A, b) with A phi = b, the
    source b compatible (zero mean)."""
    nx, ny, nz = n
    d = (cell[0], cell[1], cell[2])
    N = nx * ny * nz
    idx = np.arange(N).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    b = np.zeros(N)
    diag = np.zeros(N)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        w = 1.0 / (d[a] * d[a])
        n_a = (nx, ny, nz)[a]
        E = Esol[a]
        for side in (+1, -1):
            # cells whose neighbour on this side exists
            sl_in = [slice(None)] * 3
            sl_nb = [slice(None)] * 3
            sl_bd = [slice(None)] * 3
            if side > 0:
                sl_in[ax] = slice(0, n_a - 1)
                sl_nb[ax] = slice(1, n_a)
                sl_bd[ax] = slice(n_a - 1, n_a)
            else:
                sl_in[ax] = slice(1, n_a)
                sl_nb[ax] = slice(0, n_a - 1)
                sl_bd[ax] = slice(0, 1)
            i_in = idx[tuple(sl_in)].ravel()
            i_nb = idx[tuple(sl_nb)].ravel()
            rows.append(i_in)
            cols.append(i_nb)
            vals.append(np.full(i_in.size, w))
            np.add.at(diag, i_in, -w)
            # surface faces on this side: flux d phi / d x_a = E_sol,a of the cell
            i_bd = idx[tuple(sl_bd)].ravel()
            Eb = E[tuple(sl_bd)].ravel()
            # divergence term (flux_plus - flux_minus) / d_a with the known flux moved to b
            b[i_bd] -= side * Eb / d[a]
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    A = coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
    return A, b - b.mean()


def solve_phi(n, cell, Esol, tol=1e-13):
    """phi_E with zero mean (conjugate gradients on the negative semi-definite system)."""
    A, b = neumann_system(n, cell, Esol)
    phi, info = cg(-A, -b, rtol=tol, atol=0.0, maxiter=20000)
    if info != 0:
        raise RuntimeError("phi_E did not converge")
    phi -= phi.mean()
    nx, ny, nz = n
    return phi.reshape(nz, ny, nx)


def grad_with_ghosts(phi, Esol, cell):
    """Cell-centred gradient of phi; a missing neighbour is the ghost value of the
    boundary condition (phi + d E_sol,a on the + side, phi - d E_sol,a on the - side)."""
    g = np.empty((3,) + phi.shape)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        d = cell[a]
        n_a = phi.shape[ax]
        plus = np.roll(phi, -1, axis=ax)
        minus = np.roll(phi, 1, axis=ax)
        last = [slice(None)] * 3
        first = [slice(None)] * 3
        last[ax] = slice(n_a - 1, n_a)
        first[ax] = slice(0, 1)
        plus[tuple(last)] = phi[tuple(last)] + d * Esol[a][tuple(last)]
        minus[tuple(first)] = phi[tuple(first)] - d * Esol[a][tuple(first)]
        g[a] = (plus - minus) / (2 * d)
    return g


def eddy_field(dBdt, cell, sigma, S=None, return_all=False):
    """Steps 1-4 for a magnet whose cells carry dB/dt (3, nz, ny, nx) in T/s:
    H_eddy in A/m (and E_sol, phi_E, E_irrot, J with return_all)."""
    _, nz, ny, nx = dBdt.shape
    n = (nx, ny, nz)
    if S is None:
        S = self_S_window(n, cell)
    Esol = -cross_S(dBdt, S)
    phi = solve_phi(n, cell, Esol)
    Eirr = -grad_with_ghosts(phi, Esol, cell)
    J = sigma * (Esol + Eirr)
    H = cross_S(J, S)
    if return_all:
        return dict(H=H, Esol=Esol, phi=phi, Eirr=Eirr, J=J)
    return H


def current_field_on_other(J, cell, o_s, o_t, n_t, u, target_is_slider, kernel=None):
    """The field (A/m) of currents J (A/m^2, (3, nz, ny, nx)) of one magnet
    inside the other, at its displaced cell centres (3, nz_t, ny_t, nx_t).

    On the nodes n of the box around the target, (J x S)_a(n) = sum_j
    S(n - r_j) . R_a J(r_j) with R_x J = (0, -J_z, J_y), R_y J = (J_z, 0,
    -J_x), R_z J = (-J_y, J_x, 0), i.e. the potential sum of Sec. III.A with
    the rearranged vector as the source; each component is then interpolated
    by the cubic B-spline (mirror ends) at the displaced centres.  `kernel`:
    the S window of the box (fields.potential_kernel_window), else computed."""
    from .fields import box_for_target, potential_conv, target_positions
    from .spline import evaluate, prefilter_3d
    z = np.zeros_like(J[0])
    R = (np.stack([z, -J[2], J[1]]), np.stack([J[2], z, -J[0]]), np.stack([-J[1], J[0], z]))
    box_lo, box_dims = box_for_target(n_t, o_t, o_s, u, target_is_slider)
    pos = target_positions(n_t, o_t, o_s, u, target_is_slider) - np.asarray(box_lo, float)
    out = []
    for a in range(3):
        node = potential_conv(R[a], cell, box_lo, box_dims, kernel=kernel)
        out.append(evaluate(prefilter_3d(node), pos)[0])
    return np.stack(out)


class EddyCoupledSystem:
    """dynamics.System with the eddy fields of conducting magnets in H_eff.

    Reading of the coupling (the section gives the field computation, not
    its place in the time step): explicit and lagged by one accepted step.
    After step n the flux density of magnet g,
        B_n = mu0 (H_demag + H_stray + H_ext + Ms y5),
    is taken from the step's last field evaluation (the first-same-as-last
    stage at the 5th-order solution y5), dB/dt = (B_n - B_{n-1}) / dt_n, and
    H_eddy(dB/dt) of steps 1-4 is added to H_eff in every stage of step n + 1.
    The currents of a conducting magnet also act on the other magnet: their
    field there (current_field_on_other, at the displacement of the same
    last evaluation) is added to the other magnet's H_eff in the same way,
    whether or not that magnet conducts.
    No eddy field before the first step, nor before a second B exists.
    sigma: conductivity of each magnet (S/m, 0 = insulating)."""

    def __init__(self, system, sigma):
        self.sys = system
        self.sigma = tuple(float(s) for s in sigma)
        self.Heddy = [None, None]
        self.B_prev = [None, None]
        self.last_B = None
        self.last_u = None
        self.S = {}

    def fields(self, m0, m1, x):
        from .dynamics import anisotropy_field, exchange_field
        from .interaction import stray_interaction
        s = self.sys
        u = s.displacement(x)
        self.last_u = u
        M0, M1 = s.mat[0]["Ms"] * m0, s.mat[1]["Ms"] * m1
        on1 = stray_interaction(M0, M1, s.cell, s.offsets[0], s.offsets[1], u, True, kernel_cache=s.cache)
        on0 = stray_interaction(M1, M0, s.cell, s.offsets[1], s.offsets[0], u, False, kernel_cache=s.cache)
        H, B = [], []
        for g, (m, stray) in enumerate(((m0, on0["H"]), (m1, on1["H"]))):
            p = s.mat[g]
            hd = s.demag(g, m) + stray + s.H_ext[:, None, None, None]
            B.append(MU0 * (hd + p["Ms"] * m))
            h = hd + exchange_field(m, p["Ms"], p["Aex"], s.cell)
            h = h + anisotropy_field(m, p["Ms"], p["Ku"], p["ku_axis"])
            if self.Heddy[g] is not None:
                h = h + self.Heddy[g]
            H.append(h)
        self.last_B = B
        return H, on1, on0

    def rhs(self, t, y):
        from .dynamics import llg_rhs
        m0, m1, x, v = y
        H, on1, _ = self.fields(m0, m1, x)
        me = self.sys.mech
        F = float(np.dot(on1["F"], self.sys.e))
        acc = (me["k"] * (me["v_drive"] * t + me.get("x0_spring", 0.0) - x)
               - me["gamma_v"] * me["mass"] * v + F) / me["mass"]
        return [llg_rhs(m0, H[0], self.sys.mat[0]["alpha"]), llg_rhs(m1, H[1], self.sys.mat[1]["alpha"]), v, acc]

    def accept(self, dt):
        """After an accepted step (last evaluation at y5): update the eddy fields,
        each magnet's own and those of the other magnet's currents."""
        s = self.sys
        own, J = [None, None], [None, None]
        for g in (0, 1):
            B = self.last_B[g]
            if self.sigma[g] > 0.0 and self.B_prev[g] is not None:
                _, nz, ny, nx = B.shape
                if g not in self.S:
                    self.S[g] = self_S_window((nx, ny, nz), s.cell)
                r = eddy_field((B - self.B_prev[g]) / dt, s.cell, self.sigma[g], S=self.S[g], return_all=True)
                own[g], J[g] = r["H"], r["J"]
            self.B_prev[g] = B
        if J[0] is None and J[1] is None:
            return
        for t in (0, 1):
            H = own[t]
            g = 1 - t
            if J[g] is not None:
                from .fields import box_for_target, potential_kernel_window
                n_t = tuple(s.shapes[t])
                lo, dims = box_for_target(n_t, s.offsets[t], s.offsets[g], self.last_u, t == 1)
                key = ("X", g, tuple(lo), tuple(dims))
                if key not in self.S:
                    self.S[key] = potential_kernel_window(tuple(s.shapes[g]), s.cell, lo, dims)
                cross = current_field_on_other(J[g], s.cell, s.offsets[g], s.offsets[t], n_t, self.last_u, t == 1,
                                               kernel=self.S[key])
                H = cross if H is None else H + cross
            self.Heddy[t] = H


def run_fixed_eddy(coupled, y0, dt, nsteps, t0=0.0):
    """dynamics.run_fixed for an EddyCoupledSystem: fixed-dt Dormand-Prince
    steps with first-same-as-last reuse, the eddy fields updated after each."""
    from .dynamics import dp45_step, normalise
    t, y, k1 = t0, list(y0), None
    for _ in range(nsteps):
        y5, _, k7 = dp45_step(coupled, t, y, dt, k1)
        coupled.accept(dt)
        y = [normalise(y5[0]), normalise(y5[1]), y5[2], y5[3]]
        t += dt
        k1 = k7
    return t, y
