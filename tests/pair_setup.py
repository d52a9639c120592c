"""Shared set-up of a film pair on the CUDA path and on the CPU oracle (tests only)."""

import numpy as np

MU0 = 4e-7 * np.pi


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gpu_pair(fp, m0, m1, margin=4, adaptive=False, rtol=1e-5, mech=True, stream=None):
    """MovingMagnets context for a workloads.FilmPair with the given unit m arrays,
    on `stream` (a torch.cuda.Stream; default: the current stream)."""
    import torch
    from paper_1801_04181_gb300 import MovingMagnets

    st = stream if stream is not None else torch.cuda.current_stream()
    mm = MovingMagnets(margin=margin, adaptive=adaptive, rtol=rtol, stream=st)
    for g, (n, mat, m) in enumerate(((fp.n_base, fp.mat_base, m0), (fp.n_slider, fp.mat_slider, m1))):
        mm.set_grid(g, n, fp.cell, fp.offsets[g])
        mm.set_material(g, mat.Ms, mat.Aex, mat.Ku, mat.ku_axis, mat.alpha)
        # the tensor is made on the context's stream, which the library's copy follows
        with torch.cuda.stream(st):
            mt = torch.as_tensor(np.ascontiguousarray(m), dtype=torch.float32, device="cuda")
        mm.set_magnetization(g, mt)
    mm.set_external_field(fp.H_ext)
    if mech:
        me = fp.mech
        mm.set_mechanics(me.mass, me.k, me.v_drive, me.gamma_v, me.dir, me.x0_spring)
    mm.set_displacement(tuple(u * c for u, c in zip(fp.u0, fp.cell)))
    return mm


def oracle_system(fp):
    from oracle.dynamics import System

    return System([fp.n_base, fp.n_slider], fp.cell, fp.offsets,
                  [fp.mat_base.as_dict(), fp.mat_slider.as_dict()], fp.mech.as_dict(), u0=fp.u0,
                  H_ext=fp.H_ext)


def _S_chunk(args):
    from oracle.kernels import S_kernel
    X, Y, Z, cell = args
    return S_kernel(X, Y, Z, *cell)


def _N_chunk(args):
    from oracle.kernels import N_kernel
    X, Y, Z, cell = args
    return N_kernel(X, Y, Z, *cell)


def _window(fun, lo, length, cell, pool):
    dx, dy, dz = cell
    jobs = []
    for iz in range(length[2]):
        Y, X = np.meshgrid(np.arange(length[1]) + lo[1], np.arange(length[0]) + lo[0], indexing="ij")
        Z = np.full_like(X, iz + lo[2])
        jobs.append((X * dx, Y * dy, Z * dz, cell))
    return np.stack(pool.map(fun, jobs))


def oracle_kernel_windows(n_s, cell, box_lo, box_dims, pool):
    """The oracle's S window of a box and N window of a source grid, one z plane per pool task.

    Same values as oracle.fields.potential_kernel_window / demag_kernel_window,
    computed in parallel; pass a multiprocessing pool made with 'spawn'.
    """
    d_lo = [box_lo[a] - (n_s[a] - 1) for a in range(3)]
    d_len = [box_dims[a] + n_s[a] - 1 for a in range(3)]
    S = _window(_S_chunk, d_lo, d_len, cell, pool)
    N = _window(_N_chunk, [-(n - 1) for n in n_s], [2 * n - 1 for n in n_s], cell, pool)
    return S, N


def force_scale(hess_n, M_t, cell):
    """mu0 V sum_i |M_i| ||Hess_i||: the size of the terms that cancel in Eq. (EQForce)."""
    d = np.asarray(cell, float)
    hess = hess_n / d[:, None] / d[None, :]
    Mt = np.moveaxis(M_t, 0, -1)
    return MU0 * d.prod() * np.sum(np.linalg.norm(Mt, axis=-1) * np.linalg.norm(hess, axis=(-2, -1)))
