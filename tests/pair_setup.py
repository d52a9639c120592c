"""Shared set-up of a film pair on the CUDA path and on the CPU oracle (tests only)."""

import numpy as np

MU0 = 4e-7 * np.pi


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gpu_pair(fp, m0, m1, margin=4, adaptive=False, rtol=1e-5, mech=True, stream=None, precision="fp32",
             integrator="rk45"):
    """MovingMagnets context for a workloads.FilmPair with the given unit m arrays,
    on `stream` (a torch.cuda.Stream; default: the current stream)."""
    from paper_1801_04181_gb300 import pair_context

    return pair_context(fp, m0, m1, margin=margin, adaptive=adaptive, rtol=rtol, mech=mech, stream=stream,
                        precision=precision, integrator=integrator)


def oracle_system(fp):
    from oracle.dynamics import System

    return System([fp.n_base, fp.n_slider], fp.cell, fp.offsets,
                  [fp.mat_base.as_dict(), fp.mat_slider.as_dict()], fp.mech.as_dict(), u0=fp.u0,
                  H_ext=fp.H_ext)


def oracle_kernel_windows(n_s, cell, box_lo, box_dims, pool):
    """The oracle's S window of a box and N window of a source grid, in parallel."""
    from oracle.fields import kernel_windows_pooled

    return kernel_windows_pooled(n_s, cell, box_lo, box_dims, pool)


def force_scale(hess_n, M_t, cell):
    """mu0 V sum_i |M_i| ||Hess_i||: the size of the terms that cancel in Eq. (EQForce)."""
    d = np.asarray(cell, float)
    hess = hess_n / d[:, None] / d[None, :]
    Mt = np.moveaxis(M_t, 0, -1)
    return MU0 * d.prod() * np.sum(np.linalg.norm(Mt, axis=-1) * np.linalg.norm(hess, axis=(-2, -1)))
