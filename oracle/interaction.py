"""Stray field of one magnet at the displaced cells of the other, FP64 (test infrastructure only).

Steps, in the paper's order (Sec. II.A, III, III.A):
  1. potential phi of the source on the box around the displaced target
     (fields.potential_conv, or potential_direct on tiny grids);
  2. B-spline prefilter of phi on the box (spline.prefilter_3d);
  3. 64-term evaluation of grad phi and of its Hessian at every displaced
     target centre (spline.evaluate);
  4. H = -grad phi (Sec. II.A), the force of Eq. (EQForce),
        F_t = mu0 V sum_i (M_t(x_i) . grad) H_s(x_i) = -mu0 V sum_i Hess(phi) M_t(x_i),
     and the interaction energy E = -mu0 V sum_i M_t . H_s = mu0 V sum_i M_t . grad phi.
Derivatives in node units are divided by the cell size of their axis.
"""

import numpy as np

from . import MU0
from .fields import (MARGIN, box_for_target, potential_conv, potential_direct, potential_kernel_window,
                     target_positions)
from .spline import evaluate, prefilter_3d


def stray_interaction(M_s, M_t, cell, o_s, o_t, u, target_is_slider, direct=False,
                      return_box=False, kernel_cache=None, margin=MARGIN):
    """Stray field of source s on target t and the force/energy on t.

    M_s, M_t: (3, nz, ny, nx) in A/m; cell (dx, dy, dz) in m; o_s, o_t lattice
    offsets (cells, x y z); u slider displacement (cells, x y z).
    Returns dict(H=(3, nz_t, ny_t, nx_t) A/m, F=(3,) N, E=J, box=..., phi=..., coef=...).
    """
    n_t = (M_t.shape[3], M_t.shape[2], M_t.shape[1])
    box_lo, box_dims = box_for_target(n_t, o_t, o_s, u, target_is_slider, margin=margin)
    if direct:
        phi = potential_direct(M_s, cell, box_lo, box_dims)
    else:
        kernel = None
        if kernel_cache is not None:
            key = ("S", M_s.shape, tuple(cell), box_lo, box_dims)
            if key not in kernel_cache:
                n_s = (M_s.shape[3], M_s.shape[2], M_s.shape[1])
                kernel_cache[key] = potential_kernel_window(n_s, cell, box_lo, box_dims)
            kernel = kernel_cache[key]
        phi = potential_conv(M_s, cell, box_lo, box_dims, kernel=kernel)
    coef = prefilter_3d(phi)
    pos = target_positions(n_t, o_t, o_s, u, target_is_slider) - np.asarray(box_lo, float)
    _, grad_n, hess_n = evaluate(coef, pos)
    d = np.asarray(cell, dtype=np.float64)
    grad = grad_n / d                         # (nz, ny, nx, 3), A/m
    hess = hess_n / d[:, None] / d[None, :]   # (nz, ny, nx, 3, 3), A/m^2
    H = -np.moveaxis(grad, -1, 0)
    Mt = np.moveaxis(M_t, 0, -1)              # (nz, ny, nx, 3)
    V = d.prod()
    E = MU0 * V * np.sum(Mt * grad)
    F = -MU0 * V * np.einsum("zyxab,zyxa->b", hess, Mt)
    out = dict(H=H, F=F, E=E, box_lo=box_lo, box_dims=box_dims)
    if return_box:
        out.update(phi=phi, coef=coef, grad_n=grad_n, hess_n=hess_n)
    return out
