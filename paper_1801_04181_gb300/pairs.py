"""Set-up of a MovingMagnets context from a pair description (marshalling only).

A pair description is any object with the fields of workloads.FilmPair:
n_base, n_slider (nx, ny, nz), cell (m), offsets (two lattice offsets in
cells), mat_base / mat_slider (Ms, Aex, Ku, ku_axis, alpha), mech (mass, k,
v_drive, gamma_v, dir, x0_spring), H_ext (A/m) and u0 (slider displacement in
cells).  Nothing here computes: every value goes to the C ABI as given.
"""

import numpy as np
import torch

from . import MovingMagnets


def pair_context(desc, m0, m1, margin=4, adaptive=False, rtol=1e-5, mech=True, stream=None, precision="fp32",
                 integrator="rk45"):
    """A MovingMagnets context for `desc` with unit magnetisations m0, m1
    ((3, nz, ny, nx) arrays or tensors), on `stream` (a torch.cuda.Stream;
    default: the current stream).  mech=False leaves the slider fixed.  A
    description with `periodic` (and `pbc_images`) set gets periodic in-plane
    boundaries.  precision: "fp32" or "mixed" (tensor-core y transforms);
    integrator: "rk45" or "euler" (fixed dt)."""
    st = stream if stream is not None else torch.cuda.current_stream()
    mm = MovingMagnets(margin=margin, adaptive=adaptive, rtol=rtol, stream=st,
                       periodic=getattr(desc, "periodic", 0), pbc_images=getattr(desc, "pbc_images", 2),
                       precision=precision, integrator=integrator)
    for g, (n, mat, m) in enumerate(((desc.n_base, desc.mat_base, m0), (desc.n_slider, desc.mat_slider, m1))):
        mm.set_grid(g, n, desc.cell, desc.offsets[g])
        mm.set_material(g, mat.Ms, mat.Aex, mat.Ku, mat.ku_axis, mat.alpha)
        # the tensor is made on the context's stream, which the library's copy follows
        with torch.cuda.stream(st):
            if isinstance(m, torch.Tensor):
                mt = m.to(device="cuda", dtype=torch.float32).contiguous()
            else:
                mt = torch.as_tensor(np.ascontiguousarray(m), dtype=torch.float32, device="cuda")
        mm.set_magnetization(g, mt)
    mm.set_external_field(desc.H_ext)
    if mech:
        me = desc.mech
        mm.set_mechanics(me.mass, me.k, me.v_drive, me.gamma_v, me.dir, me.x0_spring)
    mm.set_displacement(tuple(u * c for u, c in zip(desc.u0, desc.cell)))
    return mm
