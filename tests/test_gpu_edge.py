"""Degenerate and limiting geometries on the GPU against the oracle.

* single-cell magnets (the demag field is the self term, the potential box is
  all margin);
* line magnets (one cell across in y and z) and a one-cell-wide film;
* the planner's size limit: an x extent whose FFT line no longer fits one
  shared-memory pass is refused with MM_ENOTSUP, not run.
"""

import numpy as np
import pytest

import workloads
from oracle import fields as OF
from oracle.interaction import stray_interaction
from tests.pair_setup import force_scale, gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _pair(n0, n1, gap, u, seed, lateral=(0, 0)):
    fp, _, _ = workloads.film_pair_plain(n=n0, gap=gap, seed=seed)
    fp.n_slider = n1
    fp.u0 = u
    fp.lateral = lateral
    return fp, workloads.random_unit(n0, seed), workloads.random_unit(n1, seed + 3)


@pytest.mark.parametrize("n0,n1,gap,u,lateral", [
    ((1, 1, 1), (1, 1, 1), 1, (0.4, 0.3, 0.0), (0, 0)),      # single cells
    ((17, 1, 1), (13, 1, 1), 2, (0.7, 0.0, 0.0), (2, 0)),     # lines along x
    ((9, 1, 3), (11, 1, 2), 1, (1.3, 0.45, 0.0), (-1, 0)),    # one cell across in y
    ((1, 12, 2), (1, 9, 1), 2, (0.2, 0.6, 0.0), (0, 1)),      # one cell across in x
])
def test_degenerate_geometries_match_oracle(n0, n1, gap, u, lateral):
    fp, m0, m1 = _pair(n0, n1, gap, u, 31, lateral)
    mm = gpu_pair(fp, m0, m1, mech=False)
    for src in (0, 1):
        t = 1 - src
        H = mm.compute_stray_field(src).double().cpu().numpy()
        F, E = mm.get_force(t)
        Ms = fp.mat_base.Ms
        M_s, M_t = Ms * (m0 if src == 0 else m1), Ms * (m1 if t == 1 else m0)
        ref = stray_interaction(M_s, M_t, fp.cell, fp.offsets[src], fp.offsets[t], u, t == 1, return_box=True)
        assert rel_l2(H, ref["H"]) < TOL
        scale = force_scale(ref["hess_n"], M_t, fp.cell)
        assert np.max(np.abs(np.array(F) - ref["F"])) < TOL * scale
        assert abs(E - ref["E"]) < TOL * abs(ref["E"]) + 1e-6 * scale * fp.cell[0]
        Hd = mm.compute_demag(src).double().cpu().numpy()
        assert rel_l2(Hd, OF.demag_conv(M_s, fp.cell)) < TOL
    mm.close()


def test_single_cube_cell_demag_is_one_third():
    """A single cubic cell: N = 1/3 on the diagonal, so H = -M/3."""
    fp, m0, m1 = _pair((1, 1, 1), (1, 1, 1), 3, (0.0, 0.0, 0.0), 5)
    mm = gpu_pair(fp, m0, m1, mech=False)
    H = mm.compute_demag(0).double().cpu().numpy()[:, 0, 0, 0]
    mm.close()
    ref = -fp.mat_base.Ms * m0[:, 0, 0, 0] / 3.0
    assert np.max(np.abs(H - ref)) < 1e-6 * fp.mat_base.Ms


def test_oversized_line_is_refused():
    from paper_1801_04181_gb300 import MMError

    fp, m0, m1 = _pair((4000, 2, 1), (4000, 2, 1), 1, (0.0, 0.0, 0.0), 2)
    with pytest.raises(MMError) as e:
        mm = gpu_pair(fp, m0, m1, mech=False)
        mm.compute_stray_field(0)
    assert e.value.status == -7  # MM_ENOTSUP: the FFT line does not fit one shared-memory pass
