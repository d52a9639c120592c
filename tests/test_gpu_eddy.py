"""Eddy currents on the GPU against the oracle (oracle/eddy.py): the current
density J and the field H_eddy of a conducting magnet for a given dB/dt.

E_sol and H_eddy come from the FP32 potential path (the usual 1e-5 bar); the
electric potential is solved in FP64 to a residual of 1e-9 of its source, so
J and H_eddy carry the FP32 bar too.
"""

import numpy as np
import pytest
import torch

import workloads
from oracle import eddy as OE
from tests.pair_setup import gpu_pair, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ctx(n, cell=(2e-9, 2e-9, 2e-9), gap=3, seed=0):
    fp, _, _ = workloads.film_pair_plain(n=n, gap=gap, seed=seed)
    fp.cell = cell
    m0, m1 = workloads.random_unit(n, seed), workloads.random_unit(n, seed + 1)
    return fp, gpu_pair(fp, m0, m1, mech=False)


@pytest.mark.parametrize("n,kind", [((12, 10, 7), "random"), ((12, 10, 7), "uniform"), ((20, 16, 2), "random"),
                                    ((9, 9, 9), "uniform")])
def test_eddy_field_matches_oracle(n, kind):
    fp, mm = _ctx(n)
    rng = np.random.default_rng(7)
    nx, ny, nz = n
    if kind == "random":
        B = rng.standard_normal((3, nz, ny, nx)) * 1e9
    else:
        B = np.zeros((3, nz, ny, nx))
        B[0], B[2] = 4e8, 1e9
    sigma = 1e6
    Bt = torch.as_tensor(B, dtype=torch.float32, device="cuda")
    for mag in (0, 1):
        H, J, sweeps = mm.eddy_field(mag, Bt, sigma)
        ref = OE.eddy_field(B.astype(np.float32).astype(np.float64), fp.cell, sigma, return_all=True)
        assert rel_l2(J.double().cpu().numpy(), ref["J"]) < TOL, sweeps
        assert rel_l2(H.double().cpu().numpy(), ref["H"]) < TOL
        assert sweeps > 0
    mm.close()


def test_eddy_field_of_no_change_is_zero():
    fp, mm = _ctx((8, 7, 3))
    B = torch.zeros((3, 3, 7, 8), dtype=torch.float32, device="cuda")
    H, J, sweeps = mm.eddy_field(0, B, 1e6)
    assert sweeps == 0 and float(H.abs().max()) == 0.0 and float(J.abs().max()) == 0.0
    mm.close()
