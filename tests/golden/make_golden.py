"""Writes tests/golden/oracle_regression.json: values of the FP64 oracle on one
small seeded case, as a regression guard for the oracle (test infrastructure).

The paper prints no worked example with numbers, so there is nothing of the
paper's to store; the pins proper are the closed forms, identities and brute
force of tests/test_oracle_*.py.  This file only freezes what the pinned
oracle computes today, so an unnoticed change to it shows up.  It calls only
oracle/ (and the seeded input generators of workloads/).

    python tests/golden/make_golden.py
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads  # noqa: E402
from oracle import dynamics as D  # noqa: E402
from oracle.interaction import stray_interaction  # noqa: E402
from oracle.kernels import N_kernel, S_kernel  # noqa: E402

CELL = (4e-9, 3e-9, 2e-9)


def case():
    """The frozen case: kernel values at a few offsets, a 5x4x2 source above a
    4x3x2 target (gap 1, displaced by (0.37, 0.21, 0)), stray field, force,
    energy, one fixed-dt Dormand-Prince step of the pair."""
    offs = np.array([[0, 0, 0], [1, 0, 0], [2, -1, 3], [-5, 4, 1], [20, -3, 7]], dtype=np.float64)
    X, Y, Z = (offs[:, a] * CELL[a] for a in range(3))
    S = S_kernel(X, Y, Z, *CELL)
    N = N_kernel(X, Y, Z, *CELL)
    n_s, n_t = (5, 4, 2), (4, 3, 2)
    m_s = workloads.random_unit(n_s, 21)
    m_t = workloads.random_unit(n_t, 22)
    o_s, o_t = (0, 0, 0), (1, 0, 3)
    u = (0.37, 0.21, 0.0)
    r = stray_interaction(8e5 * m_s, 1.1e6 * m_t, CELL, o_s, o_t, u, True)
    fp, m0, m1 = workloads.film_pair_stick_slip(n=(6, 5, 2), gap=2, seed=23)
    fp.u0 = (0.3, 0.0, 0.0)
    sysm = D.System([fp.n_base, fp.n_slider], fp.cell, fp.offsets,
                    [fp.mat_base.as_dict(), fp.mat_slider.as_dict()], fp.mech.as_dict(), u0=fp.u0)
    t, y = D.run_fixed(sysm, [m0, m1, 0.0, 0.0], 2e-14, 1)
    return {
        "S": np.asarray(S).tolist(), "N": np.asarray(N).tolist(),
        "H_stray": np.asarray(r["H"]).ravel().tolist(), "F": np.asarray(r["F"]).tolist(), "E": float(r["E"]),
        "step_m0": np.asarray(y[0]).ravel().tolist(), "step_m1": np.asarray(y[1]).ravel().tolist(),
        "step_x": float(y[2]), "step_v": float(y[3]), "step_t": float(t),
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(case(), f, indent=0)
        f.write("\n")
