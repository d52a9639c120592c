"""Plain FP64 CPU oracle for the moving-magnet stray-field path (arXiv:1801.04181).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, tables or constant
generators) and never reads a value produced by the CUDA path.

Each function follows one passage of the paper (cited by section / equation)
and is written for a reader to check by eye: closed forms, direct sums, plain
linear convolutions (scipy ``fftconvolve`` as a library primitive), a banded
solve for the spline and explicit 64-term tensor sums for its evaluation.

Modules
-------
kernels      cell-integrated scalar-potential kernel S and demag tensor N (Sec. III.A)
fields       potential on a box, self-demag field, box convention (Sec. II.A, III.A)
spline       cubic B-spline prefilter (banded solve) and 64-term evaluation (Sec. III.A)
interaction  stray field, Eq. (EQForce) force and interaction energy (Sec. III)
dynamics     exchange/anisotropy/Zeeman, LLG (Sec. II eq. 1), DP45 + slider EOM (Sec. III, IV.B)
mixed        split-bfloat16 arithmetic of the reduced-precision form and its error bound

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants or brute force; none is "parity unpinned".
"""

import math

MU0 = 4e-7 * math.pi
GAMMA_LL = 1.7595e11  # rad / (s T); gamma0 = MU0 * GAMMA_LL in m / (A s)
