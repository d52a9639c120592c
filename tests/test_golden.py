"""Regression guard of the oracle (CPU): tests/golden/oracle_regression.json,
written by tests/golden/make_golden.py from the oracle alone, must still come
out of it.  The paper prints no worked example, so the stored values are the
pinned oracle's own (see make_golden.py); a change to the oracle's arithmetic
that moves them must be deliberate, with the passage that justifies it."""

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_reproduces_its_stored_values():
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    now = mod.case()
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        ref = json.load(f)
    assert set(now) == set(ref)
    for k in ref:
        a, b = np.asarray(now[k], dtype=np.float64), np.asarray(ref[k], dtype=np.float64)
        scale = max(np.max(np.abs(b)), 1e-300)
        assert np.max(np.abs(a - b)) <= 1e-10 * scale, k  # FFT and BLAS builds differ in the last bits
