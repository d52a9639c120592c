"""The C-ABI library builds, loads and exports every entry point of include/mm.h (no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "mm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1801_04181_gb300.build import build

    path = build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_header_function():
    from paper_1801_04181_gb300 import _native

    bound = {n for n, _, _ in _native.SIGNATURES}
    assert set(header_functions()) == bound


def test_status_strings_and_defaults(lib):
    from paper_1801_04181_gb300 import _native

    L = _native.load()
    assert L.mm_status_string(0) == b"ok"
    assert L.mm_status_string(-4).startswith(b"displacement")
    opt = _native.mm_options()
    L.mm_default_options(ctypes.byref(opt))
    assert opt.margin == 4 and opt.adaptive == 1 and opt.rtol == 1e-5


def test_null_context_is_rejected_without_gpu(lib):
    from paper_1801_04181_gb300 import _native

    L = _native.load()
    assert L.mm_create(None, None) == _native.MM_EINVAL
    assert L.mm_set_displacement(None, None) == _native.MM_EINVAL
    assert L.mm_launch_count(None) == 0


def test_new_entry_points_reject_null_context_without_gpu(lib):
    """The batch, power and diagnostics calls validate their arguments before any CUDA work."""
    from paper_1801_04181_gb300 import _native

    L = _native.load()
    d = (ctypes.c_double * 2)()
    x = ctypes.c_double()
    assert L.mm_get_power(None, ctypes.byref(x), d, ctypes.byref(x)) == _native.MM_EINVAL
    assert L.mm_field_div_curl(None, None, 4, 4, 4, 1e-9, 1e-9, 1e-9, ctypes.byref(x),
                               ctypes.byref(x)) == _native.MM_EINVAL
    assert L.mm_step_batch(None, 1, 1, None, None, None) == _native.MM_EINVAL
    assert L.mm_assign_lanes(None, 0, 1, None) == 0
