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


def test_noalloc_argument_checks_without_gpu(lib):
    """mm_spline_field_noalloc checks its arguments on the host before any CUDA
    call: the pointers below are never dereferenced."""
    from paper_1801_04181_gb300 import _native

    L = _native.load()
    dummy = ctypes.c_void_p(0x1000)  # non-null, never touched
    dims = _native._i3(20, 20, 8)
    lo = _native._ll3(0, 0, 0)

    def call(pos, nx=8, ny=8, nz=2, d=(1e-9, 1e-9, 1e-9), Ms=1e6, dims=dims, lo=lo, FE=dummy):
        return L.mm_spline_field_noalloc(dummy, dims, lo, _native._d3(*pos), dummy, nx, ny, nz, *d, Ms,
                                         None, FE, None)

    assert call((2.0, 2.0, 2.0), FE=None) == _native.MM_EINVAL          # no force/energy output
    assert call((2.0, 2.0, 2.0), nz=0) == _native.MM_EINVAL             # empty target
    assert call((2.0, 2.0, 2.0), nz=5) == _native.MM_EINVAL             # more layers than a chunk
    assert call((2.0, 2.0, 2.0), Ms=0.0) == _native.MM_EINVAL
    assert call((2.0, 2.0, 2.0), d=(1e-9, -1e-9, 1e-9)) == _native.MM_EINVAL
    assert call((float("nan"), 2.0, 2.0)) == _native.MM_EINVAL
    assert call((2.0 ** 31, 2.0, 2.0)) == _native.MM_EINVAL             # beyond the int lattice
    assert call((2.0, 2.0, 2.0), dims=_native._i3(3, 20, 8)) == _native.MM_EINVAL
    assert call((2.0, 2.0, 2.0), lo=_native._ll3(-(1 << 62), 0, 0)) == _native.MM_EINVAL
    assert call((15.0, 2.0, 2.0)) == _native.MM_ERANGE                  # support leaves the box
    # 65536 tiles of 32 x 8 columns is the limit of the fixed scratch
    assert call((1.5, 1.5, 1.5), nx=4097, ny=4096, nz=1) == _native.MM_ETOOBIG
    # a tile count that wraps a 32-bit product must still be refused
    assert call((1.5, 1.5, 1.5), nx=2 ** 31 - 1, ny=2 ** 31 - 1, nz=4) == _native.MM_ETOOBIG


def test_autotune_entry_points_without_gpu(lib):
    """mm_autotune rejects a null context before any CUDA work; a length that
    was never tuned has no tuned plan."""
    from paper_1801_04181_gb300 import _native

    L = _native.load()
    n = ctypes.c_int(-1)
    assert L.mm_autotune(None, 4, 3, ctypes.byref(n)) == _native.MM_EINVAL
    r = (ctypes.c_int * 8)()
    assert L.mm_get_tuned_plan(1234567, r, ctypes.byref(n)) == _native.MM_ESTATE
    assert L.mm_get_tuned_plan(540, None, ctypes.byref(n)) == _native.MM_EINVAL
