"""ctypes binding of libmm (include/mm.h): same names, argument marshalling only.

Loading fails loudly when lib/libmm.so is missing: there is no CPU fallback.
"""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmm.so")

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA, MM_ERANGE, MM_ETIMEOUT, MM_ESTATE, MM_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
MM_ETOOBIG = -8


MM_PERIODIC_X, MM_PERIODIC_Y = 1, 2
MM_FP32, MM_MIXED = 0, 1
MM_RK45, MM_EULER = 0, 1


class mm_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("margin", C.c_int), ("adaptive", C.c_int),
                ("rtol", C.c_double), ("dt_min", C.c_double), ("dt_max", C.c_double),
                ("stream", C.c_void_p), ("periodic", C.c_int), ("pbc_images", C.c_int),
                ("integrator", C.c_int)]


_d3 = C.c_double * 3
_ll3 = C.c_longlong * 3
_i3 = C.c_int * 3

# (name, restype, argtypes)
SIGNATURES = [
    ("mm_default_options", None, [C.POINTER(mm_options)]),
    ("mm_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(mm_options)]),
    ("mm_destroy", None, [C.c_void_p]),
    ("mm_last_error", C.c_char_p, [C.c_void_p]),
    ("mm_status_string", C.c_char_p, [C.c_int]),
    ("mm_set_grid", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                              C.c_double, C.POINTER(C.c_longlong)]),
    ("mm_set_material", C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double,
                                  C.POINTER(C.c_double), C.c_double]),
    ("mm_set_external_field", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("mm_set_mechanics", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.POINTER(C.c_double), C.c_double]),
    ("mm_set_magnetization", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_get_magnetization", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_upload_magnetization", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_download_magnetization", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_set_displacement", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("mm_set_slider_state", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double]),
    ("mm_get_slider_state", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]),
    ("mm_compute_potential", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t,
                                       C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    ("mm_compute_stray_field", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_compute_demag", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_compute_fields", C.c_int, [C.c_void_p]),
    ("mm_get_force", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("mm_backward_energy", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p, C.c_void_p]),
    ("mm_compute_torque", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("mm_step", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("mm_step_batch", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    ("mm_fft_plan", C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("mm_autotune", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    ("mm_get_tuned_plan", C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("mm_assign_lanes", C.c_int, [C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(C.c_int)]),
    ("mm_get_power", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("mm_compute_stray_field_fd4", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_compute_stray_field_componentwise", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_eddy_field", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                C.POINTER(C.c_int)]),
    ("mm_set_conductivity", C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    ("mm_get_eddy_field", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mm_eddy_field_on_other", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("mm_field_div_curl", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("mm_get_step_stats", C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    ("mm_get_attempt_log", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("mm_clear_attempt_log", C.c_int, [C.c_void_p]),
    ("mm_get_state", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    ("mm_set_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("mm_eval_kernel_fp64", C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                      C.c_void_p]),
    ("mm_get_plan_info", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    ("mm_set_timing", C.c_int, [C.c_void_p, C.c_int]),
    ("mm_get_timing", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    ("mm_reset_timing", C.c_int, [C.c_void_p]),
    ("mm_launch_count", C.c_longlong, [C.c_void_p]),
    ("mm_spline_field_noalloc", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                          C.POINTER(C.c_double), C.c_void_p, C.c_int, C.c_int, C.c_int,
                                          C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
]

_lib = None


def load(path=LIB_PATH):
    """Load libmm and declare every entry point; raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmm.so is not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class MMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (status_name(status), status, msg))
        self.status = status


def status_name(s):
    return {0: "MM_OK", -1: "MM_EINVAL", -2: "MM_ENOMEM", -3: "MM_ECUDA", -4: "MM_ERANGE",
            -5: "MM_ETIMEOUT", -6: "MM_ESTATE", -7: "MM_ENOTSUP", -8: "MM_ETOOBIG"}.get(s, "MM_?")
