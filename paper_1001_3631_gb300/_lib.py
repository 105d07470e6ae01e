"""ctypes binding of libteuk.so (include/teuk.h).  Argument marshalling only: every
step of the time loop runs in the library's CUDA kernels.  There is no fallback:
if the library is missing this module raises."""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
# TEUK_LIB_VARIANT=check loads the checked build (device-side index checks, TEUK_EBOUNDS)
LIB_PATH = os.path.join(HERE, "libteuk_check.so" if os.environ.get("TEUK_LIB_VARIANT") == "check"
                        else "libteuk.so")
HEADER = os.path.join(ROOT, "include", "teuk.h")

TEUK_OK, TEUK_EINVAL, TEUK_ENOMEM, TEUK_ECUDA, TEUK_EUNSTABLE, TEUK_ETIMEOUT, TEUK_ESTATE, TEUK_EBOUNDS = range(8)
TEUK_FP64, TEUK_FP32, TEUK_FP32_KAHAN, TEUK_FP64_DF = 0, 1, 2, 3
STATUS_NAMES = {0: "TEUK_OK", 1: "TEUK_EINVAL", 2: "TEUK_ENOMEM", 3: "TEUK_ECUDA",
                4: "TEUK_EUNSTABLE", 5: "TEUK_ETIMEOUT", 6: "TEUK_ESTATE", 7: "TEUK_EBOUNDS"}


class teuk_params(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int), ("m", ctypes.c_int),
                ("M", ctypes.c_double), ("a", ctypes.c_double),
                ("rstar_min", ctypes.c_double), ("rstar_max", ctypes.c_double),
                ("n_rstar", ctypes.c_int), ("n_theta", ctypes.c_int),
                ("courant", ctypes.c_double), ("dt_rule", ctypes.c_int), ("dt", ctypes.c_double),
                ("rstar_ext", ctypes.c_double), ("prec", ctypes.c_int),
                ("wave_capacity", ctypes.c_int64),
                ("slab_col0", ctypes.c_int), ("slab_ncols", ctypes.c_int)]


class teuk_orbit(ctypes.Structure):
    _fields_ = [("r0", ctypes.c_double),
                ("sigma_rstar_cells", ctypes.c_double), ("sigma_theta_cells", ctypes.c_double),
                ("sigma_rstar_abs", ctypes.c_double), ("sigma_theta_abs", ctypes.c_double)]


class TeukError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None

_P, _I, _L, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_PROTOS = {
    "teuk_create": (_I, [ctypes.POINTER(teuk_params), _I, _P, ctypes.POINTER(_P)]),
    "teuk_set_source": (_I, [_P, _I, ctypes.POINTER(teuk_orbit), _P, _L]),
    "teuk_set_trajectory": (_I, [_P, _I, ctypes.POINTER(teuk_orbit), _P, _L]),
    "teuk_mode_sum": (_I, [_P, _P, _I, _L, _L, _P]),
    "teuk_radiated_flux": (_I, [_P, _L, _L, _P]),
    "teuk_set_state": (_I, [_P, _I, _P, _L]),
    "teuk_get_state": (_I, [_P, _I, _P]),
    "teuk_step_n": (_I, [_P, _L]),
    "teuk_extract": (_I, [_P, _I, _P, _P, _L, ctypes.POINTER(_L), ctypes.POINTER(_L)]),
    "teuk_adjoint_n": (_I, [_P, _I, _L, _L, _L, _P, _P, _P, _P]),
    "teuk_sync": (_I, [_P]),
    "teuk_checked_build": (_I, []),
    "teuk_save_state": (_I, [_P, _I, ctypes.c_char_p]),
    "teuk_load_state": (_I, [_P, _I, ctypes.c_char_p]),
    "teuk_check_selftest": (_I, [_P]),
    "teuk_get_time": (_I, [_P, _I, ctypes.POINTER(_L), ctypes.POINTER(_D)]),
    "teuk_set_tiling": (_I, [_P, _I, _I]),
    "teuk_set_resident": (_I, [_P, _I]),
    "teuk_set_resident_shape": (_I, [_P, _I, _I]),
    "teuk_set_blocked": (_I, [_P, _I, _I]),
    "teuk_set_allocator": (_I, [_P, _P, _P]),
    "teuk_slab_halo_bytes": (_I, [_P, _I, ctypes.POINTER(_L)]),
    "teuk_slab_export": (_I, [_P, _I, _I, _P]),
    "teuk_slab_import": (_I, [_P, _I, _I, _P]),
    "teuk_get_geometry": (_I, [_P, _I, _P]),
    "teuk_set_instance_tiling": (_I, [_P, _I, _I]),
    "teuk_autotune": (_I, [_P, _I, _P]),
    "teuk_set_fault_injection": (_I, [_P, _L, ctypes.c_longlong]),
    "teuk_set_fill_fault": (_I, [_P, _I, _I]),
    "teuk_kernel_launches": (_L, [_P]),
    "teuk_destroy": (None, [_P]),
    "teuk_last_error": (ctypes.c_char_p, [_P]),
    "teuk_waveform_sum_noalloc": (_I, [_P, _L, _I, _P, _P]),
}
TEUK_NOALLOC_MAX_RECORDS = 65536
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def header_functions():
    """Names of the functions declared in include/teuk.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(teuk_[a-z_0-9]+)\s*\(", txt)))


def load():
    """Load libteuk.so (raises if it was not built: there is no CPU path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s not built; run paper_1001_3631_gb300.build.build()"
                              % os.path.basename(LIB_PATH))
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            if not hasattr(lib, name):
                continue
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def check(status, ctx=None):
    if status != TEUK_OK:
        msg = load().teuk_last_error(ctx)
        raise TeukError(status, msg.decode() if msg else "")
    return status


def ptr(a):
    """Host pointer of a C-contiguous numpy array (or None)."""
    if a is None:
        return None
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data_as(ctypes.c_void_p)


def __getattr__(name):
    # teuk_* names resolve to the C functions themselves
    if name.startswith("teuk_"):
        return getattr(load(), name)
    raise AttributeError(name)
