"""ctypes view of the C ABI declared in include/sdc.h (argument marshalling only).

Every step of the path runs in the CUDA library; this module converts torch
tensors to device pointers and status codes to exceptions.  It fails loudly
when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsdc_swe.so")

SDC_FP64, SDC_MIXED_FP32, SDC_MIXED_BF16X3, SDC_MIXED_BF16X6 = 0, 1, 2, 3
SDC_OK, SDC_EINVAL, SDC_ENOMEM, SDC_ECUDA, SDC_EDIVERGED, SDC_ESTATE, SDC_EUNSUPPORTED = range(7)
SDC_OPT_QDELTA_RULE = 1
SDC_OPT_SERIAL_IMPLICIT = 3
SDC_SERIAL_IMPLICIT_EULER, SDC_SERIAL_IMPLICIT_LU = 0, 1
SDC_OPT_METHOD = 2
SDC_QDELTA_CLAMPED, SDC_QDELTA_LITERAL, SDC_QDELTA_MIN_SR_NS, SDC_QDELTA_IMPLICIT_EULER, SDC_QDELTA_MIN_SR_S = range(5)
SDC_METHOD_DSDC, SDC_METHOD_SERIAL_SDC, SDC_METHOD_IMEX2 = 0, 1, 2
SDC_OPT_LEGENDRE = 4
SDC_OPT_CHAINS = 5
SDC_OPT_PDL = 6
SDC_LEGENDRE_TABLE, SDC_LEGENDRE_RECURRENCE = 0, 1


class SdcPhys(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_double), ("omega", ctypes.c_double),
                ("gravity", ctypes.c_double), ("mean_depth", ctypes.c_double)]


class SdcError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_P, _I, _D, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
SIGNATURES = {
    "sdc_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, _D, ctypes.POINTER(SdcPhys), _I, _P]),
    "sdc_destroy": (_I, [_P]),
    "sdc_set_option": (_I, [_P, _I, _I]),
    "sdc_ncoef": (_I, [_P]),
    "sdc_step": (_I, [_P, _P, _P, ctypes.POINTER(_D)]),
    "sdc_run": (_I, [_P, _P, _I]),
    "sdc_tendency": (_I, [_P, _P, _P, _I]),
    "sdc_tendency_adjoint": (_I, [_P, _P, _P, _P, _I]),
    "sdc_step_adjoint": (_I, [_P, _P, _P, _P]),
    "sdc_run_adjoint": (_I, [_P, _P, _I, _I, _P, _P, ctypes.POINTER(_LL)]),
    "sdc_adjoint_run": (_I, [_P, _P, _I, _I, _P, ctypes.POINTER(_D), _P]),
    "sdc_spec_to_grid": (_I, [_P, _P, _P]),
    "sdc_grid_to_spec": (_I, [_P, _P, _P]),
    "sdc_grid_coords": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "sdc_collocation": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "sdc_counters": (_I, [_P, ctypes.POINTER(_LL), ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "sdc_save": (_I, [_P, _P, _LL, ctypes.c_char_p]),
    "sdc_qdelta": (_I, [_I, _I, _I, ctypes.POINTER(_D)]),
    "sdc_load": (_I, [_P, _P, ctypes.POINTER(_LL), ctypes.c_char_p]),
    "sdc_launches_per_step": (_I, [_P, ctypes.POINTER(_I)]),
    "sdc_sync": (_I, [_P]),
    "sdc_profile_step": (_I, [_P, _P, ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "sdc_spec_to_grid_static": (_I, [_I, _I, _I, _P, _P, _P]),
    "sdc_fp64_fma_rate": (_I, [_I, _I, _P, _P, ctypes.POINTER(_D)]),
    "sdc_strerror": (ctypes.c_char_p, [_I]),
    "sdc_last_error": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load libsdc_swe.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != SDC_OK:
        lib = load()
        raise SdcError(status, where, lib.sdc_last_error().decode(errors="replace"))
