"""GB300-native node-parallel diagonal IMEX SDC for rotating shallow water on the sphere.

The hot path (spherical-harmonic tendencies, collocation quadrature, per-mode
implicit solves, residuals) runs in hand-written CUDA kernels for sm_103a
behind the C ABI of include/sdc.h; ``Solver`` is its thin Python face.
"""
from ._lib import (LIB_PATH, SDC_FP64, SDC_METHOD_DSDC, SDC_METHOD_IMEX2, SDC_METHOD_SERIAL_SDC, SDC_MIXED_BF16X3,
                   SDC_MIXED_BF16X6, SDC_MIXED_FP32, SDC_QDELTA_CLAMPED, SDC_QDELTA_IMPLICIT_EULER,
                   SDC_QDELTA_LITERAL, SDC_QDELTA_MIN_SR_NS, SDC_QDELTA_MIN_SR_S, SDC_SERIAL_IMPLICIT_EULER,
                   SDC_SERIAL_IMPLICIT_LU, SDC_LEGENDRE_TABLE, SDC_LEGENDRE_RECURRENCE, SdcError, load)

__all__ = ["Solver", "SDC_FP64", "SDC_MIXED_FP32", "SDC_MIXED_BF16X3", "SDC_MIXED_BF16X6", "SDC_QDELTA_CLAMPED",
           "SDC_QDELTA_LITERAL", "SDC_QDELTA_MIN_SR_NS", "SDC_QDELTA_IMPLICIT_EULER", "SDC_QDELTA_MIN_SR_S",
           "SDC_METHOD_DSDC", "SDC_METHOD_SERIAL_SDC", "SDC_METHOD_IMEX2", "SDC_SERIAL_IMPLICIT_EULER",
           "SDC_SERIAL_IMPLICIT_LU", "SDC_LEGENDRE_TABLE", "SDC_LEGENDRE_RECURRENCE", "SdcError", "LIB_PATH", "load"]


def __getattr__(name):
    if name == "Solver":
        from .solver import Solver
        return Solver
    raise AttributeError(name)
