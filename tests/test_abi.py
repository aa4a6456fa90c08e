"""The C ABI library loads, exports every symbol include/sdc.h declares, and
rejects invalid arguments before touching the GPU (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "sdc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_2403_20135_gb300 as pkg
    from paper_2403_20135_gb300 import build as b
    if not os.path.exists(pkg.LIB_PATH):
        b.build()
    return pkg.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2403_20135_gb300 import _lib
    assert set(names) == set(_lib.SIGNATURES), "binding and header disagree"


def test_strerror(lib):
    assert lib.sdc_strerror(0) == b"ok"
    assert lib.sdc_strerror(1) == b"invalid argument"
    assert lib.sdc_strerror(99) == b"unknown status"


@pytest.mark.parametrize("args,msg", [
    ((0, 48, 96, 3, 3, 600.0), b"truncation"),
    ((31, 47, 96, 3, 3, 600.0), b"nlat"),
    ((31, 46, 96, 3, 3, 600.0), b"nlat"),
    ((31, 48, 90, 3, 3, 600.0), b"nlon"),
    ((31, 48, 80, 3, 3, 600.0), b"nlon"),
    ((31, 48, 96, 0, 3, 600.0), b"nodes"),
    ((31, 48, 96, 9, 3, 600.0), b"nodes"),
    ((31, 48, 96, 3, 0, 600.0), b"sweeps"),
    ((31, 48, 96, 3, 3, 0.0), b"dt"),
    ((31, 48, 96, 3, 3, float("nan")), b"dt"),
])
def test_create_rejects_invalid_sizes(lib, args, msg):
    from paper_2403_20135_gb300 import _lib
    h = ctypes.c_void_p(123)
    ph = _lib.SdcPhys(6.371e6, 7.292e-5, 9.80616, 1e4)
    st = lib.sdc_create(ctypes.byref(h), *args, ctypes.byref(ph), 0, None)
    assert st == _lib.SDC_EINVAL
    assert h.value is None
    assert msg in lib.sdc_last_error()


def test_null_arguments(lib):
    from paper_2403_20135_gb300 import _lib
    assert lib.sdc_create(None, 31, 48, 96, 3, 3, 600.0, None, 0, None) == _lib.SDC_EINVAL
    h = ctypes.c_void_p()
    assert lib.sdc_create(ctypes.byref(h), 31, 48, 96, 3, 3, 600.0, None, 0, None) == _lib.SDC_EINVAL
    assert lib.sdc_destroy(None) == _lib.SDC_OK
    assert lib.sdc_ncoef(None) == -1
    assert lib.sdc_step(None, None, None, None) == _lib.SDC_EINVAL
    assert lib.sdc_run(None, None, 1) == _lib.SDC_EINVAL


@pytest.mark.parametrize("M", range(1, 9))
def test_host_qdelta_coefficients_match_oracle(lib, M):
    """sdc_qdelta (host only, no GPU): the diagonal of every rule at sweeps 1..6
    against the oracle, which finds MIN-SR-S by a different formulation and
    solver (characteristic-polynomial root with scipy against the library's
    damped Newton on the principal-minor expansion)."""
    from oracle import sdc as osdc
    from paper_2403_20135_gb300 import _lib
    names = {_lib.SDC_QDELTA_CLAMPED: "clamped", _lib.SDC_QDELTA_LITERAL: "literal",
             _lib.SDC_QDELTA_MIN_SR_NS: "min-sr-ns", _lib.SDC_QDELTA_IMPLICIT_EULER: "ie",
             _lib.SDC_QDELTA_MIN_SR_S: "min-sr-s"}
    out = (ctypes.c_double * M)()
    for rule, name in names.items():
        coll = osdc.Collocation(M, name)
        for k in range(1, 7):
            assert lib.sdc_qdelta(M, rule, k, out) == 0
            # the MIN-SR-S root is ill-conditioned (a coalescing eigenvalue): 1e-10 at M = 8
            tol = 1e-10 if name == "min-sr-s" else 1e-13
            np.testing.assert_allclose(np.array(out[:]), coll.qdelta(k), rtol=tol, atol=1e-14)


def test_host_qdelta_rejects_bad_arguments(lib):
    out = (ctypes.c_double * 8)()
    assert lib.sdc_qdelta(0, 0, 1, out) == 1
    assert lib.sdc_qdelta(9, 0, 1, out) == 1
    assert lib.sdc_qdelta(4, 0, 0, out) == 1
    assert lib.sdc_qdelta(4, 5, 1, out) == 1
    assert lib.sdc_qdelta(4, 0, 1, None) == 1
