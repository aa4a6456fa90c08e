"""Checkpoint and resume of a state through the C ABI (sdc_save / sdc_load):
bitwise round trip, a header that parses as JSON with the context's sizes,
resume equal bit for bit to an uninterrupted run, and rejection of files of
another truncation, truncated files and foreign files (GPU only)."""
import json

import numpy as np
import pytest

import swe_inputs as si
from oracle import sht, swe
from tests.helpers import to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solver(T, J, L, M=3, K=3, dt=600.0):
    from paper_2403_20135_gb300 import Solver
    return Solver(T, J, L, M, K, dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH)


def _state(T, J, L):
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    u = swe.initial_state(si.Workload("c", 0, T, J, L, 3, 3, 600.0, 1, 1, (100.0, 100.0)), o)
    return torch.from_numpy(u).to("cuda")


def test_round_trip_and_header(tmp_path):
    T, J, L = 21, 34, 72
    s = _solver(T, J, L)
    u = _state(T, J, L)
    path = str(tmp_path / "u.sdc")
    s.save(u, path, step=17)
    with open(path, "rb") as f:
        hdr = json.loads(f.readline())
    assert hdr["format"] == "sdc-swe-state-1" and hdr["truncation"] == T and hdr["nlat"] == J
    assert hdr["nlon"] == L and hdr["step"] == 17 and hdr["ncoef"] == s.ncoef
    assert hdr["fields"] == ["phi", "zeta", "div"] and hdr["bytes"] == 3 * s.ncoef * 16
    v, step = s.load(path)
    assert step == 17
    np.testing.assert_array_equal(to_numpy(v), to_numpy(u))


def test_resume_equals_uninterrupted_run(tmp_path):
    T, J, L = 21, 34, 72
    s = _solver(T, J, L)
    u0 = _state(T, J, L)
    full = s.run(u0.clone(), 5)
    part = s.run(u0.clone(), 3)
    path = str(tmp_path / "u3.sdc")
    s.save(part, path, step=3)
    s2 = _solver(T, J, L)                       # a fresh context, as after a restart
    v, step = s2.load(path)
    assert step == 3
    s2.run(v, 2)
    np.testing.assert_array_equal(to_numpy(v), to_numpy(full))


def test_rejects_foreign_and_damaged_files(tmp_path):
    from paper_2403_20135_gb300 import SdcError
    s21 = _solver(21, 34, 72)
    s31 = _solver(31, 48, 96)
    p31 = str(tmp_path / "t31.sdc")
    s31.save(_state(31, 48, 96), p31)
    with pytest.raises(SdcError):
        s21.load(p31)                           # another truncation
    p21 = str(tmp_path / "t21.sdc")
    s21.save(_state(21, 34, 72), p21)
    data = open(p21, "rb").read()
    cut = str(tmp_path / "cut.sdc")
    open(cut, "wb").write(data[:-16])
    with pytest.raises(SdcError):
        s21.load(cut)                           # truncated data
    foreign = str(tmp_path / "foreign.sdc")
    open(foreign, "wb").write(b'{"format": "other"}\n' + b"\0" * 64)
    with pytest.raises(SdcError):
        s21.load(foreign)
    with pytest.raises(SdcError):
        s21.load(str(tmp_path / "missing.sdc"))
