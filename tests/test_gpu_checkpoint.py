"""Checkpoint and resume of a state through the C ABI (sdc_save / sdc_load):
bitwise round trip, a header that parses as JSON with the context's sizes,
resume equal bit for bit to an uninterrupted run, and rejection of files of
another truncation or configuration, truncated files and foreign files
(GPU only)."""
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


@pytest.mark.parametrize("other", [dict(dt=300.0), dict(M=4), dict(K=4), dict(L=96)])
def test_rejects_another_configuration(tmp_path, other):
    """A file saved under another step size, node or sweep count or grid (same
    truncation) is refused: its step index would not be a model time here."""
    from paper_2403_20135_gb300 import SdcError
    T, J, L = 21, 34, 72
    kw = dict(M=3, K=3, dt=600.0, L=L)
    kw.update(other)
    s_other = _solver(T, J, kw["L"], M=kw["M"], K=kw["K"], dt=kw["dt"])
    path = str(tmp_path / "other.sdc")
    s_other.save(torch.zeros(3, s_other.ncoef, dtype=torch.complex128, device="cuda"), path, step=4)
    with pytest.raises(SdcError) as e:
        _solver(T, J, L).load(path)
    assert e.value.status == 1
    assert "another configuration" in str(e.value)


def test_rejects_other_physical_constants(tmp_path):
    from paper_2403_20135_gb300 import SdcError, Solver
    T, J, L = 21, 34, 72
    s = Solver(T, J, L, 3, 3, 600.0, si.RADIUS, si.OMEGA, si.GRAVITY, 2.0 * si.MEAN_DEPTH)
    path = str(tmp_path / "deep.sdc")
    s.save(torch.zeros(3, s.ncoef, dtype=torch.complex128, device="cuda"), path)
    with pytest.raises(SdcError):
        _solver(T, J, L).load(path)
