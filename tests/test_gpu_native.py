"""Device primitives checked by small native programs under tests/native,
built with nvcc for sm_103a at test time:

* the integer-pipe FP64 <-> FP32 conversions (csrc/convert.cuh) against the
  hardware conversions, bit for bit (all binary32 values, a seeded binary64
  sample with ties, edge cases);
* the bounded mbarrier wait (csrc/async_copy.cuh): a phase nothing completes
  makes the wait give up and report it, the context stays usable.
"""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]
pytestmark = pytest.mark.gpu


def _build_and_run(tmp_path, name):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / name
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-I",
                    str(ROOT / "paper_2403_20135_gb300" / "csrc"), str(ROOT / "tests" / "native" / f"{name}.cu"),
                    "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)


def test_integer_conversions_match_hardware(tmp_path):
    r = _build_and_run(tmp_path, "convert_check")
    assert r.returncode == 0, r.stdout + r.stderr
    assert "f32_to_f64 mismatches 0" in r.stdout and "mismatches 0 sample, 0 edge" in r.stdout, r.stdout


def test_bounded_wait_gives_up_and_reports(tmp_path):
    r = _build_and_run(tmp_path, "wait_check")
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "expired wait returned 0" in r.stdout and "completed wait returned 1" in r.stdout, r.stdout
