"""The integer-pipe FP64 <-> FP32 conversions used by the mixed-precision
kernels (csrc/convert.cuh) against the hardware conversions, bit for bit
(tests/native/convert_check.cu: all binary32 values, a seeded binary64 sample
with ties, and edge cases)."""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]


@pytest.mark.gpu
def test_integer_conversions_match_hardware(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "convert_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-I",
                    str(ROOT / "paper_2403_20135_gb300" / "csrc"), str(ROOT / "tests" / "native" / "convert_check.cu"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "f32_to_f64 mismatches 0" in r.stdout and "mismatches 0 sample, 0 edge" in r.stdout, r.stdout
