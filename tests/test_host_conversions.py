"""The FP32 <-> int64 conversions of the deposits (one FP32 -> int32
conversion and a shift) and of the fixed-point loader (integer pipe),
csrc/common.cuh, equal round-to-nearest-even conversions on ~4.4e7 floats
and ~2e7 integers (halfway cases, the split's boundaries and extremes
included).  Host code compiled with nvcc; no GPU needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_conversions_match_round_to_nearest(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "conversion_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "conversion_check.cu")], check=True,
                   capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert " 0 mismatches; " in out.stdout and out.stdout.strip().endswith(" 0 mismatches")
