"""The GPU's Fourier mode selection and binning for rank-order matching
(csrc/rom.cuh ModeSel: integer |k| threshold, integer bin edges), compiled
for the host, selects the same modes into the same bins as the oracle
(Sec. 2.3.2: 100 |k| bins, k >= 0.1 h/Mpc, canonical half-space modes).
No GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import projection as OP

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = [(16, 20.0), (32, 150.0), (64, 300.0), (128, 500.0), (256, 500.0), (128, 100.0)]


def test_mode_bins_match_oracle(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "rom_bins_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-o", exe,
                    os.path.join(HERE, "rom_bins_check.cu")], check=True, capture_output=True)
    args = [str(v) for nb in CASES for v in nb]
    out = subprocess.run([exe] + args, capture_output=True, text=True, timeout=300, check=True).stdout.splitlines()
    assert len(out) == len(CASES)
    for (n, box), line in zip(CASES, out):
        got = np.array([int(v) for v in line.split()])
        np.testing.assert_array_equal(got, OP.fourier_bin_counts(n, box), err_msg=f"n={n} box={box}")
