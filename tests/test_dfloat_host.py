"""Double-float arithmetic of the mixed-precision structure factors, checked
on the host: tests/dfloat_check.cu compiles the kernels' own
__host__ __device__ functions (exact phase reduction from the integer
coordinates of G and the split fractional coordinates of P, sin/cos by table
and Taylor series, Hermite polynomial products) for the CPU and compares
them with long double and with a plain double evaluation."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_double_float_phase_and_polynomials(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "dfloat_check")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-o", exe, os.path.join(HERE, "dfloat_check.cu")],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    phase, poly, twosum = (float(x) for x in out)
    assert phase < 5e-14, phase  # absolute error of cos and sin of the phase
    assert poly < 1e-13, poly    # relative to the block's largest element
    assert twosum == 0.0, twosum
