"""The bit-level helpers of `csrc/f32conv.cuh`, compiled for the host (`tests/f32conv_host.cu`):
the FP64 <-> FP32 conversions of the FP32-arithmetic Gram-Schmidt passes and the split-TF32
operands (integer operations on the IEEE-754 layouts, truncation toward zero) against the
C library's conversions on two million random values and the edge cases, and the
fixed-point form whose 6-bit groups are the slices of the FP64-accurate GEMM against the
FP64 multiply-truncate loop that defines them.  No GPU."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.cpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bit_conversions_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "f32conv_host")
    cmd = [nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1610_02244_gb300", "csrc"),
           os.path.join(ROOT, "tests", "f32conv_host.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "mismatches 0" in r.stdout
