"""The exact double-to-float narrowing of the FP32 Q assembly
(csrc/bits.cuh), compiled for the host with nvcc and checked against the
float -> double widening on every exponent, subnormals, zeros, infinities and
NaNs (tests/bits_check.cu). No GPU is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_narrow_exact_inverts_the_widening(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "bits_check")
    src = os.path.join(ROOT, "tests", "bits_check.cu")
    inc = os.path.join(ROOT, "paper_2208_12569_gb300", "csrc")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", inc, src, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    n, bad = (int(v) for v in out.stdout.split())
    assert out.returncode == 0 and bad == 0 and n > 30_000_000
