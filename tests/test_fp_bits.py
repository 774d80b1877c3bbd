"""CPU check of the integer float32 <-> float64 conversions the multiplier update uses on
the GPU (csrc/fp_bits.cuh): compiled for the host and compared bit for bit with the host's
IEEE 754 conversions (every float32 pattern widened; 160 million doubles narrowed,
including exact ties and the overflow and underflow edges)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_16154_gb300", "csrc")


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    return inc if os.path.exists(os.path.join(inc, "cuda_runtime.h")) else None


def test_integer_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "fp_bits_check")
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CSRC}", f"-I{inc}",
                    os.path.join(ROOT, "tests", "fp_bits_check.cpp"), "-o", exe], check=True)
    res = subprocess.run([exe, "20000000"], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0 and res.stdout.strip() == "ok", res.stdout
