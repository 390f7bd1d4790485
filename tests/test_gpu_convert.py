"""The integer-pipe FP64 <-> FP32 conversions (csrc/convert.cuh) against the hardware conversions.

The mixed step converts every value it loads or stores with these helpers; the
probe compares them bit for bit with __double2float_rn and the exact widening
on 2^26 random FP64 inputs (ties included), special values and all 2^32 FP32
patterns."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_conversions_match_hardware(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(ROOT, "tests", "convert_check.cu")
    exe = str(tmp_path / "convert_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    print(res.stdout)
    assert res.returncode == 0, res.stdout + res.stderr
