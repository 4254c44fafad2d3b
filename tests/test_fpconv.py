"""The integer float <-> double conversions (csrc/fpconv.cuh) against the C
conversions: every binary32 value, and 1e8 random binary64 patterns (host code,
no GPU needed)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_integer_float_conversions_match_ieee(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fpconv_check")
    src = os.path.join(HERE, "native", "fpconv_check.cu")
    subprocess.run([nvcc, "-O2", "-std=c++17", src, "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
