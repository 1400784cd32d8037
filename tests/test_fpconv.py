"""The integer binary32 <-> binary64 conversions that the FP64 M-step tail uses
instead of the conversion instructions (gmmsp_fpconv.cuh), checked on the host
against the C casts: every binary32 encoding for the widening, rounding
boundaries (exact values, ties, one ulp either side, overflow and underflow
thresholds) and random encodings for the narrowing."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_integer_conversions_match_the_casts(tmp_path):
    exe = str(tmp_path / "fpconv_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1612_08792_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fpconv_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
    assert "widen 4278190082" in out.stdout  # 2^32 encodings less the 2 (2^23 - 1) subnormals
