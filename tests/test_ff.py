"""The double-float arithmetic of the mixed-precision kernels (csrc/ff.h),
compiled for the host and checked against long double: the binary64 split
(within 2^-46), sums (within 2^-44 of the operands' size), products, fused
multiply-adds and reciprocals (within 2^-44 relative) on random operands
over sixty binades, and the split of zeros, infinities and range edges."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_against_long_double(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "ff_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_2603_08079_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "ff_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
