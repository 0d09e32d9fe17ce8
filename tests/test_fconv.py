"""The integer binary64 <-> binary32 conversions of the mixed-precision
kernels (csrc/fconv.h), compiled for the host and compared bit for bit with
the host's own conversions (round to nearest, ties to even) on random bit
patterns, exact ties and their neighbours, and the binary32 range edges."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_conversions_match_the_host(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "fconv_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2603_08079_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "fconv_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
