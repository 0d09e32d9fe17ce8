"""The host helpers that keep bodies given with a non-diagonal second moment
in their principal frames (csrc/principal_frame.h), compiled for the host:
the cyclic Jacobi eigen-decomposition reconstructs random SPD matrices
(repeated, nearly repeated and already diagonal spectra included) with an
orthonormal, proper rotation, and the affine-part change of frame goes
there and back exactly."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_principal_frames_on_the_host(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "frame_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_2603_08079_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "frame_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
