"""The structured inverse of Hbar_A = M_A/h^2 + Kbar_A (Eq. abd_final) that
every per-body kernel applies (csrc/hbar_inv.h: 16 numbers per body in a
principal rest frame), compiled for the host and expanded to 12x12, against
the inverse of the oracle's dense Hbar_A (its mass matrix pinned by
quadrature, its stiffness by finite differences of the energy), over random
bodies from near-rigid to soft, light to heavy, and time steps from 1e-4 to
1e-1 s.  A body whose Hbar_A is not positive definite is refused."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def expand(v):
    """The 12x12 inverse from the 16 numbers: h^2/m on the translation, the
    3x3 block of A's diagonal entries q[0], q[4], q[8], and the 2x2 blocks
    of the transpose pairs (q1, q3), (q2, q6), (q5, q7)."""
    X = np.zeros((12, 12))
    for i in (9, 10, 11):
        X[i, i] = v[0]
    d = (0, 4, 8)
    S = np.array([[v[1], v[2], v[3]], [v[2], v[4], v[5]], [v[3], v[5], v[6]]])
    for r in range(3):
        for c in range(3):
            X[d[r], d[c]] = S[r, c]
    for base, (p, q) in ((7, (1, 3)), (10, (2, 6)), (13, (5, 7))):
        X[p, p], X[p, q], X[q, p], X[q, q] = v[base], v[base + 1], v[base + 1], v[base + 2]
    return X


def test_structured_inverse_against_the_oracle(ora, tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "hbar_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2603_08079_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "hbar_check.cpp"), "-o", str(exe)], check=True)
    rng = np.random.default_rng(11)
    bodies = []
    for _ in range(300):
        sides = rng.uniform(0.05, 3.0, 3)
        rho = 10.0 ** rng.uniform(1.0, 4.5)
        V = float(np.prod(sides))
        m = rho * V
        s = m * sides ** 2 / 12.0  # box second moments about the centre
        E = 10.0 ** rng.uniform(4.0, 11.0)
        nu = rng.uniform(0.0, 0.49)
        h = 10.0 ** rng.uniform(-4.0, -1.0)
        bodies.append((m, *s, V, E, nu, h))
    bodies.append((1.0, 1.0, 1.0, 1.0, 1.0, 1e8, 0.5, 1e-2))  # nu = 1/2: lambda infinite
    text = "\n".join(" ".join("%.17g" % x for x in b) for b in bodies) + "\n"
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
    assert len(out) == len(bodies)
    worst = 0.0
    for b, line in zip(bodies[:-1], out[:-1]):
        m, s0, s1, s2, V, E, nu, h = b
        S6 = np.array([s0, s1, s2, 0.0, 0.0, 0.0])
        H = ora.system_matrix(m, S6, V, E, nu, h)
        X = expand(np.array([float(x) for x in line.split()]))
        Hi = np.linalg.inv(H)
        # both sides are exact to rounding times the conditioning of H
        err = np.abs(X - Hi).max() / np.abs(Hi).max() / np.linalg.cond(H)
        worst = max(worst, err)
        # and as an inverse: X H = I to the conditioning of H
        assert np.abs(X @ H - np.eye(12)).max() <= 1e-12 * np.linalg.cond(H)
    assert worst < 1e-14, worst
    assert out[-1] == "fail"
