"""The MABD_DEBUG build of the library (index checks in the kernels that
gather by an index read from memory: a joint's bodies, tree links, the joint
graph): on valid scenes it reports no error and gives the release build's
results.  It runs in a child process, since a process loads one build."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import gpu_solver, gpu_step, need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + '/tests')
from paper_2603_08079_gb300 import scenes, mabd
from parity_util import gpu_solver, gpu_step
from test_gpu_debug_build import cases
out = {}
for name, sc, kw in cases():
    s = gpu_solver(sc, **kw)
    try:
        q, qd = scenes.perturb_state(sc, seed=1, rot=0.05, vel=0.2)
        q1, qd1, lam, st = gpu_step(s, q, qd)
    finally:
        s.close()
    out[name + '_qd'] = qd1
    out[name + '_lam'] = lam
np.savez(sys.argv[2], **out)
"""


def cases():
    return [("chain", scenes.long_chain(300, seed=1), {}),
            ("tree", scenes.random_tree(500, seed=2), {"precision": "mixed_fp32_dual"}),
            ("batch", scenes.assemblies(16, seed=3), {}),
            ("net", scenes.jittered_net(5, 5, 3, seed=4), {"precision": "mixed"})]


def test_debug_build_matches_release(tmp_path):
    need_gpu()
    out = tmp_path / "debug.npz"
    env = dict(os.environ, MABD_LIB="debug")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(out)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    dbg = np.load(out)
    for name, sc, kw in cases():
        s = gpu_solver(sc, **kw)
        try:
            q, qd = scenes.perturb_state(sc, seed=1, rot=0.05, vel=0.2)
            q1, qd1, lam, st = gpu_step(s, q, qd)
        finally:
            s.close()
        np.testing.assert_allclose(dbg[name + "_qd"], qd1, rtol=0, atol=1e-12 * max(1.0, np.abs(qd1).max()))
        np.testing.assert_allclose(dbg[name + "_lam"], lam, rtol=0, atol=1e-12 * max(1.0, np.abs(lam).max()))
