"""Element-wise parity at full size from a perturbed state: every body's
velocity and every joint's multipliers against the oracle's, with the floor
1e-3 of the largest (parity_util.elementwise), next to the normwise bound,
for the default chain form, the FP64 form and the tree and net workloads.
The element-wise bound is ten times the normwise one."""
import os

import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_elementwise, gpu_solver, gpu_step, need_gpu, oracle_step, rel

pytestmark = pytest.mark.gpu

PARAMS = os.path.join(os.path.dirname(__file__), "..", "paper_2603_08079_gb300", "data", "lpc_params.npy")

CASES = [
    ("chain1m", "fp64", 1e-9), ("chain1m", "mixed_fp32_dual", 1e-6), ("chain1m", "mixed", 1e-6),
    ("tree256k", "fp64", 1e-9), ("tree256k", "mixed_fp32_dual", 1e-6),
    ("net64x64x16", "fp64", 1e-9), ("net64x64x16", "mixed", 1e-6),
]


def scene(name):
    if name == "chain1m":
        return scenes.long_chain(1 << 20, seed=1)
    if name == "tree256k":
        return scenes.random_tree(262144, seed=2)
    return scenes.jittered_net(64, 64, 16, seed=4)


@pytest.mark.parametrize("name,form,tol", CASES)
def test_full_size_elementwise(ora, name, form, tol):
    need_gpu()
    sc = scene(name)
    q, qd = scenes.perturb_state(sc, seed=7, rot=0.02, vel=0.2)
    kw = {"precision": form, "pcg_max_iters": 20000}
    s = gpu_solver(sc, **kw)
    try:
        if name == "net64x64x16" and form != "fp64" and os.path.exists(PARAMS):
            s.set_preconditioner(np.load(PARAMS).astype(np.float32))
        q1, qd1, lam, st = gpu_step(s, q, qd)
    finally:
        s.close()
    oq1, oqd1, olam, ost = oracle_step(ora, sc, q, qd)
    e_qd, e_lam = rel(qd1, oqd1), rel(lam, olam)
    print(f"{name} {form}: normwise qdot {e_qd:.3e}, lambda {e_lam:.3e}")
    assert e_qd <= tol and e_lam <= tol, (e_qd, e_lam)
    assert_elementwise(sc, qd1, oqd1, lam, olam, tol=10 * tol)
