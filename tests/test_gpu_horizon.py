"""Trajectories: the configurations' step counts run in one call on the GPU
against the oracle's own trajectory from the same initial state, on copies of
the paper-shaped scenes small enough for the oracle (the same generators):
the chain, the tree and the net in their benchmarked forms."""
import os

import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import gpu_solver, need_gpu, rel

pytestmark = pytest.mark.gpu

PARAMS = os.path.join(os.path.dirname(__file__), "..", "paper_2603_08079_gb300", "data", "lpc_params.npy")


def run_both(ora, sc, n, **kw):
    s = gpu_solver(sc, **kw)
    try:
        if kw.get("precision") == "mixed" and os.path.exists(PARAMS):
            s.set_preconditioner(np.load(PARAMS).astype(np.float32))
        s.step(n)
        st = s.step(1, stats=True)[0]
        q, qd = s.get_state()
    finally:
        s.close()
    oq, oqd, _, ost = ora.run(sc, n + 1)
    return rel(q, oq), rel(qd, oqd), st, ost[-1]


def test_chain_100_steps_default_form(ora):
    """65,536-body pulley chain (the 1M chain's generator), 100 + 1 steps at
    h = 1e-2 s in the default form: positions within 1e-9 and velocities
    within 1e-5 of the oracle's trajectory."""
    need_gpu()
    sc = scenes.long_chain(65536, seed=1)
    eq, eqd, st, ost = run_both(ora, sc, 100, precision="mixed_fp32_dual")
    print(f"chain 100 steps: q {eq:.3e}, qdot {eqd:.3e}, joint residual {st['joint_residual']:.2e} "
          f"(oracle {ost['joint_residual']:.2e})")
    assert eq < 1e-9 and eqd < 1e-5
    assert st["joint_residual"] < 10 * ost["joint_residual"] + 1e-9


def test_tree_100_steps_mixed(ora):
    """20,000-body tree (the 262,144-body tree's generator), 100 + 1 steps at
    h = 5e-3 s, FP32 elimination with one FP64 sweep."""
    need_gpu()
    sc = scenes.random_tree(20000, seed=2)
    eq, eqd, st, ost = run_both(ora, sc, 100, precision="mixed_fp32_dual")
    print(f"tree 100 steps: q {eq:.3e}, qdot {eqd:.3e}")
    assert eq < 1e-9 and eqd < 1e-5


def test_net_100_steps_learned_preconditioner(ora):
    """16x16x8 jittered net, 100 + 1 steps at h = 1e-2 s, FP32 PCG with the
    learned preconditioner and one FP64 sweep."""
    need_gpu()
    sc = scenes.jittered_net(16, 16, 8, seed=4)
    eq, eqd, st, ost = run_both(ora, sc, 100, precision="mixed")
    print(f"net 100 steps: q {eq:.3e}, qdot {eqd:.3e}")
    assert eq < 1e-9 and eqd < 1e-5
