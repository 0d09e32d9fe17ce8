"""Steps replayed from CUDA graphs (the default without statistics) give
the same states as direct launches, for every solver."""
import os

import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import gpu_solver, need_gpu, oracle_step, rel

pytestmark = pytest.mark.gpu


def _run(sc, nsteps, graphs, **kw):
    old = os.environ.get("MABD_NO_GRAPHS")
    os.environ["MABD_NO_GRAPHS"] = "0" if graphs else "1"
    try:
        s = gpu_solver(sc, **kw)
    finally:
        if old is None:
            del os.environ["MABD_NO_GRAPHS"]
        else:
            os.environ["MABD_NO_GRAPHS"] = old
    try:
        s.step(nsteps)            # no statistics: graph replay when enabled
        q, qd = s.get_state()
        lam = s.get_lambda()
    finally:
        s.close()
    return q, qd, lam


@pytest.mark.parametrize("name", ["chain", "tree", "net"])
def test_graph_replay_equals_direct_launches(ora, name):
    need_gpu()
    kw = {}
    if name == "chain":
        sc = scenes.long_chain(3001, seed=1)
    elif name == "tree":
        sc = scenes.random_tree(2000, seed=2)
    else:
        sc = scenes.jittered_net(8, 8, 4, seed=4)
        kw = {"pcg_rtol": 1e-14, "pcg_max_iters": 20000}
    qg, qdg, lg = _run(sc, 5, True, **kw)
    qn, qdn, ln = _run(sc, 5, False, **kw)
    np.testing.assert_array_equal(qg, qn)
    np.testing.assert_array_equal(qdg, qdn)
    np.testing.assert_array_equal(lg, ln)
    # and one graph step from the initial state agrees with the oracle
    q1, qd1, l1 = _run(sc, 1, True, **kw)
    oq, oqd, olam, _ = oracle_step(ora, sc, sc["q"], sc["qdot"])
    assert rel(qd1, oqd) <= 1e-9 and rel(l1, olam) <= 1e-9
