"""GPU parity of the graph path (dual-space block-Jacobi PCG) against the
CPU oracle, one step from identical states."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, need_gpu, rel

pytestmark = pytest.mark.gpu

PCG = {"pcg_rtol": 1e-14, "pcg_max_iters": 20000}


@pytest.mark.parametrize("dims", [(3, 3, 2), (6, 6, 3), (10, 10, 4), (16, 16, 8)])
def test_jittered_net(ora, dims):
    """Closed-loop ball-joint network on a jittered lattice, bottom layer fixed."""
    need_gpu()
    sc = scenes.jittered_net(*dims, seed=4)
    s = gpu_solver(sc, **PCG)
    try:
        assert s.info()["solver"] == "pcg"
        e_qd, e_lam, st, ost = assert_parity(ora, sc, sc["q"], sc["qdot"], solver=s)
        assert st["pcg_iters"] > 0 and st["pcg_rel_residual"] <= 1e-14
        q, qd = scenes.perturb_state(sc, seed=1, rot=0.05, vel=0.2)
        assert_parity(ora, sc, q, qd, solver=s)
    finally:
        s.close()


@pytest.mark.parametrize("seed", range(4))
def test_loops_and_graphs(ora, seed):
    need_gpu()
    for topo, M in (("loop", 5 + seed), ("graph", 6 + 3 * seed)):
        sc = scenes.random_small(topo, M, seed=seed)
        q, qd = scenes.perturb_state(sc, seed=seed, rot=0.2)
        assert_parity(ora, sc, q, qd, gpu_kw=PCG)


def test_pcg_on_a_chain_matches_the_direct_solvers(ora):
    need_gpu()
    sc = scenes.long_chain(500, seed=1)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.05)
    assert_parity(ora, sc, q, qd, gpu_kw=dict(PCG, solver="pcg"))


def test_iteration_cap_is_reported(ora):
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.jittered_net(4, 4, 3, seed=4)
    s = gpu_solver(sc, pcg_max_iters=2)
    try:
        with pytest.raises(mabd.MabdError) as e:
            s.step(1, stats=True)
        assert e.value.code == 8
    finally:
        s.close()


def test_full_size_net(ora):
    """64x64x16 lattice (65,536 bodies, 4,096 fixed), ~128k ball joints."""
    need_gpu()
    sc = scenes.jittered_net(64, 64, 16, seed=4)
    e_qd, e_lam, st, ost = assert_parity(ora, sc, sc["q"], sc["qdot"], gpu_kw=PCG)
    assert st["joint_residual"] < 1e-7  # Table 1, joint-net row
