"""GPU parity of the loop solver (Sec. 5.4, Case III: one joint of a closed
loop is the breaker, the others form a chain solved by block cyclic
reduction, the breaker's multipliers come from the chain's Schur complement)
against the FP64 CPU oracle, one step from identical states."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, gpu_step, need_gpu, oracle_step, rel

pytestmark = pytest.mark.gpu


def ring(M, seed, hinge_frac=0.5):
    return scenes.random_small("loop", M, seed=seed, pin=False, hinge_frac=hinge_frac)


@pytest.mark.parametrize("M", [3, 4, 5, 8, 17, 100, 1000, 4099])
def test_random_rings(ora, M):
    need_gpu()
    sc = ring(M, seed=M)
    s = gpu_solver(sc)
    try:
        inf = s.info()
        assert inf["topology"] == "loop" and inf["solver"] == "loop"
        q, qd = scenes.perturb_state(sc, seed=M + 1, rot=0.1, vel=0.3)
        assert_parity(ora, sc, q, qd, solver=s)
        assert_parity(ora, sc, sc["q"], sc["qdot"], solver=s)
    finally:
        s.close()


@pytest.mark.parametrize("hinge_frac", [0.0, 1.0])
def test_all_ball_and_all_hinge_rings(ora, hinge_frac):
    """A ball breaker (3 rhs passes) and a hinge breaker (5 passes)."""
    need_gpu()
    for M in (6, 57):
        sc = ring(M, seed=3 + M, hinge_frac=hinge_frac)
        q, qd = scenes.perturb_state(sc, seed=2, rot=0.2, vel=0.2)
        assert_parity(ora, sc, q, qd)
        assert_parity(ora, sc, q, qd, residual_rhs=0)


def test_loop_solver_matches_pcg(ora):
    """The same ring through the FP64 PCG path: the two exact dual solves agree."""
    need_gpu()
    sc = ring(300, seed=9)
    q, qd = scenes.perturb_state(sc, seed=4, rot=0.1, vel=0.3)
    out = {}
    for name, kw in (("loop", {}), ("pcg", dict(solver="pcg", pcg_rtol=1e-14, pcg_max_iters=20000))):
        s = gpu_solver(sc, **kw)
        try:
            assert s.info()["solver"] == name
            _, out[name + "_qd"], out[name + "_lam"], _ = gpu_step(s, q, qd)
        finally:
            s.close()
    assert rel(out["loop_qd"], out["pcg_qd"]) < 1e-9 and rel(out["loop_lam"], out["pcg_lam"]) < 1e-9


def test_large_ring(ora):
    need_gpu()
    sc = ring(65537, seed=1)
    q, qd = scenes.perturb_state(sc, seed=6, rot=0.05, vel=0.2)
    e_qd, e_lam, st, _ = assert_parity(ora, sc, q, qd)
    assert st["lin_residual"] < 1e-9


def test_loop_solver_is_fp64_only():
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = ring(12, seed=2)
    with pytest.raises(mabd.MabdError):
        gpu_solver(sc, solver="loop", precision="mixed")
    s = gpu_solver(sc, precision="mixed")  # AUTO: the mixed PCG path
    try:
        assert s.info()["solver"] == "pcg"
    finally:
        s.close()


@pytest.mark.parametrize("M", [3, 10, 4096])
def test_pulley_ring(ora, M):
    """The pulley-cable chain closed into a loop (scenes.ring_chain)."""
    need_gpu()
    sc = scenes.ring_chain(M, seed=1)
    q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.2)
    assert_parity(ora, sc, q, qd)


def test_full_size_pulley_ring(ora):
    """1,048,576 bodies closed into one loop, the launch configuration the
    benchmark's loop workload times."""
    need_gpu()
    sc = scenes.ring_chain(1 << 20, seed=1)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.05, vel=0.2)
    e_qd, e_lam, st, _ = assert_parity(ora, sc, q, qd)
    assert st["lin_residual"] < 1e-8
