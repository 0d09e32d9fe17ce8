"""GPU parity of the chain path (Sec. 5.2) against the CPU oracle, one step
from identical states, through the C ABI."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, gpu_step, need_gpu, oracle_step, rel

pytestmark = pytest.mark.gpu


def test_chain64_along_oracle_trajectory(ora):
    """64 unit cubes, ball joints, body 0 pinned (the plain FP64 chain):
    parity at several states of the oracle's own 200-step trajectory."""
    need_gpu()
    sc = scenes.chain_cubes(64)
    S = ora.Scene(sc)
    q, qd = sc["q"], sc["qdot"]
    states = {}
    for n in range(200):
        if n in (0, 1, 10, 50, 120, 199):
            states[n] = (q, qd)
        q, qd, _, _ = ora.step(S, q, qd)
    solver = gpu_solver(sc)
    try:
        assert solver.info()["topology"] == "chain"
        for n, (q0, qd0) in states.items():
            e_qd, e_lam, st, ost = assert_parity(ora, sc, q0, qd0, solver=solver)
            assert st["joint_residual"] < 1e-12 and st["lin_residual"] < 1e-12
    finally:
        solver.close()


def test_chain64_free_run_200_steps(ora):
    """200 GPU steps in one call: every ball joint stays closed to round-off
    and the trajectory follows the oracle's."""
    need_gpu()
    sc = scenes.chain_cubes(64)
    solver = gpu_solver(sc)
    try:
        st = solver.step(200, stats=True)
        q, qd = solver.get_state()
    finally:
        solver.close()
    assert max(s["joint_residual"] for s in st) < 1e-11
    oq, oqd, _, _ = ora.run(sc, 200)
    assert rel(qd, oqd) < 1e-7
    assert rel(q, oq) < 1e-9


@pytest.mark.parametrize("M", [1, 2, 3, 5, 17, 64, 255, 1000, 4097, 65537])
def test_long_chain_parity_ragged_sizes(ora, M):
    """The pulley-cable chain (alternating ball/hinge, both ends pinned) at
    sizes that span one to many reduction levels and ragged tails."""
    need_gpu()
    sc = scenes.long_chain(M, seed=1)
    q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.2)
    assert_parity(ora, sc, sc["q"], sc["qdot"])
    assert_parity(ora, sc, q, qd)


@pytest.mark.parametrize("seed", range(6))
def test_random_mixed_chains(ora, seed):
    need_gpu()
    M = [2, 3, 8, 13, 31, 40][seed]
    sc = scenes.random_small("chain", M, seed=seed, hinge_frac=0.5)
    q, qd = scenes.perturb_state(sc, seed=seed, rot=0.3)
    assert_parity(ora, sc, q, qd)
    # the same chain turned rigidly: exercises arbitrary hinge axes and rotations
    Q = scenes.random_rotations(np.random.default_rng(seed), 1)[0]
    sc2 = scenes.rotate_scene(sc, Q)
    q2, qd2 = scenes.perturb_state(sc2, seed=seed + 50, rot=0.1)
    assert_parity(ora, sc2, q2, qd2)


def test_chain_variants(ora):
    """One pin, no pin, a fixed end body (its joint becomes one-sided) and the
    printed zero bottom rhs (residual_rhs = 0)."""
    need_gpu()
    sc = scenes.chain_cubes(20)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.2)
    assert_parity(ora, sc, q, qd)
    assert_parity(ora, sc, q, qd, residual_rhs=0)
    free = scenes.random_small("chain", 9, seed=4, pin=False)
    q, qd = scenes.perturb_state(free, seed=5, rot=0.2)
    assert_parity(ora, free, q, qd)
    fx = scenes.random_small("chain", 9, seed=6)
    fx["fixed"][0] = 1          # its world pin would have no free body: drop it
    fx["qdot"][0] = 0.0
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        fx[k] = fx[k][1:]
    q, qd = scenes.perturb_state(fx, seed=7, rot=0.2)
    assert_parity(ora, fx, q, qd)


def test_bodies_without_joints(ora):
    need_gpu()
    sc = scenes.random_small("chain", 5, seed=2)
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        sc[k] = sc[k][:0]
    q, qd = scenes.perturb_state(sc, seed=1, rot=1.0, vel=2.0)
    assert_parity(ora, sc, q, qd)


def test_inverted_body_is_reported_not_silent(ora):
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.chain_cubes(4)
    solver = gpu_solver(sc)
    try:
        q = sc["q"].copy()
        q[2, 0:3] *= -1.0  # reflect one column: det A < 0
        solver.set_state(q, sc["qdot"])
        with pytest.raises(mabd.MabdError) as e:
            solver.step(1, stats=True)
        assert e.value.code == 6
        solver.set_state(sc["q"], sc["qdot"])  # the context stays usable
        solver.step(1, stats=True)
    finally:
        solver.close()


def test_full_size_pulley_chain(ora):
    """1,048,576 bodies / 1,048,577 joints (4,194,305 dual rows), in the
    launch configuration the benchmark times: every output compared."""
    need_gpu()
    sc = scenes.long_chain(1 << 20, seed=1)
    e_qd, e_lam, st, ost = assert_parity(ora, sc, sc["q"], sc["qdot"])
    assert st["joint_residual"] < 1e-5  # Table 1, huge pulley row


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_polar_iteration_count(ora, precision):
    """mabd_step_stats.polar_iterations: one Newton step where A is a
    rotation already (the first step does not move it), three where A
    carries a 1e-3 symmetric stretch (steps ~1e-3, ~5e-7, then below the
    1e-9 stopping size); the step stays within parity either way."""
    need_gpu()
    sc = scenes.chain_cubes(16)
    s = gpu_solver(sc, precision=precision)
    try:
        _, _, _, st = gpu_step(s, sc["q"], sc["qdot"])
        assert st[0]["polar_iterations"] == 1.0
        q, qd = scenes.perturb_state(sc, seed=4, rot=0.3, vel=0.1)
        rng = np.random.default_rng(9)
        for j in range(len(q)):
            E = rng.standard_normal((3, 3)) * 1e-3
            A = q[j, :9].reshape(3, 3).T @ (np.eye(3) + 0.5 * (E + E.T))  # q stacks A's columns
            q[j, :9] = A.T.reshape(9)
        _, _, _, st = gpu_step(s, q, qd)
        assert 3.0 <= st[0]["polar_iterations"] <= 4.0
    finally:
        s.close()
    assert_parity(ora, sc, q, qd, tol=1e-9 if precision == "fp64" else 1e-6, gpu_kw={"precision": precision})
