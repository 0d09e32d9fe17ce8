"""GPU parity of scenes with prismatic joints (Sec. 4.5: 5 rows on three
point pairs in a frame that follows body a) against the FP64 CPU oracle, one
step from identical states; such scenes take the PCG solver."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, gpu_step, need_gpu, oracle_step, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("topo,M", [("chain", 2), ("chain", 9), ("tree", 12), ("loop", 15), ("free", 30)])
def test_prismatic_joint_scenes(ora, topo, M):
    need_gpu()
    for seed in range(3):
        sc = scenes.random_small(topo, M, seed=seed, prism_frac=0.5 if M > 2 else 1.0)
        if not (sc["jtype"] == scenes.PRISMATIC).any():
            continue
        s = gpu_solver(sc)
        try:
            assert s.info()["solver"] == "pcg"
            q, qd = scenes.perturb_state(sc, seed=seed + 7, rot=0.2, vel=0.3)
            assert_parity(ora, sc, q, qd, solver=s)
            assert_parity(ora, sc, sc["q"], sc["qdot"], solver=s)
        finally:
            s.close()
        q, qd = scenes.perturb_state(sc, seed=seed + 8, rot=0.1, vel=0.2)
        assert_parity(ora, sc, q, qd, residual_rhs=0)
        assert_parity(ora, sc, q, qd, tol=1e-6, gpu_kw={"precision": "mixed"})


def dual_condition(ora, sc, q, qd):
    """2-norm condition number of the dual matrix G H^-1 G^T (dense, oracle)."""
    S = ora.Scene(sc)
    Hw, f, G, c = ora.assemble_dense(S, q, qd)
    free = np.flatnonzero(sc["fixed"] == 0)
    idx = np.concatenate([np.arange(12 * j, 12 * j + 12) for j in free])
    Hinv = np.zeros((len(idx), len(idx)))
    for n, j in enumerate(free):
        Hinv[12 * n:12 * n + 12, 12 * n:12 * n + 12] = np.linalg.inv(Hw[j])
    G = G[:, idx]
    return float(np.linalg.cond(G @ Hinv @ G.T))


@pytest.mark.parametrize("seed", range(4))
def test_all_joint_types_together(ora, seed):
    """Ball, hinge, universal and prismatic joints in one random graph,
    rigidly turned.  Its cycles of 4- and 5-row joints nearly repeat
    constraints (dual condition numbers 1e5..4e7 here), so the bound on
    the FP64 result grows with the condition number beyond 1e5: PCG stops
    on a residual of 1e-13 relative."""
    need_gpu()
    sc = scenes.random_small("graph", 40, seed=seed, univ_frac=0.3, prism_frac=0.3)
    assert set(np.unique(sc["jtype"])) == {0, 1, 2, 3}
    Q = scenes.random_rotations(np.random.default_rng(seed), 1)[0]
    sc = scenes.rotate_scene(sc, Q)
    q, qd = scenes.perturb_state(sc, seed=seed + 3, rot=0.15, vel=0.3)
    kappa = dual_condition(ora, sc, q, qd)
    tol = 1e-9 * max(1.0, kappa / 1e5)
    assert_parity(ora, sc, q, qd, tol=tol, gpu_kw={"pcg_max_iters": 20000})


def test_inversion_reported_on_both_sides(ora):
    """A random graph whose cycles of prismatic joints over-constrain it:
    one step from this state inverts a body (det A <= 0) in the oracle, and
    the library reports MABD_ERR_INVERTED for the same step."""
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.random_small("graph", 20, seed=0, prism_frac=0.5)
    q, qd = scenes.perturb_state(sc, seed=7, rot=0.2, vel=0.3)
    with pytest.raises(RuntimeError, match="inverted"):
        oracle_step(ora, sc, q, qd)
    s = gpu_solver(sc, pcg_max_iters=20000)
    try:
        with pytest.raises(mabd.MabdError) as e:
            gpu_step(s, q, qd)
        assert e.value.code == 6
    finally:
        s.close()


def test_slider_keeps_its_line(ora):
    """A body on a prismatic joint to the world, pulled by gravity along a
    tilted axis: over ten steps the GPU and the oracle agree, the body slides
    along the axis, and its joint points stay on their lines (the five rows
    of C(q) below 1e-8 after every step)."""
    need_gpu()
    sc = scenes.random_small("chain", 1, seed=3, prism_frac=1.0)
    assert sc["jtype"][0] == scenes.PRISMATIC and sc["body_b"][0] == scenes.WORLD
    sc["anchor_b"][0] = sc["q"][0, 9:] + sc["anchor_a"][0]   # satisfied at rest (A = I)
    s = gpu_solver(sc)
    try:
        s.set_state(sc["q"], sc["qdot"])
        st = s.step(10, stats=True)
        g_q, g_qd = s.get_state()
    finally:
        s.close()
    o_q, o_qd, _, ost = ora.run(sc, 10)
    assert rel(g_q, o_q) < 1e-9 and rel(g_qd, o_qd) < 1e-9
    # one Newton iteration per step leaves a second-order residual
    assert max(x["joint_residual"] for x in st) < 1e-8
    assert max(x["joint_residual"] for x in ost) < 1e-8
    a = sc["axis_a"][0]
    A = g_q[0, :9].reshape(3, 3).T
    d = A @ sc["anchor_a"][0] + g_q[0, 9:] - sc["anchor_b"][0]
    assert abs(np.dot(d, a)) > 1e-3                          # it slid
    assert np.linalg.norm(d - np.dot(d, a) * a) < 1e-10      # along the line


def test_prismatic_joints_refuse_other_solvers_and_bad_frames():
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.random_small("chain", 8, seed=1, prism_frac=1.0)
    for solver in ("chain", "tree", "loop"):
        with pytest.raises(mabd.MabdError) as e:
            gpu_solver(sc, solver=solver)
        assert e.value.code == 10
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    bad["ref_a"][2] = bad["axis_a"][2] * 2.0              # reference along the axis
    with pytest.raises(mabd.MabdError) as e:
        gpu_solver(bad)
    assert e.value.code == 1
