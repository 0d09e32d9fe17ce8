"""GPU parity of scenes with universal joints (Sec. 4.4: 4 rows, the ball
rows in the frame R_U plus one row on body b alone) against the FP64 CPU
oracle, one step from identical states; such scenes take the PCG solver."""
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("topo,M", [("chain", 2), ("chain", 9), ("tree", 12), ("graph", 20), ("loop", 15),
                                    ("free", 30)])
def test_universal_joint_scenes(ora, topo, M):
    need_gpu()
    for seed in range(3):
        sc = scenes.random_small(topo, M, seed=seed, univ_frac=0.5 if M > 2 else 1.0)
        if not (sc["jtype"] == scenes.UNIVERSAL).any():
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


def test_all_universal_chain(ora):
    need_gpu()
    sc = scenes.random_small("chain", 40, seed=4, pin=False, univ_frac=1.0)
    assert (sc["jtype"] == scenes.UNIVERSAL).all()
    q, qd = scenes.perturb_state(sc, seed=5, rot=0.15, vel=0.3)
    assert_parity(ora, sc, q, qd)
    assert_parity(ora, sc, q, qd, tol=1e-6, gpu_kw={"precision": "mixed_fp32_dual"})


def test_universal_joints_refuse_other_solvers():
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.random_small("chain", 8, seed=1, univ_frac=1.0)
    for solver in ("chain", "tree", "loop"):
        with pytest.raises(mabd.MabdError) as e:
            gpu_solver(sc, solver=solver)
        assert e.value.code == 10
