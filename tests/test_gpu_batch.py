"""GPU parity of the batched form: thousands of independent assemblies
(each a random tree on a fixed, randomly posed base) stepped together as one
forest by the tree path."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 7, 64])
def test_small_batches(ora, n):
    need_gpu()
    sc = scenes.assemblies(n, seed=3)
    s = gpu_solver(sc)
    try:
        assert s.info()["solver"] == "tree"
        assert_parity(ora, sc, sc["q"], sc["qdot"], solver=s)
        q, qd = scenes.perturb_state(sc, seed=n, rot=0.05, vel=0.3)
        assert_parity(ora, sc, q, qd, solver=s)
    finally:
        s.close()


def test_full_batch_of_4096_assemblies(ora):
    """144,619 links / 140,523 joints: every output compared with the oracle."""
    need_gpu()
    sc = scenes.assemblies(4096, seed=3)
    q, qd = scenes.perturb_state(sc, seed=1, rot=0.02, vel=0.2)
    assert_parity(ora, sc, q, qd)


def test_batch_runs_many_steps_in_one_call(ora):
    """100 steps replayed from the step's CUDA graph stay finite and keep the
    joints closed to Table 1's loosest printed tolerance (the oracle's own
    residual on this scene after 100 steps is 1e-6 to 3e-6; the config's
    1000-step run, shortened)."""
    need_gpu()
    sc = scenes.assemblies(256, seed=3)
    s = gpu_solver(sc)
    try:
        s.step(100)
        st = s.step(1, stats=True)[0]
        q, qd = s.get_state()
    finally:
        s.close()
    assert np.all(np.isfinite(q)) and np.all(np.isfinite(qd))
    assert st["joint_residual"] < 1e-5


F32 = {"precision": "mixed_fp32_dual", "solver": "tree"}


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_full_batch_elementwise(ora, form):
    """The full 4,096-assembly batch from a perturbed state, each body's
    velocity and each joint's multipliers against the oracle's (floor 1e-3
    of the largest), in the FP64 form (1e-9) and the mixed form (1e-6)."""
    from parity_util import assert_elementwise, gpu_step, oracle_step, rel

    need_gpu()
    sc = scenes.assemblies(4096, seed=3)
    q, qd = scenes.perturb_state(sc, seed=2, rot=0.03, vel=0.3)
    kw = F32 if form == "mixed" else {}
    tol = 1e-6 if form == "mixed" else 1e-9
    s = gpu_solver(sc, **kw)
    try:
        sched = s.tree_schedule()
        q1, qd1, lam, st = gpu_step(s, q, qd)
    finally:
        s.close()
    oq1, oqd1, olam, ost = oracle_step(ora, sc, q, qd)
    print(form, sched, "normwise", rel(qd1, oqd1), rel(lam, olam))
    assert rel(qd1, oqd1) <= tol and rel(lam, olam) <= tol
    assert_elementwise(sc, qd1, oqd1, lam, olam, tol=10 * tol)


def test_full_batch_horizon(ora):
    """The full batch in the mixed form, 200 steps at h = 2e-3 s in one call,
    against the oracle's 200 steps from the same state: the state at the end
    agrees to 1e-6 normwise (velocities) and 1e-8 (positions)."""
    need_gpu()
    sc = scenes.assemblies(4096, seed=3)
    n = 200
    s = gpu_solver(sc, **F32)
    try:
        s.step(n)
        q, qd = s.get_state()
    finally:
        s.close()
    oq, oqd, _, _ = ora.run(sc, n)
    from parity_util import rel

    eq, eqd = rel(q, oq), rel(qd, oqd)
    print(f"after {n} steps: q {eq:.3e}, qdot {eqd:.3e}")
    assert eqd < 1e-6 and eq < 1e-8
