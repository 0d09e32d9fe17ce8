"""GPU parity of the mixed-precision tree form (MABD_MIXED_FP32_DUAL on the
tree solver) against the FP64 CPU oracle: the body-space elimination of
Sec. 5.3 in FP32, refined to the FP64 system by FP64 residual-correction
sweeps; the bound is 1e-6 normwise on qdot_{n+1} and lambda for one step from
an identical state."""
import os

import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, gpu_step, need_gpu, oracle_step, rel

pytestmark = pytest.mark.gpu

F32 = {"precision": "mixed_fp32_dual", "solver": "tree"}
TOL = 1e-6


@pytest.fixture
def forced():
    keys = ("MABD_TREE_MODE",)
    old = {k: os.environ.get(k) for k in keys}

    def set_(key, v):
        os.environ[key] = str(v)

    yield set_
    for k, v in old.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def drop_joints(sc, keep):
    keep = np.asarray(keep)
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        sc[k] = sc[k][keep]
    return sc


@pytest.mark.parametrize("M", [1, 2, 7, 100, 1000, 20000])
def test_random_hinge_tree(ora, M):
    need_gpu()
    sc = scenes.random_tree(M, seed=2)
    s = gpu_solver(sc, **F32)
    try:
        inf = s.info()
        assert inf["solver"] == "tree" and inf["precision"] == "mixed_fp32_dual"
        assert_parity(ora, sc, sc["q"], sc["qdot"], solver=s, tol=TOL)
        q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.3)
        assert_parity(ora, sc, q, qd, solver=s, tol=TOL)
    finally:
        s.close()


@pytest.mark.parametrize("seed", range(4))
def test_trees_forests_and_fixed_bases(ora, seed):
    """Mixed ball/hinge trees, forests of free trees, rigidly turned scenes,
    a fixed base body, both rhs readings (residual_rhs 1 and 0)."""
    need_gpu()
    for topo, M in (("tree", 6 + 5 * seed), ("free", 4 + 3 * seed)):
        sc = scenes.random_small(topo, M, seed=seed)
        Q = scenes.random_rotations(np.random.default_rng(seed), 1)[0]
        sc = scenes.rotate_scene(sc, Q)
        q, qd = scenes.perturb_state(sc, seed=seed + 10, rot=0.2)
        assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)
        assert_parity(ora, sc, q, qd, tol=TOL, residual_rhs=0, gpu_kw=F32)
    tr = scenes.random_tree(300, seed=seed, joint="mixed")
    q, qd = scenes.perturb_state(tr, seed=seed, rot=0.1)
    assert_parity(ora, tr, q, qd, tol=TOL, gpu_kw=F32)
    fb = scenes.random_tree(60, seed=7 + seed, joint="mixed")
    fb["fixed"][0] = 1
    fb = drop_joints(fb, np.arange(1, len(fb["jtype"])))
    q, qd = scenes.perturb_state(fb, seed=2, rot=0.1)
    assert_parity(ora, fb, q, qd, tol=TOL, gpu_kw=F32)


def test_root_with_two_world_joints(ora):
    need_gpu()
    sc = scenes.random_small("tree", 8, seed=3)
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        sc[k] = np.concatenate([sc[k], sc[k][:1]])
    sc["jtype"][-1] = 1 - sc["jtype"][0]
    sc["anchor_a"][-1] = sc["anchor_a"][0] * -0.5
    sc["anchor_b"][-1] = sc["anchor_b"][0] + 0.3
    q, qd = scenes.perturb_state(sc, seed=4, rot=0.1)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)


def test_level_scheduled_path(ora, forced):
    """The FP32 elimination, one launch per level."""
    need_gpu()
    forced("MABD_TREE_MODE", "levels")
    for sc in (scenes.random_tree(3000, seed=2), scenes.random_small("tree", 30, seed=7),
               scenes.assemblies(16, seed=3)):
        q, qd = scenes.perturb_state(sc, seed=11, rot=0.05, vel=0.3)
        assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)


@pytest.mark.parametrize("mode", ["forest128", "forest64", "forest32"])
def test_persistent_forest_kernel(ora, forced, mode):
    need_gpu()
    forced("MABD_TREE_MODE", mode)
    for sc in (scenes.assemblies(24, seed=5), scenes.random_tree(500, seed=4, joint="mixed")):
        s = gpu_solver(sc, **F32)
        try:
            assert s.tree_schedule()["path"] == mode
            q, qd = scenes.perturb_state(sc, seed=3, rot=0.05, vel=0.3)
            assert_parity(ora, sc, q, qd, solver=s, tol=TOL)
        finally:
            s.close()


def test_sweeps_refine_to_the_fp64_system(ora):
    """The FP32 elimination alone is FP32-accurate; the FP64 sweeps restore
    the FP64 system's solution."""
    need_gpu()
    sc = scenes.random_tree(5000, seed=3, joint="mixed")
    q, qd = scenes.perturb_state(sc, seed=5, rot=0.05, vel=0.3)
    _, oqd, olam, _ = oracle_step(ora, sc, q, qd)
    e = {}
    for sweeps in (0, 1, 2):
        s = gpu_solver(sc, refine_steps=sweeps, **F32)
        try:
            _, qd1, lam, st = gpu_step(s, q, qd)
        finally:
            s.close()
        e[sweeps] = max(rel(qd1, oqd), rel(lam, olam))
    assert e[0] > 1e-8 and e[1] <= TOL and e[2] < e[1], e


def test_full_size_tree(ora):
    """262,144 bodies, 262,143 hinges + a world ball (1,310,718 dual rows)."""
    need_gpu()
    sc = scenes.random_tree(262144, seed=2)
    e_qd, e_lam, st, _ = assert_parity(ora, sc, sc["q"], sc["qdot"], tol=TOL, gpu_kw=F32)
    assert st["joint_residual"] < 1e-6


def test_full_batch_of_4096_assemblies(ora):
    need_gpu()
    sc = scenes.assemblies(4096, seed=3)
    q, qd = scenes.perturb_state(sc, seed=1, rot=0.05, vel=0.3)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)


def test_plain_mixed_form_is_refused_on_trees():
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.random_tree(50, seed=1)
    with pytest.raises(mabd.MabdError) as e:
        gpu_solver(sc, precision="mixed", solver="tree")
    assert "MABD_MIXED_FP32_DUAL" in str(e.value)
