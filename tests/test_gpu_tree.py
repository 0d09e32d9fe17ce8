"""GPU parity of the tree path (Sec. 5.3, level-scheduled body-space
elimination) against the CPU oracle, one step from identical states."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, need_gpu, rel

pytestmark = pytest.mark.gpu


def drop_joints(sc, keep):
    keep = np.asarray(keep)
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        sc[k] = sc[k][keep]
    return sc


@pytest.mark.parametrize("M", [1, 2, 7, 100, 1000, 20000])
def test_random_hinge_tree(ora, M):
    """The random tree workload (Poisson(1.8) children, hinges, root pinned)."""
    need_gpu()
    sc = scenes.random_tree(M, seed=2)
    s = gpu_solver(sc, solver="tree")
    try:
        assert s.info()["solver"] == "tree"
        assert_parity(ora, sc, sc["q"], sc["qdot"], solver=s)
        q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.3)
        assert_parity(ora, sc, q, qd, solver=s)
    finally:
        s.close()


@pytest.mark.parametrize("seed", range(5))
def test_mixed_trees_and_forests(ora, seed):
    need_gpu()
    for topo, M in (("tree", 6 + 5 * seed), ("free", 4 + 3 * seed)):
        sc = scenes.random_small(topo, M, seed=seed)
        Q = scenes.random_rotations(np.random.default_rng(seed), 1)[0]
        sc = scenes.rotate_scene(sc, Q)
        q, qd = scenes.perturb_state(sc, seed=seed + 10, rot=0.2)
        assert_parity(ora, sc, q, qd, gpu_kw={"solver": "tree"})
    tr = scenes.random_tree(300, seed=seed, joint="mixed")
    q, qd = scenes.perturb_state(tr, seed=seed, rot=0.1)
    assert_parity(ora, tr, q, qd)


def test_root_with_two_world_joints(ora):
    need_gpu()
    sc = scenes.random_small("tree", 8, seed=3)
    # a second world joint on the root (body 0): both are eliminated together
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        sc[k] = np.concatenate([sc[k], sc[k][:1]])
    sc["jtype"][-1] = 1 - sc["jtype"][0]
    sc["anchor_a"][-1] = sc["anchor_a"][0] * -0.5
    sc["anchor_b"][-1] = sc["anchor_b"][0] + 0.3
    q, qd = scenes.perturb_state(sc, seed=4, rot=0.1)
    assert_parity(ora, sc, q, qd, gpu_kw={"solver": "tree"})


def test_fixed_base_assembly(ora):
    """A fixed base body: its joints become one-sided and each subtree hanging
    from it is a tree of its own (the batched-assembly shape)."""
    need_gpu()
    sc = scenes.random_tree(60, seed=7, joint="mixed")
    sc["fixed"][0] = 1
    sc = drop_joints(sc, np.arange(1, len(sc["jtype"])))  # drop the world pin of body 0
    Q = scenes.random_rotations(np.random.default_rng(1), 1)[0]
    sc = scenes.rotate_scene(sc, Q)
    q, qd = scenes.perturb_state(sc, seed=2, rot=0.1)
    assert_parity(ora, sc, q, qd, gpu_kw={"solver": "tree"})


def test_chain_through_the_tree_solver(ora):
    need_gpu()
    sc = scenes.chain_cubes(40)
    q, qd = scenes.perturb_state(sc, seed=1, rot=0.2)
    assert_parity(ora, sc, q, qd, gpu_kw={"solver": "tree"})
    assert_parity(ora, sc, q, qd, gpu_kw={"solver": "tree"}, residual_rhs=0)


def test_full_size_tree(ora):
    """262,144 bodies, 262,143 hinges + a world ball (1,310,718 dual rows)."""
    need_gpu()
    sc = scenes.random_tree(262144, seed=2)
    e_qd, e_lam, st, ost = assert_parity(ora, sc, sc["q"], sc["qdot"])
    assert st["joint_residual"] < 1e-6  # Table 1, tree rows


@pytest.fixture
def forced_variant():
    """Sets MABD_TREE_MODE for the contexts created inside the test."""
    import os
    keys = ("MABD_TREE_MODE",)
    old = {k: os.environ.get(k) for k in keys}

    def set_(v, key="MABD_TREE_MODE"):
        os.environ[key] = str(v)

    yield set_
    for k, v in old.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def test_level_scheduled_path(ora, forced_variant):
    """One launch per level (lane group per body): hinge and mixed trees, a
    root with two world joints, a fixed-base assembly batch."""
    need_gpu()
    forced_variant("levels")
    cases = [scenes.random_tree(3000, seed=2),
             scenes.random_small("tree", 30, seed=7),
             scenes.assemblies(16, seed=3)]
    for sc in cases:
        s = gpu_solver(sc, solver="tree")
        try:
            sched = s.tree_schedule()
            assert sched["path"] == "levels" and sched["levels"] > 0
            q, qd = scenes.perturb_state(sc, seed=11, rot=0.05, vel=0.3)
            assert_parity(ora, sc, q, qd, solver=s)
        finally:
            s.close()


@pytest.mark.parametrize("mode", ["forest128", "forest64", "forest32"])
def test_persistent_forest_kernel(ora, forced_variant, mode):
    """One block per tree, both passes in one launch: forests of fixed-base
    assemblies (many small trees), a single large tree, mixed joints, and
    several steps in one call."""
    need_gpu()
    forced_variant(mode, "MABD_TREE_MODE")
    for sc in (scenes.assemblies(64, seed=3), scenes.random_tree(3000, seed=2),
               scenes.random_small("free", 9, seed=4), scenes.random_small("tree", 30, seed=7)):
        s = gpu_solver(sc, solver="tree")
        try:
            assert s.tree_schedule()["path"] == mode
            q, qd = scenes.perturb_state(sc, seed=5, rot=0.05, vel=0.3)
            assert_parity(ora, sc, q, qd, solver=s)
        finally:
            s.close()
    sc = scenes.assemblies(32, seed=5)
    s = gpu_solver(sc, solver="tree")
    try:
        s.step(20)
        q, qd = s.get_state()
    finally:
        s.close()
    oq, oqd, _, _ = ora.run(sc, 20)
    assert rel(qd, oqd) < 1e-7


def test_tuned_schedule(ora):
    """The tuner picks a path; the tuned step keeps parity."""
    need_gpu()
    for sc in (scenes.random_tree(20000, seed=2), scenes.assemblies(256, seed=3)):
        s = gpu_solver(sc, solver="tree")
        try:
            sched = s.tree_schedule()
            assert sched["levels"] > 0 and sched["path"] in ("levels", "forest128", "forest64", "forest32")
            assert_parity(ora, sc, sc["q"], sc["qdot"], solver=s)
        finally:
            s.close()
