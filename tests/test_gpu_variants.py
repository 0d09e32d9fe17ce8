"""GPU parity of the paper's step variants (FP64 form) against the oracle,
one step from identical states, through the C ABI:

- MABD_ROTATION_NORMALIZED: the unconstrained solve of every body by Alg. 1
  (Sec. 3.4, Eq. len_preserving) on each solver (chain, tree, loop, PCG);
- MABD_JACOBIAN_FULL: the frame term of Eq. constraint_gradient (Sec. 5.1,
  frame attached to body a, Eq. r_gradient) on the tree and PCG solvers.

States carry a strain of 1e-3 (so that A is not a rotation and Alg. 1
differs from the polar step) and joint gaps (so that the frame term is not
zero); each case also checks that the variant moves the oracle's result by
far more than the tolerance."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import gpu_solver, gpu_step, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL = 1e-9


def dual_condition(ora, sc, q, qd, **modes):
    """2-norm condition number of G H^-1 G^T of the variant (dense, oracle)."""
    Hw, f, G, c = ora.assemble_dense(ora.Scene(sc, **modes), q, qd)
    free = np.flatnonzero(sc["fixed"] == 0)
    idx = np.concatenate([np.arange(12 * j, 12 * j + 12) for j in free])
    Hinv = np.zeros((len(idx), len(idx)))
    for n, j in enumerate(free):
        Hinv[12 * n:12 * n + 12, 12 * n:12 * n + 12] = np.linalg.inv(Hw[j])
    G = G[:, idx]
    return float(np.linalg.cond(G @ Hinv @ G.T))


def variant_parity(ora, sc, q, qd, modes, expect=None, tol=TOL, **gpu_kw):
    """GPU step against the oracle's step of the same variant; returns the
    relative change that the variant makes to the oracle's qdot_{n+1}."""
    s = gpu_solver(sc, **modes, **gpu_kw)
    try:
        info = s.info()
        for key, v in modes.items():
            assert info[key] == v
        if expect is not None:
            assert info["solver"] == expect
        q1, qd1, lam, st = gpu_step(s, q, qd)
    finally:
        s.close()
    _, oqd1, olam, ost = ora.step(ora.Scene(sc, 1, **modes), q, qd, "auto")
    e_qd, e_lam = rel(qd1, oqd1), rel(lam, olam)
    print(f"{info['solver']} {modes}: qdot {e_qd:.2e}, lambda {e_lam:.2e} (tol {tol:.1e})")
    assert e_qd <= tol and e_lam <= tol, (e_qd, e_lam)
    # |G dq + C(q_n)| with the variant's G (the full gradient's frame term
    # included): the step meets its own linearized constraints
    assert st[0]["lin_residual"] < 1e-8, st[0]["lin_residual"]
    _, bqd1, _, _ = ora.step(ora.Scene(sc, 1), q, qd, "auto")
    return rel(oqd1, bqd1)


NORMALIZED = {"rotation_mode": "normalized"}
FULL = {"jacobian_mode": "full"}


@pytest.mark.parametrize("case", ["chain", "long chain", "tree", "batch", "loop", "net"])
def test_normalized_rotation_on_every_solver(ora, case):
    need_gpu()
    solver = {"chain": "chain", "long chain": "chain", "tree": "tree", "batch": "tree",
              "loop": "loop", "net": "pcg"}[case]
    sc = {"chain": lambda: scenes.random_small("chain", 40, seed=1),
          "long chain": lambda: scenes.long_chain(4096, seed=3),
          "tree": lambda: scenes.random_tree(1500, seed=2, joint="mixed"),
          "batch": lambda: scenes.assemblies(24, seed=3),
          "loop": lambda: scenes.ring_chain(96, seed=1),
          "net": lambda: scenes.jittered_net(6, 6, 4, seed=4)}[case]()
    q, qd = scenes.perturb_state(sc, seed=5, rot=0.1, vel=0.3, strain=1e-3)
    moved = variant_parity(ora, sc, q, qd, NORMALIZED, expect=solver)
    assert moved > 1e-7, moved


def test_normalized_rotation_with_every_joint_type(ora):
    """Ball, hinge, universal and prismatic joints on the PCG solver (the
    bound grows with the dual's condition number beyond 1e5, as for the
    polar form of these graphs)."""
    need_gpu()
    sc = scenes.random_small("graph", 30, seed=2, univ_frac=0.3, prism_frac=0.3)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.1, vel=0.3, strain=1e-3)
    kappa = dual_condition(ora, sc, q, qd, **NORMALIZED)
    moved = variant_parity(ora, sc, q, qd, NORMALIZED, expect="pcg",
                           tol=TOL * max(1.0, kappa / 1e5), pcg_max_iters=20000)
    assert moved > 1e-7


def test_normalized_rotation_over_steps(ora):
    """Twenty steps of a tree: the state fed back each step."""
    need_gpu()
    sc = scenes.random_tree(400, seed=5, joint="mixed")
    q, qd = scenes.perturb_state(sc, seed=2, rot=0.05, vel=0.2, strain=1e-3)
    s = gpu_solver(sc, **NORMALIZED)
    try:
        s.set_state(q, qd)
        s.step(20)
        q1, qd1 = s.get_state()
    finally:
        s.close()
    oq, oqd, _, _ = ora.run(sc, 20, q=q, qd=qd, **NORMALIZED)
    assert rel(qd1, oqd) < 1e-7 and rel(q1, oq) < 1e-9


@pytest.fixture
def tree_mode():
    import os
    old = os.environ.get("MABD_TREE_MODE")

    def set_(v):
        if v is None:
            os.environ.pop("MABD_TREE_MODE", None)
        else:
            os.environ["MABD_TREE_MODE"] = v

    yield set_
    set_(old)


@pytest.mark.parametrize("solver", ["tree", "pcg"])
@pytest.mark.parametrize("case", ["hinge tree", "mixed tree", "batch", "hinge tree normalized"])
def test_full_gradient_on_trees(ora, case, solver):
    """The frame term on hinge rows, in the tree solver's elimination (its
    rows, and the parent's rows in the downward pass) and in the PCG."""
    need_gpu()
    modes = dict(FULL)
    if case == "hinge tree":
        sc = scenes.random_tree(400, seed=2)
    elif case == "mixed tree":
        sc = scenes.random_tree(300, seed=3, joint="mixed")
    elif case == "batch":
        sc = scenes.assemblies(12, seed=4)
    else:
        sc = scenes.random_tree(300, seed=4)
        modes.update(NORMALIZED)
    q, qd = scenes.perturb_state(sc, seed=6, rot=0.05, vel=0.3, strain=1e-3)
    kappa = dual_condition(ora, sc, q, qd, **modes)
    moved = variant_parity(ora, sc, q, qd, modes, expect=solver, tol=TOL * max(1.0, kappa / 1e5),
                           **({"solver": "pcg", "pcg_max_iters": 20000} if solver == "pcg" else {}))
    assert moved > 1e-6, moved


@pytest.mark.parametrize("mode", ["levels", "forest64", "forest32"])
def test_full_gradient_on_every_tree_path(ora, tree_mode, mode):
    """AUTO picks the tree solver for a tree; both the level schedule and
    the persistent kernel carry the frame term."""
    need_gpu()
    tree_mode(mode)
    sc = scenes.assemblies(16, seed=5)
    q, qd = scenes.perturb_state(sc, seed=2, rot=0.05, vel=0.3, strain=1e-3)
    s = gpu_solver(sc, **FULL)
    try:
        assert s.info()["solver"] == "tree" and s.tree_schedule()["path"] == mode
        _, qd1, lam, _ = gpu_step(s, q, qd)
    finally:
        s.close()
    _, oqd1, olam, _ = ora.step(ora.Scene(sc, 1, **FULL), q, qd, "auto")
    kappa = dual_condition(ora, sc, q, qd, **FULL)
    tol = TOL * max(1.0, kappa / 1e5)
    assert rel(qd1, oqd1) <= tol and rel(lam, olam) <= tol, (rel(qd1, oqd1), rel(lam, olam))


def test_full_gradient_on_pcg_prismatic(ora):
    """The frame term on prismatic rows (a graph: AUTO picks PCG)."""
    need_gpu()
    sc = scenes.random_small("graph", 30, seed=1, hinge_frac=0.0, prism_frac=0.5, gap=0.01)
    q, qd = scenes.perturb_state(sc, seed=6, rot=0.05, vel=0.3, strain=1e-3)
    kappa = dual_condition(ora, sc, q, qd, **FULL)
    moved = variant_parity(ora, sc, q, qd, FULL, expect="pcg", tol=TOL * max(1.0, kappa / 1e5),
                           pcg_max_iters=20000)
    assert moved > 1e-6, moved


def test_variants_are_refused_where_not_built():
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    tree = scenes.random_tree(30, seed=1)
    cases = [(scenes.random_small("chain", 12, seed=2), dict(FULL, solver="chain"), "PCG"),
             (scenes.ring_chain(12, seed=1), dict(FULL, solver="loop"), "PCG"),
             (scenes.random_small("graph", 12, seed=1, univ_frac=0.5), FULL, "universal"),
             (tree, dict(NORMALIZED, precision="mixed_fp32_dual"), "FP64"),
             (scenes.chain_cubes(8), dict(FULL, precision="mixed"), "FP64")]
    for sc, kw, word in cases:
        with pytest.raises(mabd.MabdError) as e:
            gpu_solver(sc, **kw)
        assert e.value.code == 10 and word in str(e.value), str(e.value)
