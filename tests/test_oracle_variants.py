"""Pins of the oracle's two step variants (no GPU):

- rotation_mode "normalized": the unconstrained solve by Alg. 1 (Sec. 3.4,
  Eq. len_preserving), every world <-> rest rotation of a 3-block replaced by
  A (or A^T) rescaled to keep the block's length;
- jacobian_mode "full": the constraint gradient of Eq. constraint_gradient
  with the joint frame attached to body alpha (Eq. pcpr, r_gradient), the
  rotation's derivative taken from the polar factor's differential.

Each is pinned by something other than its own formula: a reduction to the
polar step where the map is exactly a rotation (rigid and uniformly scaled
bodies), first-order agreement in the strain, equivariance under a turn of
the whole scene, central differences of C(q), and the dense KKT solve."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rel(x, y):
    x, y = np.ravel(x), np.ravel(y)
    return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)


def _step(ora, sc, q, qd, solver="dense", **modes):
    return ora.step(ora.Scene(sc, **modes), q, qd, solver)


def _turn_state(Q, x):
    """A 12-vector (or a stack) of affine coordinates turned by Q."""
    x = np.asarray(x).reshape(-1, 12)
    out = np.empty_like(x)
    for j, v in enumerate(x):
        out[j, :9] = (Q @ v[:9].reshape(3, 3).T).T.reshape(9)
        out[j, 9:] = Q @ v[9:]
    return out


# ---------------------------------------------------------------------------
# Alg. 1
# ---------------------------------------------------------------------------
def test_alg1_equals_polar_on_rigid_states(ora):
    """With A a rotation, A^T f_k has the length of f_k and A dp_k that of
    dp_k: Alg. 1 is the polar step (Eq. abd_final) exactly."""
    for sc in (scenes.random_tree(30, seed=2, joint="mixed"), scenes.chain_cubes(12),
               scenes.assemblies(2, seed=3)):
        q, qd = scenes.perturb_state(sc, seed=1, rot=0.4, vel=0.5, strain=0.0)
        a = _step(ora, sc, q, qd)
        b = _step(ora, sc, q, qd, rotation_mode="normalized")
        assert rel(b[1], a[1]) < 1e-12 and rel(b[2], a[2]) < 1e-12


def test_alg1_equals_polar_for_a_uniform_scale(ora):
    """A = s R (s != 1): the normalised map sends v to R v exactly although A
    is not a rotation, so a free body's step is the polar one; taking A
    without the rescaling, or rescaling the squared lengths, would be off by
    a factor s^+-1."""
    sc = scenes.single_body(sides=(1.0, 2.0, 0.5))
    R = scenes.axis_angle(np.array([1.0, 2.0, -0.5]), 0.7)
    q = sc["q"].copy()
    q[0, :9] = (1.003 * R).T.reshape(9)
    qd = np.random.default_rng(4).standard_normal((1, 12))
    a = _step(ora, sc, q, qd)
    b = _step(ora, sc, q, qd, rotation_mode="normalized")
    assert rel(b[1], a[1]) < 1e-12


def test_alg1_single_body_against_its_definition_of_lengths(ora):
    """The building block itself: u's blocks keep the lengths of
    Hbar^{-1} f~'s blocks, f~'s blocks those of f (Alg. 1), and for a
    rotation A the result is diag4(A) Hbar^{-1} diag4(A^T) f."""
    sc = scenes.single_body(sides=(1.0, 1.5, 0.7))
    H = ora.system_matrix(sc["mass"][0], sc["second_moment"][0], sc["volume"][0],
                          sc["young"][0], sc["poisson"][0], sc["h"])
    L = ora.cholesky12(H)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(12) * 1e3
    Rt = scenes.axis_angle(rng.standard_normal(3), 1.1)
    u = ora.alg1_solve(L, Rt, f)
    D = np.kron(np.eye(4), Rt)
    np.testing.assert_allclose(u, D @ np.linalg.solve(H, D.T @ f), rtol=1e-12, atol=1e-18)
    S = np.eye(3) + 0.05 * np.array([[0.3, 0.1, -0.2], [0.1, -0.4, 0.05], [-0.2, 0.05, 0.2]])
    A = Rt @ S
    u = ora.alg1_solve(L, A, f)
    ft = np.concatenate([A.T @ f[3 * k:3 * k + 3] * np.linalg.norm(f[3 * k:3 * k + 3]) /
                         np.linalg.norm(A.T @ f[3 * k:3 * k + 3]) for k in range(4)])
    dp = np.linalg.solve(H, ft)
    for k in range(4):
        assert abs(np.linalg.norm(u[3 * k:3 * k + 3]) - np.linalg.norm(dp[3 * k:3 * k + 3])) <= \
            1e-12 * np.linalg.norm(dp[3 * k:3 * k + 3])
        c = np.dot(u[3 * k:3 * k + 3], A @ dp[3 * k:3 * k + 3])
        assert c > 0 and abs(c / np.linalg.norm(A @ dp[3 * k:3 * k + 3]) -
                             np.linalg.norm(u[3 * k:3 * k + 3])) < 1e-10 * np.linalg.norm(u[3 * k:3 * k + 3])
    # a zero block stays zero
    f0 = f.copy()
    f0[3:6] = 0.0
    assert np.all(np.isfinite(ora.alg1_solve(L, A, f0)))


def test_alg1_departs_from_polar_with_the_strain(ora):
    """Away from rigid states the two steps differ, by an amount that goes
    to zero with the strain of A (Eq. len_preserving is exact at A = R)."""
    sc = scenes.random_tree(20, seed=4)
    d = []
    for strain in (4e-3, 2e-3, 1e-3, 5e-4):
        q, qd = scenes.perturb_state(sc, seed=2, rot=0.3, vel=0.3, strain=strain)
        a = _step(ora, sc, q, qd)
        b = _step(ora, sc, q, qd, rotation_mode="normalized")
        d.append(rel(b[1], a[1]))
    assert d[0] > 1e-6
    for x, y in zip(d, d[1:]):
        assert 1.5 < x / y < 4.5, d


@pytest.mark.parametrize("mode", [{"rotation_mode": "normalized"}, {"jacobian_mode": "full"}])
def test_variants_are_equivariant(ora, mode):
    """Turning the whole scene (poses, velocities, world anchors and axes,
    gravity) turns the step's result: no world axis is special in either
    variant (a transposed A or R would break this)."""
    sc = scenes.random_tree(16, seed=6, joint="mixed")
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.3, vel=0.4, strain=2e-3)
    sc = dict(sc, q=q, qdot=qd)
    Q = scenes.random_rotations(np.random.default_rng(8), 1)[0]
    sr = scenes.rotate_scene(sc, Q)
    sr["gravity"] = Q @ np.asarray(sc["gravity"], dtype=np.float64)
    a = _step(ora, sc, q, qd, **mode)
    b = _step(ora, sr, sr["q"], sr["qdot"], **mode)
    # (lambda is not compared: ball rows are world axes and the hinge's
    # x~, z~ are one basis of the plane normal to the axis, neither turns)
    assert rel(b[1], _turn_state(Q, a[1])) < 1e-11


# ---------------------------------------------------------------------------
# full constraint gradient
# ---------------------------------------------------------------------------
def _fd_check(ora, sc, q, ks, h=1e-6):
    """max |G - dC/dq| over the joints ks, for the full and the frozen G, C
    evaluated with the frame attached at q (central differences)."""
    Sf = ora.Scene(sc, jacobian_mode="full")
    S0 = ora.Scene(sc)
    qf = np.asarray(q, dtype=np.float64).reshape(-1)
    worst_full = worst_frozen = scale = 0.0
    for k in ks:
        _, Ga, Gb = ora.joint_eval(Sf, qf, k)
        _, Ga0, _ = ora.joint_eval(S0, qf, k)
        for body, G, G0 in ((sc["body_a"][k], Ga, Ga0), (sc["body_b"][k], Gb, None)):
            if body < 0:
                continue
            FD = np.zeros_like(G)
            for l in range(12):
                qp, qm = qf.copy(), qf.copy()
                qp[12 * body + l] += h
                qm[12 * body + l] -= h
                FD[:, l] = (ora.joint_eval_attached(Sf, qf, qp, k) -
                            ora.joint_eval_attached(Sf, qf, qm, k)) / (2 * h)
            scale = max(scale, np.abs(FD).max())
            worst_full = max(worst_full, np.abs(G - FD).max())
            if G0 is not None:
                worst_frozen = max(worst_frozen, np.abs(G0 - FD).max())
    return worst_full / scale, worst_frozen / scale


@pytest.mark.parametrize("case", ["hinge tree", "mixed tree", "prismatic graph"])
def test_full_gradient_matches_central_differences(ora, case):
    """Eq. constraint_gradient against central differences of C(q) with the
    frame attached to alpha (strained bodies, so that P != I matters); the
    frozen-frame gradient misses the frame's term, which grows with the gaps."""
    if case == "hinge tree":
        sc = scenes.random_tree(8, seed=3)
    elif case == "mixed tree":
        sc = scenes.random_tree(8, seed=5, joint="mixed")
    else:
        sc = scenes.random_small("graph", 10, seed=2, hinge_frac=0.0, prism_frac=0.6, gap=0.01)
    q, _ = scenes.perturb_state(sc, seed=4, rot=0.3, vel=0.0, strain=3e-3)
    q = q.copy()
    q[:, 9:] += np.random.default_rng(1).standard_normal((len(q), 3)) * 0.05
    ks = [k for k in range(len(sc["jtype"])) if sc["jtype"][k] in (1, 3)]
    assert ks
    e_full, e_frozen = _fd_check(ora, sc, q, ks)
    assert e_full < 1e-7, e_full
    assert e_frozen > 1e-3, e_frozen


def test_full_equals_frozen_where_the_gaps_vanish(ora):
    """The frame's term multiplies the gaps of the point pairs: at an
    assembled state both gradients coincide."""
    sc = scenes.random_tree(12, seed=2, joint="mixed")
    Sf, S0 = ora.Scene(sc, jacobian_mode="full"), ora.Scene(sc)
    for k in range(len(sc["jtype"])):
        c, Ga, Gb = ora.joint_eval(Sf, sc["q"], k)
        _, Ga0, Gb0 = ora.joint_eval(S0, sc["q"], k)
        assert np.abs(c).max() < 1e-12
        np.testing.assert_allclose(Ga, Ga0, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(Gb, Gb0)


@pytest.mark.parametrize("mode", [{"rotation_mode": "normalized"}, {"jacobian_mode": "full"},
                                  {"rotation_mode": "normalized", "jacobian_mode": "full"}])
def test_variant_solvers_agree_with_the_dense_kkt(ora, mode):
    """Chain (block Thomas), tree (body-space elimination) and CG reach the
    dense KKT solution of the variant's system; the linearized residual
    G dq + C(q_n) vanishes with the variant's G."""
    # assembled or nearly assembled scenes (the random scenes' hinges miss
    # by about a body size, where the frame's term turns bodies inside out)
    for sc, solvers in (
            (scenes.random_small("chain", 9, seed=2, hinge_frac=0.0, prism_frac=0.6, gap=0.01),
             ("chain", "cg")),
            (scenes.random_tree(12, seed=4, joint="mixed"), ("tree", "cg")),
            (scenes.random_small("graph", 12, seed=1, hinge_frac=0.0, prism_frac=0.5, gap=0.01),
             ("cg",))):
        q, qd = scenes.perturb_state(sc, seed=3, rot=0.1, vel=0.3, strain=1e-3)
        ref = _step(ora, sc, q, qd, "dense", **mode)
        assert ref[3]["lin_residual"] < 1e-10
        for s in solvers:
            r = _step(ora, sc, q, qd, s, **mode)
            assert rel(r[1], ref[1]) < 1e-9 and rel(r[2], ref[2]) < 1e-8, (s, mode)


def test_full_and_frozen_newton_steps(ora):
    """One step from a perturbed assembled tree.  The frozen frame keeps the
    anchor rows linear in q (the gap is affine in q, Eq. cp_coordinate), so
    the step closes them exactly; the full gradient makes those rows
    depend on alpha's rotation and leaves a residual of order
    |rotation of alpha| x |gap|.  Both residuals are second order in the
    perturbation."""
    sc = scenes.random_tree(30, seed=2)
    res = {}
    for rot in (0.01, 0.02):
        q, qd = scenes.perturb_state(sc, seed=5, rot=rot, vel=0.0)
        for mode in ("frozen", "full"):
            q1, _, _, st = _step(ora, sc, q, qd, jacobian_mode=mode)
            S = ora.Scene(sc)
            gap1 = 0.0
            for k in range(len(sc["jtype"])):
                c, _, _ = ora.joint_eval(S, q1, k)
                gap1 = max(gap1, np.abs(c[:3]).max())  # anchor rows: |R_H d1| = |d1|
            res[(rot, mode)] = (gap1, st["joint_residual"])
    assert res[(0.01, "frozen")][0] < 1e-12 and res[(0.02, "frozen")][0] < 1e-12
    assert res[(0.01, "full")][0] > 1e-8
    for mode in ("frozen", "full"):
        r = res[(0.02, mode)][1] / res[(0.01, mode)][1]
        assert 3.0 < r < 5.0, (mode, r)


def test_variant_arguments_are_checked(ora):
    sc = scenes.random_small("graph", 8, seed=1, univ_frac=0.5)
    assert np.any(sc["jtype"] == 2)
    with pytest.raises(RuntimeError):
        _step(ora, sc, sc["q"], sc["qdot"], jacobian_mode="full")
    S = ora.Scene(scenes.chain_cubes(4))
    S.s.rotation_mode = 2
    with pytest.raises(RuntimeError):
        ora.step(S, scenes.chain_cubes(4)["q"], scenes.chain_cubes(4)["qdot"])
