"""Learned block preconditioner of the mixed PCG path: its normalized dual
blocks and its training gradient against the CPU oracle (oracle/lpc.py),
training itself, and what the trained network does for the dual solve."""
import os

import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, need_gpu, rel

pytestmark = pytest.mark.gpu

MIXED = {"precision": "mixed"}
TOL = 1e-6
PARAMS = os.path.join(os.path.dirname(__file__), "..", "paper_2603_08079_gb300", "data", "lpc_params.npy")


@pytest.fixture(scope="module")
def lpc():
    from oracle import lpc as L
    return L


def trained_params():
    if not os.path.exists(PARAMS):
        pytest.skip("no trained parameters")
    return np.load(PARAMS).astype(np.float32)


def capture(sc, q, qd):
    from paper_2603_08079_gb300 import mabd
    s = gpu_solver(sc, **MIXED)
    s.set_state(q, qd)
    t = mabd.LpcTrainer()
    b = t.capture(s)
    return s, t, b


def test_blocks_match_oracle(ora, lpc):
    """Joint graph bit-exact; the normalized blocks E (FP32 on the GPU) within
    1e-5 of the oracle's FP64 ones."""
    need_gpu()
    sc = scenes.jittered_net(4, 4, 3, seed=7)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.2, vel=0.1)
    s, t, b = capture(sc, q, qd)
    try:
        ent, ones = lpc.joint_graph(sc)
        K = len(ent)
        nnz = sum(len(e) for e in ent)
        off, nbr, E = t.blocks(b, K, nnz)
        np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum([len(e) for e in ent])]))
        np.testing.assert_array_equal(nbr, [n for e in ent for (n, _, _, _) in e])
        C, St = lpc.normalized(lpc.dual_dense(sc, q, qd))
        Eo = np.array([blk for row in lpc.blocks(St, ent) for blk in row])
        assert rel(E, Eo) <= 1e-5
    finally:
        t.close()
        s.close()


def test_loss_and_gradient_match_oracle(ora, lpc):
    """The GPU's loss and gradient (BF16 tensor-core layers, FP32 backward)
    against the oracle's FP64 dense backpropagation with the same BF16
    rounding of the layer inputs, same probe vectors and parameters."""
    need_gpu()
    sc = scenes.jittered_net(4, 4, 3, seed=7)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.2, vel=0.1)
    s, t, b = capture(sc, q, qd)
    try:
        ent, ones = lpc.joint_graph(sc)
        C, St = lpc.normalized(lpc.dual_dense(sc, q, qd))
        E = lpc.blocks(St, ent)
        for seed, kind in ((0, "frobenius"), (1, "kaporin"), (2, "kaporin")):
            theta = scenes.lpc_init_params(seed)
            pr = lpc.unpack(theta.astype(np.float64))
            rng = np.random.default_rng(seed)
            pr["Wa"][:] = rng.standard_normal(pr["Wa"].shape) * 0.2
            pr["Wb"][:] = rng.standard_normal(pr["Wb"].shape) * 0.2
            pr["wd"][:] = rng.standard_normal(pr["wd"].shape) * 0.02
            theta = lpc.pack(pr).astype(np.float32)
            V = scenes.lpc_probe(2, len(ent), seed=10 + seed)
            L_gpu, g_gpu = t.loss_grad(b, theta, V=V, kind=kind)
            L_ora, g_ora = lpc.loss_grad(theta.astype(np.float64), St, E, ent, ones, V.astype(np.float64),
                                         kind=kind)
            assert abs(L_gpu - L_ora) <= 1e-4 * max(abs(L_ora), 1e-2), (kind, L_gpu, L_ora)
            assert rel(g_gpu, g_ora) <= 2e-3, rel(g_gpu, g_ora)
    finally:
        t.close()
        s.close()


def test_training_lowers_the_loss_on_held_out_systems():
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.net_collection(6, seed=21)
    s = gpu_solver(sc, **MIXED)
    t = mabd.LpcTrainer()
    try:
        for c in range(6):
            qq, qqd = scenes.perturb_state(sc, seed=c, rot=0.3, vel=0.5)
            s.set_state(qq, qqd)
            s.step(1)
            t.capture(s)
        p0 = scenes.lpc_init_params(0)
        held = 5
        before = np.mean([t.loss_grad(held, p0, seed=k, grad=False)[0] for k in range(4)])
        p, losses = t.train(p0, 300, lr=1e-3, nv=2, seed=3)
        assert np.all(np.isfinite(losses)) and np.mean(losses[-30:]) < np.mean(losses[:30])
        after = np.mean([t.loss_grad(held, p, seed=k, grad=False)[0] for k in range(4)])
        assert after < before - 0.05 * abs(before), (before, after)
    finally:
        t.close()
        s.close()


@pytest.mark.parametrize("dims", [(6, 6, 3), (16, 16, 8)])
def test_learned_preconditioner_step_parity(ora, dims):
    """The mixed step with the learned preconditioner stays within 1e-6 of
    the FP64 oracle (the preconditioner changes only the iteration count)."""
    need_gpu()
    p = trained_params()
    sc = scenes.jittered_net(*dims, seed=4)
    s = gpu_solver(sc, **MIXED)
    try:
        s.set_preconditioner(p)
        q, qd = scenes.perturb_state(sc, seed=2, rot=0.05, vel=0.2)
        assert_parity(ora, sc, q, qd, solver=s, tol=TOL)
    finally:
        s.close()


@pytest.mark.parametrize("dims", [(6, 6, 3), (24, 24, 8)])
def test_normalized_and_matrix_free_solves_agree(ora, dims, monkeypatch):
    """The learned-preconditioner step solved in the normalized dual space
    (one cooperative launch per solve over the stored blocks E) and by the
    matrix-free per-body S-apply: both within 1e-6 of the oracle, with
    iteration counts within a few of each other (the same iteration in exact
    arithmetic; FP32 rounding and the partial sums' blocking differ)."""
    from parity_util import gpu_step, oracle_step
    need_gpu()
    p = trained_params()
    sc = scenes.jittered_net(*dims, seed=4)
    q, qd = scenes.perturb_state(sc, seed=2, rot=0.05, vel=0.2)
    res = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("MABD_PCG_NORMALIZED", mode)
        s = gpu_solver(sc, **MIXED)
        try:
            s.set_preconditioner(p)
            q1, qd1, lam, st = gpu_step(s, q, qd)
        finally:
            s.close()
        res[mode] = (qd1, lam, st[0]["pcg_iters"])
    _, oqd, olam, _ = oracle_step(ora, sc, q, qd)
    for mode, (qd1, lam, it) in res.items():
        assert rel(qd1, oqd) <= TOL and rel(lam, olam) <= TOL, (mode, rel(qd1, oqd), rel(lam, olam))
    i1, i0 = res["1"][2], res["0"][2]
    assert abs(i1 - i0) <= max(4, i0 // 10), (i1, i0)


def test_warm_start_from_the_previous_multipliers(monkeypatch):
    """The step's first solve starts from the previous step's multipliers:
    over steps 2-6 of a net it needs fewer FP32 PCG iterations than from
    zero, and the trajectories agree to the mixed bound."""
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    p = trained_params()
    sc = scenes.jittered_net(16, 16, 8, seed=4)
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("MABD_PCG_WARM", mode)
        s = gpu_solver(sc, **MIXED)
        try:
            s.set_preconditioner(p)
            s.step(1)
            its = [s.step(1, stats=True)[0]["pcg_iters"] for _ in range(5)]
            q, qd = s.get_state()
        finally:
            s.close()
        out[mode] = (sum(its), q, qd)
    print("iterations over steps 2-6: warm", out["1"][0], "cold", out["0"][0])
    assert out["1"][0] < out["0"][0]
    assert rel(out["1"][2], out["0"][2]) <= TOL and rel(out["1"][1], out["0"][1]) <= 1e-9


@pytest.mark.parametrize("dims", [(16, 16, 8), (64, 64, 16)])
def test_learned_beats_block_jacobi(dims):
    """Fewer FP32 PCG iterations per step than block Jacobi on nets the
    network never saw (held-out seed and sizes), same accuracy target."""
    need_gpu()
    from paper_2603_08079_gb300.train_lpc import pcg_iterations
    p = trained_params()
    sc = scenes.jittered_net(*dims, seed=4)
    it_bj, it_init, it_learned = pcg_iterations(sc, scenes.lpc_init_params(0), p)
    print("pcg iterations (block Jacobi, untrained, trained)", dims, it_bj, it_init, it_learned)
    assert it_learned < 0.9 * it_bj, (it_bj, it_learned)
    assert it_learned <= 1.05 * it_init, (it_init, it_learned)   # training does not undo the structure


def test_untrained_parameters_stay_exact(ora):
    """Arbitrary (large random) parameters: the step is still within 1e-6 of
    the oracle (the preconditioner is SPD by construction; a learned solve
    that misses the tolerance is redone with block Jacobi)."""
    need_gpu()
    sc = scenes.jittered_net(6, 6, 3, seed=4)
    p = (np.random.default_rng(0).standard_normal(scenes.lpc_param_count()) * 3.0).astype(np.float32)
    s = gpu_solver(sc, **MIXED, pcg_max_iters=3000)
    try:
        s.set_preconditioner(p)
        q, qd = scenes.perturb_state(sc, seed=2, rot=0.05, vel=0.2)
        assert_parity(ora, sc, q, qd, solver=s, tol=TOL)
        assert s.lpc_fallbacks() >= 0
    finally:
        s.close()


def test_learned_preconditioner_needs_the_mixed_ball_graph_path():
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    p = scenes.lpc_init_params(0)
    sc = scenes.jittered_net(3, 3, 2, seed=4)
    s = gpu_solver(sc)                      # FP64 form
    try:
        with pytest.raises(mabd.MabdError) as e:
            s.set_preconditioner(p)
        assert e.value.code == 10
    finally:
        s.close()
    hinge = scenes.random_small("graph", 8, seed=1, hinge_frac=1.0)
    s = gpu_solver(hinge, **MIXED)
    try:
        with pytest.raises(mabd.MabdError) as e:
            s.set_preconditioner(p)
        assert e.value.code == 10
    finally:
        s.close()
