"""GPU parity of the mixed-precision form against the FP64 CPU oracle.

The mixed form solves the same linearized KKT system as the FP64 form:
per-body and per-joint products in FP32, the dual solve (FP64 block cyclic
reduction on chains, FP32 PCG on graphs), then FP64 residual-correction
sweeps (iterative refinement).
Its stated bound is 1e-6 normwise relative error on qdot_{n+1} and lambda
for one step from an identical state."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, gpu_step, need_gpu, oracle_step, rel

pytestmark = pytest.mark.gpu

MIXED = {"precision": "mixed"}
TOL = 1e-6


def mixed_errors(ora, sc, q, qd, **kw):
    solver = gpu_solver(sc, **dict(MIXED, **kw))
    try:
        assert solver.info()["precision"] == dict(MIXED, **kw)["precision"]
        _, qd1, lam, st = gpu_step(solver, q, qd)
    finally:
        solver.close()
    _, oqd1, olam, _ = oracle_step(ora, sc, q, qd, kw.get("residual_rhs", 1))
    return rel(qd1, oqd1), (rel(lam, olam) if len(olam) else 0.0), st[0]


def test_mixed_chain64_along_oracle_trajectory(ora):
    need_gpu()
    sc = scenes.chain_cubes(64)
    S = ora.Scene(sc)
    q, qd = sc["q"], sc["qdot"]
    states = {}
    for n in range(120):
        if n in (0, 1, 10, 50, 119):
            states[n] = (q, qd)
        q, qd, _, _ = ora.step(S, q, qd)
    solver = gpu_solver(sc, **MIXED)
    try:
        for q0, qd0 in states.values():
            _, _, st, _ = assert_parity(ora, sc, q0, qd0, solver=solver, tol=TOL)
            assert st["joint_residual"] < 1e-10
    finally:
        solver.close()


@pytest.mark.parametrize("M", [1, 2, 3, 5, 17, 64, 255, 1000, 4097, 65537])
def test_mixed_long_chain_ragged_sizes(ora, M):
    need_gpu()
    sc = scenes.long_chain(M, seed=1)
    q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.2)
    assert_parity(ora, sc, sc["q"], sc["qdot"], tol=TOL, gpu_kw=MIXED)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=MIXED)


@pytest.mark.parametrize("seed", range(6))
def test_mixed_random_chains(ora, seed):
    need_gpu()
    M = [2, 3, 8, 13, 31, 40][seed]
    sc = scenes.random_small("chain", M, seed=seed, hinge_frac=0.5)
    q, qd = scenes.perturb_state(sc, seed=seed, rot=0.3)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=MIXED)
    Q = scenes.random_rotations(np.random.default_rng(seed), 1)[0]
    sc2 = scenes.rotate_scene(sc, Q)
    q2, qd2 = scenes.perturb_state(sc2, seed=seed + 50, rot=0.1)
    assert_parity(ora, sc2, q2, qd2, tol=TOL, gpu_kw=MIXED)


def test_mixed_chain_variants(ora):
    """Printed zero bottom rhs, no pin, a fixed end body, a single joint and
    bodies without joints."""
    need_gpu()
    sc = scenes.chain_cubes(20)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.2)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=MIXED)
    assert_parity(ora, sc, q, qd, tol=TOL, residual_rhs=0, gpu_kw=MIXED)
    free = scenes.random_small("chain", 9, seed=4, pin=False)
    q, qd = scenes.perturb_state(free, seed=5, rot=0.2)
    assert_parity(ora, free, q, qd, tol=TOL, gpu_kw=MIXED)
    fx = scenes.random_small("chain", 9, seed=6)
    fx["fixed"][0] = 1
    fx["qdot"][0] = 0.0
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        fx[k] = fx[k][1:]
    q, qd = scenes.perturb_state(fx, seed=7, rot=0.2)
    assert_parity(ora, fx, q, qd, tol=TOL, gpu_kw=MIXED)
    one = scenes.chain_cubes(1)                 # one body, one world ball: a single dual row block
    q, qd = scenes.perturb_state(one, seed=8, rot=0.3, vel=1.0)
    assert_parity(ora, one, q, qd, tol=TOL, gpu_kw=MIXED)
    bare = scenes.random_small("chain", 5, seed=2)
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        bare[k] = bare[k][:0]
    q, qd = scenes.perturb_state(bare, seed=1, rot=1.0, vel=2.0)
    assert_parity(ora, bare, q, qd, tol=TOL, gpu_kw=MIXED)


def test_refinement_sweeps_reduce_the_error(ora):
    """Without a sweep the result carries the FP32 products' error; each FP64
    correction sweep shrinks it, and the reported FP64 residual entering the
    last sweep shrinks with it."""
    need_gpu()
    sc = scenes.long_chain(4097, seed=1)
    q, qd = scenes.perturb_state(sc, seed=11, rot=0.05, vel=0.2)
    e = {}
    for s in (0, 1, 2):
        e_qd, e_lam, st = mixed_errors(ora, sc, q, qd, refine_steps=s)
        e[s] = (max(e_qd, e_lam), st["refine_residual"])
    assert e[0][0] > 1e-9, e          # the FP32 products alone are not FP64-accurate
    assert e[1][0] <= TOL and e[2][0] <= TOL, e
    assert e[1][0] < 1e-2 * e[0][0], e
    assert e[0][1] == 0.0 and 0.0 < e[2][1] < e[1][1], e


NET_SWEEPS = 1


@pytest.mark.parametrize("dims", [(3, 3, 2), (6, 6, 3), (10, 10, 4), (16, 16, 8)])
def test_mixed_jittered_net(ora, dims):
    """Closed-loop ball-joint net: FP32 PCG for each dual solve, FP64
    residual-correction sweeps."""
    need_gpu()
    sc = scenes.jittered_net(*dims, seed=4)
    errs = {}
    for sweeps in (1, 2):
        e_qd, e_lam, st = mixed_errors(ora, sc, sc["q"], sc["qdot"], refine_steps=sweeps)
        errs[sweeps] = (e_qd, e_lam, st["pcg_iters"], st["refine_residual"])
    assert max(errs[NET_SWEEPS][:2]) <= TOL, errs
    assert max(errs[2][:2]) < max(errs[1][:2]), errs   # a second sweep still gains
    q, qd = scenes.perturb_state(sc, seed=1, rot=0.05, vel=0.2)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=dict(MIXED, refine_steps=NET_SWEEPS))


@pytest.mark.parametrize("seed", range(4))
def test_mixed_loops_and_graphs(ora, seed):
    need_gpu()
    for topo, M in (("loop", 5 + seed), ("graph", 6 + 3 * seed)):
        sc = scenes.random_small(topo, M, seed=seed)
        q, qd = scenes.perturb_state(sc, seed=seed, rot=0.2)
        assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=dict(MIXED, refine_steps=NET_SWEEPS))


def test_mixed_full_size_net(ora):
    """64x64x16 lattice (65,536 bodies, 4,096 fixed), ~128k ball joints."""
    need_gpu()
    sc = scenes.jittered_net(64, 64, 16, seed=4)
    e_qd, e_lam, st = mixed_errors(ora, sc, sc["q"], sc["qdot"], refine_steps=NET_SWEEPS)
    assert max(e_qd, e_lam) <= TOL


@pytest.mark.parametrize("dims", [(6, 6, 3), (24, 24, 8)])
def test_persistent_and_per_launch_pcg_agree(ora, dims, monkeypatch):
    """The FP32 PCG as one cooperative launch per solve (device-side loop and
    convergence test) and as one launch per step of an iteration: both meet
    the oracle at the mixed bound; their iteration counts differ by at most a
    few (the partial sums are blocked differently)."""
    need_gpu()
    sc = scenes.jittered_net(*dims, seed=4)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.05, vel=0.2)
    res = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("MABD_PCG_PERSIST", mode)
        s = gpu_solver(sc, **dict(MIXED, refine_steps=NET_SWEEPS))
        try:
            q1, qd1, lam, st = gpu_step(s, q, qd)
        finally:
            s.close()
        res[mode] = (qd1, lam, st[0]["pcg_iters"])
    _, oqd, olam, _ = oracle_step(ora, sc, q, qd)
    for mode, (qd1, lam, it) in res.items():
        assert rel(qd1, oqd) <= TOL and rel(lam, olam) <= TOL, (mode, rel(qd1, oqd), rel(lam, olam))
    assert abs(res["1"][2] - res["0"][2]) <= max(3, res["0"][2] // 20), (res["1"][2], res["0"][2])


def test_mixed_rejects_other_topologies():
    """MABD_MIXED (FP64 dual elimination) has no tree form: the tree's mixed
    form is MABD_MIXED_FP32_DUAL (tests/test_gpu_tree_mixed.py)."""
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.random_small("tree", 12, seed=3)
    with pytest.raises(mabd.MabdError) as err:
        gpu_solver(sc, **MIXED)
    assert err.value.code == 10


def test_mixed_full_size_pulley_chain(ora):
    """1,048,576 bodies / 4,194,305 dual rows in the launch configuration the
    benchmark times (one correction sweep): every output compared."""
    need_gpu()
    sc = scenes.long_chain(1 << 20, seed=1)
    e_qd, e_lam, st, _ = assert_parity(ora, sc, sc["q"], sc["qdot"], tol=TOL, gpu_kw=MIXED)
    assert st["joint_residual"] < 1e-5


# ---------------------------------------------------------------------------
# mixed form with the chain's cyclic reduction in FP32 (MABD_MIXED_FP32_DUAL)
# ---------------------------------------------------------------------------
F32 = {"precision": "mixed_fp32_dual"}


@pytest.mark.parametrize("M", [1, 2, 3, 17, 255, 4097, 65537])
def test_fp32_reduction_long_chain(ora, M):
    need_gpu()
    sc = scenes.long_chain(M, seed=1)
    q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.2)
    assert_parity(ora, sc, sc["q"], sc["qdot"], tol=TOL, gpu_kw=F32)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)


@pytest.mark.parametrize("seed", range(3))
def test_fp32_reduction_random_chains(ora, seed):
    need_gpu()
    M = [3, 13, 40][seed]
    sc = scenes.random_small("chain", M, seed=seed, hinge_frac=0.5)
    q, qd = scenes.perturb_state(sc, seed=seed, rot=0.3)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)
    assert_parity(ora, sc, q, qd, tol=TOL, residual_rhs=0, gpu_kw=F32)


def test_fp32_reduction_sweeps(ora):
    """The FP32 reduction alone is FP32-accurate; the FP64 sweeps restore
    the FP64 system's solution."""
    need_gpu()
    sc = scenes.long_chain(4097, seed=1)
    q, qd = scenes.perturb_state(sc, seed=11, rot=0.05, vel=0.2)
    e = {}
    for sweeps in (0, 1, 2):
        e_qd, e_lam, st = mixed_errors(ora, sc, q, qd, refine_steps=sweeps, **{"precision": "mixed_fp32_dual"})
        e[sweeps] = max(e_qd, e_lam)
    assert e[0] > 1e-8 and e[1] <= TOL and e[2] < e[1], e


def test_fp32_reduction_on_the_pcg_path(ora):
    need_gpu()
    sc = scenes.jittered_net(6, 6, 3, seed=4)
    assert_parity(ora, sc, sc["q"], sc["qdot"], tol=TOL, gpu_kw=F32)


def test_fp32_reduction_full_size_pulley_chain(ora):
    need_gpu()
    sc = scenes.long_chain(1 << 20, seed=1)
    e_qd, e_lam, st, _ = assert_parity(ora, sc, sc["q"], sc["qdot"], tol=TOL, gpu_kw=F32)
    assert st["joint_residual"] < 1e-5
