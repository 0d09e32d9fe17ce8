"""GPU parity of the segment-tiled chain step against the FP64 CPU oracle.

With MABD_CHAIN_SEG=1 the mixed form with the FP32 reduction and one
correction sweep runs the chain in tiles of joints (mabd_info.seg_tile): one
CTA per tile does the tile's per-body and
per-joint work and eliminates the tile's rows by block cyclic reduction in
shared memory; the tiles' first rows form a smaller block-tridiagonal system,
reduced by tiles of 256 rows (MABD_SEG_UP_T sets that size, so that small
chains here exercise several levels).  Bound: 1e-6 normwise relative error on
qdot_{n+1} and lambda for one step from an identical state (the mixed form's
bound), plus per-body and per-joint errors against a stated floor
(parity_util.elementwise)."""
import os

import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import (assert_elementwise, assert_parity, gpu_solver, gpu_step, need_gpu, oracle_step,
                         rel)

pytestmark = pytest.mark.gpu

F32 = {"precision": "mixed_fp32_dual"}
TOL = 1e-6


@pytest.fixture(autouse=True)
def seg_on():
    """The segment-tiled step is chosen with MABD_CHAIN_SEG=1."""
    old = os.environ.get("MABD_CHAIN_SEG")
    os.environ["MABD_CHAIN_SEG"] = "1"
    yield
    if old is None:
        os.environ.pop("MABD_CHAIN_SEG", None)
    else:
        os.environ["MABD_CHAIN_SEG"] = old


@pytest.fixture
def env():
    saved = {k: os.environ.get(k) for k in ("MABD_SEG_UP_T", "MABD_CHAIN_SEG")}

    def set_(k, v):
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = str(v)

    yield set_
    for k, v in saved.items():
        set_(k, v)


def seg_levels(sc, **kw):
    s = gpu_solver(sc, **dict(F32, **kw))
    try:
        return s.info()["seg_levels"]
    finally:
        s.close()


def seg_tile(sc):
    s = gpu_solver(sc, **F32)
    try:
        return s.info()["seg_tile"]
    finally:
        s.close()


def flip_joints(sc, every=2):
    """The same chain with body a and body b swapped on every `every`-th joint
    between two bodies (a hinge then takes its frame from the other body)."""
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    for k in range(0, len(sc["jtype"]), every):
        if sc["body_b"][k] < 0:
            continue
        for x, y in (("body_a", "body_b"), ("anchor_a", "anchor_b"), ("axis_a", "axis_b")):
            out[x][k], out[y][k] = sc[y][k].copy(), sc[x][k].copy()
    return out


def permute_bodies(sc, seed):
    """The same scene with its bodies numbered in a random order."""
    M = len(sc["mass"])
    perm = np.random.default_rng(seed).permutation(M)   # new id i holds old body perm[i]
    inv = np.empty(M, dtype=np.int64)
    inv[perm] = np.arange(M)
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    for key in ("mass", "second_moment", "volume", "young", "poisson", "fixed", "q", "qdot"):
        out[key] = sc[key][perm].copy()
    for key in ("body_a", "body_b"):
        v = sc[key]
        out[key] = np.where(v < 0, v, inv[np.maximum(v, 0)])
    return out


@pytest.mark.parametrize("M", [1, 2, 3, 126, 127, 128, 129, 255, 256, 257, 1000, 40000])
def test_seg_long_chain_sizes(ora, M):
    """Pulley chains (both ends pinned, K = M + 1 joints) across tile edges:
    one tile, a ragged last tile, two upper levels (40,000 bodies)."""
    need_gpu()
    sc = scenes.long_chain(M, seed=1)
    assert seg_levels(sc) >= 1
    q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.2)
    assert_parity(ora, sc, sc["q"], sc["qdot"], tol=TOL, gpu_kw=F32)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)


@pytest.mark.parametrize("ut", [2, 4, 32])
@pytest.mark.parametrize("M", [300, 2100])
def test_seg_upper_levels(ora, env, ut, M):
    """Small upper tiles: 2,100 bodies with tiles of 2 rows above the first
    level is five levels of tile reduction before the single-CTA top."""
    need_gpu()
    env("MABD_SEG_UP_T", ut)
    sc = scenes.long_chain(M, seed=2)
    T0 = seg_tile(sc)
    P0 = (M + 1 + T0 - 1) // T0
    want, n = 1, P0
    while n > ut:
        n = (n + ut - 1) // ut
        want += 1
    assert seg_levels(sc) == want
    q, qd = scenes.perturb_state(sc, seed=M + ut, rot=0.05, vel=0.2)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)


@pytest.mark.parametrize("seed", range(6))
def test_seg_random_chains(ora, seed):
    """Random boxes and gaps, balls and hinges, pinned or free ends, joints
    with body a on either side, bodies numbered in any order, rigidly turned
    copies and the printed zero bottom rhs."""
    need_gpu()
    M = [2, 5, 130, 300, 700, 1500][seed]
    sc = scenes.random_small("chain", M, seed=seed, hinge_frac=0.5, pin=seed % 3 != 2)
    if seed % 2:
        sc = flip_joints(sc)
    if seed >= 3:
        sc = permute_bodies(sc, seed)
    assert seg_levels(sc) >= 1
    q, qd = scenes.perturb_state(sc, seed=seed, rot=0.3)
    assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)
    assert_parity(ora, sc, q, qd, tol=TOL, residual_rhs=0, gpu_kw=F32)
    Q = scenes.random_rotations(np.random.default_rng(seed), 1)[0]
    sc2 = scenes.rotate_scene(sc, Q)
    q2, qd2 = scenes.perturb_state(sc2, seed=seed + 50, rot=0.1)
    assert_parity(ora, sc2, q2, qd2, tol=TOL, gpu_kw=F32)


def test_seg_one_sided_ends(ora):
    """A chain pinned at its first body only, one pinned at its last body
    only (the world joint closes the joint order), and a single body held by
    two world joints."""
    need_gpu()
    base = scenes.random_small("chain", 200, seed=9, hinge_frac=0.5)
    keep_first = [k for k in range(len(base["jtype"])) if k != len(base["jtype"]) - 1]
    keep_last = list(range(1, len(base["jtype"])))
    for keep in (keep_first, keep_last):
        sc = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
        for key in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
            sc[key] = base[key][keep]
        assert seg_levels(sc) >= 1
        q, qd = scenes.perturb_state(sc, seed=len(keep), rot=0.2)
        assert_parity(ora, sc, q, qd, tol=TOL, gpu_kw=F32)
    one = scenes.random_small("chain", 1, seed=3)
    two = scenes.concat_scenes([one])
    for key in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        two[key] = np.concatenate([one[key], one[key]])
    two["anchor_a"][1] = -two["anchor_a"][1]
    two["anchor_b"][1] = two["q"][0, 9:12] + two["anchor_a"][1] + 0.01
    assert seg_levels(two) >= 1
    q, qd = scenes.perturb_state(two, seed=2, rot=0.2)
    assert_parity(ora, two, q, qd, tol=TOL, gpu_kw=F32)


def test_seg_matches_level_path(ora, env):
    """The tiled step and the level-by-level reduction of the same form reach
    the same FP64 system's solution."""
    need_gpu()
    sc = scenes.long_chain(5000, seed=5)
    q, qd = scenes.perturb_state(sc, seed=6, rot=0.05, vel=0.2)
    out = {}
    for flag in ("1", "0"):
        env("MABD_CHAIN_SEG", flag)
        s = gpu_solver(sc, **F32)
        try:
            assert (s.info()["seg_levels"] > 0) == (flag == "1")
            out[flag] = gpu_step(s, q, qd)
        finally:
            s.close()
    _, oqd1, olam, _ = oracle_step(ora, sc, q, qd)
    for flag in ("1", "0"):
        assert rel(out[flag][1], oqd1) <= TOL and rel(out[flag][2], olam) <= TOL
    assert rel(out["1"][1], out["0"][1]) <= 2 * TOL
    assert rel(out["1"][2], out["0"][2]) <= 2 * TOL


def test_seg_chain64_trajectory(ora):
    """The 64-cube chain pinned at body 0, from states along a 120-step
    oracle trajectory."""
    need_gpu()
    sc = scenes.chain_cubes(64)
    S = ora.Scene(sc)
    q, qd = sc["q"], sc["qdot"]
    states = []
    for n in range(120):
        if n in (0, 1, 10, 50, 119):
            states.append((q, qd))
        q, qd, _, _ = ora.step(S, q, qd)
    solver = gpu_solver(sc, **F32)
    try:
        assert solver.info()["seg_levels"] == 1
        for q0, qd0 in states:
            _, _, st, _ = assert_parity(ora, sc, q0, qd0, solver=solver, tol=TOL)
            assert st["joint_residual"] < 1e-10
            assert st["refine_residual"] > 0.0 and st["polar_iterations"] >= 1.0
    finally:
        solver.close()


def test_seg_steps_follow_the_oracle(ora):
    """Ten steps in one call (replayed from the step's CUDA graph) against ten
    oracle steps."""
    need_gpu()
    sc = scenes.long_chain(3000, seed=7)
    q, qd = scenes.perturb_state(sc, seed=8, rot=0.05, vel=0.2)
    S = ora.Scene(sc)
    oq, oqd = q, qd
    for _ in range(10):
        oq, oqd, olam, _ = ora.step(S, oq, oqd)
    s = gpu_solver(sc, **F32)
    try:
        s.set_state(q, qd)
        s.step(10)
        q1, qd1 = s.get_state()
        lam = s.get_lambda()
    finally:
        s.close()
    assert rel(qd1, oqd) <= 1e-5 and rel(lam, olam) <= 1e-5


def test_seg_full_size_pulley_chain_perturbed(ora):
    """1,048,576 bodies (two or three tile levels) from a perturbed state, in
    the launch configuration the benchmark times: normwise and per body / per
    joint."""
    need_gpu()
    sc = scenes.long_chain(1 << 20, seed=1)
    assert seg_levels(sc) >= 2
    q, qd = scenes.perturb_state(sc, seed=12, rot=0.02, vel=0.1)
    solver = gpu_solver(sc, **F32)
    try:
        q1, qd1, lam, st = gpu_step(solver, q, qd)
    finally:
        solver.close()
    _, oqd1, olam, ost = oracle_step(ora, sc, q, qd)
    assert rel(qd1, oqd1) <= TOL and rel(lam, olam) <= TOL
    assert_elementwise(sc, qd1, oqd1, lam, olam, tol=1e-5)
    # the perturbed joints do not close in one linearized step: the same
    # nonlinear residual as the oracle's
    assert abs(st[0]["joint_residual"] - ost["joint_residual"]) <= 1e-3 * ost["joint_residual"]


def test_seg_thirty_steps_follow_the_oracle(ora):
    """30 steps of a 20,000-body pulley chain from a moving state (many tiles,
    every level of the tiles' reduction carrying nonzero right-hand sides):
    the state stays with the oracle's trajectory and the joints stay closed
    as the oracle's do."""
    need_gpu()
    sc = scenes.long_chain(20000, seed=3)
    q, qd = scenes.perturb_state(sc, seed=4, rot=0.01, vel=0.3)
    S = ora.Scene(sc)
    oq, oqd = q, qd
    for _ in range(30):
        oq, oqd, olam, ost = ora.step(S, oq, oqd)
    s = gpu_solver(sc, **F32)
    try:
        s.set_state(q, qd)
        s.step(29)
        st = s.step(1, stats=True)[0]
        q1, qd1 = s.get_state()
        lam = s.get_lambda()
    finally:
        s.close()
    assert rel(qd1, oqd) <= 1e-5 and rel(lam, olam) <= 1e-5
    assert st["joint_residual"] <= 2 * ost["joint_residual"] + 1e-12
