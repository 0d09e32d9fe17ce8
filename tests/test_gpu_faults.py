"""Host-side fault injection through the C ABI: calls out of order, invalid
bodies and joints, and a context that stays usable after each non-sticky
error.  Every failure is made on the host (bad arguments, wrong call order);
nothing here faults, traps or stalls the GPU.  A context needs a device,
hence the gpu mark."""
import ctypes as C

import numpy as np
import pytest

from paper_2603_08079_gb300 import mabd, scenes
from parity_util import need_gpu

pytestmark = pytest.mark.gpu

OK, INVALID_ARG, BAD_STATE, NOT_SPD, UNSUPPORTED = 0, 1, 2, 5, 10


class Ctx:
    """A bare context through the C ABI (library allocator, default stream)."""

    def __init__(self, h=1e-2, **cfg_fields):
        self.lib = mabd.load()
        cfg = mabd.Config()
        self.lib.mabd_config_default(C.byref(cfg))
        cfg.h = h
        for k, v in cfg_fields.items():
            setattr(cfg, k, v)
        self.ctx = C.c_void_p()
        assert self.lib.mabd_create(C.byref(cfg), C.byref(self.ctx)) == OK

    def add_bodies(self, b):
        return self.lib.mabd_add_bodies(self.ctx, len(b), b.ctypes.data_as(C.c_void_p), None)

    def add_joints(self, j):
        return self.lib.mabd_add_joints(self.ctx, len(j), j.ctypes.data_as(C.c_void_p), None)

    def prefactor(self):
        return self.lib.mabd_prefactor(self.ctx)

    def step(self, n=1):
        return self.lib.mabd_step(self.ctx, n, None)

    def get_state(self, M):
        q = np.empty((M, 12))
        qd = np.empty((M, 12))
        return self.lib.mabd_get_state(self.ctx, q.ctypes.data_as(C.c_void_p), qd.ctypes.data_as(C.c_void_p))

    def close(self):
        assert self.lib.mabd_destroy(self.ctx) == OK


@pytest.fixture
def chain():
    sc = scenes.long_chain(12, seed=3)
    return sc, mabd.body_array(sc), mabd.joint_array(sc)


def test_call_order(chain):
    need_gpu()
    sc, b, j = chain
    c = Ctx()
    try:
        assert c.step() == BAD_STATE               # step before prefactor
        assert c.add_bodies(b) == OK
        assert c.add_joints(j) == OK
        assert c.step() == BAD_STATE
        assert c.prefactor() == OK
        assert c.add_bodies(b[:1]) == BAD_STATE    # the scene is frozen
        assert c.add_joints(j[:1]) == BAD_STATE
        assert c.prefactor() == BAD_STATE          # only once
        assert c.step(2) == OK                     # still usable
        assert c.get_state(len(b)) == OK
    finally:
        c.close()


BAD_BODIES = [
    ("mass", 0.0, INVALID_ARG), ("mass", -2.0, INVALID_ARG), ("volume", 0.0, INVALID_ARG),
    ("young", 0.0, INVALID_ARG), ("young", -1e8, INVALID_ARG), ("poisson", 0.5, INVALID_ARG),
    ("poisson", 0.7, INVALID_ARG), ("poisson", -0.1, INVALID_ARG), ("mass", np.nan, INVALID_ARG),
    ("q", np.inf, INVALID_ARG), ("qdot", np.nan, INVALID_ARG), ("second_moment", 0.0, INVALID_ARG),
    ("fixed", 2, INVALID_ARG),
]


@pytest.mark.parametrize("field,value,code", BAD_BODIES)
def test_invalid_bodies_are_rejected_and_the_context_stays_usable(chain, field, value, code):
    need_gpu()
    sc, b, j = chain
    bad = b.copy()
    arr = bad[field]
    if arr.ndim > 1:
        arr[5, 0] = value
    else:
        arr[5] = value
    c = Ctx()
    try:
        assert c.add_bodies(bad) == code
        # nothing of the rejected call was kept: the good scene goes through
        assert c.add_bodies(b) == OK
        assert c.add_joints(j) == OK
        assert c.prefactor() == OK
        assert c.step() == OK
    finally:
        c.close()


def test_second_moment_must_be_positive_definite(chain):
    """A non-diagonal second moment is accepted (the body is kept in its
    principal frame); one with a negative principal moment is refused."""
    need_gpu()
    sc, b, j = chain
    bad = b.copy()
    s0 = bad["second_moment"][3, 0]
    bad["second_moment"][3, :] = [s0, s0, s0, 2.0 * s0, 0.0, 0.0]  # eigenvalues 3, -1, 1 (x s0)
    turned = b.copy()
    turned["second_moment"][3, 3] = 0.1 * turned["second_moment"][3, 0]
    c = Ctx()
    try:
        assert c.add_bodies(bad) == INVALID_ARG
        assert c.add_bodies(turned) == OK
        assert c.add_joints(j) == OK
        assert c.prefactor() == OK
        assert c.step() == OK
    finally:
        c.close()


@pytest.mark.parametrize("case", ["tree", "chain", "graph"])
def test_bodies_given_off_their_principal_axes(ora, case):
    """Rest frames turned off the principal axes (non-diagonal second
    moments, turned anchors and axes): the library keeps each body in its
    principal frame and returns states in the caller's frame.  Parity with
    the oracle, which takes the second moments as given, and with the same
    scene given in principal frames."""
    need_gpu()
    from parity_util import assert_parity, gpu_solver, gpu_step, rel
    if case == "tree":
        sc0 = scenes.random_tree(200, seed=2, joint="mixed")
    elif case == "chain":
        sc0 = scenes.random_small("chain", 30, seed=5)
    else:
        sc0 = scenes.random_small("graph", 20, seed=1, univ_frac=0.3, prism_frac=0.3)
    sc = scenes.turn_rest_frames(sc0, seed=3)
    tr = sc["second_moment"][:, :3].sum(axis=1)
    assert np.all(np.abs(sc["second_moment"][:, 3:]).max(axis=1) > 1e-3 * tr)
    q, qd = scenes.perturb_state(sc, seed=4, rot=0.1, vel=0.3)
    # the graph's dual has cond(S) = 2.5e5: the 1e-9 bound scaled beyond 1e5
    tol = 1e-9 if case != "graph" else 3e-9
    assert_parity(ora, sc, q, qd, tol=tol, gpu_kw={"pcg_max_iters": 20000})
    if case != "graph":
        assert_parity(ora, sc, q, qd, tol=1e-6, gpu_kw={"precision": "mixed_fp32_dual"})
    # the same state in the principal frames of sc0 (A Q^T -> A)
    Q = scenes.random_rotations(np.random.default_rng(3), len(q))
    q0, qd0 = q.copy(), qd.copy()
    for k in range(len(q)):
        q0[k, :9] = (q[k, :9].reshape(3, 3).T @ Q[k]).T.reshape(9)
        qd0[k, :9] = (qd[k, :9].reshape(3, 3).T @ Q[k]).T.reshape(9)
    s, s0 = gpu_solver(sc, pcg_max_iters=20000), gpu_solver(sc0, pcg_max_iters=20000)
    try:
        _, qd1, lam, _ = gpu_step(s, q, qd)
        _, qd01, lam0, _ = gpu_step(s0, q0, qd0)
        s.set_state(q, qd)
        qr, qdr = s.get_state()
    finally:
        s.close()
        s0.close()
    np.testing.assert_allclose(qr, q, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(qdr, qd, rtol=1e-13, atol=1e-13)
    back = qd1.copy()
    for k in range(len(q)):
        back[k, :9] = (qd1[k, :9].reshape(3, 3).T @ Q[k]).T.reshape(9)
    assert rel(back, qd01) < tol and rel(lam, lam0) < tol


@pytest.mark.parametrize("case", ["a_out_of_range", "b_out_of_range", "negative", "same_body",
                                  "two_fixed"])
def test_invalid_joint_ids_fail_at_prefactor(chain, case):
    need_gpu()
    sc, b, j = chain
    bodies = b.copy()
    bad = j.copy()
    M = len(b)
    if case == "a_out_of_range":
        bad["body_a"][4] = M
    elif case == "b_out_of_range":
        bad["body_b"][4] = M + 7
    elif case == "negative":
        bad["body_a"][4] = -3
    elif case == "same_body":
        bad["body_b"][4] = bad["body_a"][4]
    else:
        bodies["fixed"][4] = bodies["fixed"][5] = 1
        bad["body_a"][5], bad["body_b"][5] = 4, 5
    c = Ctx()
    try:
        assert c.add_bodies(bodies) == OK
        assert c.add_joints(bad) == OK             # ids are checked when the scene is frozen
        assert c.prefactor() == INVALID_ARG
        assert c.step() == BAD_STATE               # not frozen by the failed prefactor
    finally:
        c.close()


def test_invalid_joint_descriptions(chain):
    need_gpu()
    sc, b, j = chain
    h = int(np.nonzero(sc["jtype"] == 1)[0][0])
    for field, value in (("axis_a", 0.0), ("axis_len", 0.0), ("axis_len", np.inf), ("anchor_b", np.nan),
                         ("type", 7)):
        bad = j.copy()
        arr = bad[field]
        if arr.ndim > 1:
            arr[h, :] = value
        else:
            arr[h] = value
        c = Ctx()
        try:
            assert c.add_bodies(b) == OK
            assert c.add_joints(bad) == INVALID_ARG, field
            assert c.add_joints(j) == OK
            assert c.prefactor() == OK
            assert c.step() == OK
        finally:
            c.close()


def test_overflowing_body_is_not_spd(chain):
    """A mass so small that h^2/m overflows leaves Hbar^{-1} non-finite:
    NOT_SPD at prefactor, on the host, before any step."""
    need_gpu()
    sc, b, j = chain
    bad = b.copy()
    bad["mass"][2] = 1e-320
    c = Ctx()
    try:
        assert c.add_bodies(bad) == OK
        assert c.add_joints(j) == OK
        assert c.prefactor() == NOT_SPD
    finally:
        c.close()


def test_solver_topology_mismatch_is_unsupported():
    need_gpu()
    sc = scenes.random_small("tree", 9, seed=1)
    c = Ctx(solver=1)                              # the chain solver on a tree
    try:
        assert c.add_bodies(mabd.body_array(sc)) == OK
        assert c.add_joints(mabd.joint_array(sc)) == OK
        assert c.prefactor() == UNSUPPORTED
    finally:
        c.close()
