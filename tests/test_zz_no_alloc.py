"""mabd_chain_step_noalloc: the chain step for callers that cannot allocate
device memory (their intermediates live in the library's fixed device
array).  Checked against the allocating mabd_step and against the FP64 CPU
oracle on the same chains and states, two calls in a row, through the C
ABI; and every class of invalid input it must reject.  Collected last on
purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2603_08079_gb300 import mabd, scenes
from parity_util import need_gpu, rel

pytestmark = pytest.mark.gpu

TOL = 1e-9  # the FP64 parity tolerance used by every GPU test


def _lib():
    lib = mabd.load()
    P = C.c_void_p
    lib.mabd_chain_step_noalloc.argtypes = [C.POINTER(mabd.Config), C.c_int32, P, C.c_int32, P, P, P, P]
    lib.mabd_chain_step_noalloc.restype = C.c_int32
    return lib


def _cfg(lib, sc, stream):
    cfg = mabd.Config()
    lib.mabd_config_default(C.byref(cfg))
    cfg.h = float(sc["h"])
    for i in range(3):
        cfg.gravity[i] = float(sc["gravity"][i])
    cfg.stream = C.c_void_p(stream.cuda_stream)
    return cfg


def _noalloc_step(lib, sc, q, qd, torch):
    """One call: the caller owns inputs and outputs (device tensors)."""
    st = dict(sc, q=q, qdot=qd)
    b = mabd.body_array(st)
    j = mabd.joint_array(sc)
    M, K = len(b), len(j)
    rows = scenes.dual_rows(sc)
    db = torch.from_numpy(b.view(np.uint8).copy()).cuda()
    dj = torch.from_numpy(j.view(np.uint8).copy()).cuda()
    dq = torch.empty(12 * M, dtype=torch.float64, device="cuda")
    dqd = torch.empty(12 * M, dtype=torch.float64, device="cuda")
    dl = torch.empty(max(rows, 1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    cfg = _cfg(lib, sc, stream)
    code = lib.mabd_chain_step_noalloc(C.byref(cfg), M, db.data_ptr(), K, dj.data_ptr(),
                                       dq.data_ptr(), dqd.data_ptr(), dl.data_ptr())
    assert code == 0, mabd.STATUS.get(code, code)
    return dq.cpu().numpy().reshape(M, 12), dqd.cpu().numpy().reshape(M, 12), dl.cpu().numpy()[:rows]


def _drop_joints(sc, keep):
    out = dict(sc)
    for k in ("jtype", "body_a", "body_b", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
        out[k] = sc[k][keep]
    return out


def _scene(which):
    if which == "chain64":
        return scenes.chain_cubes(64)                     # one pin, ball joints
    if which == "pulley257":
        return scenes.long_chain(257, seed=1)             # both pins, ball / hinge
    if which == "pulley4096":
        return scenes.long_chain(4096, seed=1)            # the largest chain it takes
    if which == "right_pin":
        sc = scenes.long_chain(200, seed=4)               # only the last body pinned
        return _drop_joints(sc, list(range(1, len(sc["jtype"]))))
    return scenes.random_small("chain", 31, seed=2, pin=False)  # no pin


@pytest.mark.parametrize("which", ["chain64", "pulley257", "pulley4096", "free31", "right_pin"])
def test_noalloc_step_matches_mabd_step(ora, which):
    torch = need_gpu()
    lib = _lib()
    sc = _scene(which)
    q, qd = scenes.perturb_state(sc, seed=9, rot=0.05, vel=0.2)
    ref = mabd.Solver(sc)
    S = ora.Scene(sc)
    try:
        for call in range(2):                           # two calls in a row
            ref.set_state(q, qd)
            ref.step(1)
            rq, rqd = ref.get_state()
            rlam = ref.get_lambda()
            nq, nqd, nlam = _noalloc_step(lib, sc, q, qd, torch)
            assert rel(nqd, rqd) <= TOL, (call, rel(nqd, rqd))
            assert rel(nlam, rlam) <= TOL, (call, rel(nlam, rlam))
            assert rel(nq, rq) <= TOL
            oq, oqd, olam, _ = ora.step(S, q, qd)       # and the FP64 oracle from the same state
            assert rel(nqd, oqd) <= TOL, (call, rel(nqd, oqd))
            assert rel(nlam, olam) <= TOL, (call, rel(nlam, olam))
            q, qd = nq, nqd                             # the next call starts from this output
    finally:
        ref.close()


BAD_BODY = [("mass", np.inf), ("mass", np.nan), ("volume", np.inf), ("young", np.inf),
            ("second_moment", np.nan), ("q", np.nan), ("qdot", np.inf), ("mass", -1.0),
            ("poisson", 0.5)]
BAD_JOINT = [("anchor_a", np.nan), ("anchor_b", np.inf), ("axis_a", np.nan), ("axis_b", np.inf),
             ("axis_len", np.inf)]


@pytest.mark.parametrize("field,value", BAD_BODY + BAD_JOINT)
def test_noalloc_rejects_invalid_values(field, value):
    """Each class of value that mabd_add_bodies / mabd_add_joints reject is
    rejected here too (INVALID_ARG), not carried into the step."""
    torch = need_gpu()
    lib = _lib()
    sc = scenes.long_chain(9, seed=3)                 # balls and hinges, both pins
    b = mabd.body_array(sc)
    j = mabd.joint_array(sc)
    if (field, value) in BAD_BODY:
        arr = b[field]
        if arr.ndim > 1:
            arr[4, 0] = value
        else:
            arr[4] = value
    else:
        k = int(np.nonzero(sc["jtype"] == 1)[0][0])   # a hinge (it has an axis length)
        arr = j[field]
        if arr.ndim > 1:
            arr[k, 1] = value
        else:
            arr[k] = value
    stream = torch.cuda.current_stream()
    db = torch.from_numpy(b.view(np.uint8).copy()).cuda()
    dj = torch.from_numpy(j.view(np.uint8).copy()).cuda()
    out = torch.zeros(12 * len(b) + 64, dtype=torch.float64, device="cuda")
    code = lib.mabd_chain_step_noalloc(C.byref(_cfg(lib, sc, stream)), len(b), db.data_ptr(), len(j),
                                       dj.data_ptr(), out.data_ptr(), out.data_ptr(), out.data_ptr())
    assert code == 1, (field, value, code)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    torch = need_gpu()
    lib = _lib()
    M = 4097
    stream = torch.cuda.current_stream()
    sc = scenes.chain_cubes(2)
    cfg = _cfg(lib, sc, stream)
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    assert lib.mabd_chain_step_noalloc(C.byref(cfg), M, p, M, p, p, p, p) == 1
    # a joint list that is not in path order is rejected too
    sc = scenes.chain_cubes(8)
    j = mabd.joint_array(sc)
    j["body_a"][3], j["body_b"][3] = 5, 6
    b = mabd.body_array(sc)
    db = torch.from_numpy(b.view(np.uint8).copy()).cuda()
    dj = torch.from_numpy(j.view(np.uint8).copy()).cuda()
    out = torch.empty(12 * 8 + 64, dtype=torch.float64, device="cuda")
    code = lib.mabd_chain_step_noalloc(C.byref(_cfg(lib, sc, stream)), 8, db.data_ptr(), 8,
                                       dj.data_ptr(), out.data_ptr(), out.data_ptr(), out.data_ptr())
    assert code == 1
