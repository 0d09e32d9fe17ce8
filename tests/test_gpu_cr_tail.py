"""GPU parity of the chain's block cyclic reduction with its small levels in
one single-CTA launch per pass (elimination or right-hand-side pass, top
row, back-substitution), against the FP64 CPU oracle.

MABD_CR_TAIL=<rows> moves every level with at most that many rows into the
tail (0: none), for either precision of the reduction; the FP32 reduction
uses the tail by default."""
import os

import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import assert_parity, gpu_solver, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture
def tail_rows():
    old = os.environ.get("MABD_CR_TAIL")

    def set_(v):
        if v is None:
            os.environ.pop("MABD_CR_TAIL", None)
        else:
            os.environ["MABD_CR_TAIL"] = str(v)

    yield set_
    set_(old)


def tail_info(sc, **kw):
    s = gpu_solver(sc, **kw)
    try:
        inf = s.info()
    finally:
        s.close()
    return inf["cr_levels"], inf["cr_tail_level"]


@pytest.mark.parametrize("rows", [1, 2, 5, 64, 1 << 30])
@pytest.mark.parametrize("M", [1, 2, 17, 1000, 4097])
def test_fp64_reduction_with_tail(ora, tail_rows, rows, M):
    """FP64 elimination pass through the tail, from the top row only up to
    the whole chain in one CTA (1e-9)."""
    need_gpu()
    tail_rows(rows)
    sc = scenes.long_chain(M, seed=3)
    nl, l0 = tail_info(sc)
    assert l0 < nl
    q, qd = scenes.perturb_state(sc, seed=M + rows % 97, rot=0.05, vel=0.2)
    assert_parity(ora, sc, q, qd, tol=1e-9)


@pytest.mark.parametrize("rows", [3, 1 << 30])
@pytest.mark.parametrize("M", [2, 255, 4097])
def test_fp64_reduction_rhs_pass_with_tail(ora, tail_rows, rows, M):
    """Mixed form: the FP64 right-hand-side passes of the correction sweeps
    through the tail (1e-6, the mixed form's bound)."""
    need_gpu()
    tail_rows(rows)
    sc = scenes.long_chain(M, seed=5)
    q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.2)
    assert_parity(ora, sc, q, qd, tol=1e-6, gpu_kw={"precision": "mixed", "refine_steps": 2})


@pytest.mark.parametrize("rows", [None, 0, 1, 9, 1 << 30])
@pytest.mark.parametrize("M", [1, 3, 40, 4097, 65537])
def test_fp32_reduction_with_tail(ora, tail_rows, rows, M):
    """FP32 reduction: default bound, tail off, top row only, a small tail
    and the whole chain in one CTA, on chains of mixed joint types."""
    need_gpu()
    if rows == 1 << 30 and M > 4097:
        pytest.skip("one CTA for 2^15 rows per level is covered at 4097")
    tail_rows(rows)
    sc = scenes.long_chain(M, seed=7) if M > 40 else scenes.random_small("chain", M, seed=M, hinge_frac=0.5)
    kw = {"precision": "mixed_fp32_dual"}
    nl, l0 = tail_info(sc, **kw)
    if rows == 0:
        assert l0 == nl
    else:
        assert l0 < nl
    q, qd = scenes.perturb_state(sc, seed=M, rot=0.05, vel=0.2)
    assert_parity(ora, sc, q, qd, tol=1e-6, gpu_kw=kw)
    assert_parity(ora, sc, q, qd, tol=1e-6, residual_rhs=0, gpu_kw=kw)


def test_tail_default_only_for_fp32(tail_rows):
    """Without MABD_CR_TAIL the FP64 reduction launches every level and the
    FP32 reduction starts its tail at the first level of at most 512 rows."""
    need_gpu()
    tail_rows(None)
    sc = scenes.long_chain(100000, seed=1)
    K = len(sc["jtype"])
    nl, l0 = tail_info(sc)
    assert l0 == nl
    nl32, l032 = tail_info(sc, precision="mixed_fp32_dual")
    assert nl32 == nl
    # level sizes halve, rounding up, from K (+ 1 leading identity row)
    for off in (0, 1):
        N, sizes = K + off, []
        while True:
            sizes.append(N)
            if N == 1:
                break
            N = (N + 1) // 2
        if len(sizes) == nl:
            assert l032 == next(l for l, n in enumerate(sizes) if n <= 512)
