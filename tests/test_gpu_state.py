"""State transfer through the C ABI (mabd_set_state / mabd_get_state) with
pageable and page-locked host arrays (aligned and not): the same state,
non-finite input rejected without touching the device state, bit-exact
round trips."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes
from parity_util import gpu_solver, need_gpu

pytestmark = pytest.mark.gpu


def pinned(shape):
    import torch
    return torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()


@pytest.mark.parametrize("topo", ["chain", "tree", "graph"])
def test_pinned_and_pageable_round_trips(topo):
    need_gpu()
    from paper_2603_08079_gb300 import mabd
    sc = scenes.random_small(topo, 37, seed=5)
    q, qd = scenes.perturb_state(sc, seed=2, rot=0.3, vel=0.5)
    s = gpu_solver(sc)
    try:
        M = len(sc["mass"])
        pq, pqd = pinned((M, 12)), pinned((M, 12))
        pq[:], pqd[:] = q, qd
        s.set_state(pq, pqd)
        a, b = s.get_state()                 # pageable out
        np.testing.assert_array_equal(a, q)
        np.testing.assert_array_equal(b, qd)
        oq, oqd = pinned((M, 12)), pinned((M, 12))
        s.get_state(oq, oqd)                 # pinned out
        np.testing.assert_array_equal(oq, q)
        np.testing.assert_array_equal(oqd, qd)
        # a step from pinned input equals a step from pageable input
        s.set_state(pq, pqd)
        s.step(1)
        s.get_state(oq, oqd)
        s.set_state(q, qd)
        s.step(1)
        a, b = s.get_state()
        np.testing.assert_array_equal(oq, a)
        np.testing.assert_array_equal(oqd, b)
        # non-finite pinned input: rejected, state unchanged
        bad = pinned((M, 12))
        bad[:] = q
        bad[3, 5] = np.nan
        with pytest.raises(mabd.MabdError) as e:
            s.set_state(bad, pqd)
        assert e.value.code == 1
        c, d = s.get_state()
        np.testing.assert_array_equal(c, a)
        np.testing.assert_array_equal(d, b)
    finally:
        s.close()


def test_unaligned_pinned_view():
    """A pinned array viewed at an 8-byte offset (not 16-byte aligned)."""
    need_gpu()
    sc = scenes.random_small("chain", 9, seed=1)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.2, vel=0.2)
    s = gpu_solver(sc)
    try:
        M = len(sc["mass"])
        buf = pinned(12 * M + 1)
        view = buf[1:].reshape(M, 12)
        view[:] = q
        s.set_state(view, qd)
        a, _ = s.get_state()
        np.testing.assert_array_equal(a, q)
        out = pinned(12 * M + 1)
        ov = out[1:].reshape(M, 12)
        s.get_state(ov, None)
        np.testing.assert_array_equal(ov, q)
    finally:
        s.close()
