"""Pins of the learned-preconditioner oracle (oracle/lpc.py), CPU only."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes


@pytest.fixture(scope="module")
def lpc(ora):
    from oracle import lpc as L
    return L


@pytest.fixture(scope="module")
def small_system(ora, lpc):
    sc = scenes.jittered_net(3, 3, 3, seed=7)
    q, qd = scenes.perturb_state(sc, seed=3, rot=0.2, vel=0.1)
    S = lpc.dual_dense(sc, q, qd)
    ent, ones = lpc.joint_graph(sc)
    C, St = lpc.normalized(S)
    E = lpc.blocks(St, ent)
    return sc, S, C, St, E, ent, ones


def test_bf16_rounding_cases(lpc):
    """Round to nearest bfloat16 (8 significant bits), ties to even."""
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -(1 + 3 * 2 ** -8),
                  3.0, 2.0 ** -130, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -(1 + 2 ** -6), 3.0, 2.0 ** -130, 0.0])
    np.testing.assert_array_equal(lpc.bf16(x), want)
    v = np.random.default_rng(0).standard_normal(1000)
    r = lpc.bf16(v)
    assert np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8 * (1 + 1e-12))


def test_normalized_dual(small_system, lpc):
    """Unit diagonal blocks, E_nk = E_kn^T, zero blocks between joints that
    share no free body."""
    sc, S, C, St, E, ent, ones = small_system
    K = len(ent)
    for k in range(K):
        np.testing.assert_allclose(St[3 * k:3 * k + 3, 3 * k:3 * k + 3], np.eye(3), atol=1e-12)
    adj = np.zeros((K, K), dtype=bool)
    for k in range(K):
        for (n, _, _, _) in ent[k]:
            adj[k, n] = True
    for k in range(K):
        for n in range(K):
            blk = St[3 * k:3 * k + 3, 3 * n:3 * n + 3]
            if n != k and not adj[k, n]:
                assert np.max(np.abs(blk)) < 1e-12
            elif adj[k, n]:
                np.testing.assert_allclose(blk, St[3 * n:3 * n + 3, 3 * k:3 * k + 3].T, atol=1e-12)


def test_block_jacobi_special_case(small_system, lpc):
    """alpha = 0 and s = 1 (zero heads, a very negative gate offset) leave
    G = I: the loss is |S~ V - V|^2 / N and M^{-1} is blockdiag(D_k^{-1})."""
    sc, S, C, St, E, ent, ones = small_system
    p = lpc.unpack(scenes.lpc_init_params(1).astype(np.float64))
    p["Wa"][:] = 0.0
    p["Wb"][:] = 0.0
    p["we"][:] = 0.0
    p["ce"][:] = -60.0
    p["wd"][:] = 0.0
    p["cd"][:] = 0.0
    theta = lpc.pack(p)
    V = scenes.lpc_probe(2, len(ent), seed=5).astype(np.float64)
    Vm = V.reshape(2, -1).T
    want = np.sum((St @ Vm - Vm) ** 2) / Vm.size
    assert abs(lpc.loss(theta, St, E, ent, ones, V, kind="frobenius") - want) <= 1e-12 * want
    # Kaporin: log(tr(V^T S~ V) / N) with s = 1; with many probes tr(V^T S~ V)/N
    # tends to tr(S~)/n = 1 (unit diagonal blocks), so the loss tends to 0
    wantk = np.log(np.sum(Vm * (St @ Vm)) / Vm.size)
    assert abs(lpc.loss(theta, St, E, ent, ones, V, kind="kaporin") - wantk) <= 1e-12 * max(1.0, abs(wantk))
    Vmany = scenes.lpc_probe(4000, len(ent), seed=8).astype(np.float64)
    assert abs(lpc.loss(theta, St, E, ent, ones, Vmany, kind="kaporin")) < 0.02
    Minv = lpc.preconditioner(theta, S, ent, ones)
    K = len(ent)
    Dinv = np.zeros_like(S)
    for k in range(K):
        Dinv[3 * k:3 * k + 3, 3 * k:3 * k + 3] = np.linalg.inv(S[3 * k:3 * k + 3, 3 * k:3 * k + 3])
    np.testing.assert_allclose(Minv, Dinv, rtol=1e-10, atol=1e-10 * np.max(np.abs(Dinv)))


@pytest.mark.parametrize("kind", ["frobenius", "kaporin"])
def test_gradient_by_finite_differences(small_system, lpc, kind):
    """Central differences of the loss (FP64 network, no bf16 rounding)
    against the dense backpropagation, coordinate by coordinate."""
    sc, S, C, St, E, ent, ones = small_system
    theta = scenes.lpc_init_params(2).astype(np.float64)
    p = lpc.unpack(theta)
    rng = np.random.default_rng(4)
    p["Wa"][:] = rng.standard_normal(p["Wa"].shape) * 0.3
    p["Wb"][:] = rng.standard_normal(p["Wb"].shape) * 0.3
    p["wd"][:] = rng.standard_normal(p["wd"].shape) * 0.05
    p["we"][:] = [0.3, -0.2]
    theta = lpc.pack(p)
    V = scenes.lpc_probe(2, len(ent), seed=6).astype(np.float64)
    L0, g = lpc.loss_grad(theta, St, E, ent, ones, V, use_bf16=False, kind=kind)
    assert abs(L0 - lpc.loss(theta, St, E, ent, ones, V, use_bf16=False, kind=kind)) <= 1e-13 * abs(L0)
    # every head parameter, and samples of each layer's weights and biases
    offs, o = {}, 0
    for name, shape in lpc.SIZES:
        offs[name] = (o, o + int(np.prod(shape)))
        o += int(np.prod(shape))
    idx = list(range(offs["Wa"][0], lpc.NPARAM))
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        lo, hi = offs[name]
        idx += list(rng.choice(np.arange(lo, hi), size=12, replace=False))
    checked = 0
    for i in idx:
        eps = 1e-6 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (lpc.loss(tp, St, E, ent, ones, V, use_bf16=False, kind=kind) -
              lpc.loss(tm, St, E, ent, ones, V, use_bf16=False, kind=kind)) / (2 * eps)
        assert abs(fd - g[i]) <= 2e-5 * max(abs(fd), 1e-3 * np.max(np.abs(g))), (i, fd, g[i])
        checked += 1
    assert checked > 150


def test_preconditioner_is_spd_and_pcg_solves(small_system, lpc):
    """For random parameters M^{-1} is symmetric positive definite, and CG
    preconditioned with it reaches the exact dual solution."""
    sc, S, C, St, E, ent, ones = small_system
    for seed in range(3):
        theta = scenes.lpc_init_params(seed).astype(np.float64)
        p = lpc.unpack(theta)
        p["Wa"][:] = np.random.default_rng(seed).standard_normal(p["Wa"].shape)
        p["Wb"][:] = np.random.default_rng(seed + 9).standard_normal(p["Wb"].shape)
        Minv = lpc.preconditioner(lpc.pack(p), S, ent, ones)
        np.testing.assert_allclose(Minv, Minv.T, atol=1e-12 * np.max(np.abs(Minv)))
        assert np.min(np.linalg.eigvalsh(Minv)) > 0.0
        b = np.random.default_rng(seed).standard_normal(S.shape[0])
        x = np.zeros_like(b)
        r = b.copy()
        z = Minv @ r
        d = z.copy()
        rz = r @ z
        for _ in range(10 * len(b)):
            Sd = S @ d
            a = rz / (d @ Sd)
            x += a * d
            r -= a * Sd
            if np.linalg.norm(r) <= 1e-13 * np.linalg.norm(b):
                break
            z = Minv @ r
            rz, rz_old = r @ z, rz
            d = z + (rz / rz_old) * d
        np.testing.assert_allclose(x, np.linalg.solve(S, b), rtol=1e-9, atol=1e-9 * np.linalg.norm(x))
