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


def _path_graph(K, seed):
    """A path of K joints (joint k shares body k+1 with joint k+1) with random
    coupling blocks E_k,k+1 = B, E_k+1,k = B^T, the first joint one-sided."""
    rng = np.random.default_rng(seed)
    ent = [[] for _ in range(K)]
    E = [[] for _ in range(K)]
    for k in range(K - 1):
        B = rng.standard_normal((3, 3)) * 0.3
        ent[k].append((k + 1, k + 1, 1, 0))
        E[k].append(B)
        ent[k + 1].insert(0, (k, k + 1, 0, 1))
        E[k + 1].insert(0, B.T.copy())
    ones = np.zeros(K, dtype=bool)
    ones[0] = True
    return E, ent, ones


def _net_params(lpc, seed):
    p = lpc.unpack(scenes.lpc_init_params(seed).astype(np.float64))
    rng = np.random.default_rng(seed + 100)
    p["Wa"][:] = rng.standard_normal(p["Wa"].shape) * 0.3
    p["Wb"][:] = rng.standard_normal(p["Wb"].shape) * 0.3
    p["wd"][:] = rng.standard_normal(p["wd"].shape) * 0.1
    for l in (1, 2, 3):
        p["b%d" % l][:] = rng.standard_normal(p["b%d" % l].shape) * 0.1
    return lpc.pack(p)


@pytest.mark.parametrize("use_bf16", [False, True])
def test_network_is_local(lpc, use_bf16):
    """Three mean-aggregation layers over features of one-hop blocks: a
    joint's state, scale and gates depend on the coupling blocks within four
    hops only.  Changing a block six hops away leaves them bit-identical,
    while the joints next to that block change (a global or mis-indexed
    aggregation would break the first, a dropped one the second)."""
    K = 24
    E, ent, ones = _path_graph(K, seed=1)
    theta = _net_params(lpc, 3)
    base = lpc.forward(theta, E, ent, ones, use_bf16=use_bf16)
    E2 = [[b.copy() for b in row] for row in E]
    B = np.random.default_rng(9).standard_normal((3, 3))
    E2[16][1] = B            # block (16, 17)
    E2[17][0] = B.T.copy()   # block (17, 16)
    pert = lpc.forward(theta, E2, ent, ones, use_bf16=use_bf16)
    for k in range(K):
        far = min(abs(k - 16), abs(k - 17)) >= 6
        same = np.array_equal(base["h3"][k], pert["h3"][k]) and base["s"][k] == pert["s"][k]
        if far:
            assert same, k
            for i, (n, _, _, _) in enumerate(ent[k]):
                if n < k:
                    assert base["alpha"][(k, i)] == pert["alpha"][(k, i)]
        elif k in (15, 16, 17, 18):
            assert not same, k


def test_network_acts_per_component(lpc):
    """Two disjoint graphs numbered one after the other give the outputs of
    each graph alone (no message crosses between components, and the
    lower-neighbour features keep their order)."""
    E1, ent1, ones1 = _path_graph(7, seed=2)
    E2, ent2, ones2 = _path_graph(11, seed=3)
    off = len(ent1)
    ent = ent1 + [[(n + off, j + off, s, t) for (n, j, s, t) in row] for row in ent2]
    E = E1 + E2
    ones = np.concatenate([ones1, ones2])
    theta = _net_params(lpc, 4)
    both = lpc.forward(theta, E, ent, ones, use_bf16=False)
    a = lpc.forward(theta, E1, ent1, ones1, use_bf16=False)
    b = lpc.forward(theta, E2, ent2, ones2, use_bf16=False)
    np.testing.assert_allclose(both["h3"], np.vstack([a["h3"], b["h3"]]), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(both["s"], np.concatenate([a["s"], b["s"]]), rtol=1e-13)
    for (k, i), v in a["alpha"].items():
        assert abs(both["alpha"][(k, i)] - v) <= 1e-13
    for (k, i), v in b["alpha"].items():
        assert abs(both["alpha"][(k + off, i)] - v) <= 1e-13
