"""Learned block preconditioner of the dual PCG: the plain CPU definition.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): the tests, `smoke()`
and the benchmark's CPU legs may use it; the library never does.

The paper has no learned part; this extends its dual solve for closed loops
and irregular networks (Sec. 5.5, Eq. dual).  What is computed, in FP64 and
with dense matrices (small systems only):

* the dual S = sum over free bodies j of G_j H_j^{-1} G_j^T, from the
  oracle's own dense assembly (H_j and G in world coordinates);
* D_k the 3x3 diagonal blocks, C_k = L_k^{-1} for D_k = L_k L_k^T, and the
  normalized dual S~ = C S C^T; E_kn = S~_kn for joints sharing a free body;
* features of joint k (in this order): 1, degree/8, lower degree/8,
  one-sided flag, sum |E_kn|_F^2, max |E_kn|_F, sum tr E_kn, sum over
  lower neighbours n < k of |E_kn|_F^2;
* three layers h' = relu([r(h), r(mean_{n~k} h_n)] r(W) + b) where r() rounds
  to bfloat16 (round to nearest even) when `bf16` is set, as the GPU feeds
  its tensor cores;
* heads s_k = exp(clip(wd.h_k + cd, -8, 8)), a = h Wa, b = h Wb,
  alpha_kn = 1.5 sigmoid(a_k.b_n + we0 |E_kn|_F + we1 tr E_kn + ce) for n < k;
* G = diag(s)(I - A), A_kn = alpha_kn E_kn (n < k); M^{-1} = C^T G^T G C;
* with X = G S~ G^T, n = 3K and probe vectors V (nv columns): the Frobenius
  objective L = |X V - V|_F^2 / (nv n), or Kaporin's objective
  L = log(tr(V^T X V) / (nv n)) - (2/K) sum_k log s_k (the log of Kaporin's
  condition number (tr X / n)^n / det X, per row and up to the constant
  log det S~ / n; det G = prod s_k^3 since G is block triangular);
* the gradient with respect to every parameter by dense backpropagation
  (dL/dG = (D V^T + V D^T) G S~ with D = dL/dY, Y = X V; the GPU uses the
  sparse chain rule instead).

The paper prints no values for this part (the network design is this
project's reading); the tests pin this module against the mathematics
instead: finite differences of the loss for every parameter, the
block-Jacobi special case (zero heads and a closed gate leave G = I, so
M^{-1} is the inverse of the diagonal blocks), the symmetry and
definiteness of M^{-1}, and the network's structure (outputs depend on the
coupling blocks within four hops only; disjoint graphs are processed
independently).
"""
from __future__ import annotations

import numpy as np

from . import Scene, assemble_dense

F, H, R = 8, 64, 8
SIZES = (("W1", (2 * F, H)), ("b1", (H,)), ("W2", (2 * H, H)), ("b2", (H,)),
         ("W3", (2 * H, H)), ("b3", (H,)), ("Wa", (H, R)), ("Wb", (H, R)),
         ("wd", (H,)), ("cd", (1,)), ("we", (2,)), ("ce", (1,)))
NPARAM = int(sum(np.prod(s) for _, s in SIZES))


def unpack(theta) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even), through float32."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# the normalized dual and its joint graph
# ---------------------------------------------------------------------------
def joint_graph(sc: dict):
    """Adjacency of joints sharing a free body: per joint a list of
    (neighbour, body, own side, neighbour side), sorted by (neighbour, body);
    and the one-sided flags."""
    K = len(sc["jtype"])
    fixed = np.asarray(sc["fixed"]) != 0
    inc: dict[int, list] = {}
    ones = np.zeros(K, dtype=bool)
    for k in range(K):
        a, b = int(sc["body_a"][k]), int(sc["body_b"][k])
        nfree = 0
        if not fixed[a]:
            inc.setdefault(a, []).append((k, 0))
            nfree += 1
        if b >= 0 and not fixed[b]:
            inc.setdefault(b, []).append((k, 1))
            nfree += 1
        ones[k] = nfree == 1
    ent = [[] for _ in range(K)]
    for j, lst in inc.items():
        for k, s in lst:
            for n, t in lst:
                if n != k:
                    ent[k].append((n, j, s, t))
    for k in range(K):
        ent[k].sort(key=lambda e: (e[0], e[1]))
    return ent, ones


def dual_dense(sc: dict, q, qd) -> np.ndarray:
    """S = sum over free bodies of G_j H_j^{-1} G_j^T (3K x 3K, ball joints)."""
    S_ = Scene(sc)
    Hw, f, G, c = assemble_dense(S_, q, qd)
    n = G.shape[0]
    S = np.zeros((n, n))
    fixed = np.asarray(sc["fixed"]) != 0
    for j in range(len(sc["mass"])):
        if fixed[j]:
            continue
        Gj = G[:, 12 * j:12 * j + 12]
        if not np.any(Gj):
            continue
        S += Gj @ np.linalg.solve(Hw[j], Gj.T)
    return 0.5 * (S + S.T)


def normalized(S: np.ndarray):
    """C (3K x 3K block diagonal of the inverse lower Cholesky factors) and
    S~ = C S C^T."""
    n = S.shape[0]
    K = n // 3
    C = np.zeros_like(S)
    for k in range(K):
        L = np.linalg.cholesky(S[3 * k:3 * k + 3, 3 * k:3 * k + 3])
        C[3 * k:3 * k + 3, 3 * k:3 * k + 3] = np.linalg.inv(L)
    return C, C @ S @ C.T


def blocks(St: np.ndarray, ent) -> list:
    """E_kn for every adjacency entry (in the graph's order)."""
    return [[St[3 * k:3 * k + 3, 3 * n:3 * n + 3] for (n, _, _, _) in ent[k]] for k in range(len(ent))]


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def features(E, ent, ones) -> np.ndarray:
    K = len(ent)
    x = np.zeros((K, F))
    for k in range(K):
        n2 = [float(np.sum(e * e)) for e in E[k]]
        x[k, 0] = 1.0
        x[k, 1] = len(ent[k]) / 8.0
        lower = [i for i, e in enumerate(ent[k]) if e[0] < k]
        x[k, 2] = len(lower) / 8.0
        x[k, 3] = 1.0 if ones[k] else 0.0
        x[k, 4] = sum(n2)
        x[k, 5] = max([np.sqrt(v) for v in n2], default=0.0)
        x[k, 6] = sum(float(np.trace(e)) for e in E[k])
        x[k, 7] = sum(n2[i] for i in lower)
    return x


def mean_operator(ent) -> np.ndarray:
    K = len(ent)
    Nm = np.zeros((K, K))
    for k in range(K):
        d = len(ent[k])
        for (n, _, _, _) in ent[k]:
            Nm[k, n] += 1.0 / d
    return Nm


def forward(theta, E, ent, ones, use_bf16: bool = True) -> dict:
    p = unpack(theta)
    r = bf16 if use_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    Nm = mean_operator(ent)
    x = features(E, ent, ones)
    cache = {"x": x, "Nm": Nm}
    h = x
    for l in (1, 2, 3):
        A = np.concatenate([r(h), r(Nm @ h)], axis=1)
        W = r(p["W%d" % l])
        pre = A @ W + p["b%d" % l]
        cache["A%d" % l], cache["Wr%d" % l], cache["pre%d" % l] = A, W, pre
        h = np.maximum(pre, 0.0)
        cache["h%d" % l] = h
    d = h @ p["wd"] + p["cd"][0]
    s = np.exp(np.clip(d, -8.0, 8.0))
    a, b = h @ p["Wa"], h @ p["Wb"]
    K = len(ent)
    alpha = {}
    for k in range(K):
        for i, (n, _, _, _) in enumerate(ent[k]):
            if n < k:
                e = E[k][i]
                z = a[k] @ b[n] + p["we"][0] * np.sqrt(np.sum(e * e)) + p["we"][1] * np.trace(e) + p["ce"][0]
                alpha[(k, i)] = 1.5 / (1.0 + np.exp(-z))
    cache.update(d=d, s=s, a=a, b=b, alpha=alpha)
    return cache


def G_matrix(cache, E, ent) -> np.ndarray:
    """G = diag(s)(I - A) as a dense 3K x 3K matrix."""
    K = len(ent)
    A = np.zeros((3 * K, 3 * K))
    for (k, i), al in cache["alpha"].items():
        n = ent[k][i][0]
        A[3 * k:3 * k + 3, 3 * n:3 * n + 3] += al * E[k][i]
    return np.repeat(cache["s"], 3)[:, None] * (np.eye(3 * K) - A), A


def _objective(kind: str, Y, Vm, s, K):
    if kind == "frobenius":
        return float(np.sum((Y - Vm) ** 2) / Vm.size)
    return float(np.log(np.sum(Vm * Y) / Vm.size) - 2.0 / K * np.sum(np.log(s)))


def loss(theta, St, E, ent, ones, V, use_bf16: bool = True, kind: str = "kaporin") -> float:
    """V: probe vectors [nv][K][3]."""
    cache = forward(theta, E, ent, ones, use_bf16)
    G, _ = G_matrix(cache, E, ent)
    Vm = np.asarray(V, dtype=np.float64).reshape(V.shape[0], -1).T
    Y = G @ St @ G.T @ Vm
    return _objective(kind, Y, Vm, cache["s"], len(ent))


def loss_grad(theta, St, E, ent, ones, V, use_bf16: bool = True, kind: str = "kaporin"):
    """Loss and its gradient (a flat vector in the parameter layout)."""
    p = unpack(theta)
    cache = forward(theta, E, ent, ones, use_bf16)
    G, A = G_matrix(cache, E, ent)
    K = len(ent)
    Vm = np.asarray(V, dtype=np.float64).reshape(V.shape[0], -1).T
    Y = G @ St @ G.T @ Vm
    s = cache["s"]
    L = _objective(kind, Y, Vm, s, K)
    if kind == "frobenius":
        D = 2.0 * (Y - Vm) / Vm.size
    else:
        D = Vm / np.sum(Vm * Y)
    dG = (D @ Vm.T + Vm @ D.T) @ G @ St
    IA = np.eye(3 * K) - A
    ds = np.array([np.sum(dG[3 * k:3 * k + 3] * IA[3 * k:3 * k + 3]) for k in range(K)])
    if kind != "frobenius":
        ds = ds - 2.0 / (K * s)
    dA = -np.repeat(s, 3)[:, None] * dG
    g = {name: np.zeros(shape) for name, shape in SIZES}
    a, b = cache["a"], cache["b"]
    da, db = np.zeros_like(a), np.zeros_like(b)
    for (k, i), al in cache["alpha"].items():
        n = ent[k][i][0]
        e = E[k][i]
        dal = float(np.sum(dA[3 * k:3 * k + 3, 3 * n:3 * n + 3] * e))
        dz = dal * al * (1.0 - al / 1.5)
        da[k] += dz * b[n]
        db[n] += dz * a[k]
        g["we"][0] += dz * np.sqrt(np.sum(e * e))
        g["we"][1] += dz * np.trace(e)
        g["ce"][0] += dz
    d = cache["d"]
    dd = np.where((d > -8.0) & (d < 8.0), ds * s, 0.0)
    h3 = cache["h3"]
    g["Wa"] = h3.T @ da
    g["Wb"] = h3.T @ db
    g["wd"] = h3.T @ dd
    g["cd"][0] = np.sum(dd)
    dh = da @ p["Wa"].T + db @ p["Wb"].T + np.outer(dd, p["wd"])
    Nm = cache["Nm"]
    for l in (3, 2, 1):
        dpre = dh * (cache["pre%d" % l] > 0.0)
        g["W%d" % l] = cache["A%d" % l].T @ dpre
        g["b%d" % l] = np.sum(dpre, axis=0)
        dAin = dpre @ cache["Wr%d" % l].T
        kin = dAin.shape[1] // 2
        dh = dAin[:, :kin] + Nm.T @ dAin[:, kin:]
    return L, pack(g)


def preconditioner(theta, S, sc_ent, ones, use_bf16: bool = True) -> np.ndarray:
    """M^{-1} = C^T G^T G C for the dual S (dense)."""
    C, St = normalized(S)
    E = blocks(St, sc_ent)
    cache = forward(theta, E, sc_ent, ones, use_bf16)
    G, _ = G_matrix(cache, E, sc_ent)
    return C.T @ G.T @ G @ C
