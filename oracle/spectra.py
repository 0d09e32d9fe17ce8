"""Spectral estimates of the dual matrix S = G H^{-1} G^T (Sec. 5, Eq. dual)
of a scene at a state -- TEST INFRASTRUCTURE ONLY (a report of the
conditioning beside each parity target; the CUDA path never uses it).

S is applied matrix-free from the oracle's own routines: the constraint
Jacobian G from ``joint_eval`` (frame frozen at q, Eq. pcpq) as a sparse
matrix over the free bodies, and per free body the world-frame inverse
H_A^{-1} = diag4(R) Hbar_A^{-1} diag4(R^T) (Eq. abd_final, the rest-frame
system matrix turned by the body's rotation, as ``assemble_dense`` builds
H_A).  ``dense_dual`` forms S explicitly for small scenes; ``lanczos``
runs the plain three-term Lanczos recurrence (no reorthogonalisation: the
extreme Ritz values still converge, spurious copies only repeat them) and
returns the extreme eigenvalues of its tridiagonal matrix.  After m steps
the largest Ritz value is a lower bound of lambda_max and the smallest an
upper bound of lambda_min, so the reported cond is a lower bound of cond(S)
unless the smallest pair has converged (its residual is reported).

    python -m oracle.spectra [--steps 300] [--small]
prints the estimates for the parity workloads.
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import Scene, body_rhs, joint_eval, system_matrix


def _diag4(R: np.ndarray) -> np.ndarray:
    """blockdiag(R, R, R, R) acting on the 12-vector of an affine body whose
    first nine entries stack the columns of A (Eq. abd_dof) and the last
    three are the translation: each 3-block is rotated by R."""
    D = np.zeros((12, 12))
    for b in range(4):
        D[3 * b:3 * b + 3, 3 * b:3 * b + 3] = R
    return D


def dual_operator(sc: dict, q=None, qd=None):
    """(n, apply) with apply(x) = S x for the scene at (q, qd)."""
    import scipy.sparse as sp

    q = np.asarray(sc["q"] if q is None else q, dtype=np.float64).reshape(-1)
    qd = np.asarray(sc["qdot"] if qd is None else qd, dtype=np.float64).reshape(-1)
    S_ = Scene(sc)
    M, K = S_.M, S_.K
    fixed = np.asarray(sc["fixed"]) != 0
    free = np.flatnonzero(~fixed)
    col_of = -np.ones(M, dtype=np.int64)
    col_of[free] = np.arange(len(free))
    Hinv = np.zeros((len(free), 12, 12))
    for i, j in enumerate(free):
        Hb = system_matrix(sc["mass"][j], sc["second_moment"][j], sc["volume"][j], sc["young"][j],
                           sc["poisson"][j], sc["h"])
        _, R = body_rhs(S_, int(j), q, qd)
        D = _diag4(R)
        Hinv[i] = D @ np.linalg.inv(Hb) @ D.T
    rows, cols, vals = [], [], []
    r0 = 0
    a_ids = np.asarray(sc["body_a"])
    b_ids = np.asarray(sc["body_b"])
    for k in range(K):
        c, Ga, Gb = joint_eval(S_, q, k)
        C = len(c)
        for body, Gs in ((int(a_ids[k]), Ga), (int(b_ids[k]), Gb)):
            if body < 0 or fixed[body]:
                continue
            cc = 12 * col_of[body]
            rr, ci = np.meshgrid(np.arange(C), np.arange(12), indexing="ij")
            rows.append((r0 + rr).ravel())
            cols.append((cc + ci).ravel())
            vals.append(Gs.ravel())
        r0 += C
    n = r0
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, 12 * len(free)))
    GT = G.T.tocsr()

    def apply(x):
        y = (GT @ x).reshape(-1, 12)
        y = np.einsum("bij,bj->bi", Hinv, y).reshape(-1)
        return G @ y

    return n, apply


def dense_dual(sc: dict, q=None, qd=None) -> np.ndarray:
    """S formed column by column (small scenes)."""
    n, apply = dual_operator(sc, q, qd)
    S = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[i] = 1.0
        S[:, i] = apply(e)
        e[i] = 0.0
    return 0.5 * (S + S.T)


def lanczos(apply, n: int, steps: int = 300, seed: int = 0):
    """(lambda_min Ritz, lambda_max Ritz, residual of the smallest pair,
    residual of the largest pair, steps taken) of the plain Lanczos
    recurrence started from a seeded random vector."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    v_prev = np.zeros(n)
    alpha, beta = [], []
    b = 0.0
    for _ in range(min(steps, n)):
        w = apply(v) - b * v_prev
        a = float(v @ w)
        w -= a * v
        alpha.append(a)
        b = float(np.linalg.norm(w))
        if b <= 1e-14 * max(abs(a), 1.0):
            break
        beta.append(b)
        v_prev, v = v, w / b
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    th, Y = np.linalg.eigh(T)
    bl = beta[m - 1] if len(beta) >= m else 0.0
    res = np.abs(bl * Y[-1, :])  # |beta_m e_m^T y|: residual of each Ritz pair
    return float(th[0]), float(th[-1]), float(res[0]), float(res[-1]), m


def cond_estimate(sc: dict, q=None, qd=None, steps: int = 300, dense_limit: int = 1500) -> dict:
    t0 = time.time()
    n, apply = dual_operator(sc, q, qd)
    if n <= dense_limit:
        w = np.linalg.eigvalsh(dense_dual(sc, q, qd))
        return {"n": n, "lmin": float(w[0]), "lmax": float(w[-1]), "cond": float(w[-1] / w[0]),
                "method": "dense", "secs": time.time() - t0}
    lo, hi, rlo, rhi, m = lanczos(apply, n, steps)
    return {"n": n, "lmin": lo, "lmax": hi, "cond": hi / lo, "res_min": rlo, "res_max": rhi,
            "method": f"Lanczos {m} steps", "secs": time.time() - t0}


def _workloads(small: bool):
    from paper_2603_08079_gb300 import scenes
    out = [("chain64 (plain FP64 config)", scenes.chain_cubes(64))]
    if small:
        out += [("chain 65,536", scenes.long_chain(65536, seed=0)),
                ("tree 20,000", scenes.random_tree(20000, seed=2)),
                ("batch 256", scenes.assemblies(256, seed=3)),
                ("net 16x16x8", scenes.jittered_net(16, 16, 8, seed=4))]
    else:
        out += [("chain 1,048,576", scenes.long_chain(1 << 20, seed=0)),
                ("tree 262,144", scenes.random_tree(262144, seed=2)),
                ("batch 4,096", scenes.assemblies(4096, seed=3)),
                ("net 64x64x16", scenes.jittered_net(64, 64, 16, seed=4))]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--small", action="store_true")
    a = ap.parse_args()
    for name, sc in _workloads(a.small):
        r = cond_estimate(sc, steps=a.steps)
        extra = f", residuals {r['res_min']:.1e} / {r['res_max']:.1e}" if "res_min" in r else ""
        print(f"{name}: n = {r['n']}, lambda in [{r['lmin']:.3e}, {r['lmax']:.3e}], "
              f"cond = {r['cond']:.3e} ({r['method']}{extra}; {r['secs']:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
