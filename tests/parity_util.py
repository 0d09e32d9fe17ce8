"""Helpers for the GPU parity tests: one step on the GPU through the C ABI
and one step of the CPU oracle from the same state."""
import numpy as np
import pytest


def rel(x, ref):
    x = np.asarray(x, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    n = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (n if n > 0 else 1.0)


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_solver(sc, **kw):
    from paper_2603_08079_gb300 import mabd
    return mabd.Solver(sc, **kw)


def gpu_step(solver, q, qd, n=1):
    solver.set_state(q, qd)
    st = solver.step(n, stats=True)
    q1, qd1 = solver.get_state()
    return q1, qd1, solver.get_lambda(), st


def oracle_step(ora, sc, q, qd, residual_rhs=1, solver="auto"):
    S = ora.Scene(sc, residual_rhs)
    return ora.step(S, q, qd, solver)


def assert_parity(ora, sc, q, qd, solver=None, tol=1e-9, residual_rhs=1, gpu_kw=None):
    """GPU and oracle from the same (q, qd): qdot_{n+1} = dq/h and lambda agree
    normwise to tol (the FP64 bound)."""
    gpu_kw = dict(gpu_kw or {})
    gpu_kw.setdefault("residual_rhs", residual_rhs)
    own = solver is None
    if own:
        solver = gpu_solver(sc, **gpu_kw)
    try:
        q1, qd1, lam, st = gpu_step(solver, q, qd)
    finally:
        if own:
            solver.close()
    oq1, oqd1, olam, ost = oracle_step(ora, sc, q, qd, residual_rhs)
    e_qd = rel(qd1, oqd1)
    e_lam = rel(lam, olam) if len(olam) else 0.0
    fixed = np.asarray(sc["fixed"]) != 0
    np.testing.assert_array_equal(q1[fixed], np.asarray(q)[fixed])
    assert e_qd <= tol, f"qdot rel err {e_qd:.3e}"
    assert e_lam <= tol, f"lambda rel err {e_lam:.3e}"
    return e_qd, e_lam, st[0], ost


def elementwise(sc, qd, oqd, lam, olam, floor=1e-3):
    """Per-body and per-joint relative errors against the oracle: body j's is
    |qd_j - oqd_j| / max(|oqd_j|, floor * max_i |oqd_i|) over its 12 velocity
    components, joint k's the same over its rows of lambda (Euclidean norms).
    The floor keeps bodies and joints that carry almost nothing (the middle of
    a long chain in free fall, an unloaded joint) from dividing by ~0.
    Returns (worst body, worst joint)."""
    from paper_2603_08079_gb300 import scenes

    qd = np.asarray(qd, dtype=np.float64).reshape(-1, 12)
    oqd = np.asarray(oqd, dtype=np.float64).reshape(-1, 12)
    nb = np.linalg.norm(oqd, axis=1)
    eb = np.linalg.norm(qd - oqd, axis=1)
    body = float((eb / np.maximum(nb, floor * max(nb.max(), 1e-300))).max()) if len(nb) else 0.0
    rows = scenes.joint_rows(sc["jtype"])
    if len(rows) == 0:
        return body, 0.0
    off = np.concatenate([[0], np.cumsum(rows)[:-1]])
    lam = np.asarray(lam, dtype=np.float64).ravel()
    olam = np.asarray(olam, dtype=np.float64).ravel()
    nj = np.sqrt(np.add.reduceat(olam ** 2, off))
    ej = np.sqrt(np.add.reduceat((lam - olam) ** 2, off))
    joint = float((ej / np.maximum(nj, floor * max(nj.max(), 1e-300))).max())
    return body, joint


def assert_elementwise(sc, qd, oqd, lam, olam, tol, floor=1e-3):
    body, joint = elementwise(sc, qd, oqd, lam, olam, floor)
    print(f"elementwise (floor {floor:g} of the largest): body {body:.3e}, joint {joint:.3e}")
    assert body <= tol and joint <= tol, (body, joint)
    return body, joint
