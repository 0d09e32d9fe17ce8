"""CPU FP64 oracle for one M-ABD step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never links, loads or calls it, and it shares no code with it.

``mabd_oracle.c`` is plain single-threaded C built with ``gcc -O2
-ffp-contract=off``; this module compiles it (``build()``) and wraps it with
ctypes.  Functions cite the paper section / equation they follow.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mabd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmabd_oracle.so")

SOLVERS = {"auto": 0, "chain": 1, "tree": 2, "cg": 3, "dense": 4}
ERRORS = {0: "ok", 1: "invalid argument", 5: "not SPD", 6: "inverted (det A <= 0)",
          7: "non-finite", 8: "no convergence", 10: "topology"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (host build, any architecture)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mabd_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [("M", C.c_int64), ("K", C.c_int64), ("h", C.c_double), ("g", C.c_double * 3),
                ("residual_rhs", C.c_int32),
                ("mass", C.c_void_p), ("second_moment", C.c_void_p), ("volume", C.c_void_p),
                ("young", C.c_void_p), ("poisson", C.c_void_p), ("fixed", C.c_void_p),
                ("jtype", C.c_void_p), ("body_a", C.c_void_p), ("body_b", C.c_void_p),
                ("anchor_a", C.c_void_p), ("anchor_b", C.c_void_p), ("axis_a", C.c_void_p),
                ("axis_b", C.c_void_p), ("axis_len", C.c_void_p), ("ref_a", C.c_void_p),
                ("ref_b", C.c_void_p), ("rotation_mode", C.c_int32), ("jacobian_mode", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("lin_residual", C.c_double), ("joint_residual", C.c_double),
                ("solver_used", C.c_int32), ("cg_iters", C.c_int32),
                ("cg_rel_residual", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        d = C.c_double
        _lib.ora_mass_matrix.argtypes = [d, P, P]
        _lib.ora_stiffness_matrix.argtypes = [d, d, d, P]
        _lib.ora_system_matrix.argtypes = [d, P, d, d, d, d, P]
        _lib.ora_cholesky12.argtypes = [P, P]
        _lib.ora_polar.argtypes = [P, P, P]
        _lib.ora_elastic_stress.argtypes = [P, d, d, P]
        _lib.ora_elastic_stress.restype = None
        _lib.ora_body_rhs.argtypes = [P, C.c_int64, P, P, P, P]
        _lib.ora_hinge_frame.argtypes = [P, P]
        _lib.ora_hinge_frame.restype = None
        _lib.ora_joint_eval.argtypes = [P, P, C.c_int64, P, P, P, P]
        _lib.ora_dual_rows.argtypes = [P]
        _lib.ora_dual_rows.restype = C.c_int64
        _lib.ora_topology.argtypes = [P]
        _lib.ora_assemble_dense.argtypes = [P, P, P, P, P, P, P]
        _lib.ora_step.argtypes = [P, C.c_int32, P, P, P, P, P, P]
        _lib.ora_alg1_solve.argtypes = [P, P, P, P]
        _lib.ora_alg1_solve.restype = None
        _lib.ora_joint_eval_attached.argtypes = [P, P, P, C.c_int64, P]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


ROTATION_MODES = {"polar": 0, "normalized": 1}
JACOBIAN_MODES = {"frozen": 0, "full": 1}


class Scene:
    """Keeps contiguous copies of a scene dict alive behind an ``ora_scene``.
    rotation_mode "normalized": the unconstrained solve by Alg. 1 (Sec. 3.4);
    jacobian_mode "full": the constraint gradient of Eq. constraint_gradient
    with the joint frame attached to body alpha (Sec. 5.1)."""

    def __init__(self, sc: dict, residual_rhs: int = 1, rotation_mode: str = "polar",
                 jacobian_mode: str = "frozen"):
        f64 = lambda k: np.ascontiguousarray(sc[k], dtype=np.float64)
        K = len(sc["jtype"])
        ref = lambda k: np.ascontiguousarray(sc.get(k, np.zeros((K, 3))), dtype=np.float64)
        self.arrays = {
            "mass": f64("mass"), "second_moment": f64("second_moment"), "volume": f64("volume"),
            "young": f64("young"), "poisson": f64("poisson"),
            "fixed": np.ascontiguousarray(sc["fixed"], dtype=np.int32),
            "jtype": np.ascontiguousarray(sc["jtype"], dtype=np.int32),
            "body_a": np.ascontiguousarray(sc["body_a"], dtype=np.int64),
            "body_b": np.ascontiguousarray(sc["body_b"], dtype=np.int64),
            "anchor_a": f64("anchor_a"), "anchor_b": f64("anchor_b"), "axis_a": f64("axis_a"),
            "axis_b": f64("axis_b"), "axis_len": f64("axis_len"),
            "ref_a": ref("ref_a"), "ref_b": ref("ref_b"),
        }
        self.M = len(self.arrays["mass"])
        self.K = len(self.arrays["jtype"])
        self.h = float(sc["h"])
        s = _Scene()
        s.M, s.K, s.h = self.M, self.K, self.h
        for i in range(3):
            s.g[i] = float(sc["gravity"][i])
        s.residual_rhs = residual_rhs
        s.rotation_mode = ROTATION_MODES[rotation_mode]
        s.jacobian_mode = JACOBIAN_MODES[jacobian_mode]
        for k, v in self.arrays.items():
            setattr(s, k, v.ctypes.data)
        self.s = s

    @property
    def ptr(self):
        return C.cast(C.pointer(self.s), C.c_void_p)

    @property
    def rows(self) -> int:
        t = self.arrays["jtype"]
        return int(np.sum(np.where((t == 1) | (t == 3), 5, np.where(t == 2, 4, 3))))


def _check(st: int, what: str):
    if st != 0:
        raise RuntimeError(f"oracle {what}: {ERRORS.get(st, st)}")


# -- Sec. 3 building blocks ---------------------------------------------------

def mass_matrix(m: float, S6) -> np.ndarray:
    """M_A = J^T M J = [[Sigma (x) I3, 0], [0, m I3]] (Sec. 3.2, Eq. newton_abd)."""
    S6 = np.ascontiguousarray(S6, dtype=np.float64)
    out = np.zeros(144)
    lib().ora_mass_matrix(m, _p(S6), _p(out))
    return out.reshape(12, 12)


def stiffness_matrix(V: float, E: float, nu: float) -> np.ndarray:
    """Rest-shape stiffness Kbar_A of the linear elastic energy (Sec. 3.3)."""
    out = np.zeros(144)
    lib().ora_stiffness_matrix(V, E, nu, _p(out))
    return out.reshape(12, 12)


def system_matrix(m, S6, V, E, nu, h) -> np.ndarray:
    """Hbar_A = M_A / h^2 + Kbar_A (Eq. abd_final)."""
    S6 = np.ascontiguousarray(S6, dtype=np.float64)
    out = np.zeros(144)
    lib().ora_system_matrix(m, _p(S6), V, E, nu, h, _p(out))
    return out.reshape(12, 12)


def cholesky12(H: np.ndarray) -> np.ndarray:
    H = np.ascontiguousarray(H, dtype=np.float64).reshape(144)
    L = np.zeros(144)
    _check(lib().ora_cholesky12(_p(H), _p(L)), "cholesky")
    return L.reshape(12, 12)


def polar(A: np.ndarray) -> tuple[np.ndarray, int]:
    """R = A (A^T A)^{-1/2} (Eq. polar), Higham's Newton iteration."""
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    R = np.zeros(9)
    it = C.c_int32(0)
    _check(lib().ora_polar(_p(A), _p(R), C.byref(it)), "polar")
    return R.reshape(3, 3), it.value


def elastic_stress(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    """P(F) = mu (F + F^T - 2I) + lambda tr(F - I) I (Sec. 3.3)."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    P = np.zeros(9)
    lib().ora_elastic_stress(_p(F), mu, lam, _p(P))
    return P.reshape(3, 3)


def hinge_frame(a) -> np.ndarray:
    """R_H = I + [v]x + [v]x^2/(1+a_y), v = a x e_y (Sec. 4.3)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    R = np.zeros(9)
    lib().ora_hinge_frame(_p(a), _p(R))
    return R.reshape(3, 3)


def body_rhs(scene: Scene, j: int, q: np.ndarray, qd: np.ndarray):
    """World-frame Newton rhs f_A of body j and its rotation R."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    qd = np.ascontiguousarray(qd, dtype=np.float64).reshape(-1)
    f = np.zeros(12)
    R = np.zeros(9)
    _check(lib().ora_body_rhs(scene.ptr, j, _p(q), _p(qd), _p(f), _p(R)), "body_rhs")
    return f, R.reshape(3, 3)


def joint_eval(scene: Scene, q: np.ndarray, k: int):
    """C_k(q), dC/dq_alpha, dC/dq_beta with the joint frame frozen (Eq. pcpq)."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    c = np.zeros(5)
    Ga = np.zeros(60)
    Gb = np.zeros(60)
    rows = C.c_int32(0)
    _check(lib().ora_joint_eval(scene.ptr, _p(q), k, _p(c), _p(Ga), _p(Gb), C.byref(rows)),
           "joint_eval")
    n = rows.value
    return c[:n], Ga.reshape(5, 12)[:n], Gb.reshape(5, 12)[:n]


def joint_eval_attached(scene: Scene, q_ref: np.ndarray, q: np.ndarray, k: int) -> np.ndarray:
    """C_k(q) with the joint frame carried by body alpha's polar rotation from
    q_ref (R_J = dR R^T, Sec. 5.1 Eq. r_gradient); its derivative at q = q_ref
    is the full gradient of Eq. constraint_gradient."""
    q_ref = np.ascontiguousarray(q_ref, dtype=np.float64).reshape(-1)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    c = np.zeros(5)
    _check(lib().ora_joint_eval_attached(scene.ptr, _p(q_ref), _p(q), k, _p(c)), "joint_eval_attached")
    t = int(scene.arrays["jtype"][k])
    return c[:(5 if t in (1, 3) else 3)]


def alg1_solve(L: np.ndarray, A: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Alg. 1 (Sec. 3.4): u from Hbar_A = L L^T, the affine matrix A and the
    world-frame force f, every block rotation by the length-preserving map of
    Eq. len_preserving."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(3, 3))
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(12)
    u = np.zeros(12)
    lib().ora_alg1_solve(_p(L), _p(A), _p(f), _p(u))
    return u


def topology(scene: Scene) -> int:
    return int(lib().ora_topology(scene.ptr))


def assemble_dense(scene: Scene, q: np.ndarray, qd: np.ndarray):
    """Dense KKT ingredients for small systems: H_A per body (world frame),
    f, the full constraint Jacobian G and C(q_n)."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    qd = np.ascontiguousarray(qd, dtype=np.float64).reshape(-1)
    M, n = scene.M, scene.rows
    Hw = np.zeros(144 * M)
    f = np.zeros(12 * M)
    G = np.zeros(n * 12 * M)
    c = np.zeros(max(n, 1))
    _check(lib().ora_assemble_dense(scene.ptr, _p(q), _p(qd), _p(Hw), _p(f), _p(G), _p(c)),
           "assemble_dense")
    return Hw.reshape(M, 12, 12), f, G.reshape(n, 12 * M), c[:n]


def step(scene: Scene, q: np.ndarray, qd: np.ndarray, solver: str = "auto"):
    """One implicit step / one Newton iteration (Eq. kkt, dual, recover).
    Returns q_{n+1}, qdot_{n+1} (M,12), lambda (rows,) and a stats dict."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    qd = np.ascontiguousarray(qd, dtype=np.float64).reshape(-1)
    q1 = np.zeros_like(q)
    qd1 = np.zeros_like(qd)
    lam = np.zeros(max(scene.rows, 1))
    st = Stats()
    _check(lib().ora_step(scene.ptr, SOLVERS[solver], _p(q), _p(qd), _p(q1), _p(qd1), _p(lam),
                          C.byref(st)), "step")
    return q1.reshape(-1, 12), qd1.reshape(-1, 12), lam[:scene.rows], st.as_dict()


def run(sc: dict, nsteps: int, solver: str = "auto", q=None, qd=None, residual_rhs: int = 1,
        **modes):
    """Advance a scene dict nsteps from (q, qd) (default: the scene's state)."""
    scene = Scene(sc, residual_rhs, **modes)
    q = sc["q"] if q is None else q
    qd = sc["qdot"] if qd is None else qd
    stats = []
    lam = None
    for _ in range(nsteps):
        q, qd, lam, s = step(scene, q, qd, solver)
        stats.append(s)
    return q, qd, lam, stats
