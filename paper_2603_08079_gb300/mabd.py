"""Python binding of the C ABI in include/mabd.h (argument marshalling only).

Every step of the solve runs in the CUDA library ``_build/libmabd.so``; this
module converts scene dictionaries (see ``scenes.py``) into the C structs,
passes PyTorch's stream and caching allocator to the library, and copies
states and multipliers between numpy arrays and the library.  There is no
CPU fallback: if the library is missing or no GPU is usable, construction
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

WORLD = -1
SOLVERS = {"auto": 0, "chain": 1, "tree": 2, "pcg": 3, "loop": 4}
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_fp32_dual": 2}
ROTATION_MODES = {"polar": 0, "normalized": 1}
JACOBIAN_MODES = {"frozen": 0, "full": 1}
TOPOLOGIES = {0: "none", 1: "chain", 2: "tree", 3: "graph", 4: "loop"}
STATUS = {0: "ok", 1: "invalid argument", 2: "call out of order", 3: "out of device memory",
          4: "CUDA error", 5: "not positive definite", 6: "inverted body", 7: "non-finite",
          8: "no convergence", 9: "timeout", 10: "unsupported"}


class MabdError(RuntimeError):
    def __init__(self, what: str, code: int, detail: str = ""):
        msg = f"{what}: {STATUS.get(code, code)} (status {code})"
        super().__init__(msg + (f" [{detail}]" if detail else ""))
        self.code = code


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [("h", C.c_double), ("gravity", C.c_double * 3), ("precision", C.c_int32),
                ("solver", C.c_int32), ("pcg_max_iters", C.c_int32), ("pcg_rtol", C.c_double),
                ("refine_steps", C.c_int32), ("residual_rhs", C.c_int32), ("stream", C.c_void_p),
                ("dev_alloc", _ALLOC), ("dev_free", _FREE), ("alloc_user", C.c_void_p),
                ("rotation_mode", C.c_int32), ("jacobian_mode", C.c_int32)]


class StepStats(C.Structure):
    _fields_ = [("lin_residual", C.c_double), ("joint_residual", C.c_double),
                ("pcg_iters", C.c_int32), ("pcg_rel_residual", C.c_double),
                ("refine_residual", C.c_double), ("polar_iterations", C.c_double)]


class Info(C.Structure):
    _fields_ = [("bodies", C.c_int64), ("joints", C.c_int64), ("dual_rows", C.c_int64),
                ("topology", C.c_int32), ("solver", C.c_int32), ("device_bytes", C.c_int64),
                ("precision", C.c_int32), ("refine_steps", C.c_int32), ("cr_levels", C.c_int32),
                ("cr_tail_level", C.c_int32), ("seg_levels", C.c_int32), ("seg_tile", C.c_int32),
                ("rotation_mode", C.c_int32), ("jacobian_mode", C.c_int32)]


# numpy mirrors of mabd_body_desc / mabd_joint_desc (C layout, natural alignment)
BODY_DTYPE = np.dtype([("mass", "f8"), ("second_moment", "f8", 6), ("volume", "f8"),
                       ("young", "f8"), ("poisson", "f8"), ("q", "f8", 12), ("qdot", "f8", 12),
                       ("fixed", "i4")], align=True)
JOINT_DTYPE = np.dtype([("type", "i4"), ("body_a", "i8"), ("body_b", "i8"), ("anchor_a", "f8", 3),
                        ("anchor_b", "f8", 3), ("axis_a", "f8", 3), ("axis_b", "f8", 3),
                        ("axis_len", "f8"), ("ref_a", "f8", 3), ("ref_b", "f8", 3)], align=True)
assert BODY_DTYPE.itemsize == 280 and JOINT_DTYPE.itemsize == 176

_lib = None

EXPORTS = ["mabd_config_default", "mabd_create", "mabd_add_bodies", "mabd_add_joints",
           "mabd_prefactor", "mabd_step", "mabd_get_state", "mabd_set_state", "mabd_get_lambda",
           "mabd_synchronize", "mabd_get_info", "mabd_profile_enable", "mabd_profile_reset",
           "mabd_kernel_times", "mabd_destroy", "mabd_status_string", "mabd_error_detail",
           "mabd_lpc_num_params", "mabd_set_preconditioner", "mabd_lpc_fallbacks",
           "mabd_lpc_create", "mabd_lpc_capture", "mabd_lpc_batch_blocks", "mabd_lpc_loss_grad",
           "mabd_lpc_train", "mabd_lpc_destroy", "mabd_tree_schedule"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmabd.so (building it in-tree with nvcc if it is missing);
    MABD_LIB=debug in the environment loads the MABD_DEBUG build instead."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("MABD_LIB") == "debug"
    path = _build.LIB_DEBUG if debug else _build.LIB
    if not os.path.exists(path) or not _build.up_to_date(debug):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build(debug=debug)
    lib = C.CDLL(path)
    P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.mabd_config_default.argtypes = [C.POINTER(Config)]
    lib.mabd_config_default.restype = None
    lib.mabd_create.argtypes = [C.POINTER(Config), C.POINTER(P)]
    lib.mabd_add_bodies.argtypes = [P, i64, P, C.POINTER(i64)]
    lib.mabd_add_joints.argtypes = [P, i64, P, C.POINTER(i64)]
    lib.mabd_prefactor.argtypes = [P]
    lib.mabd_step.argtypes = [P, i32, P]
    lib.mabd_get_state.argtypes = [P, P, P]
    lib.mabd_set_state.argtypes = [P, P, P]
    lib.mabd_get_lambda.argtypes = [P, P]
    lib.mabd_synchronize.argtypes = [P]
    lib.mabd_get_info.argtypes = [P, C.POINTER(Info)]
    lib.mabd_profile_enable.argtypes = [P, i32]
    lib.mabd_profile_reset.argtypes = [P]
    lib.mabd_kernel_times.argtypes = [P, i32, P, P, P, C.POINTER(i32)]
    lib.mabd_destroy.argtypes = [P]
    lib.mabd_status_string.argtypes = [i32]
    lib.mabd_status_string.restype = C.c_char_p
    lib.mabd_error_detail.argtypes = [P]
    lib.mabd_error_detail.restype = C.c_char_p
    u64 = C.c_uint64
    lib.mabd_lpc_num_params.argtypes = []
    lib.mabd_set_preconditioner.argtypes = [P, P]
    lib.mabd_lpc_fallbacks.argtypes = [P, C.POINTER(i32)]
    lib.mabd_lpc_create.argtypes = [C.POINTER(P)]
    lib.mabd_lpc_capture.argtypes = [P, P, C.POINTER(i32)]
    lib.mabd_lpc_batch_blocks.argtypes = [P, i32, P, P, P]
    lib.mabd_lpc_loss_grad.argtypes = [P, i32, P, i32, i32, P, u64, C.POINTER(C.c_double), P]
    lib.mabd_lpc_train.argtypes = [P, P, i32, i32, C.c_float, i32, u64, P]
    lib.mabd_lpc_destroy.argtypes = [P]
    lib.mabd_tree_schedule.argtypes = [P, P]
    for f in EXPORTS:
        if f not in ("mabd_config_default", "mabd_status_string", "mabd_error_detail"):
            getattr(lib, f).restype = i32
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def body_array(sc: dict) -> np.ndarray:
    M = len(sc["mass"])
    d = np.zeros(M, dtype=BODY_DTYPE)
    d["mass"] = sc["mass"]
    d["second_moment"] = sc["second_moment"]
    d["volume"] = sc["volume"]
    d["young"] = sc["young"]
    d["poisson"] = sc["poisson"]
    d["q"] = sc["q"]
    d["qdot"] = sc["qdot"]
    d["fixed"] = sc["fixed"]
    return d


def joint_array(sc: dict) -> np.ndarray:
    K = len(sc["jtype"])
    d = np.zeros(K, dtype=JOINT_DTYPE)
    for f in ("anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len", "body_a", "body_b"):
        d[f] = sc[f]
    for f in ("ref_a", "ref_b"):  # prismatic joints only
        if f in sc:
            d[f] = sc[f]
    d["type"] = sc["jtype"]
    return d


class Solver:
    """One M-ABD scene on one GPU (a ``mabd_ctx``)."""

    def __init__(self, sc: dict, solver: str = "auto", residual_rhs: int = 1,
                 stream=None, allocator: str = "torch", pcg_rtol: float = 1e-13,
                 pcg_max_iters: int = 2000, precision: str = "fp64", refine_steps: int = 1,
                 rotation_mode: str = "polar", jacobian_mode: str = "frozen"):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("mabd.Solver needs a CUDA device")
        self._lib = load()
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = Config()
        self._lib.mabd_config_default(C.byref(cfg))
        cfg.h = float(sc["h"])
        for i in range(3):
            cfg.gravity[i] = float(sc["gravity"][i])
        cfg.solver = SOLVERS[solver]
        cfg.residual_rhs = int(residual_rhs)
        cfg.pcg_rtol = float(pcg_rtol)
        cfg.pcg_max_iters = int(pcg_max_iters)
        cfg.precision = PRECISIONS[precision]
        cfg.refine_steps = int(refine_steps)
        cfg.rotation_mode = ROTATION_MODES[rotation_mode]
        cfg.jacobian_mode = JACOBIAN_MODES[jacobian_mode]
        cfg.stream = C.c_void_p(self.stream.cuda_stream)
        if allocator == "torch":
            dev, strm = self.device, self.stream

            def _alloc(n, user):
                return torch.cuda.caching_allocator_alloc(int(n), dev, strm)

            def _free(p, user):
                torch.cuda.caching_allocator_delete(p)

            self._cb = (_ALLOC(_alloc), _FREE(_free))
            cfg.dev_alloc, cfg.dev_free = self._cb
        self.M = len(sc["mass"])
        self.K = len(sc["jtype"])
        ctx = C.c_void_p()
        self._check("mabd_create", self._lib.mabd_create(C.byref(cfg), C.byref(ctx)))
        self.ctx = ctx
        self._cfg = cfg
        bodies = body_array(sc)
        joints = joint_array(sc)
        first = C.c_int64(0)
        self._check("mabd_add_bodies", self._lib.mabd_add_bodies(self.ctx, self.M, _ptr(bodies), C.byref(first)))
        if self.K:
            self._check("mabd_add_joints", self._lib.mabd_add_joints(self.ctx, self.K, _ptr(joints), C.byref(first)))
        self._check("mabd_prefactor", self._lib.mabd_prefactor(self.ctx))
        self.rows = int(self.info()["dual_rows"])

    def _check(self, what, st):
        if st != 0:
            detail = ""
            if getattr(self, "ctx", None):
                detail = (self._lib.mabd_error_detail(self.ctx) or b"").decode(errors="replace")
            raise MabdError(what, st, detail)

    def step(self, n: int = 1, stats: bool = False):
        if stats:
            arr = (StepStats * max(n, 1))()
            self._check("mabd_step", self._lib.mabd_step(self.ctx, n, arr))
            return [{f: getattr(s, f) for f, _ in StepStats._fields_} for s in arr[:n]]
        self._check("mabd_step", self._lib.mabd_step(self.ctx, n, None))
        return None

    def get_state(self, q: np.ndarray | None = None, qd: np.ndarray | None = None):
        q = np.empty((self.M, 12)) if q is None else q
        qd = np.empty((self.M, 12)) if qd is None else qd
        self._check("mabd_get_state", self._lib.mabd_get_state(self.ctx, _ptr(q), _ptr(qd)))
        return q, qd

    def set_state(self, q: np.ndarray, qd: np.ndarray):
        q = np.ascontiguousarray(q, dtype=np.float64)
        qd = np.ascontiguousarray(qd, dtype=np.float64)
        assert q.size == 12 * self.M and qd.size == 12 * self.M
        self._keep = (q, qd)
        self._check("mabd_set_state", self._lib.mabd_set_state(self.ctx, _ptr(q), _ptr(qd)))

    def get_lambda(self) -> np.ndarray:
        lam = np.zeros(max(self.rows, 1))
        self._check("mabd_get_lambda", self._lib.mabd_get_lambda(self.ctx, _ptr(lam)))
        return lam[:self.rows]

    def synchronize(self):
        self._check("mabd_synchronize", self._lib.mabd_synchronize(self.ctx))

    def info(self) -> dict:
        inf = Info()
        self._check("mabd_get_info", self._lib.mabd_get_info(self.ctx, C.byref(inf)))
        d = {f: getattr(inf, f) for f, _ in Info._fields_}
        d["topology"] = TOPOLOGIES.get(d["topology"], d["topology"])
        d["solver"] = {v: k for k, v in SOLVERS.items()}.get(d["solver"], d["solver"])
        d["precision"] = {v: k for k, v in PRECISIONS.items()}.get(d["precision"], d["precision"])
        d["rotation_mode"] = {v: k for k, v in ROTATION_MODES.items()}.get(d["rotation_mode"],
                                                                            d["rotation_mode"])
        d["jacobian_mode"] = {v: k for k, v in JACOBIAN_MODES.items()}.get(d["jacobian_mode"],
                                                                            d["jacobian_mode"])
        return d

    def profile(self, enable: bool):
        self._check("mabd_profile_enable", self._lib.mabd_profile_enable(self.ctx, int(enable)))

    def profile_reset(self):
        self._check("mabd_profile_reset", self._lib.mabd_profile_reset(self.ctx))

    def kernel_times(self) -> dict:
        cap = 32
        names = (C.c_char_p * cap)()
        ms = (C.c_double * cap)()
        launches = (C.c_int64 * cap)()
        count = C.c_int32(0)
        self._check("mabd_kernel_times", self._lib.mabd_kernel_times(
            self.ctx, cap, C.cast(names, C.c_void_p), C.cast(ms, C.c_void_p),
            C.cast(launches, C.c_void_p), C.byref(count)))
        return {names[i].decode(): (ms[i], launches[i]) for i in range(min(count.value, cap))}

    def set_preconditioner(self, params):
        """Learned preconditioner parameters (float32 vector) or None."""
        if params is None:
            self._check("mabd_set_preconditioner", self._lib.mabd_set_preconditioner(self.ctx, None))
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == lpc_num_params()
        self._check("mabd_set_preconditioner", self._lib.mabd_set_preconditioner(self.ctx, _ptr(p)))

    def tree_schedule(self) -> dict:
        """Levels below the roots and the path (levels, or the persistent
        kernel's block size)."""
        c = np.zeros(4, dtype=np.int32)
        self._check("mabd_tree_schedule", self._lib.mabd_tree_schedule(self.ctx, _ptr(c)))
        return {"levels": int(c[0]),
                "path": {0: "levels", 128: "forest128", 64: "forest64", 32: "forest32"}.get(int(c[3]), int(c[3]))}

    def lpc_fallbacks(self) -> int:
        n = C.c_int32(0)
        self._check("mabd_lpc_fallbacks", self._lib.mabd_lpc_fallbacks(self.ctx, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.mabd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lpc_num_params() -> int:
    return int(load().mabd_lpc_num_params())


class LpcTrainer:
    """Captured normalized dual systems and on-device training of the learned
    preconditioner (mabd_lpc_*)."""

    def __init__(self):
        self._lib = load()
        t = C.c_void_p()
        st = self._lib.mabd_lpc_create(C.byref(t))
        if st != 0:
            raise MabdError("mabd_lpc_create", st)
        self.t = t
        self.n = lpc_num_params()

    def _check(self, what, st):
        if st != 0:
            raise MabdError(what, st)

    def capture(self, solver: Solver) -> int:
        b = C.c_int32(-1)
        self._check("mabd_lpc_capture", self._lib.mabd_lpc_capture(self.t, solver.ctx, C.byref(b)))
        return b.value

    def blocks(self, batch: int, K: int, nnz: int):
        """(off [K+1], nbr [nnz], E [nnz,3,3]) of a captured batch."""
        off = np.zeros(K + 1, dtype=np.int32)
        nbr = np.zeros(max(nnz, 1), dtype=np.int32)
        E = np.zeros((max(nnz, 1), 9), dtype=np.float32)
        self._check("mabd_lpc_batch_blocks",
                    self._lib.mabd_lpc_batch_blocks(self.t, batch, _ptr(off), _ptr(nbr), _ptr(E)))
        return off, nbr[:nnz], E[:nnz].reshape(nnz, 3, 3)

    KINDS = {"frobenius": 0, "kaporin": 1}

    def loss_grad(self, batch: int, params, V=None, nv: int = 2, seed: int = 0, grad: bool = True,
                  kind: str = "kaporin"):
        p = np.ascontiguousarray(params, dtype=np.float32)
        g = np.zeros(self.n, dtype=np.float32) if grad else None
        Vp = None
        if V is not None:
            V = np.ascontiguousarray(V, dtype=np.float32)
            nv = V.shape[0]
            Vp = _ptr(V)
        loss = C.c_double(0.0)
        self._check("mabd_lpc_loss_grad", self._lib.mabd_lpc_loss_grad(
            self.t, batch, _ptr(p), self.KINDS[kind], nv, Vp, seed, C.byref(loss),
            _ptr(g) if grad else None))
        return loss.value, g

    def train(self, params, iters: int, lr: float = 1e-3, nv: int = 2, seed: int = 0,
              kind: str = "kaporin"):
        p = np.ascontiguousarray(params, dtype=np.float32).copy()
        losses = np.zeros(max(iters, 1))
        self._check("mabd_lpc_train", self._lib.mabd_lpc_train(
            self.t, _ptr(p), self.KINDS[kind], iters, C.c_float(lr), nv, seed, _ptr(losses)))
        return p, losses[:iters]

    def close(self):
        if getattr(self, "t", None):
            self._lib.mabd_lpc_destroy(self.t)
            self.t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
