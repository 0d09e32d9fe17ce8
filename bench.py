#!/usr/bin/env python3
"""Throughput of the M-ABD step on GB300: body-steps/s on the 1,048,576-body
pulley-cable chain (alternating ball / hinge joints, both ends pinned,
h = 1e-2 s), one implicit step with one Newton iteration per step, in the
chosen form (mixed precision: FP32 products and cyclic reduction, one FP64
residual-correction sweep of the FP64 system, within 1e-6 of the FP64
oracle) with the plain FP64 GPU path and the mixed form with the FP64
reduction timed beside it.  Other workloads: --workload
tree256k | net64x64x16 (mixed form with the learned preconditioner) |
batch4096.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One process per GPU; with N > 1 (torchrun) every rank steps its own
independent copy of the chain (replicas: the method's step has no exchange
between independent assemblies) and rank 0 prints one JSON line whose value
is the sum over ranks.  ``--impl reference`` times the CPU FP64 oracle on the
host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

from paper_2603_08079_gb300 import scenes

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "body-steps/s at ≤1e-6 rel err vs FP64 oracle; chosen form vs plain GPU path"
M_FULL = 1 << 20
H = 1e-2


WORKLOADS = {
    # name: (generator kwargs, description, solver, oracle sample kwargs)
    "chain1m": ("pulley-cable chain: %d boxes (sides U[0.5,1.5], rho 10^U[2,4]), %d joints "
                "(ball/hinge alternating, both ends pinned), %d dual rows, h=1e-2 s, seed 1",
                "block cyclic reduction (chain)"),
    "tree256k": ("random tree: %d boxes (sides U[0.2,1], rho 1000, Poisson(1.8) children), %d joints "
                 "(hinges, axes uniform on the sphere, root pinned), %d dual rows, h=5e-3 s, seed 2",
                 "level-scheduled body-space elimination (tree)"),
    "net64x64x16": ("jittered net: %d unit cubes on a 64x64x16 lattice (sigma 0.05, bottom layer fixed), "
                    "%d ball joints kept with p=0.7, %d dual rows, h=1e-2 s, seed 4",
                    "PCG on the dual (graph), rtol 1e-13: block Jacobi in FP64; in the mixed form FP32 "
                    "with the learned preconditioner in the normalized dual space, one cooperative launch "
                    "per solve"),
    "loop1m": ("pulley-cable loop: %d boxes (sides U[0.5,1.5], rho 10^U[2,4]) along a closed polygon, "
               "%d joints (ball/hinge alternating, the last one closing the loop, no world joints), "
               "%d dual rows, h=1e-2 s, seed 1",
               "loop Schur complement (Case III): one breaker joint, the chain of the others by block "
               "cyclic reduction"),
    "batch4096": ("4096 independent assemblies: %d links (7..64 per assembly, Poisson(1.3) branching, "
                  "fixed base with a random pose), %d hinge/ball joints, %d dual rows, h=2e-3 s, seed 3",
                  "one forest: level-scheduled body-space elimination over all assemblies, "
                  "replayed from one CUDA graph per step"),
}


def make_scene(name: str, M: int | None = None) -> dict:
    if name == "chain1m":
        return scenes.long_chain(M or M_FULL, seed=1)
    if name == "tree256k":
        return scenes.random_tree(M or 262144, seed=2)
    if name == "batch4096":
        return scenes.assemblies(M or 4096, seed=3)
    if name == "loop1m":
        return scenes.ring_chain(M or M_FULL, seed=1)
    if name == "net64x64x16":
        if M:  # a smaller lattice with the same density, for the CPU sample
            n = max(4, int(round((M / 16) ** 0.5)))
            return scenes.jittered_net(n, n, 16 if n >= 16 else 4, seed=4)
        return scenes.jittered_net(64, 64, 16, seed=4)
    raise KeyError(name)


FORMS = {
    "fp64": "FP64 throughout",
    "mixed": "FP32 per-body/per-joint products (and Gram blocks on chains, PCG iterations on "
             "graphs); polar and rhs in double-float (FP32 pairs, ~46 bits), FP64 constraint "
             "values and chain cyclic reduction, %d residual-correction sweep(s) with the primal "
             "residual in double-float and the dual residual in FP64",
    "mixed_fp32_dual": "FP32 per-body/per-joint products, Gram blocks and chain cyclic reduction "
                       "or tree elimination (FP32 PCG on graphs); polar and rhs in double-float "
                       "(FP32 pairs, ~46 bits), FP64 constraint values, %d residual-correction "
                       "sweep(s) of the FP64 system (primal residual in double-float, dual in FP64)",
}


def workload_config(M: int, K: int, rows: int, name: str = "chain1m", form: str = "fp64",
                    refine: int = 1) -> dict:
    desc, solver = WORKLOADS[name]
    fdesc = FORMS[form] % refine if form != "fp64" else FORMS[form]
    return {
        "workload": desc % (M, K, rows),
        "bodies": M, "joints": K, "dual_rows": rows, "form": form, "form_detail": fdesc,
        "solver": solver,
        "l2": "inputs larger than L2 (working set > 129 MB), no flush",
    }


LPC_PARAMS_REL = "paper_2603_08079_gb300/data/lpc_params.npy"


def use_learned(args, form: str):
    """Trained parameters of the learned preconditioner for the net workload
    in the mixed form (None otherwise or with --no-lpc)."""
    if args.no_lpc or form == "fp64" or args.workload != "net64x64x16":
        return None
    path = os.path.join(ROOT, LPC_PARAMS_REL)
    if not os.path.exists(path):
        return None
    return np.load(path).astype(np.float32)


def chosen_form(args) -> str:
    """Chains, trees and the batched forest: the FP32 elimination refined by
    FP64 sweeps; nets: the FP32 PCG (learned preconditioner) refined by FP64
    sweeps."""
    if args.precision != "auto":
        return args.precision
    if args.workload == "loop1m":
        return "fp64"  # the loop solver is FP64; the PCG path is timed beside it
    return "mixed" if args.workload == "net64x64x16" else "mixed_fp32_dual"


def max_over_ranks(ms: float, device: str = "cuda") -> float:
    """The largest of the ranks' timings (the job's time), via all_reduce MAX
    when a process group with more than one rank is up."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, M: int, steps: int, ms_max: float) -> float:
    """Whole-job body-steps/s: every rank steps its own replica of M bodies
    (weak scaling), the job lasts as long as the slowest rank."""
    return ws * M * steps / (ms_max / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def lscpu_model() -> str:
    try:
        out = subprocess.check_output(["lscpu"], text=True)
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", "mabd_clocks_%d_%d.csv" % (os.getpid(), device_index))

    def start(self):
        """Starts nvidia-smi and returns once its first sample is written, so
        that the samples cover the region timed next."""
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# algorithmic work of the dominant kernels (FP64 flops, FMA = 2)
# --------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 peak of GB300 from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk/SM
# x 2 flop x 2.07 GHz = 1.26 TFLOP/s (the nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _cr_fma(sizes: np.ndarray):
    """(FMA, eliminated rows' total size) of block cyclic reduction over all
    levels for dual rows of the given sizes (3 ball, 5 hinge)."""
    chol = {3: 7, 5: 30}
    fma_total, rows = 0, 0
    while len(sizes) > 1:
        N = len(sizes)
        odd = np.arange(1, N, 2)
        n = sizes[odd]
        l = sizes[odd - 1]
        r = np.where(odd + 1 < N, sizes[np.minimum(odd + 1, N - 1)], 0)
        fma = np.vectorize(chol.get)(n) + (l + r + 1) * n * (n + 1) // 2 + \
            (l * (l + 1) // 2 + r * (r + 1) // 2 + l * r + l + r) * n
        fma_total += int(fma.sum())
        rows += int(n.sum())
        sizes = sizes[0::2]
    return fma_total, rows


def cr_reduce_flops(jtype_chain: np.ndarray) -> float:
    """FP64 flops of block cyclic reduction over all levels (FMA = 2): for an
    eliminated row of size n with neighbours of sizes l, r (0 if absent):
    Cholesky 2*chol(n) + n rsqrt-multiplies, Ya/Yb/y triangular solves
    (l + r + 1) n(n+1)/2 FMA, Schur updates (l(l+1)/2 + r(r+1)/2 + l r + l + r) n FMA.
    The library eliminates either the chain's rows as they are or behind one
    leading identity row of size 3, whichever has fewer FMA; the same choice
    is made here."""
    sizes = scenes.joint_rows(jtype_chain)
    best = _cr_fma(sizes)
    if len(sizes) > 1:
        shifted = _cr_fma(np.concatenate([[3], sizes]))
        if shifted[0] < best[0]:
            best = shifted
    return 2.0 * best[0] + 2.0 * best[1]


def _cr_sizes(jtype_chain: np.ndarray) -> np.ndarray:
    """Level-0 row sizes with the library's choice of the leading identity row."""
    sizes = scenes.joint_rows(jtype_chain)
    if len(sizes) > 1 and _cr_fma(np.concatenate([[3], sizes]))[0] < _cr_fma(sizes)[0]:
        return np.concatenate([[3], sizes])
    return sizes


def cr_back_bytes(jtype_chain: np.ndarray, elem: int) -> float:
    """Algorithmic bytes of the back-substitution over all levels (one
    pass): an eliminated row of size n between neighbours of sizes l, r reads
    its factor (n(n+1)/2 + n l + n r + n entries) and the neighbours'
    multipliers (l + r) and writes its own (n); a kept row copies its C
    multipliers from the next level.  elem: bytes of the reduction's type;
    level 0 writes FP64 multipliers."""
    sizes = _cr_sizes(jtype_chain)
    total, level = 0.0, 0
    while len(sizes) > 1:
        N = len(sizes)
        odd = np.arange(1, N, 2)
        n = sizes[odd]
        l = sizes[odd - 1]
        r = np.where(odd + 1 < N, sizes[np.minimum(odd + 1, N - 1)], 0)
        out = 8 if level == 0 else elem
        total += float(np.sum((n * (n + 1) // 2 + n * l + n * r + n + l + r) * elem + n * out))
        even = sizes[0::2]
        total += float(np.sum(even * (elem + out)))
        sizes = sizes[0::2]
        level += 1
    return total


def mx_res_body_bytes(jtype: np.ndarray, M: int) -> float:
    """Algorithmic HBM bytes of one k_mx_res_body launch (the mixed forms'
    primal residual, first sweep, ball and hinge joints), every datum counted
    once.  Per body: R as an FP32 pair (72), FP32 Hbar^{-1} (64), the FP32
    solve u (48), fbar as an FP32 pair (96), the FP64 constants sigma, m,
    V mu, V lambda (48), incidence offset (4) read; dqb (FP64, 96) and the
    FP32 correction solve (48) written.  Per joint: its type (1), multipliers
    (8 per row), both anchors (48); a hinge also its frame (72) and second
    points (48).  Per incidence entry: joint index and side (5)."""
    jt = np.asarray(jtype)
    hinge = int(np.sum(jt == 1))
    ball = len(jt) - hinge
    per_body = 72 + 64 + 48 + 96 + 48 + 4 + 96 + 48
    per_ball = 1 + 24 + 48
    per_hinge = 1 + 40 + 48 + 72 + 48
    return float(M * per_body + ball * per_ball + hinge * per_hinge + 2 * len(jt) * 5)


def chain_gram_flops(jtype_chain: np.ndarray) -> float:
    """FP64 flops of the per-body Gram blocks (FMA = 2).  Rows are grouped by
    point; a block is E^T Mbar(p, p') E' with the 3x3 point compliance Mbar
    (30 FMA) and projections of 54 (3x3), 45 (2x3), 36 (3x2) or 30 (2x2)
    FMA; a hinge's rest-frame directions cost 36 FMA.  Per body (lower
    joint, upper joint): ball-ball 252, ball-hinge 489, hinge-ball 498,
    hinge-hinge 795 FMA."""
    t = np.asarray(jtype_chain)
    lo, up = t[:-1], t[1:]           # body j carries joints j and j+1 (both ends pinned)
    fma = np.select([(lo == 0) & (up == 0), (lo == 0) & (up == 1), (lo == 1) & (up == 0)],
                    [252, 489, 498], 795)
    return 2.0 * float(fma.sum())


def seg_bytes(name: str, jtype: np.ndarray, M: int) -> float | None:
    """Algorithmic HBM bytes of one launch of a segment-tiled chain kernel
    (the mixed form with the FP32 reduction), every datum counted once per
    launch (a tile's halo bodies and re-reads of its own data hit L2).
    Per body: q 96, qdot 96, the FP64 constants sigma, m, V mu, V lambda 48,
    the FP32 Hbar^{-1} 64, R as an FP32 pair 72 (its high part alone 36),
    the FP32 vectors u, fbar - Hbar u, dq0 and z 48 each.  Per joint: flags 1;
    C(q_n) 40 (FP64); FP64 anchors 48, and for a hinge the second points 48,
    axis 24 and frame as an FP32 pair 72 (high part 36); FP32 anchors 24 (a
    hinge 48); the tile's factors 260 (65 FP32 per row: L, Ya, Yb); its
    forward-eliminated rhs 20; the approximate multipliers 20 (FP32); the
    multipliers 40 (FP64).
      seg_body:  reads q, qdot, constants, Hbar^{-1}, the FP64 joint data;
                 writes R, u, fbar - Hbar u, the frames and C;
      seg_first: reads R (high), u, Hbar^{-1}, frames (high), C, FP32 anchors;
                 writes the factors and the rhs;
      seg_corr:  reads R, frames, Hbar^{-1}, constants, fbar - Hbar u, u, C,
                 both anchor copies, the factors and the rhs; writes the
                 approximate multipliers, dq0, z and the new rhs;
      seg_final: reads R, frames (high), Hbar^{-1}, q, dq0, z, FP32
                 anchors, the factors, the rhs and the approximate
                 multipliers; writes q, qdot and the multipliers."""
    jt = np.asarray(jtype)
    K = len(jt)
    hg = int(np.sum(jt == 1))
    fp64_pts = 48 * K + 72 * hg
    fp32_pts = 24 * K + 24 * hg
    if name == "seg_body":
        return float(M * (96 + 96 + 48 + 64) + fp64_pts + K + M * (72 + 48 + 48) + 72 * hg + 40 * K)
    if name == "seg_first":
        return float(M * (36 + 48 + 64) + 36 * hg + 40 * K + fp32_pts + K + 260 * K + 20 * K)
    if name == "seg_corr":
        return float(M * (72 + 64 + 48 + 48 + 48) + 72 * hg + 40 * K + fp64_pts + fp32_pts + K + 260 * K
                     + 20 * K + M * (48 + 48) + 20 * K + 20 * K)
    if name == "seg_final":
        return float(M * (72 + 64 + 96 + 48 + 48) + 36 * hg + fp32_pts + K + 260 * K + 20 * K + 20 * K
                     + M * (96 + 96) + 40 * K)
    return None


def tree_up_bytes(M: int, nroots: int, form: str) -> float:
    """Algorithmic HBM bytes of one step's upward elimination passes of the
    tree solver (Alg. 2 read as exact constraint-row elimination), every
    datum counted once per pass.  Per body (FP32 elimination, x2 in FP64):
    its rotation 36 (72), Hbar^{-1} 64 (128), rhs u 48 (96), its joint's
    points and frame 60 (120) read; X = Hhat^{-1} G^T 240, L_D 60, y 48,
    e 20, U = P^T L_D^{-T} 240 and v 48 written (x2 in FP64); per non-root
    body its U and v read again by its parent 288 (576).  The mixed form runs
    two passes per step (the approximate solve and the correction), the FP64
    form one."""
    s = 1 if form != "fp64" else 2
    per_body = s * (36 + 64 + 48 + 60 + 240 + 60 + 48 + 20 + 240 + 48)
    per_child = s * 288
    passes = 2 if form != "fp64" else 1
    return float(passes * (M * per_body + (M - nroots) * per_child))


def pcg_iteration_bytes(M: int, K: int, nfixed: int) -> float:
    """Algorithmic HBM bytes of one FP32 block-Jacobi PCG iteration on the
    dual (matrix-free S p, Sec. 5.5 stand-in), per ball joint: p 12, the
    two FP32 anchors 24, S p written 12, r, z, x read and written 72, the
    preconditioner's Cholesky factor 24, and its bodies' indices 8; per free
    body: R 36, Hbar^{-1} 64, the rest-frame G^T p written and read 96."""
    return float(K * (12 + 24 + 12 + 72 + 24 + 8) + (M - nfixed) * (36 + 64 + 96))


def pcgn_iteration_bytes(K: int, nnz: int) -> float:
    """Algorithmic bytes of one iteration of the normalized-space FP32 PCG
    (ball joints, S~ = I + E, learned preconditioner G^T G), every datum
    counted once per phase that touches it.  Per joint: (A) z, p_old read,
    p, q written 64; (B) r, q, x, p read, r', x, y written and C read 120;
    (C) y, r' read, z written 48.  Per stored block (nnz, both directions):
    (A) E 36 and the neighbour's z, p 32; (B, lower half) E 36, its gate 4,
    the neighbour's r, q 32; (C, upper half) E 36, its coefficient 4, the
    neighbour's y 16."""
    return float(K * (64 + 120 + 48) + nnz * (36 + 32) + nnz / 2 * (36 + 4 + 32) + nnz / 2 * (36 + 4 + 16))


def joint_graph_entries(sc: dict) -> int:
    """Entries of the joint graph (ordered pairs of joints sharing a free body)."""
    fixed = np.asarray(sc["fixed"]) != 0
    deg = np.zeros(len(fixed), dtype=np.int64)
    for ids in (np.asarray(sc["body_a"]), np.asarray(sc["body_b"])):
        ok = ids >= 0
        ok[ok] &= ~fixed[ids[ok]]
        np.add.at(deg, ids[ok], 1)
    return int(np.sum(deg * (deg - 1)))


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a
# kernel, from one ncu capture of the current kernel (scaled to the named
# workload by the bodies it processes where the capture ran a smaller chain);
# an entry is removed when its kernel changes.  Both entries: one ncu capture
# of the current build on the full chain (dram__bytes_read.sum +
# dram__bytes_write.sum), one step after three warm-up steps.
TRAFFIC: dict = {("chain1m", "mixed_fp32_dual", "mx_res_body"): 726.8e6,
                 ("chain1m", "mixed_fp32_dual", "cr_back"): 21.93e6}


def measured_hbm_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0   # the profiling recipe's fallback


def body_prep_flops(M: int, polar_iters: float, form: str) -> float:
    """FP64 flops (FMA = 2) of the per-body kernel over M bodies.  One Newton
    step of the polar iteration: cofactors 27, determinant 5, reciprocal 1,
    X <- X/2 + C/(2 det) 27, step and its squared norm 27 (87); the rest-frame
    rhs: 1/h scalings 4, M_A qdot/h + m g 18, four R^T rotations 60,
    F = R^T A 45, trace 4, V P(F) 24, subtraction 9 (164); the FP64 form also
    applies Hbar^{-1} in FP64 (36).  polar_iters: mean Newton steps per body,
    counted by the kernel (mabd_step_stats.polar_iterations)."""
    rest = 164 + (36 if form == "fp64" else 0)
    return float(M) * (rest + 87.0 * polar_iters)


def kernel_model(name: str, jtype_chain: np.ndarray, form: str = "fp64", polar_iters: float | None = None):
    """(bound, algorithmic work of one step's launches of `name`): FP64 flops
    ("alu") or HBM bytes ("hbm"), or None without a model."""
    if name == "body_prep" and polar_iters is not None:
        return "alu", body_prep_flops(len(jtype_chain) - 1, polar_iters, form)
    # mx_body_prep computes in double-float on the FP32 pipe: no FP64-flop model
    if form != "mixed_fp32_dual" and (name.startswith("cr_reduce") or name == "cr_level"):
        return "alu", cr_reduce_flops(jtype_chain)
    if name == "chain_gram":
        return "alu", chain_gram_flops(jtype_chain)
    if name == "mx_res_body" and form != "fp64":
        return "hbm", mx_res_body_bytes(jtype_chain, len(jtype_chain) - 1)
    if name.startswith("seg_") and form == "mixed_fp32_dual":
        v = seg_bytes(name, jtype_chain, len(jtype_chain) - 1)
        return ("hbm", v) if v is not None else None
    if name == "cr_back":
        passes = 1 if form == "fp64" else 2   # factorization + the correction sweep's pass
        return "hbm", passes * cr_back_bytes(jtype_chain, 4 if form == "mixed_fp32_dual" else 8)
    return None


def time_steps(solver, steps: int, warmup: int, barrier_sync, clocks=None):
    """W untimed steps, then exactly K steps between CUDA events on the
    library's stream, with a barrier and a device synchronize on both sides."""
    import torch
    stream = solver.stream
    solver.step(warmup)
    solver.synchronize()
    barrier_sync()
    if clocks is not None:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(steps)
    e1.record(stream)
    barrier_sync()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks is not None else None
    solver.synchronize()  # surfaces any device-side failure of the timed steps
    return ms, clk


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2603_08079_gb300 import mabd, scenes

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    sc = make_scene(args.workload, args.bodies if args.workload in ("chain1m", "loop1m") else None)
    M = len(sc["mass"])
    form = chosen_form(args)
    solver = mabd.Solver(sc, precision=form, refine_steps=args.refine, pcg_max_iters=20000)
    learned = use_learned(args, form)
    if learned is not None:
        solver.set_preconditioner(learned)
    info = solver.info()
    tree_sched = solver.tree_schedule() if info["solver"] == "tree" else None

    def barrier_sync():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    ms, clk = time_steps(solver, args.steps, args.warmup, barrier_sync, clocks)
    ms_max = max_over_ranks(ms)
    value = job_value(ws, M, args.steps, ms_max)

    # per-kernel times with CUDA events on the library's stream (separate pass)
    solver.profile(True)
    solver.profile_reset()
    solver.step(args.profile_steps)
    kt = solver.kernel_times()
    solver.profile(False)

    # end to end through the C ABI with host buffers: H2D state, step, D2H state
    q_h = torch.empty((M, 12), dtype=torch.float64).pin_memory().numpy()
    qd_h = torch.empty((M, 12), dtype=torch.float64).pin_memory().numpy()
    solver.get_state(q_h, qd_h)
    e2e_steps = max(1, min(args.steps, 5))
    barrier_sync()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_state(q_h, qd_h)
        solver.step(1)
        solver.get_state(q_h, qd_h)
    barrier_sync()
    e2e_s = time.perf_counter() - t0
    e2e_value = ws * M * e2e_steps / e2e_s

    # accuracy of each form against the oracle is checked by the test-suite
    # (tests/test_gpu_chain.py, tests/test_gpu_mixed.py: full-size chain);
    # here the residuals of one step are reported
    st = solver.step(1, stats=True)[0]
    solver.close()

    # the plain FP64 GPU path on the same workload (and, for the learned
    # form, the mixed form with block Jacobi), timed the same way
    plain = None
    others = {}
    if args.workload == "loop1m":
        variants = [("pcg_fp64_gpu", dict(precision="fp64", solver="pcg"), None)]
    else:
        variants = [("plain_fp64_gpu", dict(precision="fp64"), None)] if form != "fp64" else []
    if variants:
        if form == "mixed_fp32_dual" and args.workload == "chain1m":
            variants.append(("mixed_fp64_reduction_gpu", dict(precision="mixed", refine_steps=args.refine),
                             None))
            # the same form as the segment-tiled step (MABD_CHAIN_SEG=1)
            variants.append(("mixed_fp32_dual_segment_tiled_gpu",
                             dict(precision="mixed_fp32_dual", refine_steps=args.refine), "seg"))
        if learned is not None:
            variants.append(("mixed_block_jacobi_gpu", dict(precision="mixed", refine_steps=args.refine),
                             None))
        for key, kw, lp in variants:
            if lp == "seg":
                os.environ["MABD_CHAIN_SEG"] = "1"
            try:
                ref = mabd.Solver(sc, pcg_max_iters=20000, **kw)
            finally:
                os.environ.pop("MABD_CHAIN_SEG", None)
            pms, _ = time_steps(ref, args.steps, args.warmup, barrier_sync)
            extra = {}
            if lp == "seg":
                ref.profile(True)
                ref.profile_reset()
                ref.step(args.profile_steps)
                skt = ref.kernel_times()
                ref.profile(False)
                extra = {"kernels_ms_per_step": {k: round(v[0] / args.profile_steps, 4) for k, v in skt.items()},
                         "launches_per_step": sum(n for _, n in skt.values()) / args.profile_steps,
                         "seg_levels": ref.info()["seg_levels"]}
            rst = ref.step(1, stats=True)[0]
            ref.close()
            pms = max_over_ranks(pms)
            others[key] = {"value": job_value(ws, M, args.steps, pms), "unit": "body-steps/s",
                           "ms_per_step": pms / args.steps}
            others[key].update(extra)
            if rst.get("pcg_iters"):
                others[key]["pcg_iters_per_step"] = rst["pcg_iters"]
        plain = others.get("plain_fp64_gpu")

    result = None
    if rank == 0:
        dom = max(kt.items(), key=lambda kv: kv[1][0])
        dname, (dms, dn) = dom
        per_launch_ms = dms / dn
        launches_per_step = sum(n for _, n in kt.values()) / args.profile_steps
        dom_launches = dn / args.profile_steps
        model = (kernel_model(dname, sc["jtype"], form, st.get("polar_iterations"))
                 if args.workload == "chain1m" else None)
        if model is not None and model[0] == "alu":
            step_flops = model[1]
            flops = step_flops / dom_launches     # per launch, averaged over the levels
            achieved = flops / (per_launch_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                    "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
                    "traffic": TRAFFIC.get((args.workload, form, dname)), "kernel": dname,
                    "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2.07 GHz (probe measured 1.20)",
                    "kernel_ms_per_launch": round(per_launch_ms, 5),
                    "flops_per_step": step_flops, "launches_per_step": dom_launches}
            if dname in ("body_prep", "mx_body_prep"):
                roof["polar_iterations_per_body"] = round(st["polar_iterations"], 4)
        elif model is not None:
            step_bytes = model[1]
            achieved = step_bytes / dom_launches / (per_launch_ms / 1e3) / 1e9
            peak = measured_hbm_gbs()
            roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": TRAFFIC.get((args.workload, form, dname)),
                    "kernel": dname, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "kernel_ms_per_launch": round(per_launch_ms, 5),
                    "bytes_per_step": step_bytes, "launches_per_step": dom_launches}
        else:
            roof = {"bound": "alu", "achieved": None, "peak": round(FP64_PEAK_TFLOPS, 4),
                    "unit": "TFLOP/s", "frac": None, "traffic": None, "kernel": dname}
        result = {
            "metric": METRIC, "value": value, "unit": "body-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if form == "fp64" else "f32+f64",
            "data": "synthetic (seeded generator, paper-shaped %s)" % args.workload,
            "config": workload_config(M, info["joints"], info["dual_rows"], args.workload, form,
                                      args.refine),
            "e2e": {"value": e2e_value, "unit": "body-steps/s",
                    "h2d_bytes_per_step": 2 * 12 * 8 * M, "d2h_bytes_per_step": 2 * 12 * 8 * M},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "roofline": roof,
            "kernels_ms_per_step": {k: round(v[0] / args.profile_steps, 4) for k, v in kt.items()},
            "joint_residual": st["joint_residual"],
            "clocks": clk,
        }
        if form != "fp64":
            result["refine_residual"] = st["refine_residual"]
        result.update(others)
        if learned is not None:
            result["config"]["preconditioner"] = ("learned (3-layer message passing, hidden 64, BF16 "
                                                  "tensor cores), trained parameters %s" % LPC_PARAMS_REL)
        if st.get("pcg_iters"):
            result["pcg_iters_per_step"] = st["pcg_iters"]
        if tree_sched is not None:
            result["config"]["tree_schedule"] = tree_sched
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(args)
            if args.workload == "batch4096":
                result["cpu_baseline_all_cores"] = cpu_baseline_parallel(args)
    # the other paper-shaped workloads in their chosen forms (one GPU only,
    # default run of the chain)
    if ws == 1 and args.workload == "chain1m" and not args.no_sub:
        subs = {}
        for name in SUB_WORKLOADS:
            subs[name] = sub_record(name, args, barrier_sync)
        if result is not None:
            result.update(subs)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


SUB_WORKLOADS = ("tree256k", "batch4096", "net64x64x16")


def sub_record(name: str, args, barrier_sync) -> dict:
    """One of the other paper-shaped workloads, timed like the main one in
    its chosen form with the plain FP64 GPU path beside it (one GPU)."""
    from paper_2603_08079_gb300 import mabd

    sc = make_scene(name)
    M = len(sc["mass"])
    form = "mixed" if name == "net64x64x16" else "mixed_fp32_dual"
    steps = 10 if name == "net64x64x16" else args.steps
    warm = 3
    s = mabd.Solver(sc, precision=form, refine_steps=args.refine, pcg_max_iters=20000)
    sargs = argparse.Namespace(**vars(args))
    sargs.workload = name
    learned = use_learned(sargs, form)
    if learned is not None:
        s.set_preconditioner(learned)
    info = s.info()
    ms, _ = time_steps(s, steps, warm, barrier_sync)
    s.profile(True)
    s.profile_reset()
    s.step(args.profile_steps)
    kt = s.kernel_times()
    s.profile(False)
    st = s.step(1, stats=True)[0]
    sched = s.tree_schedule() if info["solver"] == "tree" else None
    s.close()
    rec = {"config": workload_config(M, info["joints"], info["dual_rows"], name, form, args.refine),
           "form": form, "ms_per_step": ms / steps, "value": M * steps / (ms / 1e3), "unit": "body-steps/s",
           "steps": steps, "warmup": warm,
           "parity": "1e-6 normwise on qdot and lambda against the FP64 oracle, one step from the same "
                     "state, full size (tests/test_gpu_tree_mixed.py, test_gpu_mixed.py, test_gpu_lpc.py)",
           "kernels_ms_per_step": {k: round(v[0] / args.profile_steps, 4) for k, v in kt.items()},
           "launches_per_step": sum(n for _, n in kt.values()) / args.profile_steps,
           "refine_residual": st["refine_residual"], "joint_residual": st["joint_residual"]}
    if learned is not None:
        rec["config"]["preconditioner"] = "learned, trained parameters %s" % LPC_PARAMS_REL
    if st.get("pcg_iters"):
        rec["pcg_iters_per_step"] = st["pcg_iters"]
    if sched is not None:
        rec["config"]["tree_schedule"] = sched
    dname, (dms, dn) = max(kt.items(), key=lambda kv: kv[1][0])
    per_launch_ms = dms / dn
    model = None
    if dname == "tree_up":
        nroots = int(np.sum(np.asarray(sc["fixed"]) != 0)) if name == "batch4096" else 1
        model = tree_up_bytes(M, nroots, form) / (dn / args.profile_steps)
    elif dname == "p32_iteration":
        nfixed = int(np.sum(np.asarray(sc["fixed"]) != 0))
        model = pcg_iteration_bytes(M, info["joints"], nfixed)
    elif dname == "p32_solve" and st.get("pcg_iters"):
        # one launch is a whole solve: its iterations times an iteration's bytes
        iters_per_launch = st["pcg_iters"] / (dn / args.profile_steps)
        model = iters_per_launch * pcgn_iteration_bytes(info["joints"], joint_graph_entries(sc))
    if model is not None:
        achieved = model / (per_launch_ms / 1e3) / 1e9
        peak = measured_hbm_gbs()
        rec["roofline"] = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                           "frac": round(achieved / peak, 4), "traffic": None, "kernel": dname,
                           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                           "kernel_ms_per_launch": round(per_launch_ms, 5), "bytes_per_launch": model}
    else:
        rec["roofline"] = {"bound": "hbm", "achieved": None, "frac": None, "kernel": dname}
    # the plain FP64 GPU path on the same workload
    ref = mabd.Solver(sc, precision="fp64", pcg_max_iters=20000)
    psteps = 3 if name == "net64x64x16" else steps
    pms, _ = time_steps(ref, psteps, warm, barrier_sync)
    ref.close()
    rec["plain_fp64_gpu"] = {"value": M * psteps / (pms / 1e3), "unit": "body-steps/s",
                             "ms_per_step": pms / psteps}
    return rec


def split_assemblies(sc: dict) -> list:
    """The batch scene's assemblies as scenes of their own: an assembly's
    bodies are contiguous from its fixed base body, its joints are those whose
    body a (the parent) lies in that range."""
    M = len(sc["mass"])
    starts = np.flatnonzero(np.asarray(sc["fixed"]) != 0)
    ends = np.append(starts[1:], M)
    owner = np.searchsorted(starts, np.asarray(sc["body_a"]), side="right") - 1
    out = []
    for a, (lo, hi) in enumerate(zip(starts, ends)):
        ks = np.flatnonzero(owner == a)
        sub = {"h": sc["h"], "gravity": sc["gravity"]}
        for key in ("mass", "second_moment", "volume", "young", "poisson", "fixed", "q", "qdot"):
            sub[key] = np.ascontiguousarray(sc[key][lo:hi])
        for key in ("jtype", "anchor_a", "anchor_b", "axis_a", "axis_b", "axis_len"):
            sub[key] = np.ascontiguousarray(sc[key][ks])
        sub["body_a"] = np.ascontiguousarray(sc["body_a"][ks] - lo)
        bb = sc["body_b"][ks]
        sub["body_b"] = np.ascontiguousarray(np.where(bb >= 0, bb - lo, bb))
        out.append(sub)
    return out


_BATCH = None


def _batch_worker_init(n: int, seed: int):
    global _BATCH
    import oracle as ora
    subs = split_assemblies(scenes.assemblies(n, seed=seed))
    _BATCH = [(sub, ora.Scene(sub)) for sub in subs]


def _batch_worker_step(rng) -> int:
    import oracle as ora
    lo, hi = rng
    for sub, S in _BATCH[lo:hi]:
        ora.step(S, sub["q"], sub["qdot"])
    return int(sum(len(sub["mass"]) for sub, _ in _BATCH[lo:hi]))


def batch_oracle_parallel(steps: int, warmup: int, n: int = 4096, seed: int = 3):
    """The oracle, as it stands, on the 4096 independent assemblies run on all
    host cores: one oracle scene per assembly, spread over spawned worker
    processes (each builds the batch in its initializer).  Returns
    (body-steps per step, seconds of the timed steps, workers)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    nch = 4 * cores
    chunks = [(i * n // nch, (i + 1) * n // nch) for i in range(nch)]
    with mp.get_context("spawn").Pool(cores, initializer=_batch_worker_init, initargs=(n, seed)) as pool:
        for _ in range(max(warmup, 1)):
            pool.map(_batch_worker_step, chunks)
        t0 = time.perf_counter()
        for _ in range(steps):
            bodies = sum(pool.map(_batch_worker_step, chunks))
        dt = time.perf_counter() - t0
    return bodies, dt, cores


def cpu_baseline_parallel(args) -> dict:
    bodies, dt, cores = batch_oracle_parallel(1, 1)
    return {"value": bodies / dt, "unit": "body-steps/s", "cores": cores, "kind": "oracle",
            "sample": "1 step of all 4096 assemblies, one oracle scene per assembly, over %d spawned "
                      "worker processes, %s" % (cores, lscpu_model()),
            "seconds": round(dt, 3)}


def cpu_baseline(args, steps: int = 1, M: int | None = None) -> dict:
    """The CPU FP64 oracle as it stands, single-threaded, on a bounded sample."""
    import oracle as ora

    if args.workload == "chain1m":
        M = M or args.cpu_bodies
        sc = scenes.long_chain(M, seed=1)
    elif args.workload == "loop1m":
        sc = scenes.ring_chain(M or args.cpu_bodies, seed=1)
    elif args.workload in ("tree256k", "batch4096"):
        sc = make_scene(args.workload)       # the full scene: a few s per oracle step
    else:
        sc = make_scene(args.workload, 16384)  # a 32x32x16 lattice of the same net
    M = len(sc["mass"])
    S = ora.Scene(sc)
    q, qd = sc["q"], sc["qdot"]
    t0 = time.perf_counter()
    for _ in range(steps):
        q, qd, _, _ = ora.step(S, q, qd)
    dt = time.perf_counter() - t0
    return {"value": M * steps / dt, "unit": "body-steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d step(s) of a %d-body %s (same generator), single thread, %s"
                      % (steps, M, args.workload, lscpu_model()),
            "seconds": round(dt, 3)}


def run_reference(args):
    """CPU oracle arm: W untimed + K timed oracle steps, each on a bounded
    sample of the chain, on the host cores (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle as ora

    cores = 1
    if args.workload == "batch4096":
        # independent assemblies: one oracle scene each, on all host cores
        M, dt, cores = batch_oracle_parallel(args.steps, args.warmup)
        sample = "each step: all 4096 assemblies, one oracle scene per assembly, %d worker processes, %s" % (
            cores, lscpu_model())
    else:
        if args.workload == "chain1m":
            sc = scenes.long_chain(args.cpu_bodies, seed=1)
        elif args.workload == "loop1m":
            sc = scenes.ring_chain(args.cpu_bodies, seed=1)
        elif args.workload == "tree256k":
            sc = make_scene(args.workload)
        else:
            sc = make_scene(args.workload, 16384)
        M = len(sc["mass"])
        S = ora.Scene(sc)
        q, qd = sc["q"], sc["qdot"]
        for _ in range(args.warmup):
            q, qd, _, _ = ora.step(S, q, qd)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            q, qd, _, _ = ora.step(S, q, qd)
        dt = time.perf_counter() - t0
        sample = "each step: a %d-body %s from the same generator, single thread, %s" % (
            M, args.workload, lscpu_model())
    value = M * args.steps / dt
    full = make_scene(args.workload) if args.workload != "chain1m" else None
    if full is None:
        cfg = workload_config(M_FULL, M_FULL + 1, 4194305, "chain1m", chosen_form(args), args.refine)
    else:
        rows = scenes.dual_rows(full)
        cfg = workload_config(len(full["mass"]), len(full["jtype"]), rows, args.workload, chosen_form(args),
                              args.refine)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "body-steps/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator, paper-shaped chain)",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": "body-steps/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "body-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--bodies", type=int, default=M_FULL)
    ap.add_argument("--workload", default="chain1m", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-bodies", type=int, default=M_FULL // 4)
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed", "mixed_fp32_dual"],
                    help="form of the step (auto: mixed with the FP32 reduction for the chain, "
                         "mixed with the learned preconditioner for the net, FP64 otherwise)")
    ap.add_argument("--refine", type=int, default=1, help="FP64 correction sweeps of the mixed form")
    ap.add_argument("--no-sub", action="store_true",
                    help="chain workload: skip the tree, batch and net records")
    ap.add_argument("--no-lpc", action="store_true",
                    help="net workload: block Jacobi instead of the learned preconditioner")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "own":
        args.warmup = 3
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
