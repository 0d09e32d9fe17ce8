"""Trains the learned block preconditioner of the mixed-precision PCG path on
dual systems that the solver itself generates, with the library's own
forward and backward kernels, and writes the parameters.

Recipe: a scene of `--nets` disjoint jittered closed-loop nets (sizes 4..10 x
4..10 x 3..6, the form of the 64x64x16 workload); `--captures` times, the
nets are put in a random perturbed state, stepped 1-3 times by the mixed
solver and the normalized dual of the resulting state is captured (one
capture = one system per net, so captures x nets systems in all); then
`--iters` Adam steps on random captures with `--nv` probe vectors each, on
Kaporin's condition number of the preconditioned dual (or the Frobenius
distance of G S~ G^T from the identity, `--kind frobenius`).

  python -m paper_2603_08079_gb300.train_lpc --out paper_2603_08079_gb300/data/lpc_params.npy
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import mabd, scenes

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "data", "lpc_params.npy")


def pcg_iterations(sc: dict, *params_list, refine_steps: int = 1) -> tuple:
    """FP32 PCG iterations of one mixed step: block Jacobi, then with each
    parameter vector given."""
    out = []
    for p in (None,) + params_list:
        s = mabd.Solver(sc, precision="mixed", refine_steps=refine_steps, pcg_max_iters=20000)
        try:
            if p is not None:
                s.set_preconditioner(p)
            out.append(s.step(1, stats=True)[0]["pcg_iters"])
        finally:
            s.close()
    return tuple(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nets", type=int, default=48)
    ap.add_argument("--captures", type=int, default=210)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nv", type=int, default=2)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--kind", default="kaporin", choices=["kaporin", "frobenius"])
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--eval", action="store_true", help="compare PCG iterations on held-out nets")
    args = ap.parse_args()

    t0 = time.time()
    sc = scenes.net_collection(args.nets, seed=10 + args.seed)
    solver = mabd.Solver(sc, precision="mixed", refine_steps=1, pcg_max_iters=20000)
    trainer = mabd.LpcTrainer()
    for c in range(args.captures):
        q, qd = scenes.perturb_state(sc, seed=1000 + c, rot=0.3, vel=0.5)
        solver.set_state(q, qd)
        solver.step(1 + c % 3)
        trainer.capture(solver)
    t1 = time.time()
    p0 = scenes.lpc_init_params(args.seed)
    params, losses = trainer.train(p0, args.iters, lr=args.lr, nv=args.nv, seed=args.seed, kind=args.kind)
    t2 = time.time()
    l_first = float(np.mean(losses[:50])) if len(losses) else None
    l_last = float(np.mean(losses[-50:])) if len(losses) else None
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, params.astype(np.float32))
    meta = {
        "systems": args.captures * args.nets, "nets": args.nets, "captures": args.captures,
        "joints_per_capture": int(len(sc["jtype"])), "iters": args.iters, "lr": args.lr,
        "nv": args.nv, "seed": args.seed, "objective": args.kind,
        "loss_first50": l_first, "loss_last50": l_last,
        "capture_s": round(t1 - t0, 2), "train_s": round(t2 - t1, 2),
    }
    if args.eval:
        ev = {}
        for name, net in (("16x16x8", scenes.jittered_net(16, 16, 8, seed=4)),
                          ("64x64x16", scenes.jittered_net(64, 64, 16, seed=4))):
            ev[name] = pcg_iterations(net, p0, params)
        meta["pcg_iterations_block_jacobi_untrained_trained"] = ev
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))
    trainer.close()
    solver.close()


if __name__ == "__main__":
    main()
