"""Run one plan configuration for a fixed number of steps, for kernel profilers.

Kernel profilers (ncu) select launches by kernel name and launch index; this
runs the 3-D Cahn-Hilliard workload from its seeded initial field for
`--warm` steps (so that the captured steps see the run's steady block states),
then `--steps` more, with direct kernel launches (no graph replay) on a
non-default stream, and prints the plan's statistics.  Every step runs in the
library's kernels; this module only drives the plan.

Example (256^3, complex64, the staged half-spectrum form, steps 500..509):
    python -m paper_2609_03922_gb300.profile_step --dims 256 256 256 --warm 500 --steps 10
The same with the spectrum stored as its half (block map on the half, S1.2):
    python -m paper_2609_03922_gb300.profile_step --dims 256 256 256 --warm 500 --steps 10 --half-storage 1
RCD (M components; dx = 0.5):
    python -m paper_2609_03922_gb300.profile_step --model rcd --components 48 --dims 128 128 128 --block 4 4 4
A batched 2-D plan of several sizes, one launch per pass phase over all of them:
    python -m paper_2609_03922_gb300.profile_step --sides 128 192 256 384 512 --fuse 1 --multi-pass 1
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=3, default=[256, 256, 256])
    ap.add_argument("--block", type=int, nargs=3, default=[8, 8, 8])
    ap.add_argument("--threshold", type=float, default=1e-6)
    ap.add_argument("--reassess", type=int, default=10)
    ap.add_argument("--mode", choices=["adaptive", "regular"], default="adaptive")
    ap.add_argument("--fuse", type=int, default=0, help="1: update fused into the last forward pass")
    ap.add_argument("--half", type=int, default=1, help="1: Hermitian half-spectrum transforms")
    ap.add_argument("--tma", type=int, default=0, help="1: staged update moved by TMA boxes")
    ap.add_argument("--tma-passes", type=int, default=1, help="0: the z inverse copies its tiles by cp.async")
    ap.add_argument("--half-storage", type=int, default=0,
                    help="1: the spectrum stored as its half kx = 0 .. N2/2 with the block map on that half")
    ap.add_argument("--precision", choices=["c64", "c128"], default="c64")
    ap.add_argument("--mean", type=float, default=0.1)
    ap.add_argument("--warm", type=int, default=500)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--model", choices=["ch", "rcd"], default="ch")
    ap.add_argument("--components", type=int, default=48, help="RCD: components M")
    ap.add_argument("--sides", type=int, nargs="*", default=None,
                    help="2-D batched CH plan instead: one run of side s per value (16^2 blocks unless --block2 is given)")
    ap.add_argument("--block2", type=int, nargs=2, default=[16, 16])
    ap.add_argument("--multi-pass", type=int, default=0, help="batched 2-D plans: 1 or 2 = one launch per pass phase")
    ap.add_argument("--predictor", type=int, default=0,
                    help="1: attach the learned predictor (untrained weights, K = 20, J = 100) to a CH plan, "
                         "so that its prediction kernels run at steps 20, 40, 60, 80")
    args = ap.parse_args(argv)

    import torch
    from paper_2609_03922_gb300 import build as B
    B.build()
    from paper_2609_03922_gb300 import spdba
    import workloads as W
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    prec = spdba.SPDBA_C64 if args.precision == "c64" else spdba.SPDBA_C128
    rdt = np.float32 if prec == spdba.SPDBA_C64 else np.float64
    dims = tuple(args.dims)
    if args.sides:
        bd = [(sd, sd) for sd in args.sides]
        c0s = [W.ch_initial_condition(d, mean=args.mean, seed=W.BASE_SEED + i).astype(rdt) for i, d in enumerate(bd)]
        with spdba.Plan(None, tuple(args.block2), threshold=args.threshold, reassess=args.reassess, batch_dims=bd,
                        precision=prec, fuse_update=args.fuse, use_graph=0, multi_pass=args.multi_pass) as plan:
            for r, c0 in enumerate(c0s):
                plan.set_field(c0, run=r)
            plan.step(args.warm)
            plan.step(args.steps)
            plan.sync()
            cfg = plan.get_config()
        print(json.dumps({"sides": args.sides, "multi_pass": cfg["multi_pass"], "fuse_update": cfg["fuse_update"]}))
        return
    kw = {}
    if args.model == "rcd":
        M = args.components
        c0 = W.rcd_initial_condition(dims, M, W.rcd_lv_homogeneous(M), 0.1, seed=W.BASE_SEED + M).astype(rdt)
        kw = dict(model=spdba.SPDBA_MODEL_RCD, components=M, dx=0.5)
    else:
        c0 = W.ch_initial_condition(dims, mean=args.mean, seed=W.BASE_SEED).astype(rdt)
    with spdba.Plan(dims, tuple(args.block), threshold=args.threshold, reassess=args.reassess, precision=prec,
                    mode=spdba.SPDBA_MODE_ADAPTIVE if args.mode == "adaptive" else spdba.SPDBA_MODE_REGULAR,
                    fuse_update=args.fuse, half_spectrum=args.half, use_graph=0, tma_update=args.tma,
                    tma_passes=args.tma_passes, half_storage=args.half_storage, **kw) as plan:
        if args.predictor:
            m = tuple(d // b for d, b in zip(dims, args.block))
            pred = spdba.Predictor(m, max_batch=1, params=spdba.predictor_init_params(0))   # outlives the plan's steps
            plan.attach_predictor(pred, 20, 100, 0.5)
        plan.set_field(c0)
        plan.step(args.warm)
        plan.step(args.steps)
        plan.sync()
        st = plan.get_stats()
    print(json.dumps({"dims": dims, "steps": st["step"], "n_active": st["n_active"],
                      "n_transition": st["n_transition"], "nblocks": st["nblocks"]}))


if __name__ == "__main__":
    main()
