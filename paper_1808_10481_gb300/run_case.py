"""Run one Hermite-leapfrog case through the C ABI and print its timing.

  python -m paper_1808_10481_gb300.run_case --dim 2 --m 3 --n 512 --steps 200 [--warmup 3]

The state lives on the device for the whole run; timing is CUDA events around
hl_step.  Used for quick experiments and as the command profiled by ncu.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--m", type=int, default=3)
    ap.add_argument("--n", type=int, nargs="+", default=[512])
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--cfl", type=float, default=0.9)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--path", type=int, default=0, help="0 auto, 1 single CTA, 2 grid launches")
    ap.add_argument("--init", choices=["gaussian", "random", "zero"], default="random")
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp32_comp", "tc_split"], default="fp64")
    ap.add_argument("--tile", type=int, default=-1, help="tile shape index (HL_OPT_TILE); -1 keeps the default")
    ap.add_argument("--split", action="store_true",
                    help="FP64 half-steps as the split pair: interpolant stored, then evolved (HL_OPT_SPLIT)")
    ap.add_argument("--mlp-rows", type=int, default=0,
                    help="instead of stepping: this many rows of MLP training steps (loss, gradient, Adam)")
    ap.add_argument("--mlp-forward", action="store_true",
                    help="with --mlp-rows: time the inference forward (hl_mlp_forward) instead of training steps")
    args = ap.parse_args(argv)
    if args.mlp_rows:
        return run_mlp(args)

    import numpy as np
    import torch

    from paper_1808_10481_gb300 import hl
    from paper_1808_10481_gb300 import inputs as I

    hl.load()
    ncell = args.n * args.dim if len(args.n) == 1 else args.n
    dt = I.cfl_dt(ncell, args.cfl)
    if args.init == "gaussian":
        st = I.gaussian_pulse(args.dim, args.m, ncell, dt, seed=args.seed)
        p, u = st.p, st.u
    elif args.init == "random":
        st = I.random_state(args.dim, args.m, ncell, seed=args.seed)
        p, u = st.p, st.u
    else:
        nq = (args.m + 1) ** args.dim
        p = np.zeros((int(np.prod(ncell)), nq))
        u = np.zeros((args.dim,) + p.shape)
    h = hl.hl_create(args.dim, args.m, ncell, dt)
    try:
        stream = torch.cuda.current_stream()
        hl.hl_set_stream(h, stream)
        if args.path:
            hl.hl_set_option(h, hl.HL_OPT_KERNEL_PATH, args.path)
        if args.tile >= 0:
            hl.hl_set_option(h, hl.HL_OPT_TILE, args.tile)
        if args.split:
            hl.hl_set_option(h, hl.HL_OPT_SPLIT, 1)
        hl.hl_set_precision(h, {"fp64": hl.HL_FP64, "fp32": hl.HL_FP32, "fp32_comp": hl.HL_FP32_COMP,
                                 "tc_split": hl.HL_TC_SPLIT}[args.precision])
        hl.hl_set_initial(h, p, u)
        if args.warmup:
            hl.hl_step(h, args.warmup)
        hl.hl_sync(h)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hl.hl_step(h, args.steps)
        e1.record(stream)
        status = hl.hl_sync(h)
        ms = e0.elapsed_time(e1)
    finally:
        hl.hl_destroy(h)
    dof = (args.dim + 1) * (args.m + 1) ** args.dim * int(np.prod(ncell))
    print(json.dumps({"dim": args.dim, "m": args.m, "n_cells": ncell, "precision": args.precision, "tile": args.tile,
                      "split": args.split,
                      "steps": args.steps, "ms": ms,
                      "ms_per_step": ms / max(args.steps, 1), "dof_updates_per_s": dof * args.steps / (ms / 1e3),
                      "status": status}))
    return 0 if status == hl.HL_OK else 1


def run_mlp(args):
    """MLP training steps on seeded random rows (the learned correction's kernels)."""
    import numpy as np
    import torch

    from paper_1808_10481_gb300 import hl

    hl.load()
    rows = args.mlp_rows
    rng = np.random.default_rng(args.seed)
    X = torch.from_numpy(rng.standard_normal((rows, hl.HL_MLP_IN)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.standard_normal((rows, hl.HL_MLP_OUT)).astype(np.float32)).cuda()
    net = hl.hl_mlp_create(args.seed)
    if args.mlp_forward:
        return run_mlp_forward(args, hl, net, X, rows)
    try:
        stream = torch.cuda.current_stream()
        hl.hl_mlp_set_stream(net, stream)
        for _ in range(args.warmup):
            hl.hl_mlp_loss_grad(net, X, T, rows, want_loss=False)
            hl.hl_mlp_adam_step(net, 1e-3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            hl.hl_mlp_loss_grad(net, X, T, rows, want_loss=False)
            hl.hl_mlp_adam_step(net, 1e-3)
        e1.record(stream)
        loss = hl.hl_mlp_loss_grad(net, X, T, rows)
        ms = e0.elapsed_time(e1)
    finally:
        hl.hl_mlp_destroy(net)
    flops = 3 * 2 * rows * (hl.HL_MLP_IN * hl.HL_MLP_HIDDEN + hl.HL_MLP_HIDDEN ** 2 + hl.HL_MLP_HIDDEN * hl.HL_MLP_OUT)
    print(json.dumps({"mlp_rows": rows, "steps": args.steps, "ms_per_step": ms / max(args.steps, 1),
                      "tflops": flops * args.steps / (ms / 1e3) / 1e12, "loss": loss}))
    return 0


def run_mlp_forward(args, hl, net, X, rows):
    """Inference forwards of `rows` rows: X read once, Y written (the correction's network call)."""
    import torch

    Y = torch.empty((rows, hl.HL_MLP_OUT), dtype=torch.float32, device=X.device)
    try:
        stream = torch.cuda.current_stream()
        hl.hl_mlp_set_stream(net, stream)
        for _ in range(args.warmup):
            hl.hl_mlp_forward(net, X, rows, Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            hl.hl_mlp_forward(net, X, rows, Y)
        e1.record(stream)
        hl.hl_mlp_params(net)          # synchronises and reports an expired tensor-core wait
        ms = e0.elapsed_time(e1)
    finally:
        hl.hl_mlp_destroy(net)
    flops = 2 * rows * (hl.HL_MLP_IN * hl.HL_MLP_HIDDEN + hl.HL_MLP_HIDDEN ** 2 + hl.HL_MLP_HIDDEN * hl.HL_MLP_OUT)
    nbytes = rows * 4 * (hl.HL_MLP_IN + hl.HL_MLP_OUT)
    us = 1e3 * ms / max(args.steps, 1)
    print(json.dumps({"mlp_rows": rows, "forward": True, "steps": args.steps, "us_per_forward": us,
                      "gbs": nbytes / (us / 1e6) / 1e9, "tflops": flops / (us / 1e6) / 1e12}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
