#!/usr/bin/env python
"""Hermite-leapfrog benchmark on GB300.

Headline workload (the default; one bench "step" = 20 consecutive leapfrog steps of it): 3D acoustics on the
periodic unit cube, 256^3 nodes per grid, m = 2 (27 scaled derivatives per node and field
component), plane wave p = cos(k.x - |k| t + phi) with seeded wave vector k = 2 pi n,
|n| <= 8, 100 leapfrog steps at C_CFL = 0.9.
Metric: DOF-updates/s = (dim+1) (m+1)^dim N^dim * leapfrog steps / time, for the FP64 path
(`value`), and for each mixed-precision mode beside its L2 error against the exact plane
wave and the time of the coarsest plain FP64 grid that is at least as accurate.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hl|reference] [--workload ...]

--impl hl (default): the CUDA library through its C ABI.  `value` is device time
(CUDA events on the library's stream) with the state resident in HBM (14.5 GB, larger
than L2); `e2e` is the same run timed on the host through hl_set_initial / hl_step /
hl_get_fields with pinned host buffers.
--impl reference: the CPU oracle (plain C, FP64, OpenMP over nodes) on the host cores,
each step a bounded sample (one leapfrog step of the same problem on a 32^3 grid).
Under torchrun every rank solves its own independently seeded problem (no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Hermite-leapfrog DOF-updates/s vs FP64 plain at equal L2 error; % roofline"
UNIT = "DOF-updates/s"
DIM, M, N, LF_STEPS = 3, 2, 256, 100
# one timed bench step: this many consecutive leapfrog steps of the 100-step run (each step does
# the full 256^3 work; the whole 100-step run is timed for e2e and for the L2 error comparison)
TIMED_LF = 20
WAVE_SEED = 3
SAMPLE_N = 32            # CPU samples: one leapfrog step of the same problem on 32^3
L2_FLUSH_BYTES = 256 << 20

# FP64 peak of one GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA per SM
# per clock x 2 flop x 2.070 GHz maximum SM clock.
N_SM = 152
FP64_FMA_PER_SM_CLK = 2
SM_MAX_GHZ = 2.070
FP64_PEAK_FLOPS = N_SM * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_GHZ * 1e9

# DRAM traffic of the dominant kernel per launch from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only while the kernel
# source is unchanged (keyed by the hash of the kernel header); per workload.
TRAFFIC_SOURCE_HASH = "5629d2e800a9a677"
# 3D: captured at 128^3 (2,097,152 nodes, 2.3 GB a launch, streaming) and scaled by the node
# count to 256^3 (x8); the FP64 kernels read and write every node's data once per launch.
TRAFFIC_BYTES = {"2d": {"p_half": 103940096, "u_half": None},
                 "3d": {"p_half": 18202758144, "u_half": 25131762688}}

WORKLOAD = ("3D acoustics p_t+div u=0, u_t+grad p=0, periodic unit cube, 256^3 nodes per grid, "
            "m=2 (27 scaled derivatives per node per field), FP64, plane wave with seeded wave vector "
            "k=2 pi n, |n|<=8, and phase, 100 leapfrog steps at C_CFL=0.9 (a timed bench step is 20 of them; "
            "e2e and the L2 errors run all 100)")
WORKLOAD_2D = ("2D acoustics p_t+div u=0, u_t+grad p=0, periodic unit square, 512x512 nodes per grid, "
               "m=3 (16 scaled derivatives per node per field), FP64, seeded Gaussian pressure pulse "
               "(width 0.05, random centre), 200 leapfrog steps per bench step at C_CFL=0.9")


def headline_config():
    """The config block both arms print (the reference arm times a bounded CPU sample of it)."""
    return {"workload": WORKLOAD, "dim": DIM, "m": M, "n_cells": [N] * DIM, "leapfrog_steps_per_step": TIMED_LF,
            "leapfrog_steps_per_run": LF_STEPS,
            "l2": "inputs larger than L2 (14.5 GB of FP64 state)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hl", "reference"], default="hl")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-seeds", type=int, default=96, help="learned workload: training seeds")
    ap.add_argument("--test-seeds", type=int, default=32, help="learned workload: held-out seeds")
    ap.add_argument("--workload", choices=["3d", "2d", "1d", "batch", "mixed3d", "mixed2d", "learned", "split3d",
                                           "modified1d", "variable1d"], default="3d",
                    help="3d: the headline line; the others measure further rows of the solver")
    return ap.parse_args()


def dofs(dim=DIM, m=M, n=N):
    return (dim + 1) * (m + 1) ** dim * n ** dim


def tc_issued_flops_per_step(dim, m, ncell):
    """Dense FP16 tensor-core flops the split mode's MMAs issue in one leapfrog step: per
    128-node tile and unit, data digit i multiplies 4 vertices' operands of K = 16 slots
    by the 32-column (2D p-half: 16) blocks of levels i .. i + nlev_i - 1 (nlev = 7, 6, 5,
    4, 3, 2: 27 level blocks)."""
    if dim not in (2, 3):
        return 0.0
    tiles = -(-ncell[0] // 128) * int(math.prod(ncell[1:]))
    lev_blocks = 27
    per_block = 4 * 128 * 16 * 2                              # vertices x M x K x 2
    if dim == 2:
        units_cols = 2 * 16 + 1 * 32                           # p-half: 2 units of N 16; u-half: 1 of N 32
    else:
        units_cols = 12 * 32 + 12 * 32                         # 12 units a half, N 32 per level
    return float(tiles * units_cols * lev_blocks * per_block)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def tc_roofline(dim, m, ncell, ms_per_step, peaks):
    fl = tc_issued_flops_per_step(dim, m, ncell)
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    ach = fl / (ms_per_step / 1e3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "peak_source": ("measured bf16 sustained (FP16 has the same dense rate)" if peaks else "fallback"),
            "flops": "dense FP16 MMA flops issued (digit pairs of 27 level blocks, padded slots included) over "
                     "the whole step time (cut, exponent and tensor-core kernels)"}


def kernel_hash():
    h = hashlib.sha256()
    for f in ("hl_fp64.cuh",):  # the FP64 kernels' source
        with open(os.path.join(ROOT, "paper_1808_10481_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            if vis and vis.split(",")[0].isdigit():
                cmd += ["-i", vis.split(",")[0]]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline_sample(target_s: float = 15.0):
    """The oracle as it stands on the host cores: leapfrog steps of the headline problem on
    a 32^3 grid (the per-node work does not depend on the grid size, so DOF-updates/s carry
    over), for about target_s seconds; and on one thread, one step of a 16^3 grid."""
    import oracle
    from paper_1808_10481_gb300 import inputs as I
    ncell = [SAMPLE_N] * DIM
    dt = I.cfl_dt(ncell)
    st = I.plane_wave(M, ncell, dt, seed=WAVE_SEED)
    t0 = time.perf_counter()
    p, u = oracle.run(DIM, M, ncell, dt, st.p, st.u, 1)
    t1 = time.perf_counter() - t0
    extra = max(0, int(target_s / max(t1, 1e-9)) - 1)
    t0 = time.perf_counter()
    if extra:
        oracle.run(DIM, M, ncell, dt, p, u, extra)
    t2 = time.perf_counter() - t0
    steps = 1 + extra
    secs = t1 + t2
    cores = oracle.threads()
    n1 = [16] * DIM
    dt1 = I.cfl_dt(n1)
    st1 = I.plane_wave(M, n1, dt1, seed=WAVE_SEED)
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.run(DIM, M, n1, dt1, st1.p, st1.u, 1)
        s1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return {"value": dofs(n=SAMPLE_N) * steps / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} leapfrog step(s) of the plane-wave problem on a {SAMPLE_N}^3 grid (m=2) in "
                      f"{secs:.1f} s (plain C oracle, OpenMP over nodes); per-node work as at 256^3",
            "single_core": {"value": dofs(n=16) / s1, "unit": UNIT, "cores": 1,
                            "sample": f"1 leapfrog step of the 16^3 m=2 problem in {s1:.1f} s on one thread"}}


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    from paper_1808_10481_gb300 import inputs as I
    ncell = [SAMPLE_N] * DIM
    dt = I.cfl_dt(ncell)
    st = I.plane_wave(M, ncell, dt, seed=WAVE_SEED)
    p, u = st.p, st.u
    for _ in range(args.warmup):
        p, u = oracle.run(DIM, M, ncell, dt, p, u, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p, u = oracle.run(DIM, M, ncell, dt, p, u, 1)
    secs = time.perf_counter() - t0
    # each step is a bounded sample of one run: one leapfrog step on 32^3 stands for the
    # 100 leapfrog steps on 256^3 at the same DOF-updates/s
    value = dofs(n=SAMPLE_N) * args.steps / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(),
        "sample": f"each step = 1 leapfrog step of the same plane-wave problem on a {SAMPLE_N}^3 grid",
        "parallelism": "host cores (OpenMP)",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"{args.steps} timed leapfrog steps of the m=2 plane-wave problem on "
                                   f"{SAMPLE_N}^3"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def fp64_flops_per_node_step(dim, m):
    """Algorithmic FP64 flops of one node and full step of the fused kernels
    (multiply-add = 2, butterfly and final additions = 1)."""
    from paper_1808_10481_gb300 import hl
    fma, add = hl.hl_op_counts(dim, m)
    return 2 * fma + add


def run_aux(args, rank=0, world=1, dist=None):
    """Measurements of the other workloads (one JSON line, printed by rank 0).  The batched
    workload shards its shots over the ranks by cost; the others run on rank 0 only."""
    import numpy as np
    import torch

    from paper_1808_10481_gb300 import build as libbuild
    from paper_1808_10481_gb300 import hl
    from paper_1808_10481_gb300 import inputs as I

    libbuild.build()
    hl.load()
    stream = torch.cuda.current_stream()
    out = {"metric": METRIC, "unit": UNIT, "dtype": "f64", "data": "synthetic", "higher_is_better": True}
    if args.workload == "1d":
        d, m, ncell, lf = 1, 3, [64], 1000
        dt = I.cfl_dt(ncell)
        st = I.standing_mode(d, m, ncell, dt, wave=[3])
        desc = "1D, 64 nodes, m=3, p=sin(2 pi 3 x), u at dt/2 from the exact standing mode, 1000 steps"
        h = hl.hl_create(d, m, ncell, dt)
        hl.hl_set_stream(h, stream)
        hl.hl_set_initial(h, st.p, st.u)
        hl.hl_step(h, min(lf, 3))
        hl.hl_sync(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hl.hl_step(h, lf)
        e1.record(stream)
        rc = hl.hl_sync(h)
        ms = e0.elapsed_time(e1)
        hl.hl_destroy(h)
        nnode = int(np.prod(ncell))
        dof = (d + 1) * (m + 1) ** d * nnode
        fl = fp64_flops_per_node_step(d, m) * nnode * lf
        out.update({"workload": args.workload, "value": dof * lf / (ms / 1e3), "ms_per_run": ms,
                    "config": {"workload": desc, "dim": d, "m": m, "n_cells": ncell, "leapfrog_steps": lf},
                    "roofline": {"bound": "alu", "achieved": fl / (ms / 1e3) / 1e12, "peak": FP64_PEAK_FLOPS / 1e12,
                                 "unit": "TFLOP/s", "frac": fl / (ms / 1e3) / FP64_PEAK_FLOPS},
                    "status": rc})
    elif args.workload in ("mixed3d", "mixed2d"):
        # each precision mode on the same problem: DOF-updates/s beside its L2 error
        if args.workload == "mixed3d":
            d, m, ncell, lf = 3, 2, [256, 256, 256], 100
            dt = I.cfl_dt(ncell)
            st = I.plane_wave(m, ncell, dt, seed=3)
            ex = I.plane_wave(m, ncell, dt, seed=3, t0=lf * dt)
            desc = "3D, 256^3 nodes per grid, m=2, plane wave |n|<=8 (seed 3), 100 steps"
        else:
            d, m, ncell, lf = 2, 3, [512, 512], 200
            dt = I.cfl_dt(ncell)
            st = I.gaussian_pulse(d, m, ncell, dt, seed=1)
            ex = None
            desc = "2D, 512^2 nodes per grid, m=3, Gaussian pulse (seed 1), 200 steps"
        nnode = int(np.prod(ncell))
        dof = (d + 1) * (m + 1) ** d * nnode
        modes = {}
        ref_p = None
        mode_list = [("fp64", hl.HL_FP64), ("fp32", hl.HL_FP32), ("fp32_comp", hl.HL_FP32_COMP)]
        if d in getattr(hl, "TC_SPLIT_DIMS", (2,)):
            mode_list.append(("tc_split", hl.HL_TC_SPLIT))
        for name, mode in mode_list:
            h = hl.hl_create(d, m, ncell, dt)
            hl.hl_set_stream(h, stream)
            hl.hl_set_precision(h, mode)
            hl.hl_set_initial(h, st.p, st.u)
            tile, _ = hl.hl_autotune(h, 1)
            hl.hl_set_option(h, hl.HL_OPT_TIMING, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hl.hl_step(h, lf)
            e1.record(stream)
            hl.hl_sync(h)
            ms = e0.elapsed_time(e1)
            kt, kc = hl.hl_kernel_times(h)
            pg, ug, _, _ = hl.hl_get_fields(h)
            hl.hl_destroy(h)
            r = {"value": dof * lf / (ms / 1e3), "ms_per_step": ms / lf, "tile": hl.TILES[tile],
                 "p_half_us": 1e3 * kt["p_half"] / max(kc["p_half"], 1),
                 "u_half_us": 1e3 * kt["u_half"] / max(kc["u_half"], 1)}
            if ex is not None:
                r["l2_err_p_vs_exact"] = I.l2_error(d, ncell, pg, ex.p)
            if ref_p is None:
                ref_p = pg
            else:
                r["max_rel_diff_vs_fp64"] = float(np.abs(pg - ref_p).max() / np.abs(ref_p).max())
            # HBM-bound modes: state bytes moved per step / step time vs measured copy bandwidth
            nq = (m + 1) ** d
            bytes_step = (3 * d + 3) * nq * 8 * nnode
            r["hbm_gbs"] = bytes_step / (ms / lf / 1e3) / 1e9
            modes[name] = r
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except OSError:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        for name in [k for k in modes if k != "fp64"]:
            modes[name]["roofline"] = {"bound": "hbm", "achieved": modes[name]["hbm_gbs"], "peak": hbm,
                                       "unit": "GB/s", "frac": modes[name]["hbm_gbs"] / hbm,
                                       "peak_source": "measured" if peaks else "fallback"}
            if name == "tc_split":
                modes[name]["roofline"] = tc_roofline(d, m, ncell, modes[name]["ms_per_step"], peaks)
        if ex is not None:
            # equal L2 error: plain FP64 on coarser grids to the same final time; each
            # mode is compared with the coarsest FP64 grid whose error is no larger
            t_end = lf * dt
            ladder = []
            for n2 in (48, 64, 80, 96, 128, 160):
                c2 = [n2] * d
                steps2 = int(math.ceil(t_end / I.cfl_dt(c2) - 1e-9))
                dt2 = t_end / steps2
                st2 = I.plane_wave(m, c2, dt2, seed=3)
                ex2 = I.plane_wave(m, c2, dt2, seed=3, t0=t_end)
                h = hl.hl_create(d, m, c2, dt2)
                hl.hl_set_stream(h, stream)
                hl.hl_set_initial(h, st2.p, st2.u)
                hl.hl_step(h, 2)
                hl.hl_set_initial(h, st2.p, st2.u)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hl.hl_step(h, steps2)
                e1.record(stream)
                hl.hl_sync(h)
                pg2, _, _, _ = hl.hl_get_fields(h)
                hl.hl_destroy(h)
                ladder.append({"n": n2, "steps": steps2, "ms_run": e0.elapsed_time(e1),
                               "l2_err_p_vs_exact": I.l2_error(d, c2, pg2, ex2.p)})
            ladder.append({"n": ncell[0], "steps": lf, "ms_run": modes["fp64"]["ms_per_step"] * lf,
                           "l2_err_p_vs_exact": modes["fp64"]["l2_err_p_vs_exact"]})
            for name in [k for k in modes if k != "fp64"]:
                e = modes[name]["l2_err_p_vs_exact"]
                ok = [r for r in ladder if r["l2_err_p_vs_exact"] <= e * 1.001]  # equal within 0.1%
                if ok:
                    r = min(ok, key=lambda r: r["ms_run"])
                    t_mode = modes[name]["ms_per_step"] * lf
                    modes[name]["fp64_at_equal_error"] = {
                        "n": r["n"], "ms_run": r["ms_run"], "l2_err_p_vs_exact": r["l2_err_p_vs_exact"],
                        "ms_run_mode": t_mode, "speedup_vs_fp64_at_equal_error": r["ms_run"] / t_mode}
            out["fp64_error_ladder"] = ladder
        # headline of the line: the fastest mode that keeps the FP64 solution (the split modes)
        best = max([k for k in ("fp32_comp", "tc_split") if k in modes], key=lambda k: modes[k]["value"])
        out.update({"workload": args.workload, "value": modes[best]["value"], "value_mode": best,
                    "config": {"workload": desc, "dim": d, "m": m, "n_cells": ncell, "leapfrog_steps": lf},
                    "modes": modes})
    elif args.workload == "learned":
        out.update(run_learned(args, n_train=args.train_seeds, n_test=args.test_seeds, dist=dist))
    elif args.workload == "split3d":
        out.update(run_split3d(hl, I, stream))
    elif args.workload in ("modified1d", "variable1d"):
        out.update(run_1d_variant(args.workload, hl, I, stream))
    else:
        from paper_1808_10481_gb300.sharding import max_over_ranks, shard_by_cost
        d, m, n_shots, lf = 2, 3, 64, 500
        rng = np.random.default_rng(2024)
        sizes_all = [int(x) for x in rng.integers(128, 1025, size=n_shots)]
        x0_all = [list(rng.random(2)) for _ in range(n_shots)]
        f0_all = [float(x) for x in rng.uniform(10.0, 20.0, size=n_shots)]
        mine = shard_by_cost([n * n for n in sizes_all], world)[rank]
        sizes = [sizes_all[i] for i in mine]
        x0 = [x0_all[i] for i in mine]
        f0 = [f0_all[i] for i in mine]
        n_shots = len(mine)
        cells = [[n, n] for n in sizes]
        dts = [I.cfl_dt(c) for c in cells]
        def run_batch(mode):
            h = hl.hl_create_batch(d, m, cells, dts)
            try:
                hl.hl_set_stream(h, stream)
                hl.hl_set_precision(h, mode)
                best, tile_ms = hl.hl_autotune(h, 2)
                hl.hl_set_sources(h, x0, [0.01] * n_shots, f0, [1.0] * n_shots)
                hl.hl_step(h, 5)
                hl.hl_sync(h)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hl.hl_step(h, lf)
                e1.record(stream)
                rc = hl.hl_sync(h)
                p_dev = torch.empty(h.nnode * h.nq, dtype=torch.float64, device="cuda")
                hl.hl_get_fields_device(h, p_dev, None)
            finally:
                hl.hl_destroy(h)
            return e0.elapsed_time(e1), rc, best, tile_ms, p_dev

        ms, rc, best, tile_ms, p64 = run_batch(hl.HL_FP64)
        ms = max_over_ranks(ms, dist, "cuda")
        nnode = sum(n * n for n in sizes_all)
        dof = (d + 1) * (m + 1) ** d * nnode
        # the same run in the mixed modes (every shot has dt/h = 0.9, so one operator table serves all)
        modes = {}
        scale = float(p64.abs().max())
        for name, mode in (("fp32", hl.HL_FP32), ("fp32_comp", hl.HL_FP32_COMP), ("tc_split", hl.HL_TC_SPLIT)):
            ms_m, rc_m, best_m, _, pm = run_batch(mode)
            ms_m = max_over_ranks(ms_m, dist, "cuda")
            modes[name] = {"value": dof * lf / (ms_m / 1e3), "ms_per_run": ms_m, "tile": hl.TILES[best_m],
                           "max_rel_diff_vs_fp64_p": float((pm - p64).abs().max()) / scale if scale > 0 else 0.0,
                           "status": rc_m}
            del pm
        fl = fp64_flops_per_node_step(d, m) * nnode * lf
        out.update({"workload": "batch", "n_gpus": world, "scaling": "strong (64 shots split by cost)", "value": dof * lf / (ms / 1e3), "ms_per_run": ms,
                    "config": {"workload": "64 independent 2D shots, n ~ U{128..1024} per axis (seed 2024), m=3, "
                                           "FP64, Ricker source per shot (f0 ~ U[10,20], sigma 0.01, seeded x0) "
                                           "from a zero field, 500 steps, one CUDA graph per run",
                               "total_nodes": nnode, "tile": hl.TILES[best], "tile_ms_per_step": tile_ms},
                    "roofline": {"bound": "alu", "achieved": fl / (ms / 1e3) / 1e12 / world,
                                 "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                                 "frac": fl / (ms / 1e3) / FP64_PEAK_FLOPS / world},
                    "mixed_modes": modes,
                    "status": rc})
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_split3d(hl, I, stream):
    """Section 6's comparison on GB300: the fused FP64 kernels against the split pair
    (interpolant stored, then evolved), 3D plane wave, m = 1/2/3 on the paper's grids
    200^3 / 130^3 / 100^3 (Table 6), time per iteration (p-half + u-half) and each form's
    algorithmic FP64 rate and HBM bandwidth per half-step."""
    import numpy as np
    import torch
    rows = {}
    for m, n in ((1, 200), (2, 130), (3, 100)):
        ncell = [n] * 3
        dt = I.cfl_dt(ncell)
        st = I.plane_wave(m, ncell, dt, seed=3)
        nq, A = (m + 1) ** 3, 2 * m + 2
        AD = A ** 3
        nnode = n ** 3
        res = {}
        for name, split in (("fused", 0), ("split", 1)):
            h = hl.hl_create(3, m, ncell, dt)
            try:
                hl.hl_set_stream(h, stream)
                hl.hl_set_option(h, hl.HL_OPT_KERNEL_PATH, 2)
                if split:
                    hl.hl_set_option(h, hl.HL_OPT_SPLIT, 1)
                else:
                    hl.hl_autotune(h, 1)
                hl.hl_set_initial(h, st.p, st.u)
                hl.hl_step(h, 3)
                hl.hl_sync(h)
                hl.hl_set_option(h, hl.HL_OPT_TIMING, 1)
                hl.hl_kernel_times(h)
                steps = 10
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hl.hl_step(h, steps)
                e1.record(stream)
                rc = hl.hl_sync(h)
                kt, kc = hl.hl_kernel_times(h)
            finally:
                hl.hl_destroy(h)
            r = {"ms_per_iteration": e0.elapsed_time(e1) / steps, "p_half_ms": kt["p_half"] / kc["p_half"],
                 "u_half_ms": kt["u_half"] / kc["u_half"], "status": rc}
            if split:
                # per half-step: interpolation reads the partner once and writes its interpolant,
                # evolution reads the interpolant and the node's own data and writes them back
                bytes_p = 8 * nnode * (3 * nq + 3 * AD + 3 * AD + 2 * nq)
                bytes_u = 8 * nnode * (nq + AD + AD + 2 * 3 * nq)
                fl_p = 2 * nnode * 3 * (3 * AD * A)
                fl_u = 2 * nnode * (3 * AD * A)
            else:
                fma, add = hl.hl_op_counts(3, m)
                bytes_p = 8 * nnode * (3 * nq + 2 * nq)
                bytes_u = 8 * nnode * (nq + 2 * 3 * nq)
                fl_p = fl_u = nnode * (fma + add / 2.0)   # half of the full step's count each
            r["p_half_gbs"] = bytes_p / (r["p_half_ms"] / 1e3) / 1e9
            r["u_half_gbs"] = bytes_u / (r["u_half_ms"] / 1e3) / 1e9
            r["p_half_interp_gflops"] = fl_p / (r["p_half_ms"] / 1e3) / 1e9
            r["u_half_interp_gflops"] = fl_u / (r["u_half_ms"] / 1e3) / 1e9
            res[name] = r
        res["split_over_fused"] = res["split"]["ms_per_iteration"] / res["fused"]["ms_per_iteration"]
        res["dof_updates_per_s_fused"] = 4 * nq * nnode / (res["fused"]["ms_per_iteration"] / 1e3)
        rows[f"m{m}_{n}^3"] = res
    return {"workload": "split3d", "value": rows["m2_130^3"]["dof_updates_per_s_fused"],
            "config": {"workload": "3D plane wave, m = 1/2/3 on 200^3/130^3/100^3 (Table 6 sizes), fused "
                                   "FP64 kernels against the split interpolation + evolution pair, 10 iterations"},
            "table6": rows,
            "note": "split rows' GB/s count the stored interpolant round trip; GFLOP/s count the "
                    "interpolation's sum-factorised multiply-adds (fused: the fused operator's)"}


def run_1d_variant(workload, hl, I, stream):
    """Throughput of the 1D method variants on a long periodic interval: the modified
    Hermite-leapfrog scheme (both fields on both grids) and the variable wave speed."""
    import math
    import numpy as np
    import torch
    m, n, steps = 3, 1 << 22, 50
    if workload == "modified1d":
        dt = 0.9 / n
        st = I.standing_mode_1d_both_grids(m, n, dt, 3)
        h = hl.hl_mod_create(m, n, dt)
        try:
            hl.hl_mod_set_stream(h, stream)
            hl.hl_mod_set_initial(h, *st)
            hl.hl_mod_step(h, 3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hl.hl_mod_step(h, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            hl.hl_mod_get_fields(h)
        finally:
            hl.hl_mod_destroy(h)
        dof = 4 * (m + 1) * n   # p and u on both grids
        desc = "modified Hermite-leapfrog, 1D, m=3, 2^22 nodes per grid, standing wave, 50 steps"
        bytes_step = 8 * n * (m + 1) * (4 + 2 * 4)    # both grids: read partner (2 fields), read+write own (2 fields)
    else:
        dt = 0.9 / n / I.c2_max()
        p, u, _, _ = I.variable_speed_wave(m, n, dt)
        h = hl.hl_create(1, m, [n], dt)
        try:
            hl.hl_set_stream(h, stream)
            hl.hl_set_wave_speed(h, I.c2_taylor_table(n, m, False), I.c2_taylor_table(n, m, True))
            hl.hl_set_initial(h, p, u.reshape(1, n, m + 1))
            hl.hl_step(h, 3)
            hl.hl_sync(h)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hl.hl_step(h, steps)
            e1.record(stream)
            hl.hl_sync(h)
        finally:
            hl.hl_destroy(h)
        dof = 2 * (m + 1) * n
        desc = "variable wave speed c^2 = 1 + sin(2 pi x)/2, 1D, m=3, 2^22 nodes, 50 steps"
        bytes_step = 8 * n * ((m + 1) * 6 + 2 * (2 * m + 2))   # fields + both c^2 tables
    ms = e0.elapsed_time(e1)
    return {"workload": workload, "value": dof * steps / (ms / 1e3), "ms_per_step": ms / steps,
            "hbm_gbs_algorithmic": bytes_step * steps / (ms / 1e3) / 1e9,
            "config": {"workload": desc, "dim": 1, "m": m, "n_cells": [n]}}


def run_learned(args, n_train=96, n_test=32, horizon=32, seed0=1000, dist=None):
    """Learned coarse-grid correction at the workload's scale: coarse 256^2 vs fine 1024^2,
    m = 3, seeded Gaussian pulses and Ricker sources; the fine FP64 solver is the reference.
    Under torchrun the training seeds are sharded over the ranks and the network trains data-
    parallel (gradients averaged by all-reduce before every Adam step); rank 0 evaluates."""
    import numpy as np
    import torch

    from paper_1808_10481_gb300 import hl
    from paper_1808_10481_gb300 import inputs as I
    from paper_1808_10481_gb300 import learned

    world = dist.get_world_size() if dist is not None else 1
    rank = dist.get_rank() if dist is not None else 0
    train_lo, train_hi = learned.shard_range(n_train, world, rank)

    nc, r = [256, 256], 4
    nf = [nc[0] * r, nc[1] * r]
    rows = nc[0] * nc[1]
    dev = "cuda"
    stream = torch.cuda.current_stream()

    def make(seed, ncell):
        rng = np.random.default_rng(seed)
        dt = I.cfl_dt(ncell)
        h = hl.hl_create(2, 3, ncell, dt)
        hl.hl_set_stream(h, stream)
        if seed % 2 == 0:
            st = I.gaussian_pulse(2, 3, ncell, dt, seed=seed, width=float(rng.uniform(0.012, 0.025)))
            hl.hl_set_initial(h, st.p, st.u)
        else:
            nq = 16
            hl.hl_set_initial(h, np.zeros((ncell[0] * ncell[1], nq)), np.zeros((2, ncell[0] * ncell[1], nq)))
            hl.hl_set_source(h, list(rng.random(2)), 0.01, float(rng.uniform(10.0, 20.0)), 1.0)
        return h

    def pair(seed):
        hc, hf = make(seed, nc), make(seed, nf)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t2 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        hl.hl_step(hc, horizon)
        t1.record(stream)
        hl.hl_step(hf, horizon * r)
        t2.record(stream)
        torch.cuda.synchronize()
        return hc, hf, t0.elapsed_time(t1), t1.elapsed_time(t2)

    per_seed = 16384
    n = (train_hi - train_lo) * per_seed
    X = torch.empty((n, hl.HL_MLP_IN), dtype=torch.float32, device=dev)
    T = torch.empty((n, hl.HL_MLP_OUT), dtype=torch.float32, device=dev)
    t_coarse = t_fine = 0.0
    wall = time.perf_counter()
    for k, i in enumerate(range(train_lo, train_hi)):
        gen_rng = np.random.default_rng(10_000 + i)    # the training nodes of seed i
        hc, hf, tc, tf = pair(seed0 + i)
        t_coarse += tc
        t_fine += tf
        nodes = torch.from_numpy(gen_rng.choice(rows, per_seed, replace=False).astype(np.int32)).to(dev)
        hl.hl_features(hc, nodes, per_seed, 1.0, 0.0, X[k * per_seed:(k + 1) * per_seed])
        hl.hl_targets(hf, r, hc, nodes, per_seed, 1.0, T[k * per_seed:(k + 1) * per_seed])
        hl.hl_destroy(hc)
        hl.hl_destroy(hf)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - wall
    # one output scale for every rank: the RMS of all training targets
    ss = torch.tensor([float(T.pow(2).sum()), float(T.numel())], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(ss)
    out_scale = float((ss[0] / ss[1]).sqrt())
    T /= out_scale
    net = hl.hl_mlp_create(7)
    hl.hl_mlp_set_stream(net, stream)
    iters, batch = 3000, 8192
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    # stream-ordered: draw, loss and gradient, gradient all-reduce (several ranks), Adam
    learned.train(net, X, T, iters, batch, lambda it: 1e-3 if it < 2000 else 2e-4, seed=0, dist=dist)
    e1.record(stream)
    final_loss = hl.hl_mlp_loss_grad(net, X[:65536].contiguous(), T[:65536].contiguous(), min(n, 65536))
    train_ms = e0.elapsed_time(e1)
    del X, T
    if rank != 0:
        hl.hl_mlp_destroy(net)
        return {}
    # held-out seeds, one pair at a time: plain error, correction, corrected error
    plain = corr = 0.0
    plain0 = corr0 = 0.0
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    corr_ms = 0.0
    Tt = torch.empty((rows, hl.HL_MLP_OUT), dtype=torch.float32, device=dev)
    for i in range(n_test):
        hc, hf, tc, tf = pair(seed0 + n_train + i)
        t_coarse += tc
        t_fine += tf
        hl.hl_targets(hf, r, hc, None, rows, 1.0, Tt)
        plain += float(Tt.pow(2).sum())
        plain0 += float(Tt[:, 0].pow(2).sum())
        e2.record(stream)
        hl.hl_apply_correction(hc, net, 1.0, 0.0, out_scale)
        e3.record(stream)
        hl.hl_targets(hf, r, hc, None, rows, 1.0, Tt)
        torch.cuda.synchronize()
        corr_ms += e2.elapsed_time(e3)
        corr += float(Tt.pow(2).sum())
        corr0 += float(Tt[:, 0].pow(2).sum())
        hl.hl_destroy(hc)
        hl.hl_destroy(hf)
    hl.hl_mlp_destroy(net)
    n_seeds = (train_hi - train_lo) + n_test   # the pairs this rank ran and timed
    dof_c = 3 * 16 * rows * horizon
    dof_f = 3 * 16 * rows * r * r * horizon * r
    return {
        "workload": "learned",
        "value": dof_c / ((t_coarse / n_seeds + corr_ms / n_test) / 1e3),
        "config": {"workload": f"learned coarse-grid correction: 2D m=3, coarse 256^2 vs fine 1024^2 (fine FP64 solver as reference), "
                               f"{n_train} training + {n_test} held-out seeds (Gaussian pulses width U[0.012,0.025] "
                               f"and Ricker sources f0 U[10,20]), horizon {horizon} coarse steps",
                   "mlp": "288-128-128-16, BF16 tensor-core products, FP32 accumulate, Adam",
                   "train_iters": iters, "batch_per_rank": batch, "train_rows": n_train * per_seed,
                   "data_parallel_ranks": world},
        "held_out_rms_err_plain": (plain / (n_test * rows * 16)) ** 0.5,
        "held_out_rms_err_corrected": (corr / (n_test * rows * 16)) ** 0.5,
        "gain_all_slots": (plain / corr) ** 0.5,
        "gain_value_slot": (plain0 / corr0) ** 0.5,
        "final_train_loss": final_loss,
        "ms_coarse_run": t_coarse / n_seeds, "ms_fine_run": t_fine / n_seeds, "ms_correction": corr_ms / n_test,
        "ms_training": train_ms, "s_data_generation": gen_s,
        "dof_updates_per_s_coarse_corrected": dof_c / ((t_coarse / n_seeds + corr_ms / n_test) / 1e3),
        "dof_updates_per_s_fine": dof_f / (t_fine / n_seeds / 1e3),
    }


def run_headline_2d(args):
    """The 2D workload line (512^2, m = 3, Gaussian pulse, 200 leapfrog steps per bench step)."""
    DIM, M, N, LF_STEPS = 2, 3, 512, 200
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    import numpy as np
    import torch

    from paper_1808_10481_gb300 import build as libbuild
    from paper_1808_10481_gb300 import hl
    from paper_1808_10481_gb300 import inputs as I

    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps are required")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    libbuild.build()
    hl.load()

    ncell = [N] * DIM
    dt = I.cfl_dt(ncell)
    st = I.gaussian_pulse(DIM, M, ncell, dt, seed=1 + rank)
    stream = torch.cuda.current_stream()
    h = hl.hl_create(DIM, M, ncell, dt)
    hl.hl_set_stream(h, stream)
    hl.hl_set_initial(h, st.p, st.u)
    tile, _ = hl.hl_autotune(h, 2)          # tile shape for this GPU and workload (untimed)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        hl.hl_step(h, LF_STEPS)
        flush.fill_(1)
    hl.hl_sync(h)
    hl.hl_set_option(h, hl.HL_OPT_TIMING, 1)
    hl.hl_kernel_times(h)  # reset

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler()
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        starts[k].record(stream)
        hl.hl_step(h, LF_STEPS)
        ends[k].record(stream)
        flush.fill_(k & 0xFF)          # untimed: evicts the state from L2 between steps
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clock = clocks.stop()
    status = hl.hl_sync(h)
    if status != hl.HL_OK:
        raise SystemExit(f"solver reported status {status}")
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ktimes, kcount = hl.hl_kernel_times(h)
    hl.hl_set_option(h, hl.HL_OPT_TIMING, 0)

    t_max_ms = dev_ms
    if dist:
        t = torch.tensor([dev_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max_ms = float(t.item())
    value = world * dofs(DIM, M, N) * LF_STEPS * args.steps / (t_max_ms / 1e3)

    # roofline of the dominant kernel (FP64 pipe): algorithmic flops per launch / mean launch time
    fma, add = hl.hl_op_counts(DIM, M)
    nnode = N ** DIM
    nz = fma / 2.0
    bfly = DIM * (1 << DIM) * (M + 1) ** DIM
    nq = (M + 1) ** DIM
    flops = {"p_half": nnode * (2 * nz + DIM * bfly + nq), "u_half": nnode * (2 * nz + bfly + DIM * nq)}
    dom = max(("p_half", "u_half"), key=lambda k: ktimes[k])
    mean_s = ktimes[dom] / kcount[dom] / 1e3
    achieved = flops[dom] / mean_s
    traffic = TRAFFIC_BYTES["2d"].get(dom) if TRAFFIC_SOURCE_HASH == kernel_hash() else None
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_FLOPS, "traffic": traffic, "kernel": dom,
                "kernel_mean_us": mean_s * 1e6,
                "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.070 GHz (unit counts and max clock)",
                "kernel_share": ktimes[dom] / max(dev_ms, 1e-9)}

    # end to end through the C ABI with pinned host buffers
    nq = (M + 1) ** DIM
    hp = torch.empty((nnode, nq), dtype=torch.float64, pin_memory=True)
    hu = torch.empty((DIM, nnode, nq), dtype=torch.float64, pin_memory=True)
    hp.copy_(torch.from_numpy(st.p))
    hu.copy_(torch.from_numpy(st.u))
    op = torch.empty_like(hp).pin_memory()
    ou = torch.empty_like(hu).pin_memory()
    e2e_n = max(1, min(args.steps, 5))
    hl.hl_set_initial(h, hp, hu)
    hl.hl_step(h, LF_STEPS)
    hl.hl_get_fields(h, op, ou)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_n):
        hl.hl_set_initial(h, hp, hu)
        hl.hl_step(h, LF_STEPS)
        hl.hl_get_fields(h, op, ou)
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * dofs(DIM, M, N) * LF_STEPS * e2e_n / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": hp.numel() * 8 + hu.numel() * 8,
           "d2h_bytes_per_step": op.numel() * 8 + ou.numel() * 8}
    hl.hl_destroy(h)

    cpu = None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "workload": "2d", "config": {"workload": WORKLOAD_2D, "dim": DIM, "m": M, "n_cells": ncell,
                       "leapfrog_steps_per_step": LF_STEPS, "l2": "flushed between timed steps (256 MiB write)",
                       "tile": hl.TILES[tile],
                       "parallelism": f"replicas x{world}: one independently seeded problem per GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock,
            "gpu_launches": int(kcount["p_half"] + kcount["u_half"] + kcount["small"]),
            "kernel_ms": ktimes,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()




def mode_list(hl, dim):
    """The mixed-precision modes the library offers for this dim (name, mode)."""
    out = [("fp32", hl.HL_FP32), ("fp32_comp", hl.HL_FP32_COMP)]
    if dim in getattr(hl, "TC_SPLIT_DIMS", (2,)):
        out.append(("tc_split", hl.HL_TC_SPLIT))
    return out


def run_headline(args):
    """The headline line: the 3D plane-wave workload, FP64 value and roofline, end to end
    through host buffers, every mixed-precision mode at its L2 error beside the plain FP64
    grid of equal error, and the oracle on the host cores."""
    import numpy as np
    import torch

    from paper_1808_10481_gb300 import build as libbuild
    from paper_1808_10481_gb300 import hl
    from paper_1808_10481_gb300 import inputs as I

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps are required")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    libbuild.build()
    hl.load()

    ncell = [N] * DIM
    nnode = N ** DIM
    nq = (M + 1) ** DIM
    dt = I.cfl_dt(ncell)
    seed = WAVE_SEED + rank
    st = I.plane_wave(M, ncell, dt, seed=seed)
    t_end = LF_STEPS * dt
    exact_end = I.plane_wave(0, ncell, dt, seed=seed, t0=t_end).p  # value slot of p at the final time
    stream = torch.cuda.current_stream()
    h = hl.hl_create(DIM, M, ncell, dt)
    hl.hl_set_stream(h, stream)
    hl.hl_set_initial(h, st.p, st.u)
    tile, _ = hl.hl_autotune(h, 1)          # tile shape for this GPU and workload (untimed)

    for _ in range(args.warmup):
        hl.hl_step(h, TIMED_LF)
    hl.hl_sync(h)
    hl.hl_set_option(h, hl.HL_OPT_TIMING, 1)
    hl.hl_kernel_times(h)  # reset

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler()
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        starts[k].record(stream)
        hl.hl_step(h, TIMED_LF)          # the 14.5 GB state does not fit the 129 MB L2
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clock = clocks.stop()
    status = hl.hl_sync(h)
    if status != hl.HL_OK:
        raise SystemExit(f"solver reported status {status}")
    dev_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    ktimes, kcount = hl.hl_kernel_times(h)
    hl.hl_set_option(h, hl.HL_OPT_TIMING, 0)
    t_max_ms = dev_ms
    if dist:
        t = torch.tensor([dev_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max_ms = float(t.item())
    value = world * dofs() * TIMED_LF * args.steps / (t_max_ms / 1e3)

    # roofline of the dominant kernel (FP64 pipe): algorithmic flops per launch / mean launch time
    fma, add = hl.hl_op_counts(DIM, M)
    nz = fma / 2.0
    bfly = DIM * (1 << DIM) * nq
    flops = {"p_half": nnode * (2 * nz + DIM * bfly + nq), "u_half": nnode * (2 * nz + bfly + DIM * nq)}
    dom = max(("p_half", "u_half"), key=lambda k_: ktimes[k_])
    mean_s = ktimes[dom] / kcount[dom] / 1e3
    achieved = flops[dom] / mean_s
    traffic = TRAFFIC_BYTES["3d"].get(dom) if TRAFFIC_SOURCE_HASH == kernel_hash() else None
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_FLOPS, "traffic": traffic, "kernel": dom,
                "kernel_mean_us": mean_s * 1e6,
                "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.070 GHz (unit counts and max clock)",
                "kernel_share": ktimes[dom] / max(dev_ms, 1e-9)}

    # end to end through the C ABI with pinned host buffers: one run from the initial data
    hp = torch.empty((nnode, nq), dtype=torch.float64, pin_memory=True)
    hu = torch.empty((DIM, nnode, nq), dtype=torch.float64, pin_memory=True)
    hp.copy_(torch.from_numpy(st.p))
    hu.copy_(torch.from_numpy(st.u))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    hl.hl_set_initial(h, hp, hu)
    hl.hl_step(h, LF_STEPS)
    hl.hl_get_fields(h, hp, hu)          # the result overwrites the input buffers
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * dofs() * LF_STEPS / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": hp.numel() * 8 + hu.numel() * 8,
           "d2h_bytes_per_step": hp.numel() * 8 + hu.numel() * 8,
           "step": "hl_set_initial + hl_step(100) + hl_get_fields from/to pinned host memory"}
    fp64_l2 = I.l2_error(DIM, ncell, hp.numpy(), exact_end)
    hl.hl_destroy(h)
    del hu

    modes = {}
    if rank == 0:
        fp64_run_ms = t_max_ms / args.steps * (LF_STEPS / TIMED_LF)   # the whole 100-step run
        modes["fp64"] = {"value": dofs() * LF_STEPS / (fp64_run_ms / 1e3), "ms_per_run": fp64_run_ms,
                         "l2_err_p_vs_exact": fp64_l2}
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except OSError:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        for name, mode in mode_list(hl, DIM):
            hm = hl.hl_create(DIM, M, ncell, dt)
            try:
                hl.hl_set_stream(hm, stream)
                hl.hl_set_precision(hm, mode)
                hl.hl_set_initial(hm, st.p, st.u)
                mtile, _ = hl.hl_autotune(hm, 1)
                hl.hl_set_initial(hm, st.p, st.u)
                hl.hl_set_option(hm, hl.HL_OPT_TIMING, 1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hl.hl_step(hm, LF_STEPS)
                e1.record(stream)
                rc = hl.hl_sync(hm)
                ms = e0.elapsed_time(e1)
                kt, kc = hl.hl_kernel_times(hm)
                hl.hl_get_fields(hm, hp, None)
            finally:
                hl.hl_destroy(hm)
            bytes_run = (3 * DIM + 3) * nq * 8 * nnode * LF_STEPS   # read + write every FP64 DOF once per step
            gbs = bytes_run / (ms / 1e3) / 1e9
            modes[name] = {"value": dofs() * LF_STEPS / (ms / 1e3), "ms_per_run": ms, "tile": hl.TILES[mtile],
                           "p_half_us": 1e3 * kt["p_half"] / max(kc["p_half"], 1),
                           "u_half_us": 1e3 * kt["u_half"] / max(kc["u_half"], 1),
                           "l2_err_p_vs_exact": I.l2_error(DIM, ncell, hp.numpy(), exact_end), "status": rc,
                           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                        "frac": gbs / hbm, "peak_source": "measured" if peaks else "fallback",
                                        "bytes": "FP64 state read and written once per leapfrog step"}}
            if name == "tc_split":
                modes[name]["roofline"] = tc_roofline(DIM, M, ncell, ms / LF_STEPS, peaks)
        # equal L2 error: plain FP64 on coarser grids to the same final time; each mode is
        # set against the fastest FP64 grid whose error is no larger (equal within 1%)
        ladder = []
        for n2 in (48, 64, 80, 96, 112, 128, 160):
            c2 = [n2] * DIM
            steps2 = int(math.ceil(t_end / I.cfl_dt(c2) - 1e-9))
            dt2 = t_end / steps2
            st2 = I.plane_wave(M, c2, dt2, seed=seed)
            ex2 = I.plane_wave(0, c2, dt2, seed=seed, t0=t_end).p
            h2 = hl.hl_create(DIM, M, c2, dt2)
            try:
                hl.hl_set_stream(h2, stream)
                hl.hl_set_initial(h2, st2.p, st2.u)
                hl.hl_step(h2, 2)
                hl.hl_set_initial(h2, st2.p, st2.u)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hl.hl_step(h2, steps2)
                e1.record(stream)
                hl.hl_sync(h2)
                pg2, _, _, _ = hl.hl_get_fields(h2)
            finally:
                hl.hl_destroy(h2)
            ladder.append({"n": n2, "steps": steps2, "ms_run": e0.elapsed_time(e1),
                           "l2_err_p_vs_exact": I.l2_error(DIM, c2, pg2, ex2)})
        ladder.append({"n": N, "steps": LF_STEPS, "ms_run": fp64_run_ms, "l2_err_p_vs_exact": fp64_l2})
        for name in [k_ for k_ in modes if k_ != "fp64"]:
            e = modes[name]["l2_err_p_vs_exact"]
            ok = [r_ for r_ in ladder if r_["l2_err_p_vs_exact"] <= e * 1.01]
            if ok:
                r_ = min(ok, key=lambda x: x["ms_run"])
                modes[name]["fp64_at_equal_error"] = {
                    "n": r_["n"], "ms_run": r_["ms_run"], "l2_err_p_vs_exact": r_["l2_err_p_vs_exact"],
                    "speedup_vs_fp64_at_equal_error": r_["ms_run"] / modes[name]["ms_per_run"]}
            else:
                modes[name]["fp64_at_equal_error"] = None
        modes["fp64_error_ladder"] = ladder
    del hp

    # 2D companion at the size of the 2D workload, where the tensor-core split mode runs: the
    # standing mode sin(48 pi x) sin(48 pi y) cos(w t) (exact solution known; 21 points per
    # wavelength, so the discretisation error sits well above rounding), 512^2, m = 3,
    # 200 steps, each mode beside the fastest plain FP64 grid of no larger L2 error
    modes_2d = None
    if rank == 0:
        modes_2d = run_modes_2d(hl, I, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(),
            "workload": "3d", "tile": hl.TILES[tile],
            "parallelism": f"replicas x{world}: one independently seeded problem per GPU",
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock,
            "gpu_launches": int(kcount["p_half"] + kcount["u_half"] + kcount["small"]),
            "kernel_ms": ktimes, "fp64_l2_err_p_vs_exact": fp64_l2,
            "modes_vs_fp64_at_equal_l2_error": modes,
            "modes_2d_vs_fp64_at_equal_l2_error": modes_2d,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_modes_2d(hl, I, stream, n=512, m=3, lf=200, wave=(24, 24)):
    """Every precision mode on the 2D standing mode at n^2, its L2 error against the exact
    solution, and the plain FP64 grid that reaches that error fastest."""
    import numpy as np
    import torch

    def run(ncell, steps, dt, mode, tune=True):
        st = I.standing_mode(2, m, ncell, dt, wave=list(wave))
        ex = I.standing_mode_exact(2, m, ncell, list(wave), steps * dt, (steps + 0.5) * dt)
        h = hl.hl_create(2, m, ncell, dt)
        try:
            hl.hl_set_stream(h, stream)
            hl.hl_set_precision(h, mode)
            hl.hl_set_initial(h, st.p, st.u)
            if tune:
                hl.hl_autotune(h, 2)
            hl.hl_step(h, 3)                       # warm-up
            hl.hl_set_initial(h, st.p, st.u)
            hl.hl_set_option(h, hl.HL_OPT_TIMING, 1)
            hl.hl_kernel_times(h)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hl.hl_step(h, steps)
            e1.record(stream)
            rc = hl.hl_sync(h)
            kt, kc = hl.hl_kernel_times(h)
            pg, _, _, _ = hl.hl_get_fields(h)
        finally:
            hl.hl_destroy(h)
        return e0.elapsed_time(e1), I.l2_error(2, ncell, pg, ex.p), rc, kt, kc

    ncell = [n, n]
    dt = I.cfl_dt(ncell)
    dof = 3 * (m + 1) ** 2 * n * n * lf
    out = {"config": f"2D standing mode sin({2 * wave[0]} pi x) sin({2 * wave[1]} pi y), {n}^2, m={m}, "
                     f"{lf} steps, C_CFL=0.9"}
    for name, mode in (("fp64", hl.HL_FP64), ("fp32", hl.HL_FP32), ("fp32_comp", hl.HL_FP32_COMP),
                       ("tc_split", hl.HL_TC_SPLIT)):
        ms, err, rc, kt, kc = run(ncell, lf, dt, mode)
        out[name] = {"value": dof / (ms / 1e3), "ms_per_run": ms, "l2_err_p_vs_exact": err, "status": rc,
                     "p_half_us": 1e3 * kt["p_half"] / max(kc["p_half"], 1),
                     "u_half_us": 1e3 * kt["u_half"] / max(kc["u_half"], 1)}
        if name == "tc_split":
            out[name]["roofline"] = tc_roofline(2, m, ncell, ms / lf, _peaks())
    t_end = lf * dt
    ladder = [{"n": n, "ms_run": out["fp64"]["ms_per_run"], "l2_err_p_vs_exact": out["fp64"]["l2_err_p_vs_exact"]}]
    for n2 in (192, 256, 320, 384, 448):
        c2 = [n2, n2]
        steps2 = int(np.ceil(t_end / I.cfl_dt(c2) - 1e-9))
        ms, err, _, _, _ = run(c2, steps2, t_end / steps2, hl.HL_FP64, tune=False)
        ladder.append({"n": n2, "ms_run": ms, "l2_err_p_vs_exact": err})
    for name in ("fp32", "fp32_comp", "tc_split"):
        ok = [r for r in ladder if r["l2_err_p_vs_exact"] <= out[name]["l2_err_p_vs_exact"] * 1.01]
        r = min(ok, key=lambda x: x["ms_run"]) if ok else None
        out[name]["fp64_at_equal_error"] = None if r is None else dict(
            r, speedup_vs_fp64_at_equal_error=r["ms_run"] / out[name]["ms_per_run"])
    out["fp64_error_ladder"] = ladder
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "3d":
        run_headline(args)
        return
    if args.workload == "2d":
        run_headline_2d(args)
        return
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.workload in ("batch", "learned") or rank == 0:
        run_aux(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
