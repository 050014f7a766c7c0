#!/usr/bin/env python3
"""Throughput of the point-source Fresnel CGH hot path on GB300.

Workload: the paper's Table 1 frame -- 1920 x 1024 pixels from N = 1024
object points (integer coordinates, z ~ U[0.5, 1.5] m, lambda = 633 nm,
p = 6.4 um, seed 0).  One step computes that hologram once by every GPU
method the build has, in the order: direct FP32 (per-axis angle tables,
whose kernel also builds the point records, then the direct point loop) and
separable split-FP16 (U/V tables, whose kernel also builds the point
records, then the tcgen05 GEMM).  value = point-pixel updates of all holograms of a
step, summed over ranks, / step time; the per-method times are in "methods".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank computes its own copy of
the workload (replicas, weak scaling); no collective touches the data path.
--impl reference times the FP64 CPU oracle on the host cores instead (the
paper ships no code, so the oracle is the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "point-pixel updates/s & ms per 1920x1024x1024 CGH, direct vs TC separable"
UNIT = "pp/s"
WORKLOAD = "cfg2_1920x1024_n1024"
MUFU_PER_CLK_PER_SM = 16     # MUFU (special-function) cosines per SM per clock
FP32_PER_CLK_PER_SM = 128    # FP32 lanes of the FMA pipe per SM per clock
# Work of the direct kernel per point-pixel update, in FP32 (FMA-pipe)
# operations: MUFU-cosine path = angle add, argument scale, accumulate (3,
# plus 1 MUFU); polynomial path = angle add, fold, square, 5 FMA (degree-5
# polynomial of the default tile), accumulate (9, no MUFU).  With a share s
# on the polynomial the FMA-pipe limit is 128 / (3 + 6 s) and the MUFU limit
# 16 / (1 - s) updates/clk/SM; they meet at s = 5/14: 16 * 14 / 9 = 24.9
# updates per clock per SM.  (Issue slots do not bind: packed FP32x2
# instructions do two of these operations per slot.)
MIXED_PP_PER_CLK_PER_SM = 16.0 * 14.0 / 9.0
# The direct adjoint per update: hardware path = angle add, argument scale,
# sin + cos (2 MUFU), 3 accumulations (G cos, the column's and the row's
# G sin: 5 FP32 ops); polynomial path = add, fold, square, 5 + 5 FMA (cos
# and sin), times u, 3 accumulations (17 FP32 ops, no MUFU).  FMA-pipe
# limit 128 / (5 + 12 s), MUFU limit 16 / (2 (1 - s)): they meet at
# s = 11/28, 224/17 = 13.2 updates per clock per SM.
ADJ_MIXED_PP_PER_CLK_PER_SM = 224.0 / 17.0
# The Eq. 2 recurrence kernel (the paper's design) per update: 1 MUFU
# cosine, 7 issue slots (2 integer adds, shift, or, FMA to radians,
# argument scale, accumulate): the MUFU binds at 16 updates/clk/SM.
RECUR_PP_PER_CLK_PER_SM = 16.0
# The FP32 separable product (angle addition) per update: 2 FP32
# multiply-adds on the FMA pipe, no MUFU: 128 / 2 = 64 updates/clk/SM.
SIMT_PP_PER_CLK_PER_SM = 64.0
# The FP32 separable adjoint per update: 4 FP32 multiply-adds (the column
# sums U, V and the row sums P, Q), no MUFU: 128 / 4 = 32 updates/clk/SM
# (the row's sincos and sums, shared by 16 updates, not counted).
BWD_SIMT_PP_PER_CLK_PER_SM = 32.0
# The paper's Table 1 (1,920 x 1,024 pixels), times in ms, for context.
PAPER_TABLE1 = {
    "N": [512, 1024, 1536, 2048, 2560, 3072, 3584],
    "cpu_one_core_eq2": [30e3, 59e3, 88e3, 115e3, 146e3, 174e3, 204e3],
    "nvidia_gtx260_cuda23": [33, 59, 85, 112, 139, 165, 192],
    "amd_hd5850_opencl_unoptimised": [215, 422, 630, 838, 1045, 1252, 1464],
    "amd_hd5850_opencl_optimised": [19, 31, 44, 56, 68, 80, 93],
}
# The paper's figure for this metric and workload (Table 1: 31 ms for the
# 1,920 x 1,024 hologram of 1,024 points, optimised OpenCL on a Radeon
# HD5850), in point-pixel updates per second: another machine, so context
# for vs_baseline, not a target.
PAPER_PP_PER_S = 1920 * 1024 * 1024 / 31e-3
NOMINAL_SMS = 152
NOMINAL_MAX_MHZ = 2070.0
FP16_OVER_BF16 = 1.0         # dense FP16 and BF16 tensor rates are equal


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="host time budget of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--split", choices=["replicas", "rows", "problems"],
                    default="replicas",
                    help="several GPUs (torchrun): replicas = every rank its own copy "
                         "of the workload (weak scaling, the default); rows = each rank "
                         "a slab of each hologram's rows (paper, large; strong "
                         "scaling); problems = each rank an LPT share of the batch "
                         "(batch64; strong scaling).  No collective on the data path.")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the built-in heuristics' shapes instead of running the "
                         "library's autotuner (cgh_tune, cgh_tune_batch) first")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (large frame, 64-hologram batch, "
                         "adjoint) that the default line reports under 'extra'")
    ap.add_argument("--methods", default=None,
                    help="comma-separated methods (default: direct,sep_fp16x3; "
                         "table1: direct,recur,sep_fp32,sep_fp16x3)")
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "large", "batch64", "adjoint", "table1"],
                    help="paper: 1920x1024x1024 (the headline line); large: "
                         "3840x2160x16384; batch64: 64 uneven holograms; adjoint: "
                         "1920x1080x4096 forward + adjoint; table1: the paper's "
                         "Table 1 sweep, N = 512..3584 at 1920x1024")
    return ap.parse_args()


def workload_desc():
    return ("1920x1024 pixels, N=1024 points, integer x_j,y_j, z_j~U[0.5,1.5] m, "
            "A_j~U[0,1], lambda=633 nm, p=6.4 um, seed 0 (the paper's Table 1 "
            "frame; synthetic cloud)")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self, t0=None, t1=None):
        """Summary of the samples; those taken in [t0, t1] (host time) if any
        landed there, else those of the loaded run just before."""
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        import datetime
        rows = []
        for ln in out.splitlines():
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        window = "timed region"
        sel = [r for r in rows if t0 is not None and t0 - 0.05 <= r[0] <= t1 + 0.05]
        if not sel:
            window = "load just before the timed region (same work)"
            sel = [r for r in rows if t0 is None or r[0] <= t0]
            sel = sel[-5:] if sel else rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[i] for _, _, _, r in sel for i in range(4)
                          if r[i].lower().startswith("active")})
        max_mhz = max(r[2] for r in rows)
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": max_mhz,
                "reasons": reasons, "samples": len(sel), "window": window}


# ------------------------------------------------------------ cpu baseline
def _oracle_rows_for(cloud, seconds):
    """Evenly spaced rows (and whole-frame repeats) worth about `seconds` of
    oracle time on all host cores."""
    import numpy as np

    import oracle
    probe = np.linspace(0, cloud.Ny - 1, min(cloud.Ny, 32)).round().astype(np.int32)
    t0 = time.perf_counter()
    oracle.forward(cloud, rows=probe)
    per_row = (time.perf_counter() - t0) / len(probe)
    nrows = int(max(1, min(cloud.Ny, seconds / max(per_row, 1e-6))))
    rows = np.unique(np.linspace(0, cloud.Ny - 1, nrows).round().astype(np.int32))
    reps = 1
    if len(rows) == cloud.Ny:
        reps = max(1, int(seconds / max(per_row * cloud.Ny, 1e-6)))
    return rows, reps


def cpu_baseline(cloud, seconds: float):
    """Time the FP64 oracle, as it stands, on about `seconds` of the workload
    (evenly spaced rows, or whole frames repeated), all host cores."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    rows, reps = _oracle_rows_for(cloud, seconds)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.forward(cloud, rows=rows)
    dt = time.perf_counter() - t0
    pp = reps * len(rows) * cloud.Nx * cloud.N
    what = (f"{len(rows)} of {cloud.Ny} rows (evenly spaced)" if reps == 1 else
            f"the whole frame {reps} times")
    return {"value": pp / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} of the {cloud.Nx}x{cloud.Ny}x{cloud.N} hologram, "
                      f"FP64 Eq. 1, OpenMP over rows; {dt:.2f} s"}


def cpu_eq2_table1(seconds: float):
    """The paper's CPU method beside Table 1's CPU column: the oracle's Eq. 2
    recurrence (FP64, one host core), timed on a few evenly spaced rows of
    each Table 1 hologram and scaled to the whole frame."""
    import numpy as np

    import oracle
    from workloads import TABLE1_POINTS, table1_cloud
    oracle.build()
    per_n = seconds / len(TABLE1_POINTS)
    ms, sample = [], None
    for n in TABLE1_POINTS:
        c = table1_cloud(n)
        probe = np.array([c.Ny // 2], dtype=np.int32)
        t0 = time.perf_counter()
        oracle.forward_recurrence(c, rows=probe, nthreads=1)
        per_row = time.perf_counter() - t0
        k = int(max(1, min(c.Ny, per_n / max(per_row, 1e-6))))
        rows = np.unique(np.linspace(0, c.Ny - 1, k).round().astype(np.int32))
        t0 = time.perf_counter()
        oracle.forward_recurrence(c, rows=rows, nthreads=1)
        dt = time.perf_counter() - t0
        ms.append(1e3 * dt / len(rows) * c.Ny)
        sample = f"{len(rows)} evenly spaced rows per hologram"
    return {"N": list(TABLE1_POINTS), "ms_whole_frame": ms, "cores": 1,
            "kind": "oracle Eq. 2 recurrence (FP64)",
            "sample": f"{sample}, scaled to 1024 rows"}


# -------------------------------------------------------------- reference
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from workloads import workload
    import numpy as np

    import oracle
    oracle.build()
    c = workload(WORKLOAD)
    cores = oracle.max_threads()
    # one step: a bounded row sample sized so the run takes ~2 minutes
    budget = 120.0 / max(1, args.steps + args.warmup)
    rows, _ = _oracle_rows_for(c, budget)
    for _ in range(args.warmup):
        oracle.forward(c, rows=rows)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.forward(c, rows=rows)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    pp = len(rows) * c.Nx * c.N
    value = pp / (ms / 1e3)
    sample = (f"{len(rows)} of {c.Ny} rows (evenly spaced) per step of the "
              f"{c.Nx}x{c.Ny}x{c.N} hologram, FP64 Eq. 1, OpenMP over rows")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(), "Nx": c.Nx, "Ny": c.Ny,
                   "N": c.N, "parallelism": "rank 0 host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- ours
def _traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    srcs = rec.get("sources") or [rec.get("source")]
    shas = rec.get("source_sha256")
    shas = shas if isinstance(shas, list) else [shas]
    if len(srcs) != len(shas):
        return None
    for rel, want in zip(srcs, shas):
        src = os.path.join(ROOT, rel or "")
        if not rel or not os.path.exists(src):
            return None
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != want:
            return None   # the kernel changed since the counters were taken
    return rec.get("dram_bytes_per_launch")


class Leg:
    """One piece of a step: a callable that enqueues its work on the stream,
    the point-pixel updates it performs, and the tensor-core flops (if any)
    of its GEMM launches."""

    def __init__(self, name, fn, pp, gemm_flops=0.0, gemm_launches=0,
                 kernel=None, method=None, N=None):
        self.name, self.fn, self.pp = name, fn, pp
        self.gemm_flops, self.gemm_launches = gemm_flops, gemm_launches
        self.kernel = kernel          # the kernel that does this leg's updates
        self.method, self.N = method or name, N
        self.problems = None          # batch legs: the problems (for the tuner)
        self.plan = None              # batch legs: what cgh_batch runs
        self.size = None              # forward legs: (N, Nx, Ny) of one call
        self.tile = None              # direct and batch legs: the direct tile used


# kernel (cgh_kernel_id name) that carries a forward method's point-pixel work
MAIN_KERNEL = {"direct": "direct", "naive": "naive", "recur": "recur",
               "sep_fp32": "simt", "sep_fp16x3": "gemm", "sep_fp16": "gemm",
               "sep_bf16": "gemm"}
GEMM_PASSES = {"sep_fp16x3": 3.0, "sep_fp16": 1.0, "sep_bf16": 1.0}
# methods whose kernels store the hologram tile by tile (into mapped host
# memory in place when the output is a pinned host buffer)
PROGRESSIVE = {"direct", "naive", "recur", "sep_fp32"}


def build_legs(cg, h, which, methods, dev, stream, shard=None):
    """The legs of one step of workload `which` (tensors on `dev`).  shard:
    None (the whole workload), ("rows", y0, rows) (a slab of each hologram's
    rows, cgh_forward_rows) or ("problems", [indices]) (those problems of
    the batch)."""
    import torch

    from workloads import batch_problems, grad_field, workload

    def dev_cloud(c):
        return (torch.from_numpy(c.xy).to(dev), torch.from_numpy(c.A).to(dev),
                torch.from_numpy(c.z).to(dev))

    legs = []

    def forward_leg(c, m, pts, A, z, name):
        out = torch.empty((c.Ny, c.Nx), dtype=torch.float32, device=dev)
        fn = (lambda m=m, out=out: cg.cgh_forward(
            pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=out, method=m, handle=h,
            stream=stream))
        mult = GEMM_PASSES.get(m, 0.0)
        leg = Leg(name, fn, c.pp, 4.0 * c.pp * mult, 1 if mult else 0,
                  kernel=MAIN_KERNEL.get(m), method=m, N=c.N)
        leg.size = (c.N, c.Nx, c.Ny)
        return leg

    def slab_leg(c, m, pts, A, z, name, y0, rows):
        out = torch.empty((max(rows, 1), c.Nx), dtype=torch.float32, device=dev)
        fn = ((lambda m=m, out=out: cg.cgh_forward_rows(
            pts, A, z, c.lam, c.p, c.Nx, y0, rows, out=out, method=m, handle=h,
            stream=stream)) if rows > 0 else (lambda: None))
        pp = rows * c.Nx * c.N
        mult = GEMM_PASSES.get(m, 0.0)
        leg = Leg(name, fn, pp, 4.0 * pp * mult, 1 if mult else 0,
                  kernel=MAIN_KERNEL.get(m), method=m, N=c.N)
        leg.size = (c.N, c.Nx, rows) if rows > 0 else None
        return leg

    if which in ("paper", "large"):
        c = workload(WORKLOAD if which == "paper" else "cfg3_3840x2160_n16384")
        pts, A, z = dev_cloud(c)
        for m in methods:
            if shard is not None and shard[0] == "rows":
                legs.append(slab_leg(c, m, pts, A, z, m, shard[1], shard[2]))
            else:
                legs.append(forward_leg(c, m, pts, A, z, m))
        return c, legs
    if which == "table1":
        from workloads import TABLE1_POINTS, table1_cloud
        for n in TABLE1_POINTS:
            c = table1_cloud(n)
            pts, A, z = dev_cloud(c)
            for m in methods:
                legs.append(forward_leg(c, m, pts, A, z, f"{m}_n{n}"))
        return c, legs
    if which == "batch64":
        clouds = batch_problems(seed=0)
        if shard is not None and shard[0] == "problems":
            clouds = [clouds[i] for i in shard[1]]
        probs = []
        for cl in clouds:
            p_, A_, z_ = dev_cloud(cl)
            probs.append(dict(points=p_, A=A_, z=z_, lam=cl.lam, p=cl.p, Nx=cl.Nx,
                              Ny=cl.Ny, out=torch.empty((cl.Ny, cl.Nx),
                                                        dtype=torch.float32,
                                                        device=dev)))
        pp = sum(cl.pp for cl in clouds)
        for m in methods:
            if m not in ("direct", "sep_fp16x3"):
                continue
            fn = ((lambda m=m: cg.cgh_batch(probs, method=m, handle=h, stream=stream))
                  if probs else (lambda: None))
            # the separable batch's timed kernel is its whole graph (prologue,
            # tables and grouped split-FP16 GEMM): 3 passes of 4 pp flops
            legs.append(Leg("batch_" + m, fn, pp,
                            12.0 * pp if m == "sep_fp16x3" else 0.0,
                            1 if m == "sep_fp16x3" else 0,
                            kernel="batch" if m == "direct" else "batch_sep"))
        for leg in legs:
            leg.problems = probs
        return (clouds[0] if clouds else batch_problems(seed=0)[0]), legs
    if which == "adjoint":
        c = workload("cfg5_1920x1080_n4096")
        pts, A, z = dev_cloud(c)
        G = torch.from_numpy(grad_field(11, c.Nx, c.Ny, scale=40.0)).to(dev)
        for m in methods:
            if m not in ("direct", "sep_fp32", "sep_fp16x3"):
                continue
            out = torch.empty((c.Ny, c.Nx), dtype=torch.float32, device=dev)
            f_fwd = (lambda m=m, out=out: cg.cgh_forward(
                pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=out, method=m, handle=h,
                stream=stream))
            f_bwd = (lambda m=m: cg.cgh_backward(
                pts, A, z, c.lam, c.p, c.Nx, c.Ny, G, method=m, handle=h,
                stream=stream))
            mult = 3.0 if m == "sep_fp16x3" else 0.0
            legs.append(Leg(m + "_fwd", f_fwd, c.pp, 4.0 * c.pp * mult, 1 if mult else 0,
                            kernel=MAIN_KERNEL[m], method=m))
            legs[-1].size = (c.N, c.Nx, c.Ny)
            legs.append(Leg(m + "_bwd", f_bwd, c.pp, 2 * 4.0 * c.pp * mult,
                            2 if mult else 0,
                            kernel={"direct": "bwd_direct", "sep_fp32": "bwd_simt"}.get(
                                m, "bwd_gemm")))
        return c, legs
    raise SystemExit(f"unknown workload {which}")


ALU_KERNELS = ("direct", "naive", "batch", "bwd_direct", "recur", "simt", "bwd_simt")
GEMM_KERNELS = ("gemm", "bwd_gemm", "batch_sep")


def alu_recipe(kernel, tile=None):
    """(updates per clk per SM at the nominal pipe rates, description, the
    same bound as a function of the measured rates (m MUFU cosines, f FP32
    multiply-adds per clk per SM), MUFU operations per update).  tile: the
    direct tile shape a direct or batch kernel ran with (its recipe)."""
    pk = tile[7] if tile else None
    if kernel in ("direct", "batch") and pk is not None and pk >= 7:
        vx, vy = tile[2], tile[3]
        # per point and thread: the angle add, the sincos argument scale, 2
        # amplitude products, 4 per row rotation (VY - 1 rows), and 2 per
        # pixel (1 for the row's first); the packed form (8) spends 2 on
        # the first pixel too
        f = 2.0 + (3.0 if pk == 7 else 4.0) / vx
        return (128.0 / f,
                f"FMA-pipe limit of the two-axis rotation recipe ({vx}x{vy} pixels a "
                f"thread{', packed pixel pairs' if pk == 8 else ''}): {f:.4g} FP32 ops "
                f"per update, 128 per clk/SM; 2 MUFU ops per {vx * vy} updates",
                lambda m, fr, f=f: fr / f, 2.0 / (vx * vy))
    if kernel in ("direct", "batch") and pk == 6:
        return (32.0,
                "MUFU limit of the row rotation recipe: a sincos (2 MUFU ops) per "
                "row of 4 pixels, 16 per clk/SM; 3 FP32 ops per update allow 42.7",
                lambda m, fr: min(2.0 * m, fr / 3.0), 0.5)
    if kernel == "simt":
        return (SIMT_PP_PER_CLK_PER_SM,
                "FMA-pipe limit of the FP32 angle-addition product: 2 FP32 "
                "multiply-adds per update, 128 per clk/SM", lambda m, f: f / 2.0, 0.0)
    if kernel == "bwd_simt":
        return (BWD_SIMT_PP_PER_CLK_PER_SM,
                "FMA-pipe limit of the FP32 angle-addition adjoint: 4 FP32 "
                "multiply-adds per update, 128 per clk/SM", lambda m, f: f / 4.0, 0.0)
    if kernel == "recur":
        return (RECUR_PP_PER_CLK_PER_SM,
                "MUFU limit of the Eq. 2 recurrence recipe: 1 hardware cosine per "
                "update at 16/clk/SM (7 issue slots per update allow 18.3)",
                lambda m, f: m, 1.0)
    if kernel == "bwd_direct":
        return (ADJ_MIXED_PP_PER_CLK_PER_SM,
                "FMA-pipe (128 FP32 ops/clk/SM) and MUFU (16 ops/clk/SM) limits of "
                "the adjoint recipe: 5 FP32 ops + 2 MUFU (sin, cos) per hardware "
                "update, 17 FP32 ops per polynomial update, best mix 11/28 -> 13.2 "
                "updates/clk/SM", lambda m, f: (f + 6.0 * m) / 17.0, 2.0)
    return (MIXED_PP_PER_CLK_PER_SM,
            "FMA-pipe (128 FP32 ops/clk/SM) and MUFU (16 cosines/clk/SM) limits "
            "of the direct recipe: 3 FP32 ops + 1 MUFU per MUFU-cosine update, "
            "9 FP32 ops per polynomial-cosine update, best mix 5/14 -> 24.9 "
            "updates/clk/SM", lambda m, f: (f + 6.0 * m) / 9.0, 1.0)


def kernel_roofline(kernel, pp, flops, ms, sms, peaks, pipe_rates=None, sm_mhz=None,
                    tile=None):
    """Roofline of one kernel from its algorithmic work per launch (pp
    point-pixel updates, or flops for a tensor-core GEMM) and its mean launch
    time in ms; tile: the direct tile shape (direct and batch kernels)."""
    if kernel in ALU_KERNELS and pp:
        per_clk, src, measured, mufu_per_pp = alu_recipe(kernel, tile)
        achieved = pp / (ms / 1e3) / 1e9
        peak = sms * per_clk * NOMINAL_MAX_MHZ * 1e6 / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Gpp/s", "frac": achieved / peak, "tile": list(tile) if tile else None,
                "peak_source": f"derived: {sms} SMs x {NOMINAL_MAX_MHZ:.0f} MHz max SM "
                               f"clock x {per_clk:.2f} updates/clk/SM ({src})"}
        if pipe_rates:
            m, f = pipe_rates["mufu_cos_per_clk_per_sm"], pipe_rates["fma_per_clk_per_sm"]
            roof["measured_pipe_rates"] = dict(pipe_rates)
            roof["peak_from_measured_rates"] = (sms * measured(m, f) * NOMINAL_MAX_MHZ
                                                * 1e6 / 1e9)
            roof["frac_of_measured_rates"] = achieved / roof["peak_from_measured_rates"]
        if mufu_per_pp:
            roof["frac_mufu_only"] = achieved / (
                sms * MUFU_PER_CLK_PER_SM / mufu_per_pp * NOMINAL_MAX_MHZ * 1e6 / 1e9)
        if sm_mhz:
            roof["frac_at_observed_clock"] = achieved / (sms * per_clk * sm_mhz * 1e6 / 1e9)
        if kernel in ("direct", "batch") and tile and tile[7] >= 6:
            # the rotation forms against the bound of the cosine-per-pixel
            # recipe they replace (above 1: faster than that recipe can be)
            roof["vs_cosine_per_pixel_bound"] = achieved / (
                sms * MIXED_PP_PER_CLK_PER_SM * NOMINAL_MAX_MHZ * 1e6 / 1e9)
        return roof
    if kernel in GEMM_KERNELS and flops:
        achieved = flops / (ms / 1e3) / 1e12
        base = peaks.get("bf16_tflops")
        src = "of measured (MEASURED_PEAKS.json bf16 burst; FP16 dense rate equal)"
        if base is None:
            base, src = 1900.0, "of fallback (1.9 PFLOP/s bf16)"
        peak = base * FP16_OVER_BF16
        return {"bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": src}
    return {"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"),
            "unit": "GB/s", "frac": None}


TUNABLE = ("direct", "sep_bf16", "sep_fp16", "sep_fp16x3")


def prepare_legs(cg, h, which, methods, dev, stream, shard=None, tune=True):
    """The legs of workload `which` that this build runs, each called once
    (sizes workspaces, captures batch graphs); the device status checked.
    tune: the library's autotuner picks the shapes first (direct tile, GEMM
    plan, batch tiles), outside any timed region."""
    import torch
    c, all_legs = build_legs(cg, h, which, methods, dev, stream, shard)
    legs = []
    tuned = set()
    for leg in all_legs:
        try:
            if tune and leg.size and leg.method in TUNABLE and \
                    (leg.method, leg.size) not in tuned:
                cg.cgh_tune(h, *leg.size, method=leg.method, stream=stream)
                tuned.add((leg.method, leg.size))
            if leg.problems and tune:
                # the batch's tiles from the autotuner (outside any timed
                # region; it synchronises)
                m = leg.method.replace("batch_", "")
                cg.cgh_tune_batch(h, leg.problems, m, stream=stream)
            if leg.problems:
                leg.plan = cg.cgh_batch_plan(h, leg.problems, leg.method.replace("batch_", ""))
                leg.tile = leg.plan["tile"]
            elif leg.size and leg.kernel == "direct":
                leg.tile = cg.cgh_direct_tile_for(h, *leg.size)
            leg.fn()
        except cg.CGHError as e:
            if e.status == cg.CGH_ERR_UNSUPPORTED:
                continue
            raise
        legs.append(leg)
    if not legs:
        raise SystemExit(f"no GPU method available for workload {which}")
    torch.cuda.synchronize()
    if cg.cgh_last_device_status(h) != cg.CGH_OK:
        raise SystemExit("device status not OK after the first calls: "
                         + cg.cgh_last_error(h))
    return c, legs


def time_legs(cg, h, legs, K, flush, stream):
    """Per leg, two passes of K calls, each call after an L2 flush: the first
    with events only around each call (ms per call, the call's kernels
    overlapping as they do in use), the second with every kernel launch of
    the handle bracketed by events as well (device time of each kernel).
    Returns {leg name: (ms per call, {kernel: (total ms, launches)})}."""
    import torch
    out = {}
    for leg in legs:
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            leg.fn()
            b.record(stream)
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        cg.cgh_kernel_timing(h, True)
        for _ in range(K):
            flush.zero_()
            leg.fn()
        torch.cuda.synchronize()
        kt = {name: cg.cgh_kernel_time(h, name) for name in cg.KERNELS}
        cg.cgh_kernel_timing(h, False)
        out[leg.name] = (ms, {k: v for k, v in kt.items() if v[1] > 0})
    return out


def leg_entries(legs, per_leg, K, sms, peaks, pipe_rates, sm_mhz):
    """The "methods" object of a line: per leg its ms per call, point-pixel
    updates per second, and its main kernel's device time per call and
    roofline fraction (the call's work over that time; a kernel launched
    more than once per call, like the adjoint's two GEMMs, is summed)."""
    res = {}
    for leg in legs:
        ms, kt = per_leg[leg.name]
        e = {"ms": ms, "pp_per_s": leg.pp / (ms / 1e3)}
        k = leg.kernel
        if k in kt:
            kms = kt[k][0] / K
            roof = kernel_roofline(k, leg.pp, leg.gemm_flops, kms, sms, peaks,
                                   pipe_rates, sm_mhz, leg.tile)
            e.update({"kernel": k, "kernel_ms_per_call": kms, "tile": leg.tile,
                      "kernel_launches_per_call": kt[k][1] / K,
                      "kernel_frac": roof["frac"], "kernel_bound": roof["bound"]})
            if "frac_of_measured_rates" in roof:
                e["kernel_frac_of_measured_rates"] = roof["frac_of_measured_rates"]
        e["kernels_ms_per_launch"] = {n: v[0] / v[1] for n, v in kt.items()}
        res[leg.name] = e
    return res


def dominant_kernel(legs, per_leg, K):
    """The kernel with the most device time over the legs, its device time
    per call of the legs it serves, and their work per call (mean pp; mean
    GEMM flops)."""
    tot = {}
    for leg in legs:
        for k, (ms, n) in per_leg[leg.name][1].items():
            t = tot.setdefault(k, [0.0, 0])
            t[0] += ms
            t[1] += n
    dom = max(tot, key=lambda k: tot[k][0])
    served = [leg for leg in legs if leg.kernel == dom and dom in per_leg[leg.name][1]]
    ncalls = K * max(1, len(served))
    dom_ms = tot[dom][0] / ncalls
    pp = statistics.mean(leg.pp for leg in served) if served else None
    flops = statistics.mean(leg.gemm_flops for leg in served) if served else 0.0
    launches = tot[dom][1] / ncalls
    tile = next((leg.tile for leg in served if leg.tile), None)
    return (dom, dom_ms, pp, flops, launches, {k: v[0] / v[1] for k, v in tot.items()},
            tile)


EXTRA_WORKLOADS = {
    "large": ("3840x2160 pixels, N=16384 continuous points, z_j~U[0.3,2.0] m, "
              "lambda=532 nm, p=3.74 um, seed 0", "direct,recur,sep_fp32,sep_bf16,"
              "sep_fp16,sep_fp16x3"),
    "batch64": ("64 holograms, Nx,Ny in {512..2048 step 128}, N~U[100,8192], lambda "
                "in {633,532,473} nm, p=8 um, seed 0; one cgh_batch call each",
                "direct,sep_fp16x3"),
    "adjoint": ("1920x1080 pixels, N=4096 continuous points, lambda=532 nm, p=6.4 um, "
                "seed 0; forward and adjoint (a seeded dL/dI field)",
                "direct,sep_fp32,sep_fp16x3"),
}


def measure_extras(cg, h, dev, stream, flush, K, sms, peaks, pipe_rates, gpu_id,
                   tune=True):
    """The other workloads, measured leg by leg (ms per hologram or batch per
    method, main kernel time and roofline fraction, the dominant kernel)."""
    import torch
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    t0 = time.time()
    extra = {}
    for which, (desc, methods) in EXTRA_WORKLOADS.items():
        c, legs = prepare_legs(cg, h, which, methods.split(","), dev, stream, tune=tune)
        for _ in range(2):
            for leg in legs:
                leg.fn()
        torch.cuda.synchronize()
        per_leg = time_legs(cg, h, legs, K, flush, stream)
        dom, dom_ms, pp, flops, nl, _, tile = dominant_kernel(legs, per_leg, K)
        roof = kernel_roofline(dom, pp, flops, dom_ms, sms, peaks, pipe_rates, tile=tile)
        e = {"workload": desc, "pp_per_call": {leg.name: leg.pp for leg in legs},
             "methods": leg_entries(legs, per_leg, K, sms, peaks, pipe_rates, None),
             "dominant_kernel": {"kernel": dom, "ms_per_call": dom_ms,
                                 "launches_per_call": nl,
                                 "frac": roof["frac"], "bound": roof["bound"],
                                 "peak": roof["peak"], "unit": roof["unit"]},
             "steps": K, "l2": "flushed before every call"}
        if which == "batch64":
            e["batch_plans"] = {leg.name: leg.plan for leg in legs if leg.plan}
        else:
            e["shapes"] = {"direct_tile": list(cg.cgh_direct_tile_for(h, c.N, c.Nx, c.Ny)),
                           "tuned": tune}
            for m in sorted({leg.method for leg in legs if leg.method in GEMM_PASSES}):
                e["shapes"]["gemm_plan_" + m] = list(cg.cgh_gemm_plan_for(h, c.N, c.Nx,
                                                                          c.Ny, m))
        if "frac_of_measured_rates" in roof:
            e["dominant_kernel"]["frac_of_measured_rates"] = roof["frac_of_measured_rates"]
        extra[which] = e
        del legs
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    t1 = time.time()
    extra["clocks"] = sampler.stop(t0, t1)
    return extra


def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_1002_0916_gb300 as cg

    dev = torch.device("cuda", local)
    h = cg.cgh_create(local)
    stream = torch.cuda.current_stream()
    if args.methods is None:
        args.methods = {"table1": "direct,recur,sep_fp32,sep_fp16x3",
                        "adjoint": "direct,sep_fp32,sep_fp16x3"}.get(args.workload,
                                                                     "direct,sep_fp16x3")
    methods = [m.strip() for m in args.methods.split(",") if m.strip()]
    shard = None
    if world > 1 and args.split == "rows" and args.workload in ("paper", "large"):
        from paper_1002_0916_gb300.sharding import row_slabs
        from workloads import workload
        Ny = workload(WORKLOAD if args.workload == "paper" else "cfg3_3840x2160_n16384").Ny
        y0, rows = row_slabs(Ny, world)[rank]
        shard = ("rows", y0, rows)
    elif world > 1 and args.split == "problems" and args.workload == "batch64":
        from paper_1002_0916_gb300.sharding import lpt_shard
        from workloads import batch_problems
        shard = ("problems", lpt_shard([cl.pp for cl in batch_problems(seed=0)], world)[rank])
    c, legs = prepare_legs(cg, h, args.workload, methods, dev, stream, shard,
                           tune=not args.no_tune)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB

    def step():
        for leg in legs:
            leg.fn()

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    # the two pipe rates the ALU rooflines are derived from, measured on this
    # device (outside the timed regions)
    pipe_rates = cg.cgh_debug_pipe_rates(h, stream=stream)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    gpu_id = (f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local))
    sampler = ClockSampler(gpu_id)
    K = args.steps
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    # keep the GPU busy with the same work while the sampler warms up, so
    # that the clock samples nearest the timed region are under this load
    t_end = time.perf_counter() + 0.5
    while time.perf_counter() < t_end:
        step()
        torch.cuda.synchronize()

    # ---- timed region 1: whole steps, events only at the step boundaries
    # (nothing between the kernels of a step, so programmatic dependent
    # launch overlaps each kernel's launch with the one before)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    n0 = cg.cgh_launch_count(h)
    t0 = time.time()
    for a, b in evs:
        flush.zero_()                       # L2 flush between timed steps
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    launches = cg.cgh_launch_count(h) - n0
    barrier()
    # ---- timed region 2: the same K steps leg by leg, each call and every
    # kernel launch bracketed by events: ms per hologram per method and the
    # dominant kernel's launch time for the roofline
    per_leg = time_legs(cg, h, legs, K, flush, stream)
    t2 = time.time()
    barrier()
    clocks = sampler.stop(t0, t2)

    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        lt = torch.tensor([float(launches)], device=dev)
        dist.all_reduce(lt, op=dist.ReduceOp.SUM)
        launches = int(lt.item())
    pp_step = sum(leg.pp for leg in legs)
    if shard is None:
        value = world * pp_step / (ms / 1e3)     # replicas: every rank the whole step
    else:
        # a split: the ranks' shares add up to one copy of the workload
        from paper_1002_0916_gb300.sharding import reduce_sum
        value = reduce_sum(pp_step, dist, dev) / (ms / 1e3)

    # ---- roofline of the dominant kernel (timed live in timed region 2)
    dom, dom_ms, pp_dom, flops_dom, nl_dom, kernels_ms, tile_dom = dominant_kernel(
        legs, per_leg, K)
    roof = kernel_roofline(dom, pp_dom, flops_dom, dom_ms, sms, peaks, pipe_rates,
                           clocks.get("sm_mhz") if clocks else None, tile_dom)
    roof["kernel"] = dom
    roof["ms_per_launch"] = dom_ms / max(nl_dom, 1e-9)
    roof["launches_per_call"] = nl_dom
    roof["timed"] = ("timed region 2: K calls of each method with every kernel launch "
                     "bracketed by CUDA events on its stream; achieved = the work of "
                     "one call / the kernel's device time per call")
    roof["traffic"] = _traffic_for(dom)

    # ---- end to end through the host-buffer C-ABI call (forward legs)
    e2e = None
    fwd_methods = [leg.name for leg in legs if leg.name in cg.METHODS]
    if fwd_methods and args.workload in ("paper", "large"):
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        hp, hA, hz = pin(c.xy), pin(c.A), pin(c.z)
        hout = {m: torch.empty((c.Ny, c.Nx), dtype=torch.float32).pin_memory()
                for m in fwd_methods}
        E = max(3, K // 2)

        def sync_step():
            # each call returns with its hologram in host memory
            for m in fwd_methods:
                cg.cgh_forward_host(hp, hA, hz, c.lam, c.p, c.Nx, c.Ny, out=hout[m],
                                    method=m, handle=h, stream=stream)

        # pipelined: the tensor-core holograms first, so that their copies to
        # the host run while the tile-by-tile kernels (which write their
        # holograms to host memory as they go) compute; one wait per step
        order = sorted(fwd_methods, key=lambda m: m in PROGRESSIVE)

        def async_step():
            for m in order:
                cg.cgh_forward_host_async(hp, hA, hz, c.lam, c.p, c.Nx, c.Ny,
                                          out=hout[m], method=m, handle=h,
                                          stream=stream)
            cg.cgh_host_wait(h, stream)

        def timed(fn):
            fn()
            barrier()
            t0 = time.perf_counter()
            for _ in range(E):
                fn()
            s = (time.perf_counter() - t0) / E
            if dist is not None:
                t = torch.tensor([s], device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                s = float(t.item())
            return s

        # pipelined, as a display loop runs: step k issues its holograms into
        # its own pair of pinned buffers, then waits (ticket) for step k - 1's,
        # whose outputs are then complete; the next step's kernels run
        # meanwhile
        hout2 = [hout, {m: torch.empty((c.Ny, c.Nx), dtype=torch.float32).pin_memory()
                        for m in fwd_methods}]

        def pipelined_steps():
            prev = None
            for k in range(E):
                for m in order:
                    cg.cgh_forward_host_async(hp, hA, hz, c.lam, c.p, c.Nx, c.Ny,
                                              out=hout2[k % 2][m], method=m, handle=h,
                                              stream=stream)
                t = cg.cgh_host_ticket(h)
                if prev is not None:
                    cg.cgh_host_wait_ticket(h, prev)
                prev = t
            cg.cgh_host_wait_ticket(h, prev)

        sync_s = timed(sync_step)
        wait_s = timed(async_step)
        pipelined_steps()
        barrier()
        t0 = time.perf_counter()
        pipelined_steps()
        e2e_s = (time.perf_counter() - t0) / E
        if dist is not None:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        npp = world * len(fwd_methods) * c.pp
        e2e = {"value": npp / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": len(fwd_methods) * c.N * 16,
               "d2h_bytes_per_step": len(fwd_methods) * c.Nx * c.Ny * 4,
               "ms_per_step": e2e_s * 1e3,
               "calls": "cgh_forward_host_async per hologram (" + ", ".join(order)
                        + ") into the step's own pinned buffers, then "
                          "cgh_host_wait_ticket for the previous step",
               "one_wait_per_step": {"value": npp / wait_s, "ms_per_step": wait_s * 1e3,
                                     "calls": "the same calls, then cgh_host_wait"},
               "synchronous": {"value": npp / sync_s, "ms_per_step": sync_s * 1e3,
                               "calls": "cgh_forward_host per hologram ("
                                        + ", ".join(fwd_methods) + ")"}}

    table1 = None
    leg_ms = {name: v[0] for name, v in per_leg.items()}
    if args.workload == "table1":
        from workloads import TABLE1_POINTS
        table1 = {"N": list(TABLE1_POINTS), "ms": {}, "pp_per_s": {},
                  "paper_table1_ms": PAPER_TABLE1,
                  "paper_source": "Table 1 of the paper (other machines; context)"}
        for m in methods:
            ms_m = [leg_ms[f"{m}_n{n}"] for n in TABLE1_POINTS if f"{m}_n{n}" in leg_ms]
            if len(ms_m) == len(TABLE1_POINTS):
                table1["ms"][m] = ms_m
                table1["pp_per_s"][m] = [n * 1920 * 1024 / (t / 1e3)
                                         for n, t in zip(TABLE1_POINTS, ms_m)]

    line = None
    if rank == 0:
        cfg = {"workload": workload_desc() if args.workload == "paper" else args.workload,
               "methods": [leg.name for leg in legs],
               "l2": "flushed: 256 MiB device write between timed steps (and before "
                     "every call of timed region 2)",
               "parallelism": ("single GPU" if world == 1 else
                               "replicas (each rank its own copy of the workload)"
                               if shard is None else
                               f"{world} ranks, each a slab of every hologram's rows "
                               "(cgh_forward_rows), no collective on the data path"
                               if shard[0] == "rows" else
                               f"{world} ranks, each an LPT share of the batch's "
                               "problems, no collective on the data path")}
        if args.workload == "batch64":
            cfg["batch_plans"] = {leg.name: leg.plan for leg in legs if leg.plan}
        if args.workload in ("paper", "large", "adjoint"):
            Ny_call = shard[2] if shard is not None and shard[0] == "rows" else c.Ny
            if Ny_call > 0:
                cfg["direct_tile"] = dict(zip(
                    ("tile_x", "tile_y", "vec_x", "vec_y", "points_per_stage",
                     "poly_pixels", "point_groups", "packed"),
                    cg.cgh_direct_tile_for(h, c.N, c.Nx, Ny_call)))
                tiling, width, tuned_plan = cg.cgh_gemm_plan_for(h, c.N, c.Nx, Ny_call,
                                                                 "sep_fp16x3")
                cfg["gemm_plan_sep_fp16x3"] = {"tiling": tiling, "width": width,
                                               "tuned": tuned_plan}
            cfg["shapes"] = ("from the library's autotuner (cgh_tune)" if not args.no_tune
                             else "the built-in heuristics")
        if args.workload == "table1":
            cfg["workload"] = ("1920x1024 pixels, N = 512, 1024, ..., 3584 points (the "
                               "paper's Table 1 sweep), otherwise the 1920x1024x1024 "
                               "recipe; one step = every N by every method")
            cfg.update({"Nx": c.Nx, "Ny": c.Ny, "N": "512..3584 step 512"})
        elif args.workload != "batch64":
            cfg.update({"Nx": c.Nx, "Ny": c.Ny, "N": c.N})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak" if shard is None else "strong",
            "vs_baseline": value / PAPER_PP_PER_S if args.workload == "paper" else None,
            "dtype": ("f32+f16x3" if any(leg.method in GEMM_PASSES for leg in legs)
                      else "f32"),
            "data": "synthetic", "config": cfg,
            "timing": ("ms_per_step, value, gpu_launches: timed region 1 (K whole steps, "
                       "CUDA events only at step boundaries); methods, "
                       "kernels_ms_per_launch, roofline: timed region 2 (the same K "
                       "steps method by method, every call and kernel launch bracketed "
                       "by events)"),
            "methods": leg_entries(legs, per_leg, K, sms, peaks, pipe_rates, None),
            "kernels_ms_per_launch": kernels_ms,
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        }
        if table1 is not None:
            line["table1"] = table1
    if (rank == 0 and world == 1 and args.workload == "paper" and not args.no_extra):
        line["extra"] = measure_extras(cg, h, dev, stream, flush, max(3, min(K, 5)),
                                       sms, peaks, pipe_rates, gpu_id,
                                       tune=not args.no_tune)
    cg.cgh_destroy(h)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and args.workload == "paper":
            line["cpu_baseline"] = cpu_baseline(c, args.cpu_seconds)
        if world == 1 and not args.no_cpu_baseline and args.workload == "table1":
            line["table1"]["cpu_eq2_one_core"] = cpu_eq2_table1(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
