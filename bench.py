#!/usr/bin/env python3
"""Throughput of the point-source Fresnel CGH hot path on GB300.

Workload: the paper's Table 1 frame -- 1920 x 1024 pixels from N = 1024
object points (integer coordinates, z ~ U[0.5, 1.5] m, lambda = 633 nm,
p = 6.4 um, seed 0).  One step computes that hologram once by every GPU
method the build has, in the order: direct FP32 (per-point prologue,
per-axis angle tables, direct point loop) and separable split-FP16 (U/V
tables, tcgen05 GEMM).  value = point-pixel updates of all holograms of a
step, summed over ranks, / step time; the per-method times are in "methods".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank computes its own copy of
the workload (replicas, weak scaling); no collective touches the data path.
--impl reference times the FP64 CPU oracle on the host cores instead (the
reference arm for this build: there is no reference GPU code).
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
MUFU_PER_CLK_PER_SM = 16     # MUFU (special-function) lanes per SM per clock
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
    ap.add_argument("--methods", default="direct,sep_fp16x3")
    return ap.parse_args()


def workload_desc():
    return ("1920x1024 pixels, N=1024 points, integer x_j,y_j, z_j~U[0.5,1.5] m, "
            "A_j~U[0,1], lambda=633 nm, p=6.4 um, seed 0 (the paper's Table 1 "
            "frame; synthetic cloud)")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for ln in out.splitlines():
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4)
                          if r[i].lower().startswith("active")})
        max_mhz = max(r[1] for r in rows)
        loaded = [r[0] for r in rows if r[0] > 0.5 * max_mhz] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max_mhz,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ cpu baseline
def cpu_baseline(cloud, seconds: float, tag: str = "cpu_baseline"):
    """Time the FP64 oracle on evenly spaced rows of the workload, sized to
    about `seconds` of host work (all cores)."""
    import numpy as np

    import oracle
    oracle.build()
    cores = oracle.max_threads()
    probe_rows = np.arange(0, cloud.Ny, max(1, cloud.Ny // 4))[:4].astype(np.int32)
    t0 = time.perf_counter()
    oracle.forward(cloud, rows=probe_rows)
    per_row = (time.perf_counter() - t0) / len(probe_rows)
    nrows = int(max(1, min(cloud.Ny, seconds / max(per_row, 1e-6))))
    rows = np.linspace(0, cloud.Ny - 1, nrows).round().astype(np.int32)
    rows = np.unique(rows)
    t0 = time.perf_counter()
    oracle.forward(cloud, rows=rows)
    dt = time.perf_counter() - t0
    pp = len(rows) * cloud.Nx * cloud.N
    return {"value": pp / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(rows)} of {cloud.Ny} rows (evenly spaced) of the "
                      f"{cloud.Nx}x{cloud.Ny}x{cloud.N} hologram, FP64 Eq. 1, "
                      f"OpenMP over rows; {dt:.2f} s"}


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
    probe = np.arange(0, c.Ny, c.Ny // 4)[:4].astype(np.int32)
    t0 = time.perf_counter()
    oracle.forward(c, rows=probe)
    per_row = (time.perf_counter() - t0) / len(probe)
    budget = 120.0 / max(1, args.steps + args.warmup)
    nrows = int(max(1, min(c.Ny, budget / max(per_row, 1e-6))))
    rows = np.linspace(0, c.Ny - 1, nrows).round().astype(np.int32)
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
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if sha != rec.get("source_sha256"):
        return None
    return rec.get("dram_bytes_per_launch")


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
    from workloads import workload

    c = workload(WORKLOAD)
    dev = torch.device("cuda", local)
    pts = torch.from_numpy(c.xy).to(dev)
    A = torch.from_numpy(c.A).to(dev)
    z = torch.from_numpy(c.z).to(dev)
    h = cg.cgh_create(local)
    stream = torch.cuda.current_stream()

    methods = []
    outs = {}
    for m in [s.strip() for s in args.methods.split(",") if s.strip()]:
        out = torch.empty((c.Ny, c.Nx), dtype=torch.float32, device=dev)
        try:
            cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=out, method=m,
                           handle=h)
        except cg.CGHError as e:
            if e.status == cg.CGH_ERR_UNSUPPORTED:
                continue
            raise
        methods.append(m)
        outs[m] = out
    if not methods:
        raise SystemExit("no GPU method available")
    torch.cuda.synchronize()
    if cg.cgh_last_device_status(h) != cg.CGH_OK:
        raise SystemExit("device status not OK after the first calls: "
                         + cg.cgh_last_error(h))

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB

    def step(evs=None):
        for i, m in enumerate(methods):
            cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=outs[m],
                           method=m, handle=h, stream=stream)
            if evs is not None:
                evs[i + 1].record(stream)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(f"GPU-{props.uuid}" if getattr(props, "uuid", None)
                           else str(local))
    K = args.steps
    evsets = [[torch.cuda.Event(enable_timing=True) for _ in range(len(methods) + 1)]
              for _ in range(K)]
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    cg.cgh_kernel_timing(h, True)
    n0 = cg.cgh_launch_count(h)
    for k in range(K):
        flush.zero_()                       # L2 flush between timed steps
        evsets[k][0].record(stream)
        step(evsets[k])
    torch.cuda.synchronize()
    launches = cg.cgh_launch_count(h) - n0
    barrier()
    clocks = sampler.stop()

    step_ms = [evs[0].elapsed_time(evs[-1]) for evs in evsets]
    meth_ms = {m: [evs[i].elapsed_time(evs[i + 1]) for evs in evsets]
               for i, m in enumerate(methods)}
    kt = {name: cg.cgh_kernel_time(h, name) for name in cg.KERNELS}
    cg.cgh_kernel_timing(h, False)
    ms = statistics.mean(step_ms)
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        lt = torch.tensor([float(launches)], device=dev)
        dist.all_reduce(lt, op=dist.ReduceOp.SUM)
        launches = int(lt.item())
    pp = c.pp
    value = world * len(methods) * pp / (ms / 1e3)

    # ---- roofline of the dominant kernel
    dom = max((k for k in kt if kt[k][1] > 0), key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / kt[dom][1]
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    sms = props.multi_processor_count
    if dom in ("direct", "naive"):
        achieved = pp / (dom_ms / 1e3) / 1e9
        peak = sms * MUFU_PER_CLK_PER_SM * NOMINAL_MAX_MHZ * 1e6 / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Gpp/s", "frac": achieved / peak,
                "peak_source": (f"derived: {sms} SMs x {MUFU_PER_CLK_PER_SM} MUFU "
                                f"cosines/clk/SM x {NOMINAL_MAX_MHZ:.0f} MHz max SM "
                                "clock (one cosine per point-pixel update)")}
        if clocks and clocks.get("sm_mhz"):
            roof["frac_at_observed_clock"] = achieved / (
                sms * MUFU_PER_CLK_PER_SM * clocks["sm_mhz"] * 1e6 / 1e9)
    elif dom == "gemm":
        mult = 3 if "sep_fp16x3" in methods else 1
        flops = 4.0 * c.N * c.Nx * c.Ny * mult
        achieved = flops / (dom_ms / 1e3) / 1e12
        base = peaks.get("bf16_tflops")
        src = "of measured (MEASURED_PEAKS.json bf16 burst; FP16 rate equal)"
        if base is None:
            base, src = 1900.0, "of fallback (1.9 PFLOP/s bf16)"
        peak = base * FP16_OVER_BF16
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": src}
    else:
        roof = {"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"),
                "unit": "GB/s", "frac": None}
    roof["kernel"] = dom
    roof["ms_per_launch"] = dom_ms
    kernel_src = {"direct": "paper_1002_0916_gb300/csrc/direct.cu",
                  "gemm": "paper_1002_0916_gb300/csrc/umma.cu"}.get(dom)
    roof["traffic"] = _traffic_for(dom) if kernel_src else None

    # ---- end to end through the host-buffer C-ABI call
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    hp, hA, hz = pin(c.xy), pin(c.A), pin(c.z)
    hout = {m: torch.empty((c.Ny, c.Nx), dtype=torch.float32).pin_memory()
            for m in methods}
    for m in methods:
        cg.cgh_forward_host(hp, hA, hz, c.lam, c.p, c.Nx, c.Ny, out=hout[m],
                            method=m, handle=h, stream=stream)
    barrier()
    E = max(3, K // 2)
    t0 = time.perf_counter()
    for _ in range(E):
        for m in methods:
            cg.cgh_forward_host(hp, hA, hz, c.lam, c.p, c.Nx, c.Ny, out=hout[m],
                                method=m, handle=h, stream=stream)
    e2e_s = (time.perf_counter() - t0) / E
    if dist is not None:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * len(methods) * pp / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": len(methods) * c.N * 16,
           "d2h_bytes_per_step": len(methods) * c.Nx * c.Ny * 4,
           "ms_per_step": e2e_s * 1e3}

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if methods == ["direct"] else "f32+f16x3",
            "data": "synthetic",
            "config": {"workload": workload_desc(), "Nx": c.Nx, "Ny": c.Ny,
                       "N": c.N, "methods": methods,
                       "l2": "flushed: 256 MiB device write between timed steps",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "methods": {m: {"ms_per_cgh": statistics.mean(meth_ms[m]),
                            "pp_per_s": pp / (statistics.mean(meth_ms[m]) / 1e3)}
                        for m in methods},
            "kernels_ms_per_launch": {k: kt[k][0] / kt[k][1]
                                      for k in kt if kt[k][1] > 0},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
        }
    cg.cgh_destroy(h)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(c, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
