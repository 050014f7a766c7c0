#!/usr/bin/env python3
"""Error of every GPU result against the FP64 oracle, per workload and
method, as a markdown table (needs a GPU; not collected by pytest).

    python tests/accuracy_report.py > accuracy.md

Forward: max |I - I_ref| / sum|A_j| and relative RMS on sampled rows (all
rows for small frames).  Adjoint: relative error per parameter group on
sampled points against the oracle gradient for the same dL/dI field.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from gpu_util import max_abs, rel_rms, sample_rows, sum_abs_A, to_dev  # noqa: E402
from workloads import batch_problems, grad_field, workload  # noqa: E402


def main():
    import torch

    import paper_1002_0916_gb300 as cg
    h = cg.cgh_create(0)
    rows_out = ["| workload | method | rows checked | max abs err / sum A | rel RMS |",
                "|---|---|---|---|---|"]
    cases = [("cfg1_256x256_n64", None), ("cfg2_1920x1024_n1024", 48),
             ("cfg3_3840x2160_n16384", 4), ("cfg5_1920x1080_n4096", 16)]
    for name, nrows in cases:
        c = workload(name)
        pts, A, z = to_dev(c)
        rows = None if nrows is None else sample_rows(c.Ny, nrows)
        ref = oracle.forward(c, rows=rows)
        for m in ("direct", "recur", "sep_fp32", "sep_fp16x3", "sep_fp16", "sep_bf16"):
            I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=m, handle=h)
            torch.cuda.synchronize()
            got = I.cpu().numpy()
            if rows is not None:
                got = got[rows]
            rows_out.append(f"| {name} | {m} | {len(ref)} | "
                            f"{max_abs(got, ref) / sum_abs_A(c):.2e} | "
                            f"{rel_rms(got, ref):.2e} |")
    # batch: a few problems
    clouds = batch_problems(seed=0)
    probs = []
    for cl in clouds:
        p_, A_, z_ = to_dev(cl)
        probs.append(dict(points=p_, A=A_, z=z_, lam=cl.lam, p=cl.p, Nx=cl.Nx,
                          Ny=cl.Ny, out=torch.empty((cl.Ny, cl.Nx), device="cuda")))
    for m in ("direct", "sep_fp16x3"):
        cg.cgh_batch(probs, method=m, handle=h)
        torch.cuda.synchronize()
        worst_abs, worst_rel = 0.0, 0.0
        for i in (0, 17, 40, 63):
            cl = clouds[i]
            rows = sample_rows(cl.Ny, 2, seed=i)
            ref = oracle.forward(cl, rows=rows)
            got = probs[i]["out"].cpu().numpy()[rows]
            worst_abs = max(worst_abs, max_abs(got, ref) / sum_abs_A(cl))
            worst_rel = max(worst_rel, rel_rms(got, ref))
        rows_out.append(f"| batch of 64 (problems 0, 17, 40, 63) | {m} | 8 | "
                        f"{worst_abs:.2e} | {worst_rel:.2e} |")
    print("\n".join(rows_out))
    print()
    # adjoint
    c = workload("cfg5_1920x1080_n4096")
    pts, A, z = to_dev(c)
    G = grad_field(11, c.Nx, c.Ny, scale=40.0)
    sel = np.sort(np.random.default_rng(3).choice(c.N, 64, replace=False))
    rp, rA, rz = oracle.grad(c, G.astype(np.float64), pts=sel)
    print("| adjoint (1920x1080x4096, 64 sampled points) | rel err A | x | y | z |")
    print("|---|---|---|---|---|")
    Gd = torch.from_numpy(G).cuda()
    for m in ("direct", "sep_fp32", "sep_fp16x3"):
        gp, gA, gz = cg.cgh_backward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, Gd,
                                     method=m, handle=h)
        torch.cuda.synchronize()
        gp, gA, gz = gp.cpu().numpy()[sel], gA.cpu().numpy()[sel], gz.cpu().numpy()[sel]

        def rel(a, b):
            return np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"| {m} | {rel(gA, rA):.2e} | {rel(gp[:, 0], rp[:, 0]):.2e} | "
              f"{rel(gp[:, 1], rp[:, 1]):.2e} | {rel(gz, rz):.2e} |")
    cg.cgh_destroy(h)


if __name__ == "__main__":
    main()
