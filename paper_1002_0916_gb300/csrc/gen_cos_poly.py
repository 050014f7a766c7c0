#!/usr/bin/env python3
"""Fit the software cosine and sine used next to the hardware (MUFU) ones in
the direct kernels, and write cos_poly.h.

cos(d) for d in [0, pi] as a polynomial in s = d^2 of degree 6 (and 5), and
sin(d) as d times a polynomial in s of degree 5, fitted by an iteratively
reweighted least-squares minimax approximation (Lawson's algorithm: repeated
weighted least squares whose weights grow where the error is largest) on a
dense grid.  The kernels fold any angle |theta| < 2 pi into [-pi, pi] first
(u = |theta| - pi: cos theta = -cos u, sin theta = -sign(theta) sin u).

    python gen_cos_poly.py            # rewrite cos_poly.h beside this file
    python gen_cos_poly.py --check    # print the error of the committed table
"""
import os
import sys

import numpy as np

DEG = 6
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "cos_poly.h")


def fit(deg=DEG, iters=200, odd=False):
    s = np.linspace(0.0, np.pi ** 2, 40001)
    d = np.sqrt(s)
    f = np.sin(d) if odd else np.cos(d)
    V = np.vander(s, deg + 1, increasing=True)
    if odd:
        V = V * d[:, None]   # absolute error of d * S(d^2)
    w = np.ones_like(s)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(V * w[:, None], f * w, rcond=None)
        e = np.abs(V @ c - f)
        w = w * (e / e.max() + 1e-3)
        w /= w.sum()
    return c


def fp32_error(c, odd=False):
    d = np.linspace(0.0, np.pi, 200001).astype(np.float32)
    s = (d * d).astype(np.float32)
    c32 = np.asarray(c, dtype=np.float32)
    p = np.full_like(s, c32[-1])
    for k in range(len(c32) - 2, -1, -1):
        p = (p * s + c32[k]).astype(np.float32)
    if odd:
        p = (p * d).astype(np.float32)
    ref = np.sin(d.astype(np.float64)) if odd else np.cos(d.astype(np.float64))
    return float(np.max(np.abs(p.astype(np.float64) - ref)))


def main():
    if "--check" in sys.argv:
        txt = open(OUT).read()
        for prefix in ("COS_C", "COS5_C", "SIN5_C"):
            vals = [float(t.split("=")[1].strip().rstrip("f;")) for t in txt.splitlines()
                    if f"constexpr float {prefix}" in t]
            print(f"{prefix}: max error on [0, pi] in FP32: "
                  f"{fp32_error(vals, odd=prefix.startswith('SIN')):.3e}")
        return
    c = fit()
    c5 = fit(5)
    s5 = fit(5, odd=True)
    lines = ["// cos_poly.h -- written by gen_cos_poly.py; do not edit.",
             "// cos(d) ~= sum_k C_k (d^2)^k for d in [0, pi] (Lawson minimax fits):",
             f"// COS_C: degree {DEG} in d^2, max error in FP32 evaluation "
             f"{fp32_error(c):.2e};",
             f"// COS5_C: degree 5 in d^2, max error in FP32 evaluation "
             f"{fp32_error(c5):.2e};",
             "// sin(d) ~= d * sum_k S_k (d^2)^k for d in [0, pi]:",
             f"// SIN5_C: degree 5 in d^2, max error in FP32 evaluation "
             f"{fp32_error(s5, odd=True):.2e}.",
             "#pragma once", "", "namespace cgh {", ""]
    for k, v in enumerate(c):
        lines.append(f"constexpr float COS_C{k} = {float(np.float32(v))!r}f;")
    lines.append("")
    for k, v in enumerate(c5):
        lines.append(f"constexpr float COS5_C{k} = {float(np.float32(v))!r}f;")
    lines.append("")
    for k, v in enumerate(s5):
        lines.append(f"constexpr float SIN5_C{k} = {float(np.float32(v))!r}f;")
    lines += ["", "}  // namespace cgh", ""]
    open(OUT, "w").write("\n".join(lines))
    print(open(OUT).read())


if __name__ == "__main__":
    main()
