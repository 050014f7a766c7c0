"""The FMA-pipe cosine polynomial of the direct kernels (cos_poly.h, fitted
by gen_cos_poly.py): its error over the folded range [0, pi], evaluated in
FP32 exactly as the kernel does, against FP64 cos."""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1002_0916_gb300", "csrc", "cos_poly.h")


def _coeffs(prefix="COS_C"):
    txt = open(HDR).read()
    return [np.float32(float(v)) for v in
            re.findall(r"constexpr float " + prefix + r"\d+ = ([-0-9.e+]+)f;", txt)]


def _kernel_cos(theta, prefix="COS_C"):
    """The kernel's fold (u = |theta| - pi, cos theta = -cos u) and Horner
    evaluation, in float32."""
    c = _coeffs(prefix)
    u = (np.abs(theta.astype(np.float32)) - np.float32(np.pi)).astype(np.float32)
    s = (u * u).astype(np.float32)
    p = np.full_like(s, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p * s + c[k]).astype(np.float32)
    return -p


def test_polynomial_error_bound():
    # the kernel feeds it theta_x + theta_y, both in [-pi, pi)
    th = np.linspace(-2 * np.pi + 1e-6, 2 * np.pi - 1e-6, 400001).astype(np.float32)
    for prefix, bound in (("COS_C", 1e-6), ("COS5_C", 2e-6)):
        err = np.abs(_kernel_cos(th, prefix).astype(np.float64)
                     - np.cos(th.astype(np.float64)))
        assert err.max() < bound, prefix


def test_polynomial_has_the_taylor_leading_terms():
    c = _coeffs()
    assert len(c) == 7
    assert abs(c[0] - 1.0) < 1e-6 and abs(c[1] + 0.5) < 1e-5
    assert abs(c[2] - 1.0 / 24) < 1e-5


def _kernel_sin(theta):
    """The adjoint kernel's sine: u = |theta| - pi, sin theta = -sign(theta)
    u S(u^2), Horner in float32."""
    c = _coeffs("SIN5_C")
    t = theta.astype(np.float32)
    u = (np.abs(t) - np.float32(np.pi)).astype(np.float32)
    s = (u * u).astype(np.float32)
    p = np.full_like(s, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p * s + c[k]).astype(np.float32)
    v = (p * u).astype(np.float32)
    return np.where(t < 0, v, -v)


def test_sine_polynomial_error_bound():
    th = np.linspace(-2 * np.pi + 1e-6, 2 * np.pi - 1e-6, 400001).astype(np.float32)
    err = np.abs(_kernel_sin(th).astype(np.float64) - np.sin(th.astype(np.float64)))
    assert err.max() < 1e-6
    c = _coeffs("SIN5_C")
    assert len(c) == 6
    assert abs(c[0] - 1.0) < 1e-5 and abs(c[1] + 1.0 / 6) < 1e-5
