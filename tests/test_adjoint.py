"""The hand-written adjoint (cgh_backward, CGHFunction) against the FP64
oracle gradient and central finite differences of the FP64 loss.

Bound: relative error ||g - g_ref|| / ||g_ref|| <= 1e-3 per parameter group
(A, x, y, z); finite differences per sampled component:
|g - fd| <= 1e-3 max(|fd|, rms(fd of that group))."""
import functools
import json
import os

import numpy as np
import pytest

from gpu_util import to_dev
from workloads import grad_field, make_cloud, workload

pytestmark = pytest.mark.gpu

METHODS = ["direct", "sep_fp32", "sep_fp16x3"]
TOL = 1e-3


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1002_0916_gb300 as cg
    return cg


@pytest.fixture(scope="module")
def h(cg):
    handle = cg.cgh_create(0)
    yield handle
    cg.cgh_destroy(handle)


def _bwd(cg, h, c, G, method):
    import torch
    pts, A, z = to_dev(c)
    Gd = torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).cuda()
    gp, gA, gz = cg.cgh_backward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, Gd,
                                 method=method, handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    return gp.cpu().numpy(), gA.cpu().numpy(), gz.cpu().numpy()


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _check_groups(got, ref, sel=None, log=None):
    gp, gA, gz = got
    rp, rA, rz = ref
    if sel is not None:
        gp, gA, gz = gp[sel], gA[sel], gz[sel]
    errs = {"A": _rel(gA, rA), "x": _rel(gp[:, 0], rp[:, 0]),
            "y": _rel(gp[:, 1], rp[:, 1]), "z": _rel(gz, rz)}
    path = os.environ.get("CGH_ACCURACY_LOG")
    if path and log is not None:
        with open(path, "a") as fh:
            fh.write(json.dumps({"workload": log[0], "method": log[1], "points": int(
                len(gA)), "grad_rel": errs}) + "\n")
    assert all(v <= TOL for v in errs.values()), errs
    return errs


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("integer", [True, False])
def test_loss_gradient_small(cg, h, oracle_mod, method, integer):
    """L = ||I - T||^2 with I, T from the FP64 oracle (T: an independent
    cloud); G = 2 (I - T); all points checked."""
    c = make_cloud(71, 300, 200, 150, integer=integer, zlo=0.3, zhi=0.9,
                   lam=532e-9, p=6.4e-6)
    t = make_cloud(72, 300, 200, 150, integer=integer, zlo=0.3, zhi=0.9,
                   lam=532e-9, p=6.4e-6)
    G = 2.0 * (oracle_mod.forward(c) - oracle_mod.forward(t))
    G32 = G.astype(np.float32)
    ref = oracle_mod.grad(c, G32.astype(np.float64))
    _check_groups(_bwd(cg, h, c, G32, method), ref)


@pytest.mark.parametrize("method", METHODS)
def test_ragged_and_edge_sizes(cg, h, oracle_mod, method):
    for (N, Nx, Ny) in [(1, 33, 17), (129, 130, 129), (255, 17, 301)]:
        c = make_cloud(N + Nx, N, Nx, Ny, integer=False, zlo=0.2, zhi=0.6,
                       lam=473e-9, p=8e-6)
        G = grad_field(N + 5, Nx, Ny)
        ref = oracle_mod.grad(c, G.astype(np.float64))
        _check_groups(_bwd(cg, h, c, G, method), ref)


@pytest.mark.parametrize("method", METHODS)
def test_cfg5_full_size_sampled_points(cg, h, method):
    """1920 x 1080, 4096 continuous points, the differentiable workload, in
    the launch configuration of a full-size call: the derivatives of Eq. 1
    (Section 1) with respect to A_j, x_j, y_j and z_j, against the FP64
    oracle gradient on 256 sampled points (every parameter group)."""
    c = workload("cfg5_1920x1080_n4096")
    G = grad_field(11, c.Nx, c.Ny, scale=40.0)
    got = _bwd(cg, h, c, G, method)
    sel, ref = _cfg5_grad_ref()
    _check_groups(got, ref, sel, log=(c.name, method))


@functools.lru_cache(maxsize=None)
def _cfg5_grad_ref():
    import oracle
    c = workload("cfg5_1920x1080_n4096")
    G = grad_field(11, c.Nx, c.Ny, scale=40.0)
    sel = np.sort(np.random.default_rng(3).choice(c.N, 256, replace=False))
    return sel, oracle.grad(c, G.astype(np.float64), pts=sel)


def test_cfg5_finite_differences(cg, h, oracle_mod):
    """Central differences of the FP64 loss ||I - T||^2 (T: the FP64
    hologram of an independent seeded 4096-point cloud) on sampled
    parameters, against every adjoint method."""
    c = workload("cfg5_1920x1080_n4096")
    T = oracle_mod.forward(workload("cfg5_1920x1080_n4096", seed=1))
    I = oracle_mod.forward(c)
    G = (2.0 * (I - T)).astype(np.float32)
    grads = {m: _bwd(cg, h, c, G, m) for m in METHODS}
    rng = np.random.default_rng(17)
    js = rng.choice(c.N, 6, replace=False)

    def single(xy, A, z):
        return oracle_mod.forward(xy=np.array([xy], np.float32),
                                  A=np.array([A], np.float32),
                                  z=np.array([z], np.float32), lam=c.lam, p=c.p,
                                  Nx=c.Nx, Ny=c.Ny)

    rows = {"A": [], "x": [], "y": [], "z": []}
    for j in js:
        xy0, A0, z0 = c.xy[j].copy(), float(c.A[j]), float(c.z[j])
        base = single(xy0, A0, z0)
        R = I - base - T
        for which in rows:
            if which == "A":
                p1, p2 = np.float32(A0 + 1e-3), np.float32(A0 - 1e-3)
                a = single(xy0, p1, z0)
                b = single(xy0, p2, z0)
                h_tot = float(p1) - float(p2)
            elif which in ("x", "y"):
                k = 0 if which == "x" else 1
                u1, u2 = xy0.copy(), xy0.copy()
                u1[k] = np.float32(xy0[k] + 0.01)
                u2[k] = np.float32(xy0[k] - 0.01)
                a, b = single(u1, A0, z0), single(u2, A0, z0)
                h_tot = float(u1[k]) - float(u2[k])
            else:
                p1, p2 = np.float32(z0 * (1 + 4e-6)), np.float32(z0 * (1 - 4e-6))
                a, b = single(xy0, A0, p1), single(xy0, A0, p2)
                h_tot = float(p1) - float(p2)
            # L(+) - L(-) = sum (a - b)(2R + a + b), no large-sum cancellation
            fd = float(np.sum((a - b) * (2 * R + a + b))) / h_tot
            rows[which].append((j, fd))
    for m in METHODS:
        gp, gA, gz = grads[m]
        for which, lst in rows.items():
            fds = np.array([v for _, v in lst])
            scale = np.sqrt(np.mean(fds ** 2))
            for (j, fd) in lst:
                g = {"A": gA[j], "x": gp[j, 0], "y": gp[j, 1], "z": gz[j]}[which]
                assert abs(g - fd) <= TOL * max(abs(fd), scale), (m, which, j, g, fd)


def test_autograd_function(cg, oracle_mod):
    import torch
    c = make_cloud(81, 120, 96, 80, integer=False, zlo=0.3, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    t = make_cloud(82, 120, 96, 80, integer=False, zlo=0.3, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    T = torch.from_numpy(oracle_mod.forward(t).astype(np.float32)).cuda()
    pts, A, z = (v.clone().requires_grad_(True) for v in to_dev(c))
    for fwd, bwd in (("direct", "direct"), ("sep_fp32", "sep_fp32"),
                     ("sep_fp16x3", "sep_fp16x3")):
        for v in (pts, A, z):
            v.grad = None
        I = cg.CGHFunction.apply(pts, A, z, c.lam, c.p, c.Nx, c.Ny, fwd, bwd)
        loss = ((I - T) ** 2).sum()
        loss.backward()
        Gref = 2.0 * (oracle_mod.forward(c) - oracle_mod.forward(t))
        ref = oracle_mod.grad(c, Gref)
        got = (pts.grad.cpu().numpy(), A.grad.cpu().numpy(), z.grad.cpu().numpy())
        _check_groups(got, ref)


def test_deterministic_and_optional_outputs(cg, h):
    import torch
    c = make_cloud(5, 200, 150, 100, integer=True, zlo=0.5, zhi=1.0,
                   lam=532e-9, p=8e-6)
    G = grad_field(6, c.Nx, c.Ny)
    for m in METHODS:
        a = _bwd(cg, h, c, G, m)
        b = _bwd(cg, h, c, G, m)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
    pts, A, z = to_dev(c)
    Gd = torch.from_numpy(G).cuda()
    gp, gA, gz = cg.cgh_backward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, Gd,
                                 handle=h, need=(False, True, False))
    torch.cuda.synchronize()
    assert gp is None and gz is None
    assert np.array_equal(gA.cpu().numpy(), _bwd(cg, h, c, G, "direct")[1])
    with pytest.raises(cg.CGHError) as e:
        cg.cgh_backward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, Gd, method="naive",
                        handle=h)
    assert e.value.status == cg.CGH_ERR_INVALID_ARG


@pytest.mark.parametrize("case", [(300, 200, 150), (129, 130, 129), (4096, 1920, 1080)])
def test_separable_adjoint_on_both_gemm_tilings(cg, oracle_mod, case):
    """The split-FP16 adjoint on one-CTA GEMM tiles and on CTA pairs: both
    within the bound of the FP64 gradient (sampled points at full size), and
    within rounding of each other."""
    N, Nx, Ny = case
    c = make_cloud(N + 3, N, Nx, Ny, integer=False, zlo=0.3, zhi=1.2,
                   lam=532e-9, p=6.4e-6)
    G = grad_field(N + 9, Nx, Ny, scale=10.0)
    sel = None if N <= 300 else np.sort(np.random.default_rng(5).choice(N, 32, replace=False))
    ref = oracle_mod.grad(c, G.astype(np.float64), pts=sel)
    got = {}
    for tiles in ("single", "pairs"):
        hh = cg.cgh_create(0)
        try:
            cg.cgh_set_gemm_tiles(hh, tiles)
            got[tiles] = _bwd(cg, hh, c, G, "sep_fp16x3")
        finally:
            cg.cgh_destroy(hh)
        _check_groups(got[tiles], ref, sel)
    for a, b in zip(got["single"], got["pairs"]):
        assert _rel(b, a) <= 1e-5


def test_direct_adjoint_staged_and_global_rows_agree(cg, oracle_mod, monkeypatch):
    """The direct adjoint reads G through shared memory (TMA-staged rows)
    where G's layout allows, else row by row from global memory: the same
    arithmetic in the same order, so the same bits; both within the bound."""
    c = make_cloud(81, 700, 200, 150, integer=False, zlo=0.3, zhi=0.9, lam=532e-9,
                   p=6.4e-6)
    G = grad_field(82, c.Nx, c.Ny)
    out = {}
    for staged in ("1", "0"):
        monkeypatch.setenv("CGH_BWD_STAGED", staged)
        hh = cg.cgh_create(0)
        try:
            out[staged] = _bwd(cg, hh, c, G, "direct")
        finally:
            cg.cgh_destroy(hh)
    for a, b in zip(out["1"], out["0"]):
        assert np.array_equal(a, b)
    _check_groups(out["1"], oracle_mod.grad(c, G.astype(np.float64)))


def test_fp32_separable_adjoint_staged_and_global_rows_agree(cg, oracle_mod, monkeypatch):
    """The FP32 separable adjoint (angle addition, per-column sums U, V and
    per-row sums P, Q) with G rows staged by TMA and read from global memory:
    the same bits, within the bound; and within FP32 rounding of the direct
    adjoint (the same sums, the cosine of each sum expanded)."""
    c = make_cloud(85, 700, 200, 157, integer=False, zlo=0.3, zhi=0.9, lam=532e-9,
                   p=6.4e-6)
    G = grad_field(86, c.Nx, c.Ny)
    out = {}
    for staged in ("1", "0"):
        monkeypatch.setenv("CGH_BWD_STAGED", staged)
        hh = cg.cgh_create(0)
        try:
            out[staged] = _bwd(cg, hh, c, G, "sep_fp32")
            if staged == "1":
                out["direct"] = _bwd(cg, hh, c, G, "direct")
        finally:
            cg.cgh_destroy(hh)
    for a, b in zip(out["1"], out["0"]):
        assert np.array_equal(a, b)
    _check_groups(out["1"], oracle_mod.grad(c, G.astype(np.float64)))
    for a, b in zip(out["1"], out["direct"]):
        assert _rel(a, b) <= 2e-5


def test_fp32_separable_adjoint_unaligned_gradient_field(cg, oracle_mod):
    """A G that starts 4 bytes past a 16-byte boundary (Nx a multiple of 4):
    both strip kernels read it row by row from global memory with scalar
    loads, and the results meet the bound."""
    import torch
    c = make_cloud(87, 200, 96, 70, integer=True, zlo=0.3, zhi=0.9, lam=532e-9,
                   p=6.4e-6)
    G = grad_field(88, c.Nx, c.Ny)
    pts, A, z = to_dev(c)
    buf = torch.zeros(c.Nx * c.Ny + 4, device="cuda")
    Gd = buf[1:1 + c.Nx * c.Ny].view(c.Ny, c.Nx)
    Gd.copy_(torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)))
    ref = oracle_mod.grad(c, G.astype(np.float64))
    for m in ("direct", "sep_fp32"):
        hh = cg.cgh_create(0)
        try:
            gp, gA, gz = cg.cgh_backward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, Gd,
                                         method=m, handle=hh)
            torch.cuda.synchronize()
            assert cg.cgh_last_device_status(hh) == cg.CGH_OK
            _check_groups((gp.cpu().numpy(), gA.cpu().numpy(), gz.cpu().numpy()), ref)
        finally:
            cg.cgh_destroy(hh)
