"""cgh_forward_noalloc: the hologram entry point that allocates nothing.

It serves callers that may not allocate GPU memory while they run (a
fixed-rate display loop for a spatial light modulator, a plug-in inside an
application that owns all device memory), so it takes its scratch from a
fixed device array instead of a handle's workspace.  These tests call it
through the C ABI and compare it with cgh_forward, twice in a row, to show
that a call is not disturbed by what the previous call left in the shared
array.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import max_abs, sum_abs_A, to_dev
from workloads import make_cloud, workload

pytestmark = pytest.mark.gpu

TOL = 1e-4  # times sum |A_j|, the direct FP32 path's bound


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1002_0916_gb300 as cg
    return cg


def _noalloc(cg, c, out):
    import torch
    pts, A, z = to_dev(c)
    st = cg.lib.cgh_forward_noalloc(
        ctypes.c_void_p(pts.data_ptr()), ctypes.c_void_p(A.data_ptr()),
        ctypes.c_void_p(z.data_ptr()), c.N, c.lam, c.p, c.Nx, c.Ny,
        ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_forward_on_two_calls_in_a_row(cg):
    import torch
    h = cg.cgh_create(0)
    try:
        clouds = [workload("cfg2_1920x1024_n1024"),
                  make_cloud(77, 301, 333, 97, integer=False, zlo=0.3,
                             zhi=0.9, lam=473e-9, p=8e-6)]
        for c in clouds:
            pts, A, z = to_dev(c)
            ref = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny,
                                 method="direct", handle=h)
            out = torch.full((c.Ny, c.Nx), float("nan"), device="cuda")
            assert _noalloc(cg, c, out) == cg.CGH_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert max_abs(got, ref.cpu().numpy()) <= TOL * sum_abs_A(c)
    finally:
        cg.cgh_destroy(h)


def test_noalloc_rejects_frames_beyond_its_scratch(cg):
    import torch
    # 2^20 points need about 512 MiB of angle tables even for a 64 x 64
    # frame: far more than the fixed array.  Nothing may be launched.
    c = make_cloud(5, 1 << 20, 64, 64, integer=True, zlo=0.5, zhi=1.0,
                   lam=532e-9, p=8e-6)
    out = torch.full((64, 64), 5.0, device="cuda")
    assert _noalloc(cg, c, out) == cg.CGH_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.all(out == 5.0)
    bad = make_cloud(5, 8, 64, 64, integer=True, zlo=0.5, zhi=1.0, lam=532e-9,
                     p=8e-6)
    bad.lam = -1.0
    assert _noalloc(cg, bad, out) == cg.CGH_ERR_INVALID_ARG
