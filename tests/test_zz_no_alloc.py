"""cgh_forward_noalloc: the hologram entry point that allocates nothing.

It serves callers that may not allocate GPU memory while they run (a
fixed-rate display loop for a spatial light modulator, a plug-in inside an
application that owns all device memory), so it takes its scratch from a
fixed device array instead of a handle's workspace.  These tests call it
through the C ABI and compare it with the FP64 oracle (Eq. 1, Section 1;
bound max |I - I_ref| <= 1e-4 sum |A_j|) and with cgh_forward, twice in a
row, to show that a call is not disturbed by what the previous call left in
the shared array; that an empty cloud gives zeros; that calls leave the
device's free memory unchanged; and that frames beyond the array are
refused.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import max_abs, sample_rows, sum_abs_A, to_dev
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


def _noalloc(cg, c, out, dev_inputs=None):
    import torch
    pts, A, z = dev_inputs if dev_inputs is not None else to_dev(c)
    st = cg.lib.cgh_forward_noalloc(
        ctypes.c_void_p(pts.data_ptr()), ctypes.c_void_p(A.data_ptr()),
        ctypes.c_void_p(z.data_ptr()), c.N, ctypes.c_double(c.lam),
        ctypes.c_double(c.p), c.Nx, c.Ny, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def _clouds():
    return [workload("cfg2_1920x1024_n1024"),
            make_cloud(77, 301, 333, 97, integer=False, zlo=0.3, zhi=0.9,
                       lam=473e-9, p=8e-6)]


def test_noalloc_matches_forward_on_two_calls_in_a_row(cg):
    import torch
    h = cg.cgh_create(0)
    try:
        for c in _clouds():
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


def test_noalloc_against_the_oracle(cg, oracle_mod):
    """The paper's Table 1 frame (1920 x 1024, 1024 points) on 48 sampled
    rows, and a ragged 333 x 97 frame of continuous points in full, each
    computed twice in a row on the shared array."""
    import torch
    for c in _clouds():
        rows = sample_rows(c.Ny, 48, seed=31) if c.Ny > 128 else None
        ref = oracle_mod.forward(c, rows=rows)
        for _ in range(2):
            out = torch.full((c.Ny, c.Nx), float("nan"), device="cuda")
            assert _noalloc(cg, c, out) == cg.CGH_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            got = got if rows is None else got[rows]
            err = max_abs(got, ref)
            assert err <= TOL * sum_abs_A(c), err


def test_noalloc_runs_a_rotation_tile(cg, oracle_mod):
    """A frame whose built-in tile is a rotation tile and whose rotation tables
    (twice the angle tables) fit the array: 1024 x 1024 with 512 points needs
    8.4 MB.  The call runs that tile; checked against cgh_forward and the
    oracle on sampled rows, twice in a row."""
    import torch
    c = make_cloud(91, 512, 1024, 1024, integer=False, zlo=0.4, zhi=1.4,
                   lam=532e-9, p=8e-6)
    h = cg.cgh_create(0)
    try:
        assert cg.cgh_direct_tile_for(h, c.N, c.Nx, c.Ny)[7] >= 6
        pts, A, z = to_dev(c)
        ref_gpu = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method="direct",
                                 handle=h).cpu().numpy()
    finally:
        cg.cgh_destroy(h)
    rows = sample_rows(c.Ny, 16, seed=5)
    ref = oracle_mod.forward(c, rows=rows)
    for _ in range(2):
        out = torch.full((c.Ny, c.Nx), float("nan"), device="cuda")
        assert _noalloc(cg, c, out) == cg.CGH_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert max_abs(got, ref_gpu) <= 1e-5 * sum_abs_A(c)
        assert max_abs(got[rows], ref) <= TOL * sum_abs_A(c)


def test_noalloc_empty_cloud_gives_zeros(cg):
    import torch
    e = torch.zeros(0, device="cuda")
    c = make_cloud(1, 0, 45, 23, integer=True, zlo=0.5, zhi=1.0, lam=532e-9,
                   p=8e-6)
    out = torch.full((c.Ny, c.Nx), 3.0, device="cuda")
    assert _noalloc(cg, c, out, dev_inputs=(e, e, e)) == cg.CGH_OK
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_noalloc_leaves_free_device_memory_unchanged(cg):
    """After a first call (which loads the kernels), further calls do not
    change the device's free memory: nothing is allocated."""
    import torch
    c = workload("cfg2_1920x1024_n1024")
    dev_inputs = to_dev(c)
    out = torch.empty((c.Ny, c.Nx), device="cuda")
    assert _noalloc(cg, c, out, dev_inputs) == cg.CGH_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert _noalloc(cg, c, out, dev_inputs) == cg.CGH_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


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
