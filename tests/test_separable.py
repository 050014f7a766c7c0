"""Parity of the separable tensor-core methods with the FP64 oracle.

Bounds (relative RMS error ||I - I_ref|| / ||I_ref||): split-FP16 <= 1e-4;
single-pass FP16 and BF16 <= 1e-2."""
import numpy as np
import pytest

from gpu_util import record, rel_rms, sample_rows, to_dev
from oracle_cache import workload_rows
from workloads import make_cloud, workload

pytestmark = pytest.mark.gpu

BOUND = {"sep_fp16x3": 1e-4, "sep_fp16": 1e-2, "sep_bf16": 1e-2}
METHODS = list(BOUND)


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1002_0916_gb300 as cg
    return cg


@pytest.fixture(scope="module", params=["auto", "single"])
def h(cg, request):
    """Every test on the default GEMM tiling (CTA pairs above 128 rows) and
    on one-CTA tiles."""
    handle = cg.cgh_create(0)
    cg.cgh_set_gemm_tiles(handle, request.param)
    yield handle
    cg.cgh_destroy(handle)


def _fwd(cg, h, c, method):
    import torch
    pts, A, z = to_dev(c)
    I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    return I.cpu().numpy()


@pytest.mark.parametrize("method", METHODS)
def test_cfg1_full_frame(cg, h, oracle_mod, method):
    c = workload("cfg1_256x256_n64")
    assert record(c.name, method, _fwd(cg, h, c, method), oracle_mod.forward(c),
                  c)[1] <= BOUND[method]


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("integer", [True, False])
def test_ragged_frames(cg, h, oracle_mod, method, integer):
    c = make_cloud(61, 257, 97, 61, integer=integer, zlo=0.05, zhi=0.5,
                   lam=532e-9, p=8e-6)
    c.xy[:, 1] = c.xy[:, 1] * 2 - 30  # points also outside the frame
    assert rel_rms(_fwd(cg, h, c, method), oracle_mod.forward(c)) <= BOUND[method]


@pytest.mark.parametrize("N", [1, 31, 32, 33, 95, 96, 97])
def test_point_counts_across_k_blocks(cg, h, oracle_mod, N):
    c = make_cloud(300 + N, N, 150, 140, integer=True, zlo=0.2, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    assert rel_rms(_fwd(cg, h, c, "sep_fp16x3"), oracle_mod.forward(c)) <= 1e-4


@pytest.mark.parametrize("method", METHODS)
def test_cfg2_paper_frame(cg, h, oracle_mod, method):
    """1920 x 1024 x 1024 (the paper's Table 1 frame, the benchmark's
    workload): GPU full frame, oracle on sampled rows."""
    c = workload("cfg2_1920x1024_n1024")
    I = _fwd(cg, h, c, method)
    rows = sample_rows(c.Ny, 40)
    assert record(c.name, method, I[rows], oracle_mod.forward(c, rows=rows),
                  c)[1] <= BOUND[method]


@pytest.mark.parametrize("method", METHODS)
def test_cfg3_large_frame(cg, h, method):
    """3840 x 2160 pixels, 16384 continuous points (Eq. 1, Section 1, in the
    separable form): the full frame on the GPU -- both K chunks of the split
    form, every wave of tiles -- and the FP64 oracle on 64 evenly spaced rows
    plus 8 random ones."""
    c = workload("cfg3_3840x2160_n16384")
    I = _fwd(cg, h, c, method)
    rows, ref = workload_rows(c.name)
    assert np.all(np.isfinite(I))
    assert record(c.name, method, I[rows], ref, c)[1] <= BOUND[method]


def test_cfg5_forward(cg, h, oracle_mod):
    c = workload("cfg5_1920x1080_n4096")
    I = _fwd(cg, h, c, "sep_fp16x3")
    rows = sample_rows(c.Ny, 8, seed=9)
    assert record(c.name, "sep_fp16x3", I[rows], oracle_mod.forward(c, rows=rows),
                  c)[1] <= 1e-4


def test_separable_agrees_with_direct(cg, h):
    c = workload("cfg2_1920x1024_n1024")
    d = _fwd(cg, h, c, "direct")
    s = _fwd(cg, h, c, "sep_fp16x3")
    assert rel_rms(s, d) <= 1e-4
    assert np.array_equal(s, _fwd(cg, h, c, "sep_fp16x3"))  # deterministic


def test_empty_and_launch_count(cg, h):
    import torch
    out = torch.full((9, 9), 1.0, device="cuda")
    e = torch.zeros(0, device="cuda")
    cg.cgh_forward(e.view(0, 2), e, e, 532e-9, 8e-6, 9, 9, out=out,
                   method="sep_fp16x3", handle=h)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    c = make_cloud(1, 40, 64, 64, integer=True, zlo=0.5, zhi=1.0, lam=532e-9,
                   p=8e-6)
    n0 = cg.cgh_launch_count(h)
    _fwd(cg, h, c, "sep_fp16x3")
    # tables (building the point records themselves), GEMM
    assert cg.cgh_launch_count(h) - n0 == 2
