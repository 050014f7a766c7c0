"""Parity of the FP32 separable method (angle addition on the FMA pipe:
cos(tx + ty) = cos tx cos ty - sin tx sin ty as an FP32 product of depth 2N)
with the FP64 oracle, through the C ABI.
Bound (FP32 paths): max |I - I_ref| <= 1e-4 sum |A_j|."""
import numpy as np
import pytest

from gpu_util import max_abs, record, sample_rows, sum_abs_A, to_dev
from oracle_cache import workload_rows
from workloads import make_cloud, workload

pytestmark = pytest.mark.gpu

TOL = 1e-4  # times sum |A_j|


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


def _fwd(cg, h, c, method="sep_fp32"):
    import torch
    pts, A, z = to_dev(c)
    I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
    torch.cuda.synchronize()
    return I.cpu().numpy()


def test_cfg1_full_frame(cg, h, oracle_mod):
    c = workload("cfg1_256x256_n64")
    err, _ = record(c.name, "sep_fp32", _fwd(cg, h, c), oracle_mod.forward(c), c)
    assert err <= TOL * sum_abs_A(c), err
    assert cg.cgh_last_device_status(h) == cg.CGH_OK


@pytest.mark.parametrize("integer", [True, False])
@pytest.mark.parametrize("Nx,Ny", [(257, 97), (129, 129), (7, 300), (1, 1),
                                   (128, 128), (300, 5)])
def test_ragged_frames(cg, h, oracle_mod, integer, Nx, Ny):
    """Frames that are not multiples of the 128 x 128 tile, points outside the
    frame; small frames take the split-K schedule."""
    c = make_cloud(77 + Nx, 45, Nx, Ny, integer=integer, zlo=0.05, zhi=0.5,
                   lam=532e-9, p=8e-6)
    c.xy[:, 1] = c.xy[:, 1] * 2 - 40
    err = max_abs(_fwd(cg, h, c), oracle_mod.forward(c))
    assert err <= TOL * sum_abs_A(c), err


@pytest.mark.parametrize("N", [1, 7, 8, 9, 63, 64, 65, 1000])
def test_point_count_edges(cg, h, oracle_mod, N):
    """Point counts around the 8-point stage; 1000 points on a small frame
    is cut into many k slices."""
    c = make_cloud(400 + N, N, 150, 90, integer=True, zlo=0.2, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    err = max_abs(_fwd(cg, h, c), oracle_mod.forward(c))
    assert err <= TOL * sum_abs_A(c)


def test_deterministic_and_unaligned_output(cg, h, oracle_mod):
    """Two calls give identical bits (the split-K partials are added in a
    fixed order); a 4-byte-aligned output takes scalar stores."""
    import torch
    c = make_cloud(5, 500, 136, 70, integer=False, zlo=0.3, zhi=0.8,
                   lam=473e-9, p=8e-6)
    I1, I2 = _fwd(cg, h, c), _fwd(cg, h, c)
    assert np.array_equal(I1, I2)
    pts, A, z = to_dev(c)
    buf = torch.zeros(136 * 70 + 1, device="cuda")
    out = buf[1:].view(70, 136)
    cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=out, method="sep_fp32",
                   handle=h)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), I1)
    assert buf[0].item() == 0.0
    assert max_abs(I1, oracle_mod.forward(c)) <= TOL * sum_abs_A(c)


def test_cfg2_paper_frame_sampled_rows(cg, h, oracle_mod):
    c = workload("cfg2_1920x1024_n1024")
    I = _fwd(cg, h, c)
    rows = sample_rows(c.Ny, 24, seed=4)
    err, _ = record(c.name, "sep_fp32", I[rows], oracle_mod.forward(c, rows=rows), c)
    assert err <= TOL * sum_abs_A(c), err
    assert max_abs(I, _fwd(cg, h, c, "direct")) <= 2e-5 * sum_abs_A(c)


def test_cfg3_large_frame_sampled_rows(cg, h):
    """3840 x 2160 pixels, 16384 continuous points (Eq. 1, Section 1, the
    cosine of the summed axis phases expanded): the full frame on the GPU,
    the FP64 oracle on 64 evenly spaced rows plus 8 random ones."""
    c = workload("cfg3_3840x2160_n16384")
    I = _fwd(cg, h, c)
    rows, ref = workload_rows(c.name)
    err, _ = record(c.name, "sep_fp32", I[rows], ref, c)
    assert err <= TOL * sum_abs_A(c), err
    assert np.all(np.isfinite(I))


def test_cfg5_continuous_sampled_rows(cg, h, oracle_mod):
    c = workload("cfg5_1920x1080_n4096")
    I = _fwd(cg, h, c)
    rows = sample_rows(c.Ny, 6, seed=22)
    err, _ = record(c.name, "sep_fp32", I[rows], oracle_mod.forward(c, rows=rows), c)
    assert err <= TOL * sum_abs_A(c), err
