"""Parity of the Eq. 2 recurrence kernel (the paper's optimised kernel design,
Section 2.1, restated) with the FP64 oracle, through the C ABI; and every
forward method at the largest point count of the paper's Table 1.
Bound (FP32 paths): max |I - I_ref| <= 1e-4 sum |A_j|."""
import numpy as np
import pytest

from gpu_util import max_abs, record, rel_rms, sample_rows, sum_abs_A, to_dev
from oracle_cache import workload_rows
from workloads import make_cloud, table1_cloud, workload

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


def _fwd(cg, h, c, method="recur"):
    import torch
    pts, A, z = to_dev(c)
    I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
    torch.cuda.synchronize()
    return I.cpu().numpy()


def test_cfg1_full_frame(cg, h, oracle_mod):
    c = workload("cfg1_256x256_n64")
    err, _ = record(c.name, "recur", _fwd(cg, h, c), oracle_mod.forward(c), c)
    assert err <= TOL * sum_abs_A(c), err
    assert cg.cgh_last_device_status(h) == cg.CGH_OK


@pytest.mark.parametrize("integer", [True, False])
@pytest.mark.parametrize("Nx,Ny", [(257, 97), (129, 17), (7, 33), (1, 1), (136, 16)])
def test_ragged_frames(cg, h, oracle_mod, integer, Nx, Ny):
    """Frames that are not multiples of the 128 x 16 group, eight-pixel
    vectors cut by the right edge, points outside the frame."""
    c = make_cloud(61 + Nx, 41, Nx, Ny, integer=integer, zlo=0.05, zhi=0.5,
                   lam=532e-9, p=8e-6)
    c.xy[:, 0] = c.xy[:, 0] * 3 - 97
    err = max_abs(_fwd(cg, h, c), oracle_mod.forward(c))
    assert err <= TOL * sum_abs_A(c), err


@pytest.mark.parametrize("N", [1, 4, 255, 256, 257, 511, 513])
def test_point_count_edges(cg, h, oracle_mod, N):
    """Point counts around the 256-point stage and the unroll by four."""
    c = make_cloud(900 + N, N, 150, 37, integer=True, zlo=0.2, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    err = max_abs(_fwd(cg, h, c), oracle_mod.forward(c))
    assert err <= TOL * sum_abs_A(c)


def test_unaligned_output(cg, h, oracle_mod):
    """An output that is 4-byte but not 16-byte aligned takes scalar stores."""
    import torch
    c = make_cloud(8, 33, 136, 11, integer=True, zlo=0.2, zhi=0.4, lam=532e-9,
                   p=8e-6)
    pts, A, z = to_dev(c)
    buf = torch.zeros(136 * 11 + 1, device="cuda")
    out = buf[1:]
    cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=out.view(11, 136),
                   method="recur", handle=h)
    torch.cuda.synchronize()
    assert max_abs(out.view(11, 136).cpu().numpy(), oracle_mod.forward(c)) \
        <= TOL * sum_abs_A(c)
    assert buf[0].item() == 0.0


def test_wide_row_large_phase(cg, h, oracle_mod):
    """The widest frame (32768 pixels) with a short depth: phases of tens of
    thousands of turns, where an FP32 running sum of radians would fail."""
    c = make_cloud(17, 24, 32768, 2, integer=False, zlo=0.02, zhi=0.05,
                   lam=473e-9, p=8e-6)
    err = max_abs(_fwd(cg, h, c), oracle_mod.forward(c))
    assert err <= TOL * sum_abs_A(c), err


def test_bad_point_skipped_and_reported(cg, h, oracle_mod):
    c = make_cloud(3, 20, 40, 30, integer=True, zlo=0.2, zhi=0.4, lam=532e-9,
                   p=8e-6)
    bad = make_cloud(3, 20, 40, 30, integer=True, zlo=0.2, zhi=0.4, lam=532e-9,
                     p=8e-6)
    bad.z[4] = -1.0
    keep = np.array([j for j in range(20) if j != 4])
    ref = oracle_mod.forward(xy=c.xy[keep], A=c.A[keep], z=c.z[keep], lam=c.lam,
                             p=c.p, Nx=c.Nx, Ny=c.Ny)
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    assert max_abs(_fwd(cg, h, bad), ref) <= TOL * sum_abs_A(c)
    assert cg.cgh_last_device_status(h) == cg.CGH_ERR_INVALID_ARG


def test_cfg2_paper_frame_sampled_rows(cg, h, oracle_mod):
    c = workload("cfg2_1920x1024_n1024")
    I = _fwd(cg, h, c)
    rows = sample_rows(c.Ny, 24, seed=3)
    err, _ = record(c.name, "recur", I[rows], oracle_mod.forward(c, rows=rows), c)
    assert err <= TOL * sum_abs_A(c), err
    # the same hologram as the per-axis-table kernel, to rounding
    assert max_abs(I, _fwd(cg, h, c, "direct")) <= 2e-5 * sum_abs_A(c)


def test_cfg3_large_frame_sampled_rows(cg, h):
    """3840 x 2160 pixels, 16384 continuous points: the Eq. 2 recurrence
    kernel over the full frame, the FP64 oracle (Eq. 1) on 64 evenly spaced
    rows plus 8 random ones."""
    c = workload("cfg3_3840x2160_n16384")
    I = _fwd(cg, h, c)
    rows, ref = workload_rows(c.name)
    err, _ = record(c.name, "recur", I[rows], ref, c)
    assert err <= TOL * sum_abs_A(c), err
    assert np.all(np.isfinite(I))


def test_cfg5_continuous_sampled_rows(cg, h, oracle_mod):
    c = workload("cfg5_1920x1080_n4096")
    I = _fwd(cg, h, c)
    rows = sample_rows(c.Ny, 6, seed=21)
    err, _ = record(c.name, "recur", I[rows], oracle_mod.forward(c, rows=rows), c)
    assert err <= TOL * sum_abs_A(c), err


@pytest.mark.parametrize("method", ["direct", "recur", "sep_fp32", "sep_fp16x3"])
def test_table1_largest_point_count(cg, h, oracle_mod, method):
    """1920 x 1024 pixels from 3584 points, the last row of the paper's
    Table 1, in the configuration the Table 1 sweep of the benchmark runs."""
    c = table1_cloud(3584)
    I = _fwd(cg, h, c, method)
    rows = sample_rows(c.Ny, 8, seed=35)
    ref = oracle_mod.forward(c, rows=rows)
    if method == "sep_fp16x3":
        assert rel_rms(I[rows], ref) <= 1e-4
    else:
        assert max_abs(I[rows], ref) <= TOL * sum_abs_A(c)
