"""cgh_forward_rows: a slab of rows of one hologram (the unit of a row split
over GPUs).  Pixel rows of Eq. 1 (Section 1) are independent, and the row
origin is folded into each point's fixed-point record exactly, so a slab
equals the same rows of the whole frame: bit for bit for the methods whose
per-pixel arithmetic does not depend on where the tiles fall, and within
the stated bounds against the FP64 oracle for every method."""
import numpy as np
import pytest

from gpu_util import max_abs, rel_rms, sum_abs_A, to_dev
from paper_1002_0916_gb300.sharding import row_slabs
from workloads import make_cloud, workload

pytestmark = pytest.mark.gpu

FP32 = ("direct", "recur", "sep_fp32", "naive")
TC = {"sep_fp16x3": 1e-4, "sep_fp16": 1e-2, "sep_bf16": 1e-2}


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


def _slabs(cg, h, c, method, world):
    import torch
    pts, A, z = to_dev(c)
    parts = []
    for y0, rows in row_slabs(c.Ny, world):
        if rows == 0:
            continue
        parts.append(cg.cgh_forward_rows(pts, A, z, c.lam, c.p, c.Nx, y0, rows,
                                         method=method, handle=h))
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    return torch.cat(parts, 0).cpu().numpy()


def _full(cg, h, c, method):
    import torch
    pts, A, z = to_dev(c)
    I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
    torch.cuda.synchronize()
    return I.cpu().numpy()


@pytest.mark.parametrize("method", list(FP32) + list(TC))
@pytest.mark.parametrize("world", [2, 3])
def test_slabs_equal_the_whole_frame(cg, h, oracle_mod, method, world):
    """A 1-, 2- or 3-way row split of a ragged frame (continuous points, some
    outside it) against the whole-frame call and the oracle."""
    c = make_cloud(515, 301, 263, 197, integer=False, zlo=0.1, zhi=0.8,
                   lam=532e-9, p=8e-6)
    c.xy[:, 1] = c.xy[:, 1] * 1.4 - 40
    got = _slabs(cg, h, c, method, world)
    ref = oracle_mod.forward(c)
    if method in FP32:
        assert max_abs(got, ref) <= 1e-4 * sum_abs_A(c)
    else:
        assert rel_rms(got, ref) <= TC[method]
    full = _full(cg, h, c, method)
    if method in ("naive", "recur"):
        # one thread's own loop per pixel: the same arithmetic wherever the
        # slab boundary falls
        assert np.array_equal(got, full), method
    elif method in TC:
        # a slab may take another GEMM tiling than the whole frame
        assert rel_rms(got, full) <= 1e-6
    else:
        assert max_abs(got, full) <= 2e-6 * sum_abs_A(c)


@pytest.mark.parametrize("method", ["direct", "sep_fp16x3"])
def test_far_slab_of_a_tall_frame(cg, h, oracle_mod, method):
    """Rows 9000 .. 9063 of a 12000-row frame of continuous points: the row
    origin shifts the records by c y0^2 - b y0 exactly (mod one turn)."""
    c = make_cloud(77, 200, 320, 12000, integer=False, zlo=0.3, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    import torch
    pts, A, z = to_dev(c)
    got = cg.cgh_forward_rows(pts, A, z, c.lam, c.p, c.Nx, 9000, 64, method=method,
                              handle=h)
    torch.cuda.synchronize()
    ref = oracle_mod.forward(c, rows=np.arange(9000, 9064))
    if method == "direct":
        assert max_abs(got.cpu().numpy(), ref) <= 1e-4 * sum_abs_A(c)
    else:
        assert rel_rms(got.cpu().numpy(), ref) <= 1e-4


def test_paper_frame_two_slabs(cg, h, oracle_mod):
    """The 1920 x 1024 x 1024 workload split in two slabs of 512 rows (the
    two-GPU row split the benchmark runs with --split rows)."""
    c = workload("cfg2_1920x1024_n1024")
    got = _slabs(cg, h, c, "direct", 2)
    rows = np.array([0, 300, 511, 512, 513, 800, 1023], np.int32)
    assert max_abs(got[rows], oracle_mod.forward(c, rows=rows)) <= 1e-4 * sum_abs_A(c)


def test_row_argument_errors(cg, h):
    import ctypes
    import torch
    out = torch.full((4, 8), 2.0, device="cuda")
    e = torch.zeros(2, device="cuda")
    L = cg.lib
    assert L.cgh_forward_rows(h, ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                              ctypes.c_void_p(e.data_ptr()), 1, 532e-9, 8e-6, 8, -1, 4,
                              ctypes.c_void_p(out.data_ptr()), 0, None) == cg.CGH_ERR_INVALID_ARG
    assert L.cgh_forward_rows(h, ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                              ctypes.c_void_p(e.data_ptr()), 1, 532e-9, 8e-6, 8, 0, 0,
                              ctypes.c_void_p(out.data_ptr()), 0, None) == cg.CGH_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.all(out == 2.0)
