"""The separable forward with operand tiles generated inside the CTA-pair
GEMM (CGH_GEMM_PAIRS_GEN): the U / V entries of the separable form of
Eq. 1 (Section 1; the phase split into its x and y parts, each stepped by
the exact fixed-point form of Eq. 2) are computed in shared memory instead
of read from tables.  Checks: bit-identical holograms to the table path at
the same tile width (same entries, same MMAs), and the stated bounds
against the FP64 oracle (relative RMS: split FP16 <= 1e-4, single-pass
FP16 / BF16 <= 1e-2) on ragged frames, point counts across K blocks, the
1920 x 1024 x 1024 frame, two K chunks and the 3840 x 2160 x 16384 frame."""
import numpy as np
import pytest

from gpu_util import rel_rms, record, sample_rows, to_dev
from oracle_cache import workload_rows
from workloads import make_cloud, workload

pytestmark = pytest.mark.gpu

BOUND = {"sep_fp16x3": 1e-4, "sep_fp16": 1e-2, "sep_bf16": 1e-2}


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


def _fwd(cg, h, c, method, tiling, width):
    import torch
    cg.cgh_set_gemm_plan(h, tiling, width)
    try:
        pts, A, z = to_dev(c)
        I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
        torch.cuda.synchronize()
        assert cg.cgh_last_device_status(h) == cg.CGH_OK
        return I.cpu().numpy()
    finally:
        cg.cgh_set_gemm_plan(h, "auto")


@pytest.mark.parametrize("method,width", [("sep_fp16x3", 112), ("sep_fp16x3", 144),
                                          ("sep_fp16x3", 160), ("sep_fp16x3", 224),
                                          ("sep_fp16x3", 256), ("sep_fp16", 112),
                                          ("sep_fp16", 256), ("sep_bf16", 112),
                                          ("sep_bf16", 256)])
def test_bit_identical_to_the_table_path(cg, h, method, width):
    """Same entries (exact fixed-point phase, same sincos and rounding) and
    the same MMAs in the same order: the generated and the table GEMM give
    the same bits, on a ragged frame with points outside it."""
    c = make_cloud(91, 421, 613, 333, integer=False, zlo=0.1, zhi=0.7,
                   lam=532e-9, p=8e-6)
    c.xy[:, 0] = c.xy[:, 0] * 1.5 - 100
    gen = _fwd(cg, h, c, method, "pairs_gen", width)
    tab = _fwd(cg, h, c, method, "pairs", width)
    assert np.all(np.isfinite(gen))
    assert np.array_equal(gen, tab)


@pytest.mark.parametrize("method", list(BOUND))
def test_cfg1_and_ragged_frames(cg, h, oracle_mod, method):
    for c in (workload("cfg1_256x256_n64"),
              make_cloud(61, 257, 97, 61, integer=True, zlo=0.05, zhi=0.5,
                         lam=532e-9, p=8e-6),
              make_cloud(62, 100, 300, 1, integer=False, zlo=0.3, zhi=0.9,
                         lam=473e-9, p=8e-6)):
        got = _fwd(cg, h, c, method, "pairs_gen", 112)
        assert record(c.name or "ragged", method + "/gen", got, oracle_mod.forward(c),
                      c)[1] <= BOUND[method]


@pytest.mark.parametrize("N", [1, 31, 32, 33, 95, 96, 97])
def test_point_counts_across_k_blocks(cg, h, oracle_mod, N):
    c = make_cloud(300 + N, N, 150, 140, integer=True, zlo=0.2, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    assert rel_rms(_fwd(cg, h, c, "sep_fp16x3", "pairs_gen", 112),
                   oracle_mod.forward(c)) <= 1e-4


@pytest.mark.parametrize("method", list(BOUND))
def test_cfg2_paper_frame(cg, h, oracle_mod, method):
    """1920 x 1024 x 1024, the paper's Table 1 frame, with the width the
    heuristic picks for it; oracle on 40 rows."""
    c = workload("cfg2_1920x1024_n1024")
    I = _fwd(cg, h, c, method, "pairs_gen", 0)
    rows = sample_rows(c.Ny, 40)
    assert record(c.name, method + "/gen", I[rows], oracle_mod.forward(c, rows=rows),
                  c)[1] <= BOUND[method]


def test_two_k_chunks(cg, h, oracle_mod):
    """10,000 points: 20,000 values of k, more than the 16,384 one split-FP16
    launch accumulates; the second launch adds its partial product into the
    first's output."""
    c = make_cloud(4242, 10000, 320, 272, integer=False, zlo=0.4, zhi=1.2,
                   lam=532e-9, p=6.4e-6)
    gen = _fwd(cg, h, c, "sep_fp16x3", "pairs_gen", 160)
    assert np.array_equal(gen, _fwd(cg, h, c, "sep_fp16x3", "pairs", 160))
    rows = sample_rows(c.Ny, 24, seed=4)
    assert rel_rms(gen[rows], oracle_mod.forward(c, rows=rows)) <= 1e-4


@pytest.mark.parametrize("method", list(BOUND))
def test_cfg3_large_frame(cg, h, method):
    """3840 x 2160 x 16384 continuous points at 256-wide pairs (both waves of
    pair tiles; two K chunks in split FP16), the FP64 oracle on 64 evenly
    spaced rows plus 8 random ones."""
    c = workload("cfg3_3840x2160_n16384")
    I = _fwd(cg, h, c, method, "pairs_gen", 256)
    rows, ref = workload_rows(c.name)
    assert np.all(np.isfinite(I))
    assert record(c.name, method + "/gen", I[rows], ref, c)[1] <= BOUND[method]


def test_plan_errors(cg, h):
    assert cg.lib.cgh_set_gemm_plan(h, 3, 200) == cg.CGH_ERR_UNSUPPORTED
    assert cg.lib.cgh_set_gemm_plan(h, 1, 256) == cg.CGH_ERR_UNSUPPORTED
    assert cg.lib.cgh_set_gemm_plan(None, 2, 112) == cg.CGH_ERR_INVALID_ARG
    cg.cgh_set_gemm_plan(h, "pairs_gen", 144)
    assert cg.cgh_gemm_plan_for(h, 1024, 1920, 1024, "sep_fp16x3") == ("pairs_gen", 144,
                                                                        False)
    cg.cgh_set_gemm_plan(h, "auto")


def test_tuned_plan_is_used(cg, oracle_mod):
    """cgh_tune on a tensor-core method measures every GEMM plan and the
    handle's later calls of that size take the fastest."""
    import torch
    hh = cg.cgh_create(0)
    try:
        c = workload("cfg2_1920x1024_n1024")
        assert cg.cgh_gemm_plan_for(hh, c.N, c.Nx, c.Ny, "sep_fp16x3")[2] is False
        tiling, width, tuned = cg.cgh_tune(hh, c.N, c.Nx, c.Ny, "sep_fp16x3")
        assert tuned and tiling in ("single", "pairs", "pairs_gen") and width >= 112
        assert cg.cgh_gemm_plan_for(hh, c.N, c.Nx, c.Ny, "sep_fp16x3") == (tiling, width,
                                                                           True)
        pts, A, z = to_dev(c)
        I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method="sep_fp16x3",
                           handle=hh)
        torch.cuda.synchronize()
        rows = sample_rows(c.Ny, 16, seed=3)
        assert rel_rms(I.cpu().numpy()[rows], oracle_mod.forward(c, rows=rows)) <= 1e-4
    finally:
        cg.cgh_destroy(hh)
