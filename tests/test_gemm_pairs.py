"""The tensor-core GEMM on CTA pairs (tcgen05 cta_group::2, 256-row tiles
over two SMs) against an FP64 CPU product of the same 16-bit operands, and
the separable methods with pair tiles against the FP64 oracle.
Bounds as the one-CTA GEMM: per element |D - ref| <= K 2^-23 (|A| |B|^T);
relative RMS: split FP16 <= 1e-4, single-pass FP16 / BF16 <= 1e-2."""
import numpy as np
import pytest

from gpu_util import rel_rms, sample_rows, to_dev
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
    cg.cgh_set_gemm_tiles(handle, "pairs")
    yield handle
    cg.cgh_destroy(handle)


@pytest.mark.parametrize("dtype", ["fp16", "bf16"])
@pytest.mark.parametrize("M,N,K", [(256, 112, 64), (200, 300, 128), (1, 1, 64),
                                   (129, 257, 192), (1024, 1920, 2048),
                                   (333, 129, 1024), (2160, 3840, 256),
                                   (1080, 1920, 256)])
def test_pair_gemm_matches_fp64_product(cg, h, dtype, M, N, K):
    import torch
    tdt = {"fp16": torch.float16, "bf16": torch.bfloat16}[dtype]
    g = torch.Generator().manual_seed(M * 5 + N * 11 + K)
    A = torch.randn(M, K, generator=g).to(tdt)
    B = torch.randn(N, K, generator=g).to(tdt)
    D = cg.cgh_debug_gemm(A.cuda(), B.cuda(), handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    A64 = A.double().numpy()
    B64 = B.double().numpy()
    ref = A64 @ B64.T
    bound = K * 2.0 ** -23 * (np.abs(A64) @ np.abs(B64).T) + 1e-30
    err = np.abs(D.cpu().double().numpy() - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_pair_gemm_structure_identity(cg, h):
    """Each row of A picks one column of B: a swapped half of A or B between
    the two CTAs, or a shifted row, changes the result exactly."""
    import torch
    M, N, K = 512, 448, 128
    A = torch.zeros(M, K, dtype=torch.float16)
    for m in range(M):
        A[m, (7 * m + 1) % K] = 1.0
    B = (torch.arange(N * K, dtype=torch.float32).reshape(N, K) % 2029).to(torch.float16)
    D = cg.cgh_debug_gemm(A.cuda(), B.cuda(), handle=h).cpu()
    assert torch.equal(D, A.float() @ B.float().T)


def _fwd(cg, h, c, method):
    import torch
    pts, A, z = to_dev(c)
    I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    return I.cpu().numpy()


@pytest.mark.parametrize("method", list(BOUND))
def test_cfg1_full_frame(cg, h, oracle_mod, method):
    c = workload("cfg1_256x256_n64")
    assert rel_rms(_fwd(cg, h, c, method), oracle_mod.forward(c)) <= BOUND[method]


@pytest.mark.parametrize("method", list(BOUND))
def test_ragged_frame(cg, h, oracle_mod, method):
    c = make_cloud(62, 257, 301, 259, integer=False, zlo=0.05, zhi=0.5,
                   lam=532e-9, p=8e-6)
    c.xy[:, 1] = c.xy[:, 1] * 2 - 30
    assert rel_rms(_fwd(cg, h, c, method), oracle_mod.forward(c)) <= BOUND[method]


@pytest.mark.parametrize("method", list(BOUND))
def test_cfg2_paper_frame_sampled_rows(cg, h, oracle_mod, method):
    c = workload("cfg2_1920x1024_n1024")
    I = _fwd(cg, h, c, method)
    rows = sample_rows(c.Ny, 16, seed=8)
    assert rel_rms(I[rows], oracle_mod.forward(c, rows=rows)) <= BOUND[method]


def test_pairs_agree_with_single_tiles(cg, h):
    """Same products, FP32 accumulation: the two tilings agree to rounding on
    the split-FP16 hologram of the 1920x1024x1024 workload."""
    import torch
    c = workload("cfg2_1920x1024_n1024")
    I_pair = _fwd(cg, h, c, "sep_fp16x3")
    h1 = cg.cgh_create(0)
    try:
        cg.cgh_set_gemm_tiles(h1, "single")
        I_one = _fwd(cg, h1, c, "sep_fp16x3")
    finally:
        cg.cgh_destroy(h1)
    assert np.max(np.abs(I_pair - I_one)) <= 1e-6 * np.max(np.abs(I_one))


@pytest.mark.parametrize("method", list(BOUND))
def test_cfg3_large_frame_sampled_rows(cg, h, method):
    """3840 x 2160 pixels, 16384 continuous points (Eq. 1, Section 1) on CTA
    pairs: both waves of pair tiles (and both K chunks in split FP16), the
    FP64 oracle on 64 evenly spaced rows plus 8 random ones."""
    c = workload("cfg3_3840x2160_n16384")
    I = _fwd(cg, h, c, method)
    rows, ref = workload_rows(c.name)
    assert np.all(np.isfinite(I))
    assert rel_rms(I[rows], ref) <= BOUND[method]


def test_tiling_argument_errors(cg, h):
    with pytest.raises(KeyError):
        cg.cgh_set_gemm_tiles(h, "bogus")
    assert cg.lib.cgh_set_gemm_tiles(h, 9) == cg.CGH_ERR_INVALID_ARG
    assert cg.lib.cgh_set_gemm_tiles(None, 0) == cg.CGH_ERR_INVALID_ARG



def test_gemm_plan(cg):
    """The tile widths the automatic plan takes: 112-column pairs at the
    paper's 1920 x 1024 (144 CTAs on 152 SMs), 144 at 1920 x 1080 (140), 256
    at 3840 x 2160 (two waves); one-CTA tiles for frames of at most 128 rows
    and when asked for."""
    hh = cg.cgh_create(0)
    try:
        assert cg.cgh_gemm_plan(hh, 1920, 1024) == ("pairs", 112)
        assert cg.cgh_gemm_plan(hh, 1920, 1080) == ("pairs", 144)
        assert cg.cgh_gemm_plan(hh, 3840, 2160) == ("pairs", 256)
        assert cg.cgh_gemm_plan(hh, 300, 100)[0] == "single"
        cg.cgh_set_gemm_tiles(hh, "single")
        assert cg.cgh_gemm_plan(hh, 1920, 1024)[0] == "single"
        with pytest.raises(cg.CGHError):
            cg.cgh_gemm_plan(hh, 0, 10)
    finally:
        cg.cgh_destroy(hh)
