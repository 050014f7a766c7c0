"""The tcgen05 GEMM on its own (cgh_debug_gemm), against an FP64 CPU
product of the same 16-bit operands.  Bound per element: FP32 accumulation
of K exact products, |D - ref| <= K 2^-23 (|A| |B|^T)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1002_0916_gb300 as cg
    return cg


@pytest.fixture(scope="module")
def h(cg):
    """A handle on the one-CTA tiling (the CTA-pair tiling has its own
    tests)."""
    handle = cg.cgh_create(0)
    cg.cgh_set_gemm_tiles(handle, "single")
    yield handle
    cg.cgh_destroy(handle)


@pytest.mark.parametrize("dtype", ["fp16", "bf16"])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 300, 128), (1, 1, 64),
                                   (129, 257, 192), (1024, 1920, 2048),
                                   (333, 129, 1024)])
def test_gemm_matches_fp64_product(cg, h, dtype, M, N, K):
    import torch
    tdt = {"fp16": torch.float16, "bf16": torch.bfloat16}[dtype]
    g = torch.Generator().manual_seed(M * 7 + N * 13 + K)
    A = torch.randn(M, K, generator=g).to(tdt)
    B = torch.randn(N, K, generator=g).to(tdt)
    D = cg.cgh_debug_gemm(A.cuda(), B.cuda(), handle=h)
    torch.cuda.synchronize()
    A64 = A.double().numpy()
    B64 = B.double().numpy()
    ref = A64 @ B64.T
    bound = K * 2.0 ** -23 * (np.abs(A64) @ np.abs(B64).T) + 1e-30
    err = np.abs(D.cpu().double().numpy() - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_gemm_structure_identity(cg, h):
    """A selects one column of B per row: catches transposed or shifted
    operand layouts exactly."""
    import torch
    M, N, K = 256, 192, 128
    A = torch.zeros(M, K, dtype=torch.float16)
    for m in range(M):
        A[m, (5 * m + 3) % K] = 1.0
    B = (torch.arange(N * K, dtype=torch.float32).reshape(N, K) % 2039).to(torch.float16)
    D = cg.cgh_debug_gemm(A.cuda(), B.cuda(), handle=h).cpu()
    ref = A.float() @ B.float().T
    assert torch.equal(D, ref)


def test_gemm_rejects_bad_shapes(cg):
    import torch
    A = torch.zeros(8, 48, dtype=torch.float16, device="cuda")
    with pytest.raises(cg.CGHError) as e:
        cg.cgh_debug_gemm(A, A)
    assert e.value.status == cg.CGH_ERR_INVALID_ARG
