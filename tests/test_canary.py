"""Every forward method writes exactly its Ny x Nx output: NaN guard bands
before and after the output stay untouched, and every output pixel is
written (finite) and within the method's bound of the FP64 oracle.  And
every forward method can be captured into a caller's CUDA graph after one
uncaptured call of the same shape, and the replay follows new input values.
(compute-sanitizer is not available; these stand in for its out-of-bounds
and uninitialised-memory checks.)"""
import numpy as np
import pytest

from gpu_util import max_abs, rel_rms, sum_abs_A, to_dev
from workloads import make_cloud

pytestmark = pytest.mark.gpu

FP32 = ["direct", "naive", "recur", "sep_fp32"]
BOUND_RMS = {"sep_fp16x3": 1e-4, "sep_fp16": 1e-2, "sep_bf16": 1e-2}
METHODS = FP32 + list(BOUND_RMS)
GUARD = 64  # floats (256 bytes: the output keeps 16-byte alignment)


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


def _check(c, got, ref, method):
    assert np.all(np.isfinite(got)), method
    if method in FP32:
        assert max_abs(got, ref) <= 1e-4 * sum_abs_A(c), method
    else:
        assert rel_rms(got, ref) <= BOUND_RMS[method], method


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("Nx,Ny,N", [(257, 131, 70), (33, 300, 9), (129, 129, 300)])
def test_guard_bands_and_full_coverage(cg, h, oracle_mod, method, Nx, Ny, N):
    import torch
    c = make_cloud(Nx * 7 + N, N, Nx, Ny, integer=(N % 2 == 0), zlo=0.1, zhi=0.8,
                   lam=532e-9, p=8e-6)
    pts, A, z = to_dev(c)
    buf = torch.full((Nx * Ny + 2 * GUARD,), float("nan"), device="cuda")
    out = buf[GUARD:GUARD + Nx * Ny].view(Ny, Nx)
    cg.cgh_forward(pts, A, z, c.lam, c.p, Nx, Ny, out=out, method=method, handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    b = buf.cpu().numpy()
    assert np.all(np.isnan(b[:GUARD])) and np.all(np.isnan(b[-GUARD:])), method
    _check(c, out.cpu().numpy(), oracle_mod.forward(c), method)


@pytest.mark.parametrize("method", METHODS)
def test_forward_captured_in_caller_graph(cg, h, oracle_mod, method):
    import torch
    Nx, Ny, N = 300, 200, 150
    c1 = make_cloud(31, N, Nx, Ny, integer=False, zlo=0.2, zhi=0.9, lam=633e-9,
                    p=6.4e-6)
    c2 = make_cloud(32, N, Nx, Ny, integer=False, zlo=0.2, zhi=0.9, lam=633e-9,
                    p=6.4e-6)
    pts, A, z = to_dev(c1)
    out = torch.full((Ny, Nx), float("nan"), device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        # one uncaptured call sizes the workspace and sets kernel attributes
        cg.cgh_forward(pts, A, z, c1.lam, c1.p, Nx, Ny, out=out, method=method,
                       handle=h)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        cg.cgh_forward(pts, A, z, c1.lam, c1.p, Nx, Ny, out=out, method=method,
                       handle=h)
    for c in (c2, c1):
        p2, A2, z2 = to_dev(c)
        pts.copy_(p2)
        A.copy_(A2)
        z.copy_(z2)
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        _check(c, out.cpu().numpy(), oracle_mod.forward(c), method)
    assert cg.cgh_last_device_status(h) == cg.CGH_OK


@pytest.mark.parametrize("method", METHODS)
def test_host_entry_point_buffer_kinds(cg, h, method):
    """cgh_forward_host with pinned (mapped, used in place) and pageable
    (staged) host buffers, in every combination of inputs and output: the
    same hologram as the device-buffer call, bit for bit."""
    import torch
    c = make_cloud(77, 120, 201, 97, integer=False, zlo=0.2, zhi=0.9, lam=532e-9,
                   p=8e-6)
    pts, A, z = to_dev(c)
    ref = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    host_in = [torch.from_numpy(np.ascontiguousarray(a)) for a in (c.xy, c.A, c.z)]
    for pin_in in (False, True):
        ins = [t.pin_memory() if pin_in else t.clone() for t in host_in]
        for pin_out in (False, True):
            out = torch.full((c.Ny, c.Nx), float("nan"))
            if pin_out:
                out = out.pin_memory()
            cg.cgh_forward_host(*ins, c.lam, c.p, c.Nx, c.Ny, out=out, method=method,
                                handle=h)
            assert np.array_equal(out.numpy(), ref), (method, pin_in, pin_out)
