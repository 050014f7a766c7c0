"""Every forward method writes exactly its Ny x Nx output: NaN guard bands
before and after the output stay untouched, and every output pixel is
written (finite) and within the method's bound of the FP64 oracle.  And
every forward method can be captured into a caller's CUDA graph after one
uncaptured call of the same shape, and the replay follows new input values.
The same for the adjoint methods' three gradient arrays.
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


ADJ = ["direct", "sep_fp32", "sep_fp16x3"]


@pytest.mark.parametrize("method", ADJ)
def test_adjoint_guard_bands(cg, h, oracle_mod, method):
    """cgh_backward writes exactly N (x, y) pairs, N dL/dA and N dL/dz: NaN
    guard bands around each output stay untouched, every entry is finite and
    within 1e-3 of the FP64 gradient."""
    import ctypes

    import torch
    from workloads import grad_field
    c = make_cloud(91, 150, 130, 90, integer=False, zlo=0.3, zhi=0.9, lam=532e-9,
                   p=8e-6)
    G = torch.from_numpy(grad_field(92, c.Nx, c.Ny)).cuda()
    pts, A, z = to_dev(c)
    N = c.N
    bufs = [torch.full((n + 2 * GUARD,), float("nan"), device="cuda")
            for n in (2 * N, N, N)]
    views = [b[GUARD:GUARD + n] for b, n in zip(bufs, (2 * N, N, N))]
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = cg.lib.cgh_backward(h, p(pts), p(A), p(z), N, c.lam, c.p, c.Nx, c.Ny, p(G),
                             p(views[0]), p(views[1]), p(views[2]),
                             cg.METHODS[method],
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == cg.CGH_OK
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    for b in bufs:
        b = b.cpu().numpy()
        assert np.all(np.isnan(b[:GUARD])) and np.all(np.isnan(b[-GUARD:])), method
    got = [v.cpu().numpy().astype(np.float64) for v in views]
    assert all(np.all(np.isfinite(g)) for g in got)
    rp, rA, rz = oracle_mod.grad(c, G.cpu().numpy().astype(np.float64))
    gp = got[0].reshape(N, 2)
    for g, want in ((got[1], rA), (gp[:, 0], rp[:, 0]), (gp[:, 1], rp[:, 1]), (got[2], rz)):
        assert np.linalg.norm(g - want) <= 1e-3 * np.linalg.norm(want), method


@pytest.mark.parametrize("method", ADJ)
def test_adjoint_captured_in_caller_graph(cg, h, oracle_mod, method):
    """After one uncaptured call of the same shape, cgh_backward can be
    captured into a caller's CUDA graph; replays follow new inputs."""
    import torch
    from workloads import grad_field
    Nx, Ny, N = 200, 120, 100
    c1 = make_cloud(93, N, Nx, Ny, integer=False, zlo=0.3, zhi=0.9, lam=633e-9, p=6.4e-6)
    c2 = make_cloud(94, N, Nx, Ny, integer=False, zlo=0.3, zhi=0.9, lam=633e-9, p=6.4e-6)
    G1 = grad_field(95, Nx, Ny)
    G2 = grad_field(96, Nx, Ny)
    pts, A, z = to_dev(c1)
    G = torch.from_numpy(G1).cuda()
    gp = torch.empty((N, 2), device="cuda")
    gA = torch.empty(N, device="cuda")
    gz = torch.empty(N, device="cuda")
    import ctypes
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    s = torch.cuda.Stream()

    def call():
        st = cg.lib.cgh_backward(h, p(pts), p(A), p(z), N, c1.lam, c1.p, Nx, Ny, p(G),
                                 p(gp), p(gA), p(gz), cg.METHODS[method],
                                 ctypes.c_void_p(s.cuda_stream))
        assert st == cg.CGH_OK

    with torch.cuda.stream(s):
        call()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call()
    for c, Gn in ((c2, G2), (c1, G1)):
        p2, A2, z2 = to_dev(c)
        pts.copy_(p2)
        A.copy_(A2)
        z.copy_(z2)
        G.copy_(torch.from_numpy(Gn))
        gA.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        rp, rA, rz = oracle_mod.grad(c, Gn.astype(np.float64))
        for got, want in ((gA, rA), (gp[:, 0], rp[:, 0]), (gp[:, 1], rp[:, 1]), (gz, rz)):
            g64 = got.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(g64 - want) <= 1e-3 * np.linalg.norm(want), method
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
