"""Edge cases of the point cloud for every forward method, against the FP64
oracle through the C ABI: the maximum point count (N = 2^24) and one past
it, degenerate clouds (coincident points, points exactly on pixels,
near-zero phase from a very distant point, zero and negative amplitudes,
points far outside the frame), points up to 3e6 pixels away with signed
amplitudes and a point near the records' Fresnel limit (forward and
adjoint).
Bounds: FP32 paths max |I - I_ref| <= 1e-4 sum|A_j|; split FP16 relative
RMS <= 1e-4 (or, where I_ref is near zero, max error <= 1e-4 sum|A_j|)."""
import numpy as np
import pytest

from gpu_util import max_abs, rel_rms, sum_abs_A, to_dev
from workloads import Cloud, make_cloud

pytestmark = pytest.mark.gpu

FP32 = ["direct", "naive", "recur", "sep_fp32"]
METHODS = FP32 + ["sep_fp16x3"]


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


def _fwd(cg, h, c, method):
    import torch
    pts, A, z = to_dev(c)
    I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    return I.cpu().numpy()


def _check(c, got, ref, method):
    tol = 1e-4 * sum_abs_A(c)
    assert np.all(np.isfinite(got))
    if method in FP32:
        assert max_abs(got, ref) <= tol, method
    else:
        assert rel_rms(got, ref) <= 1e-4 or max_abs(got, ref) <= tol, method


def _degenerate_cloud(Nx, Ny):
    rng = np.random.default_rng(2024)
    xy, A, z = [], [], []
    for _ in range(16):          # coincident points on a pixel
        xy.append((10.0, 7.0)); A.append(0.25); z.append(0.4)
    for k in range(8):           # points exactly on other pixels
        xy.append((float(3 * k), float(2 * k))); A.append(1.0); z.append(0.3 + 0.05 * k)
    xy.append((20.0, 20.0)); A.append(0.7); z.append(5.0e4)   # phase ~ 0: a plane wave
    xy.append((5.0, 5.0)); A.append(0.0); z.append(0.5)       # zero amplitude
    xy.append((30.5, 11.25)); A.append(-0.8); z.append(0.6)   # negative amplitude
    xy.append((-1.0e4, 3.0)); A.append(0.5); z.append(0.9)    # far outside the frame
    xy.append((Nx + 2.0e3, -7.5e3)); A.append(0.3); z.append(1.1)
    for _ in range(9):           # ordinary points
        xy.append((rng.uniform(0, Nx), rng.uniform(0, Ny))); A.append(rng.uniform())
        z.append(rng.uniform(0.2, 1.0))
    return Cloud(xy=np.array(xy, np.float32), A=np.array(A, np.float32),
                 z=np.array(z, np.float32), lam=532e-9, p=8e-6, Nx=Nx, Ny=Ny,
                 name="degenerate")


@pytest.mark.parametrize("method", METHODS)
def test_degenerate_cloud(cg, h, oracle_mod, method):
    c = _degenerate_cloud(131, 67)
    _check(c, _fwd(cg, h, c, method), oracle_mod.forward(c), method)


@pytest.mark.parametrize("method", ["direct", "sep_fp16x3"])
def test_all_points_coincident(cg, h, oracle_mod, method):
    """N copies of one point: the hologram is N times one Fresnel zone
    pattern, which the oracle's pins fix; any per-point indexing error shows."""
    N = 1000
    c = Cloud(xy=np.tile(np.array([[40.0, 25.0]], np.float32), (N, 1)),
              A=np.full(N, 0.5, np.float32), z=np.full(N, 0.35, np.float32),
              lam=633e-9, p=6.4e-6, Nx=97, Ny=53)
    _check(c, _fwd(cg, h, c, method), oracle_mod.forward(c), method)


@pytest.mark.parametrize("method", ["direct", "recur", "naive", "sep_fp16x3"])
def test_maximum_point_count(cg, h, oracle_mod, method):
    """N = 2^24 points (the largest N the ABI accepts) on a small frame:
    point padding, the split schedule and 64-bit table offsets at their
    limit."""
    N = 1 << 24
    c = make_cloud(24, N, 8, 8, integer=False, zlo=0.5, zhi=1.5, lam=633e-9,
                   p=6.4e-6)
    _check(c, _fwd(cg, h, c, method), oracle_mod.forward(c), method)


def test_point_count_above_the_limit_is_rejected(cg, h):
    import ctypes

    import torch
    N = (1 << 24) + 1
    pts = torch.zeros((N, 2), device="cuda")
    A = torch.zeros(N, device="cuda")
    z = torch.ones(N, device="cuda")
    out = torch.full((4, 4), 3.0, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = cg.lib.cgh_forward(h, p(pts), p(A), p(z), N, 532e-9, 8e-6, 4, 4, p(out), 0,
                            None)
    assert st == cg.CGH_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.all(out == 3.0)


@pytest.mark.parametrize("tiles", ["auto", "single"])
def test_coherent_sum_longer_than_one_k_chunk(cg, oracle_mod, tiles):
    """100,000 coincident points (every term of a pixel's sum has the same
    phase): the split-FP16 product runs in several K chunks whose partial
    products are added in FP32 with round to nearest, so the tensor cores'
    accumulation never runs over more than 16,384 values of k."""
    import torch
    N = 100000
    c = Cloud(xy=np.tile(np.array([[150.0, 60.0]], np.float32), (N, 1)),
              A=np.full(N, 0.5, np.float32), z=np.full(N, 0.8, np.float32),
              lam=633e-9, p=6.4e-6, Nx=300, Ny=200)
    hh = cg.cgh_create(0)
    try:
        cg.cgh_set_gemm_tiles(hh, tiles)
        n0 = cg.cgh_launch_count(hh)
        got = _fwd(cg, hh, c, "sep_fp16x3")
        # tables (building the records) and ceil(200,000 / 16,384) = 13
        # GEMM chunks
        assert cg.cgh_launch_count(hh) - n0 == 1 + 13
    finally:
        cg.cgh_destroy(hh)
    assert rel_rms(got, oracle_mod.forward(c)) <= 1e-4


def test_batch_with_a_problem_longer_than_one_k_chunk(cg, oracle_mod):
    """A separable batch mixing ordinary problems with one of 20,000 points
    (K = 40,000 > 16,384): the long one runs as chunked launches in the same
    graph; every hologram within the split-FP16 bound."""
    import torch
    clouds = [make_cloud(5, 300, 200, 150, integer=True, zlo=0.3, zhi=1.0,
                         lam=532e-9, p=8e-6),
              Cloud(xy=np.tile(np.array([[90.0, 40.0]], np.float32), (20000, 1)),
                    A=np.full(20000, 0.25, np.float32),
                    z=np.full(20000, 0.6, np.float32), lam=633e-9, p=8e-6,
                    Nx=180, Ny=130),
              make_cloud(6, 50, 77, 64, integer=False, zlo=0.3, zhi=1.0,
                         lam=473e-9, p=8e-6)]
    hh = cg.cgh_create(0)
    try:
        probs = []
        for cl in clouds:
            pts, A, z = to_dev(cl)
            probs.append(dict(points=pts, A=A, z=z, lam=cl.lam, p=cl.p, Nx=cl.Nx,
                              Ny=cl.Ny, out=torch.full((cl.Ny, cl.Nx), float("nan"),
                                                       device="cuda")))
        for _ in range(2):  # the first call builds the graph, the second replays it
            cg.cgh_batch(probs, method="sep_fp16x3", handle=hh)
            torch.cuda.synchronize()
            assert cg.cgh_last_device_status(hh) == cg.CGH_OK
            for cl, pr in zip(clouds, probs):
                assert rel_rms(pr["out"].cpu().numpy(), oracle_mod.forward(cl)) <= 1e-4
            for pr in probs:
                pr["out"].fill_(float("nan"))
    finally:
        cg.cgh_destroy(hh)


@pytest.mark.parametrize("method", ["recur", "sep_fp32", "sep_fp16x3", "sep_bf16"])
@pytest.mark.parametrize("Nx,Ny", [(32768, 3), (1, 4099), (5, 1), (1, 1)])
def test_extreme_frame_shapes(cg, h, oracle_mod, method, Nx, Ny):
    """The widest and the tallest frames the ABI accepts next to one-pixel
    ones, for the methods the direct tests do not cover."""
    c = make_cloud(11, 40, Nx, Ny, integer=False, zlo=0.5, zhi=1.5, lam=473e-9,
                   p=8e-6)
    got = _fwd(cg, h, c, method)
    ref = oracle_mod.forward(c)
    if method == "sep_bf16":
        assert rel_rms(got, ref) <= 1e-2 or max_abs(got, ref) <= 1e-2 * sum_abs_A(c)
    else:
        _check(c, got, ref, method)


def _bwd(cg, h, c, G, method):
    import torch
    pts, A, z = to_dev(c)
    Gd = torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).cuda()
    gp, gA, gz = cg.cgh_backward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, Gd,
                                 method=method, handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    return gp.cpu().numpy(), gA.cpu().numpy(), gz.cpu().numpy()


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("method", ["direct", "sep_fp16x3"])
def test_adjoint_many_points(cg, h, oracle_mod, method):
    """50,000 points on a small frame: many GEMM rows (2N) and many
    point-owned CTAs; oracle gradient on sampled points, bound 1e-3 per
    parameter group."""
    from workloads import grad_field
    c = make_cloud(50, 50000, 64, 48, integer=False, zlo=0.3, zhi=1.2, lam=532e-9,
                   p=8e-6)
    G = grad_field(51, c.Nx, c.Ny)
    gp, gA, gz = _bwd(cg, h, c, G, method)
    sel = np.sort(np.random.default_rng(52).choice(c.N, 24, replace=False))
    rp, rA, rz = oracle_mod.grad(c, G.astype(np.float64), pts=sel)
    for got, ref in ((gA[sel], rA), (gp[sel, 0], rp[:, 0]), (gp[sel, 1], rp[:, 1]),
                     (gz[sel], rz)):
        assert _rel(got, ref) <= 1e-3


@pytest.mark.parametrize("method", ["direct", "sep_fp16x3"])
def test_adjoint_degenerate_cloud_and_zero_gradient(cg, h, oracle_mod, method):
    """Coincident points, points on pixels, zero and negative amplitudes and
    points far outside the frame; and dL/dI = 0, whose gradient is exactly
    zero."""
    c = _degenerate_cloud(131, 67)
    from workloads import grad_field
    G = grad_field(53, c.Nx, c.Ny)
    gp, gA, gz = _bwd(cg, h, c, G, method)
    rp, rA, rz = oracle_mod.grad(c, G.astype(np.float64))
    for got, ref in ((gA, rA), (gp[:, 0], rp[:, 0]), (gp[:, 1], rp[:, 1]), (gz, rz)):
        assert _rel(got, ref) <= 1e-3
    zp, zA, zz = _bwd(cg, h, c, np.zeros_like(G), method)
    assert not np.any(zp) and not np.any(zA) and not np.any(zz)


def test_batch_of_degenerate_and_empty_problems(cg, oracle_mod):
    """A batch holding a degenerate cloud, an empty cloud and a one-pixel
    frame, by both methods."""
    import torch
    clouds = [_degenerate_cloud(131, 67),
              Cloud(xy=np.zeros((0, 2), np.float32), A=np.zeros(0, np.float32),
                    z=np.zeros(0, np.float32), lam=532e-9, p=8e-6, Nx=40, Ny=30),
              make_cloud(9, 17, 1, 1, integer=False, zlo=0.4, zhi=0.9, lam=633e-9,
                         p=8e-6)]
    hh = cg.cgh_create(0)
    try:
        for method in ("direct", "sep_fp16x3"):
            probs = []
            for cl in clouds:
                pts, A, z = to_dev(cl)
                probs.append(dict(points=pts, A=A, z=z, lam=cl.lam, p=cl.p, Nx=cl.Nx,
                                  Ny=cl.Ny, out=torch.full((cl.Ny, cl.Nx), float("nan"),
                                                           device="cuda")))
            cg.cgh_batch(probs, method=method, handle=hh)
            torch.cuda.synchronize()
            assert cg.cgh_last_device_status(hh) == cg.CGH_OK
            for cl, pr in zip(clouds, probs):
                got = pr["out"].cpu().numpy()
                if cl.N == 0:
                    assert np.count_nonzero(got) == 0
                    continue
                _check(cl, got, oracle_mod.forward(cl),
                       "direct" if method == "direct" else "sep_fp16x3")
    finally:
        cg.cgh_destroy(hh)


@pytest.mark.parametrize("method", ["sep_fp16", "sep_bf16"])
def test_coherent_sum_single_pass(cg, h, oracle_mod, method):
    """The single-pass forms accumulate up to 131,072 values of k per launch:
    100,000 coincident points (K = 200,000) take two launches and stay within
    their 1e-2 bound."""
    N = 100000
    c = Cloud(xy=np.tile(np.array([[150.0, 60.0]], np.float32), (N, 1)),
              A=np.full(N, 0.5, np.float32), z=np.full(N, 0.8, np.float32),
              lam=633e-9, p=6.4e-6, Nx=300, Ny=200)
    n0 = cg.cgh_launch_count(h)
    got = _fwd(cg, h, c, method)
    assert cg.cgh_launch_count(h) - n0 == 1 + 2  # tables, 2 chunks
    assert rel_rms(got, oracle_mod.forward(c)) <= 1e-2


def _far_and_signed_cloud(seed, Nx, Ny):
    """Random points with signed amplitudes, plus points up to 3e6 pixels
    outside the frame and one point close to the Fresnel limit of the
    records (Q = p^2 / (2 lambda z) = 0.9 turn per pixel^2: a fringe pattern
    aliased far past the Nyquist rate, still defined pixel by pixel)."""
    rng = np.random.default_rng(seed)
    lam, p = 532e-9, 8e-6
    n = 60
    xy = np.stack([rng.uniform(0, Nx, n), rng.uniform(0, Ny, n)], 1).tolist()
    A = rng.uniform(-1.0, 1.0, n).tolist()
    z = rng.uniform(0.2, 1.0, n).tolist()
    for (x, y) in [(1.0e5, 10.0), (-1.0e5, -2.5e4), (3.0e6, Ny / 2), (Nx / 2, -3.0e6)]:
        xy.append((x, y)); A.append(float(rng.uniform(-1, 1))); z.append(0.7)
    xy.append((Nx / 3, Ny / 4)); A.append(0.6); z.append(p * p / (2 * lam * 0.9))
    return Cloud(xy=np.array(xy, np.float32), A=np.array(A, np.float32),
                 z=np.array(z, np.float32), lam=lam, p=p, Nx=Nx, Ny=Ny,
                 name="far_and_signed")


@pytest.mark.parametrize("method", METHODS)
def test_far_points_signed_amplitudes_near_fresnel_limit(cg, h, oracle_mod, method):
    c = _far_and_signed_cloud(31, 96, 70)
    _check(c, _fwd(cg, h, c, method), oracle_mod.forward(c), method)


@pytest.mark.parametrize("method", ["direct", "sep_fp32", "sep_fp16x3"])
def test_adjoint_far_points_signed_amplitudes(cg, h, oracle_mod, method):
    """The adjoint of the same cloud: every parameter group within 1e-3 of
    the FP64 gradient, the far points' large offsets included."""
    import torch
    from workloads import grad_field
    c = _far_and_signed_cloud(32, 96, 70)
    G = grad_field(33, c.Nx, c.Ny)
    pts, A, z = to_dev(c)
    gp, gA, gz = cg.cgh_backward(pts, A, z, c.lam, c.p, c.Nx, c.Ny,
                                 torch.from_numpy(G).cuda(), method=method, handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    rp, rA, rz = oracle_mod.grad(c, G.astype(np.float64))
    for got, want in ((gA, rA), (gp[:, 0], rp[:, 0]), (gp[:, 1], rp[:, 1]), (gz, rz)):
        g64 = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g64 - want) <= 1e-3 * np.linalg.norm(want), method
