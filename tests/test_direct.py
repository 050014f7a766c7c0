"""Parity of the direct FP32 path (and the naive kernel) with the FP64 oracle,
through the C ABI.  Bound (FP32 paths): max |I - I_ref| <= 1e-4 sum |A_j|."""
import ctypes

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


def _fwd(cg, h, c, method="direct"):
    import torch
    pts, A, z = to_dev(c)
    I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, method=method, handle=h)
    torch.cuda.synchronize()
    return I.cpu().numpy()


@pytest.mark.parametrize("method", ["direct", "naive"])
def test_cfg1_full_frame(cg, h, oracle_mod, method):
    c = workload("cfg1_256x256_n64")
    I = _fwd(cg, h, c, method)
    err, _ = record(c.name, method, I, oracle_mod.forward(c), c)
    assert err <= TOL * sum_abs_A(c), err
    assert cg.cgh_last_device_status(h) == cg.CGH_OK


@pytest.mark.parametrize("integer", [True, False])
def test_every_tile_on_ragged_frame(cg, h, oracle_mod, integer):
    c = make_cloud(41, 257, 97, 61, integer=integer, zlo=0.05, zhi=0.5,
                   lam=532e-9, p=8e-6)
    c.xy[:, 0] = c.xy[:, 0] * 3 - 97   # points also outside the frame
    ref = oracle_mod.forward(c)
    try:
        for tile in cg.cgh_direct_tiles():
            cg.cgh_set_direct_tile(h, tile)
            err = max_abs(_fwd(cg, h, c), ref)
            assert err <= TOL * sum_abs_A(c), (tile, err)
    finally:
        cg.cgh_set_direct_tile(h, None)


@pytest.mark.parametrize("N", [1, 3, 15, 16, 17, 31, 32, 33, 63, 64, 65, 255, 256, 257])
def test_point_count_edges(cg, h, oracle_mod, N):
    c = make_cloud(100 + N, N, 70, 45, integer=True, zlo=0.2, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    err = max_abs(_fwd(cg, h, c), oracle_mod.forward(c))
    assert err <= TOL * sum_abs_A(c)


@pytest.mark.parametrize("Nx,Ny", [(32768, 3), (1, 4099), (5, 1), (1, 1)])
def test_extreme_frame_shapes(cg, h, oracle_mod, Nx, Ny):
    c = make_cloud(7, 40, Nx, Ny, integer=False, zlo=0.5, zhi=1.5,
                   lam=473e-9, p=8e-6)
    err = max_abs(_fwd(cg, h, c), oracle_mod.forward(c))
    assert err <= TOL * sum_abs_A(c)


def test_empty_cloud_gives_zeros(cg, h):
    import torch
    out = torch.full((13, 17), 7.0, device="cuda")
    e = torch.zeros(0, device="cuda")
    cg.cgh_forward(e.view(0, 2) if e.numel() else torch.zeros((0, 2), device="cuda"),
                   e, e, 532e-9, 8e-6, 17, 13, out=out, handle=h)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_cfg2_paper_frame_sampled_rows(cg, h, oracle_mod):
    """1920 x 1024 pixels, 1024 points (the paper's Table 1 frame), full GPU
    frame in the launch configuration the benchmark uses; oracle on rows."""
    c = workload("cfg2_1920x1024_n1024")
    I = _fwd(cg, h, c)
    rows = sample_rows(c.Ny, 40)
    err, _ = record(c.name, "direct", I[rows], oracle_mod.forward(c, rows=rows), c)
    assert err <= TOL * sum_abs_A(c), err
    assert np.all(np.isfinite(I))


def test_cfg3_large_frame_sampled_rows(cg, h):
    """3840 x 2160 pixels, 16384 continuous points (Eq. 1, Section 1): the
    full frame on the GPU in the launch configuration of a full-size call
    (every tile wave, the split tail), the FP64 oracle on 64 evenly spaced
    rows plus 8 random ones."""
    c = workload("cfg3_3840x2160_n16384")
    I = _fwd(cg, h, c)
    rows, ref = workload_rows(c.name)
    err, _ = record(c.name, "direct", I[rows], ref, c)
    assert err <= TOL * sum_abs_A(c), err
    assert np.all(np.isfinite(I))


def test_cfg5_continuous_sampled_rows(cg, h, oracle_mod):
    c = workload("cfg5_1920x1080_n4096")
    I = _fwd(cg, h, c)
    rows = sample_rows(c.Ny, 8, seed=9)
    err, _ = record(c.name, "direct", I[rows], oracle_mod.forward(c, rows=rows), c)
    assert err <= TOL * sum_abs_A(c), err


def test_bad_point_is_skipped_and_reported(cg, h, oracle_mod):
    c = make_cloud(3, 20, 40, 30, integer=True, zlo=0.2, zhi=0.4, lam=532e-9,
                   p=8e-6)
    bad = make_cloud(3, 20, 40, 30, integer=True, zlo=0.2, zhi=0.4, lam=532e-9,
                     p=8e-6)
    bad.z[5] = 0.0
    bad.xy[7, 0] = np.nan
    keep = np.array([j for j in range(20) if j not in (5, 7)])
    ref = oracle_mod.forward(xy=c.xy[keep], A=c.A[keep], z=c.z[keep], lam=c.lam,
                             p=c.p, Nx=c.Nx, Ny=c.Ny)
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    I = _fwd(cg, h, bad)
    assert max_abs(I, ref) <= TOL * sum_abs_A(c)
    assert cg.cgh_last_device_status(h) == cg.CGH_ERR_INVALID_ARG
    assert cg.cgh_last_device_status(h) == cg.CGH_OK  # read clears it


def test_argument_errors_leave_output_untouched(cg, h):
    import torch
    c = workload("cfg1_256x256_n64")
    pts, A, z = to_dev(c)
    out = torch.full((8, 8), 3.0, device="cuda")
    L = cg.lib
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    base = [h, p(pts), p(A), p(z), 64, 532e-9, 8e-6, 8, 8, p(out), 0, None]

    def call(**kw):
        a = list(base)
        names = ["h", "pts", "A", "z", "N", "lam", "p", "Nx", "Ny", "out", "m", "s"]
        for k, v in kw.items():
            a[names.index(k)] = v
        return L.cgh_forward(*a)

    assert call(N=-1) == cg.CGH_ERR_INVALID_ARG
    assert call(Nx=0) == cg.CGH_ERR_INVALID_ARG
    assert call(Ny=40000) == cg.CGH_ERR_INVALID_ARG
    assert call(lam=0.0) == cg.CGH_ERR_INVALID_ARG
    assert call(p=float("nan")) == cg.CGH_ERR_INVALID_ARG
    assert call(lam=float("inf")) == cg.CGH_ERR_INVALID_ARG
    assert call(out=None) == cg.CGH_ERR_INVALID_ARG
    assert call(A=None) == cg.CGH_ERR_INVALID_ARG
    assert call(m=17) == cg.CGH_ERR_INVALID_ARG
    assert call(out=ctypes.c_void_p(out.data_ptr() + 2)) == cg.CGH_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.all(out == 3.0)
    assert call() == cg.CGH_OK


def test_unaligned_output_and_odd_width(cg, h, oracle_mod):
    import torch
    c = make_cloud(8, 33, 37, 11, integer=True, zlo=0.2, zhi=0.4, lam=532e-9,
                   p=8e-6)
    pts, A, z = to_dev(c)
    buf = torch.zeros(37 * 11 + 1, device="cuda")
    out = buf[1:]  # 4-byte but not 16-byte aligned
    cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=out.view(11, 37), handle=h)
    torch.cuda.synchronize()
    assert max_abs(out.view(11, 37).cpu().numpy(), oracle_mod.forward(c)) \
        <= TOL * sum_abs_A(c)
    assert buf[0].item() == 0.0


def test_deterministic_and_host_entry_point(cg, h):
    import torch
    c = workload("cfg1_256x256_n64")
    I1 = _fwd(cg, h, c)
    I2 = _fwd(cg, h, c)
    assert np.array_equal(I1, I2)
    out = torch.empty((c.Ny, c.Nx), dtype=torch.float32).pin_memory()
    cg.cgh_forward_host(torch.from_numpy(c.xy), torch.from_numpy(c.A),
                        torch.from_numpy(c.z), c.lam, c.p, c.Nx, c.Ny, out=out,
                        handle=h)
    assert np.array_equal(out.numpy(), I1)


def test_launch_count_and_autotune(cg, h, oracle_mod):
    n0 = cg.cgh_launch_count(h)
    c = make_cloud(5, 300, 500, 300, integer=True, zlo=0.5, zhi=1.0,
                   lam=532e-9, p=8e-6)
    _fwd(cg, h, c)
    assert cg.cgh_launch_count(h) - n0 == 2   # tables (records built inside), direct
    tile = cg.cgh_tune(h, c.N, c.Nx, c.Ny)
    assert tile in cg.cgh_direct_tiles()
    err = max_abs(_fwd(cg, h, c), oracle_mod.forward(c))
    assert err <= TOL * sum_abs_A(c)


@pytest.mark.parametrize("N,Nx,Ny", [
    (4096, 32, 32),      # one tile, cut into one chunk per point stage
    (1000, 100, 70),     # a few tiles, all of them split
    (257, 1920, 1024),   # 1920 tiles: the last 96 split into uneven chunks
    (64, 33, 1),         # a single point stage: nothing to split
])
def test_split_schedule(cg, h, oracle_mod, N, Nx, Ny):
    """The tail-split schedule against the oracle and the one-CTA-per-tile
    grid: every tile shape, deterministic from call to call."""
    c = make_cloud(300 + N, N, Nx, Ny, integer=False, zlo=0.3, zhi=1.2,
                   lam=532e-9, p=8e-6)
    rows = None if Ny <= 128 else sample_rows(Ny, 6, seed=N)
    ref = oracle_mod.forward(c, rows=rows)
    tol = TOL * sum_abs_A(c)
    try:
        for tile in cg.cgh_direct_tiles()[:: 1 if Nx * Ny < 10**5 else 4]:
            cg.cgh_set_direct_tile(h, tile)
            cg.cgh_set_direct_schedule(h, "split")
            s1 = _fwd(cg, h, c)
            s2 = _fwd(cg, h, c)
            assert np.array_equal(s1, s2), tile
            cg.cgh_set_direct_schedule(h, "grid")
            g = _fwd(cg, h, c)
            assert cg.cgh_last_device_status(h) == cg.CGH_OK
            got = s1 if rows is None else s1[rows]
            assert max_abs(got, ref) <= tol, tile
            # same terms, different summation order only
            assert max_abs(s1, g) <= 1e-5 * sum_abs_A(c), tile
    finally:
        cg.cgh_set_direct_schedule(h, "auto")
        cg.cgh_set_direct_tile(h, None)


def test_schedule_argument_errors(cg, h):
    with pytest.raises(KeyError):
        cg.cgh_set_direct_schedule(h, "bogus")
    assert cg.lib.cgh_set_direct_schedule(h, 7) == cg.CGH_ERR_INVALID_ARG
    assert cg.lib.cgh_set_direct_schedule(None, 0) == cg.CGH_ERR_INVALID_ARG
    cg.cgh_set_direct_schedule(h, "auto")


def test_direct_tile_query(cg, h):
    """cgh_direct_tile_for reports the shape the handle's direct calls use: a
    compiled shape, the forced one while forced, and the tuned one after
    tuning that size."""
    tiles = cg.cgh_direct_tiles()
    auto = cg.cgh_direct_tile_for(h, 1024, 1920, 1024)
    assert auto in tiles
    forced = tiles[0] if tiles[0] != auto else tiles[1]
    try:
        cg.cgh_set_direct_tile(h, forced)
        assert cg.cgh_direct_tile_for(h, 1024, 1920, 1024) == forced
    finally:
        cg.cgh_set_direct_tile(h, None)
    assert cg.cgh_direct_tile_for(h, 1024, 1920, 1024) == auto
    tuned = cg.cgh_tune(h, 200, 96, 64)
    assert cg.cgh_direct_tile_for(h, 200, 96, 64) == tuned
    with pytest.raises(cg.CGHError):
        cg.cgh_direct_tile_for(h, 0, 8, 8)


def test_fused_records_match_prologue(cg, oracle_mod, monkeypatch):
    """The tables kernel that builds the point records itself gives the same
    hologram, bit for bit, as the prologue launch plus tables, and raises the
    same bad-point status."""
    import torch
    c = make_cloud(71, 500, 300, 170, integer=False, zlo=0.2, zhi=0.9,
                   lam=633e-9, p=6.4e-6)
    monkeypatch.setenv("CGH_DIRECT_FUSED_TABLES", "0")
    h0 = cg.cgh_create(0)
    monkeypatch.delenv("CGH_DIRECT_FUSED_TABLES")
    h1 = cg.cgh_create(0)
    try:
        n0 = cg.cgh_launch_count(h0)
        I0 = _fwd(cg, h0, c)
        assert cg.cgh_launch_count(h0) - n0 == 3   # prologue, tables, direct
        I1 = _fwd(cg, h1, c)
        assert np.array_equal(I0, I1)
        assert max_abs(I1, oracle_mod.forward(c)) <= TOL * sum_abs_A(c)
        bad = make_cloud(72, 40, 64, 64, integer=True, zlo=0.2, zhi=0.9,
                         lam=633e-9, p=6.4e-6)
        bad.z[7] = -1.0
        for hh in (h0, h1):
            _fwd(cg, hh, bad)
            assert cg.cgh_last_device_status(hh) == cg.CGH_ERR_INVALID_ARG
    finally:
        cg.cgh_destroy(h0)
        cg.cgh_destroy(h1)
