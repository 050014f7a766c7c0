"""cgh_forward_host_async / cgh_host_wait: the pipelined host-buffer entry
point gives bit for bit the holograms of the synchronous one, also when
tensor-core calls (output copied on the handle's copy stream from one of two
device buffers used in turn) and tile-by-tile calls (output written in
place) are queued back to back, when the output buffer has to grow, and it
refuses buffers that are not page-locked and stream capture."""
import numpy as np
import pytest

from workloads import make_cloud

pytestmark = pytest.mark.gpu

METHODS = ["direct", "recur", "sep_fp32", "sep_bf16", "sep_fp16", "sep_fp16x3"]


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


def _host(c, pinned=True):
    import torch
    ts = [torch.from_numpy(np.ascontiguousarray(a)) for a in (c.xy, c.A, c.z)]
    return [t.pin_memory() if pinned else t.clone() for t in ts]


def _out(c, pinned=True):
    import torch
    o = torch.full((c.Ny, c.Nx), float("nan"))
    return o.pin_memory() if pinned else o


def _sync(cg, h, c, method):
    out = _out(c)
    cg.cgh_forward_host(*_host(c), c.lam, c.p, c.Nx, c.Ny, out=out, method=method,
                        handle=h)
    return out.numpy().copy()


@pytest.mark.parametrize("method", METHODS)
def test_async_matches_sync(cg, h, method):
    c = make_cloud(11, 300, 257, 131, integer=False, zlo=0.2, zhi=0.9, lam=532e-9,
                   p=8e-6)
    ref = _sync(cg, h, c, method)
    ins, out = _host(c), _out(c)
    cg.cgh_forward_host_async(*ins, c.lam, c.p, c.Nx, c.Ny, out=out, method=method,
                              handle=h)
    cg.cgh_host_wait(h)
    assert np.array_equal(out.numpy(), ref), method
    assert cg.cgh_last_device_status(h) == cg.CGH_OK


def test_queued_calls_of_both_kinds(cg, h):
    """Seven calls queued without a wait between them: four tensor-core ones
    (so each of the two device buffers is reused while the copy out of it
    may still be pending) between three direct ones, different clouds and
    frame sizes (the buffers grow), one wait at the end."""
    plan = [("sep_fp16x3", 100, 200, 150), ("direct", 60, 200, 150),
            ("sep_fp16x3", 300, 300, 200), ("sep_bf16", 80, 128, 64),
            ("direct", 90, 333, 77), ("sep_fp16x3", 500, 640, 480),
            ("direct", 40, 64, 64)]
    clouds = [make_cloud(200 + i, n, nx, ny, integer=(i % 2 == 0), zlo=0.2, zhi=0.9,
                         lam=633e-9, p=6.4e-6) for i, (_, n, nx, ny) in enumerate(plan)]
    refs = [_sync(cg, h, c, m) for (m, *_), c in zip(plan, clouds)]
    keep = []
    for (m, *_), c in zip(plan, clouds):
        ins, out = _host(c), _out(c)
        keep.append((ins, out))
        cg.cgh_forward_host_async(*ins, c.lam, c.p, c.Nx, c.Ny, out=out, method=m,
                                  handle=h)
    cg.cgh_host_wait(h)
    for (m, *_), (_, out), ref in zip(plan, keep, refs):
        assert np.array_equal(out.numpy(), ref), m


def test_steady_pipeline_reuses_buffers(cg, h):
    """The same two holograms over and over (the benchmark's pattern): every
    repeat is exact."""
    ca = make_cloud(301, 256, 320, 240, integer=True, zlo=0.3, zhi=0.9, lam=532e-9,
                    p=8e-6)
    cb = make_cloud(302, 256, 320, 240, integer=True, zlo=0.3, zhi=0.9, lam=532e-9,
                    p=8e-6)
    ra, rb = _sync(cg, h, ca, "sep_fp16x3"), _sync(cg, h, cb, "direct")
    ia, ib = _host(ca), _host(cb)
    for _ in range(5):
        oa, ob = _out(ca), _out(cb)
        cg.cgh_forward_host_async(*ia, ca.lam, ca.p, ca.Nx, ca.Ny, out=oa,
                                  method="sep_fp16x3", handle=h)
        cg.cgh_forward_host_async(*ib, cb.lam, cb.p, cb.Nx, cb.Ny, out=ob,
                                  method="direct", handle=h)
        cg.cgh_host_wait(h)
        assert np.array_equal(oa.numpy(), ra) and np.array_equal(ob.numpy(), rb)


@pytest.mark.parametrize("which", ["points", "out"])
def test_pageable_buffers_are_refused(cg, h, which):
    c = make_cloud(12, 50, 64, 64, integer=True, zlo=0.2, zhi=0.9, lam=532e-9, p=8e-6)
    ins, out = _host(c, pinned=(which != "points")), _out(c, pinned=(which != "out"))
    n0 = cg.cgh_launch_count(h)
    with pytest.raises(cg.CGHError) as ei:
        cg.cgh_forward_host_async(*ins, c.lam, c.p, c.Nx, c.Ny, out=out,
                                  method="sep_fp16x3", handle=h)
    assert ei.value.status == cg.CGH_ERR_INVALID_ARG
    assert cg.cgh_launch_count(h) == n0
    assert np.all(np.isnan(out.numpy()))


def test_refused_inside_capture(cg, h):
    import torch
    c = make_cloud(13, 50, 64, 64, integer=True, zlo=0.2, zhi=0.9, lam=532e-9, p=8e-6)
    ins, out = _host(c), _out(c)
    cg.cgh_forward_host_async(*ins, c.lam, c.p, c.Nx, c.Ny, out=out,
                              method="sep_fp16x3", handle=h)
    cg.cgh_host_wait(h)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            with pytest.raises(cg.CGHError) as ei:
                cg.cgh_forward_host_async(*ins, c.lam, c.p, c.Nx, c.Ny, out=out,
                                          method="sep_fp16x3", handle=h, stream=s)
        finally:
            g.capture_end()   # an empty graph: nothing was enqueued
    assert ei.value.status == cg.CGH_ERR_UNSUPPORTED


def test_tickets_pipeline_two_steps_in_flight(cg):
    """A display-loop pipeline: each step issues a split-FP16 and a direct
    hologram into its own pair of pinned buffers, then waits only for the
    previous step's ticket.  Every step's outputs are exact once its ticket
    has been waited for, although the next step is already running."""
    hh = cg.cgh_create(0)
    try:
        clouds = [make_cloud(400 + k, 200, 256, 160, integer=(k % 2 == 0), zlo=0.3,
                             zhi=0.9, lam=532e-9, p=8e-6) for k in range(6)]
        refs = [(_sync(cg, hh, c, "sep_fp16x3"), _sync(cg, hh, c, "direct")) for c in clouds]
        bufs = [(_out(clouds[0]), _out(clouds[0])) for _ in range(2)]
        ins = [_host(c) for c in clouds]
        assert cg.cgh_host_ticket(hh) == 0
        prev = None
        for k, c in enumerate(clouds):
            o = bufs[k % 2]
            cg.cgh_forward_host_async(*ins[k], c.lam, c.p, c.Nx, c.Ny, out=o[0],
                                      method="sep_fp16x3", handle=hh)
            cg.cgh_forward_host_async(*ins[k], c.lam, c.p, c.Nx, c.Ny, out=o[1],
                                      method="direct", handle=hh)
            t = cg.cgh_host_ticket(hh)
            assert t == 2 * (k + 1)
            if prev is not None:
                cg.cgh_host_wait_ticket(hh, prev)
                po = bufs[(k - 1) % 2]
                assert np.array_equal(po[0].numpy(), refs[k - 1][0])
                assert np.array_equal(po[1].numpy(), refs[k - 1][1])
            prev = t
        cg.cgh_host_wait_ticket(hh, prev)
        o = bufs[(len(clouds) - 1) % 2]
        assert np.array_equal(o[0].numpy(), refs[-1][0])
        assert np.array_equal(o[1].numpy(), refs[-1][1])
        cg.cgh_host_wait_ticket(hh, 3)          # long done: returns at once
        with pytest.raises(cg.CGHError) as ei:
            cg.cgh_host_wait_ticket(hh, prev + 1)
        assert ei.value.status == cg.CGH_ERR_INVALID_ARG
    finally:
        cg.cgh_destroy(hh)


def test_tickets_beyond_the_ring(cg):
    """More calls in flight than the handle remembers: a new call first
    waits for the one CGH_HOST_TICKETS before it, and every output is
    right."""
    hh = cg.cgh_create(0)
    try:
        c = make_cloud(450, 120, 128, 96, integer=True, zlo=0.3, zhi=0.9,
                       lam=633e-9, p=6.4e-6)
        ref = _sync(cg, hh, c, "sep_fp16x3")
        ins = _host(c)
        outs = [_out(c) for _ in range(40)]
        for o in outs:
            cg.cgh_forward_host_async(*ins, c.lam, c.p, c.Nx, c.Ny, out=o,
                                      method="sep_fp16x3", handle=hh)
        cg.cgh_host_wait_ticket(hh, cg.cgh_host_ticket(hh))
        for o in outs:
            assert np.array_equal(o.numpy(), ref)
    finally:
        cg.cgh_destroy(hh)


@pytest.mark.parametrize("method", ["direct", "sep_fp16x3"])
def test_async_empty_cloud_gives_zeros(cg, h, method):
    """N = 0 through the asynchronous call: the hologram is all zeros and the
    call takes a ticket like any other."""
    import torch
    from workloads import Cloud
    c = Cloud(xy=np.zeros((0, 2), np.float32), A=np.zeros(0, np.float32),
              z=np.zeros(0, np.float32), lam=532e-9, p=8e-6, Nx=70, Ny=40, name="empty")
    ins = [torch.zeros(0).pin_memory() for _ in range(3)]
    ins[0] = torch.zeros((0, 2)).pin_memory()
    out = _out(c)
    t0 = cg.cgh_host_ticket(h)
    cg.cgh_forward_host_async(*ins, c.lam, c.p, c.Nx, c.Ny, out=out, method=method,
                              handle=h)
    assert cg.cgh_host_ticket(h) == t0 + 1
    cg.cgh_host_wait_ticket(h, t0 + 1)
    assert np.all(out.numpy() == 0.0)
