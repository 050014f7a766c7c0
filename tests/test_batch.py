"""cgh_batch: many holograms of uneven size, N and wavelength in one
persistent, graph-replayed launch.  Each hologram must equal its own
single-call result (bit for bit with the same tile shape, direct method) and
match the FP64 oracle within the method's bound."""
import numpy as np
import pytest

from gpu_util import max_abs, record, rel_rms, sample_rows, sum_abs_A, to_dev
from oracle_cache import batch_rows
from workloads import batch_problems, make_cloud

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1002_0916_gb300 as cg
    return cg


@pytest.fixture
def h(cg):
    handle = cg.cgh_create(0)
    yield handle
    cg.cgh_destroy(handle)


def _problems(clouds):
    import torch
    probs = []
    for c in clouds:
        pts, A, z = to_dev(c)
        out = torch.full((c.Ny, c.Nx), float("nan"), device="cuda")
        probs.append(dict(points=pts, A=A, z=z, lam=c.lam, p=c.p, Nx=c.Nx,
                          Ny=c.Ny, out=out))
    return probs


def _small_clouds():
    lams = (633e-9, 532e-9, 473e-9)
    shapes = [(97, 61, 257), (128, 128, 64), (33, 200, 1), (300, 17, 129),
              (64, 64, 0), (250, 190, 500), (5, 3, 31)]
    return [make_cloud(500 + i, N, Nx, Ny, integer=(i % 2 == 0), zlo=0.3,
                       zhi=1.2, lam=lams[i % 3], p=8e-6)
            for i, (Nx, Ny, N) in enumerate(shapes)]


def _batch_tiles(cg):
    """The first compiled tile and every rotation tile: the batch builds its
    tables entry by entry (`direct_table_entry`), the single call with the
    tables kernel (angles per coordinate, rotation offsets stepped by the
    first difference), so equal bits also check that the two table builders
    agree."""
    tiles = cg.cgh_direct_tiles()
    return [tiles[0]] + [t for t in tiles if t[7] >= 6]


def test_direct_batch_equals_single_calls(cg, h, oracle_mod):
    import torch
    clouds = _small_clouds()
    probs = _problems(clouds)
    refs = [oracle_mod.forward(c) if c.N else None for c in clouds]
    # the batch runs whole tiles like the one-CTA-per-tile schedule: the same
    # summation order, so the same bits
    try:
        for tile in _batch_tiles(cg):
            cg.cgh_set_direct_tile(h, tile)
            cg.cgh_set_direct_schedule(h, "grid")
            cg.cgh_batch(probs, method="direct", handle=h)
            torch.cuda.synchronize()
            assert cg.cgh_last_device_status(h) == cg.CGH_OK
            for c, pr, ref in zip(clouds, probs, refs):
                got = pr["out"].cpu().numpy()
                pts, A, z = to_dev(c)
                single = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, handle=h)
                assert np.array_equal(got, single.cpu().numpy()), tile
                cg.cgh_set_direct_schedule(h, "split")
                split = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, handle=h)
                cg.cgh_set_direct_schedule(h, "grid")
                assert max_abs(got, split.cpu().numpy()) <= 1e-5 * max(sum_abs_A(c), 1.0)
                if c.N:
                    assert max_abs(got, ref) <= 1e-4 * sum_abs_A(c), tile
                else:
                    assert np.all(got == 0)
    finally:
        cg.cgh_set_direct_schedule(h, "auto")
        cg.cgh_set_direct_tile(h, None)


def test_graph_replay_rereads_inputs(cg, h, oracle_mod):
    import torch
    clouds = _small_clouds()[:4]
    probs = _problems(clouds)
    cg.cgh_batch(probs, handle=h)
    n0 = cg.cgh_launch_count(h)
    cg.cgh_batch(probs, handle=h)            # replay of the cached graph
    assert cg.cgh_launch_count(h) - n0 == 3
    first = [pr["out"].clone() for pr in probs]
    # new amplitudes in the same buffers: the replay must see them
    for pr in probs:
        pr["A"].mul_(0.5)
    cg.cgh_batch(probs, handle=h)
    torch.cuda.synchronize()
    for f, pr in zip(first, probs):
        assert torch.allclose(pr["out"], 0.5 * f, rtol=1e-5, atol=1e-5)


def test_batch_captured_by_caller(cg, h):
    import torch
    clouds = _small_clouds()[:3]
    probs = _problems(clouds)
    cg.cgh_batch(probs, handle=h)  # sizes the workspace outside the capture
    torch.cuda.synchronize()
    ref = [pr["out"].clone() for pr in probs]
    for pr in probs:
        pr["out"].fill_(float("nan"))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            cg.cgh_batch(probs, handle=h, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for r, pr in zip(ref, probs):
        assert torch.equal(r, pr["out"])


def test_batch_argument_errors(cg, h):
    clouds = _small_clouds()[:2]
    probs = _problems(clouds)
    probs[1]["lam"] = -1.0
    with pytest.raises(cg.CGHError) as e:
        cg.cgh_batch(probs, handle=h)
    assert e.value.status == cg.CGH_ERR_INVALID_ARG
    assert "problem 1" in str(e.value)
    import ctypes
    assert cg.lib.cgh_batch(h, None, 0, 0, None) == cg.CGH_ERR_INVALID_ARG


@pytest.mark.parametrize("method", ["direct", "sep_fp16x3"])
def test_batch64_uneven_workload(cg, h, oracle_mod, method):
    """64 holograms, Nx, Ny in {512..2048 step 128}, N in [100, 8192], three
    wavelengths: the batched workload at full size, one call (each problem
    an evaluation of Eq. 1, Section 1); every one of the 64 holograms is
    checked against the FP64 oracle on 4 rows (3 evenly spaced from the
    first to the last, 1 at random)."""
    import torch
    clouds = batch_problems(seed=0)
    probs = _problems(clouds)
    try:
        cg.cgh_batch(probs, method=method, handle=h)
    except cg.CGHError as e:
        if e.status == cg.CGH_ERR_UNSUPPORTED:
            pytest.skip("method not built")
        raise
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK
    refs = batch_rows(4)
    assert len(refs) == len(clouds) == 64
    for i, c in enumerate(clouds):
        got = probs[i]["out"].cpu().numpy()
        assert np.all(np.isfinite(got)), i
        rows, ref = refs[i]
        err, rel = record(f"batch64[{i}]", method, got[rows], ref, c)
        if method == "direct":
            assert err <= 1e-4 * sum_abs_A(c), i
        else:
            assert rel <= 1e-4, i


def test_tuned_separable_batch(cg, oracle_mod):
    """cgh_tune_batch on the split-FP16 batch times both GEMM item shapes
    and later calls of these sizes use the faster (cgh_batch_plan says so);
    every hologram within the split-FP16 bound of the FP64 oracle (Eq. 1)."""
    import torch
    hh = cg.cgh_create(0)
    try:
        clouds = _small_clouds()
        probs = _problems(clouds)
        assert cg.cgh_batch_plan(hh, probs, "sep_fp16x3")["tuned"] is False
        tiling = cg.cgh_tune_batch(hh, probs, "sep_fp16x3")
        assert tiling in ("single", "pairs")
        plan = cg.cgh_batch_plan(hh, probs, "sep_fp16x3")
        assert plan["tuned"] is True and plan["gemm_tiling"] == tiling
        for pr in probs:
            pr["out"].fill_(float("nan"))
        cg.cgh_batch(probs, method="sep_fp16x3", handle=hh)
        torch.cuda.synchronize()
        assert cg.cgh_last_device_status(hh) == cg.CGH_OK
        for c, pr in zip(clouds, probs):
            got = pr["out"].cpu().numpy()
            if c.N == 0:
                assert np.count_nonzero(got) == 0
            else:
                assert rel_rms(got, oracle_mod.forward(c)) <= 1e-4
        tile = cg.cgh_tune_batch(hh, probs, "direct")
        plan = cg.cgh_batch_plan(hh, probs, "direct")
        assert plan["tuned"] is True and plan["tile"] == tile
    finally:
        cg.cgh_destroy(hh)


def test_tune_batch(cg, h):
    import torch
    clouds = _small_clouds()
    probs = _problems(clouds)
    tile = cg.cgh_tune_batch(h, probs)
    assert tile in cg.cgh_direct_tiles()
    cg.cgh_batch(probs, handle=h)
    torch.cuda.synchronize()
    assert cg.cgh_last_device_status(h) == cg.CGH_OK


@pytest.mark.parametrize("tiles", ["single", "pairs"])
def test_sep_batch_on_both_gemm_tilings(cg, oracle_mod, tiles):
    """The separable batch on one-CTA items (128 x 128) and on CTA-pair items
    (256 x 128): every hologram of an uneven small batch within the split-FP16
    bound of the FP64 oracle, and the two tilings within rounding of each
    other; a second call of the same geometry replays the graph and gives
    the same bits."""
    import torch
    clouds = _small_clouds()
    out = {}
    for t in ("single", "pairs"):
        hh = cg.cgh_create(0)
        try:
            cg.cgh_set_gemm_tiles(hh, t)
            probs = _problems(clouds)
            cg.cgh_batch(probs, method="sep_fp16x3", handle=hh)
            torch.cuda.synchronize()
            first = [p["out"].cpu().numpy() for p in probs]
            cg.cgh_batch(probs, method="sep_fp16x3", handle=hh)
            torch.cuda.synchronize()
            assert cg.cgh_last_device_status(hh) == cg.CGH_OK
            out[t] = [p["out"].cpu().numpy() for p in probs]
            for a, b in zip(first, out[t]):
                assert np.array_equal(a, b)
        finally:
            cg.cgh_destroy(hh)
    for c, got in zip(clouds, out[tiles]):
        if c.N == 0:
            assert np.count_nonzero(got) == 0
            continue
        assert rel_rms(got, oracle_mod.forward(c)) <= 1e-4
    for a, b in zip(out["single"], out["pairs"]):
        assert np.max(np.abs(a - b)) <= 1e-6 * max(1.0, float(np.max(np.abs(b))))
