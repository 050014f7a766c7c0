"""Failure handling without a GPU fault: a device wait that runs out reports
CGH_ERR_TIMEOUT through the status word and leaves the context usable; an
injected host allocation failure is reported as CGH_ERR_NOMEM with the
outputs untouched."""
import os

import numpy as np
import pytest

from gpu_util import max_abs, sum_abs_A, to_dev
from workloads import make_cloud

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1002_0916_gb300 as cg
    return cg


def test_stalled_wait_times_out_and_context_survives(cg, oracle_mod):
    import torch
    h = cg.cgh_create(0)
    try:
        s = torch.cuda.current_stream().cuda_stream
        # ~10 ms at GB300 clocks: a wait on an mbarrier that nothing sets
        assert cg.lib.cgh_debug_stalled_wait(h, 20_000_000, s) == cg.CGH_OK
        assert cg.cgh_last_device_status(h) == cg.CGH_ERR_TIMEOUT
        assert "bounded" in cg.cgh_last_error(h)
        assert cg.cgh_last_device_status(h) == cg.CGH_OK   # cleared by the read
        c = make_cloud(4, 50, 64, 48, integer=True, zlo=0.3, zhi=0.8,
                       lam=532e-9, p=8e-6)
        pts, A, z = to_dev(c)
        I = cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, handle=h)
        torch.cuda.synchronize()
        assert max_abs(I.cpu().numpy(), oracle_mod.forward(c)) <= 1e-4 * sum_abs_A(c)
    finally:
        cg.cgh_destroy(h)


def test_injected_allocation_failure(cg, monkeypatch):
    import torch
    monkeypatch.setenv("CGH_FAIL_ALLOC_AFTER", "0")
    h = cg.cgh_create(0)
    monkeypatch.delenv("CGH_FAIL_ALLOC_AFTER")
    try:
        c = make_cloud(4, 50, 64, 48, integer=True, zlo=0.3, zhi=0.8,
                       lam=532e-9, p=8e-6)
        pts, A, z = to_dev(c)
        out = torch.full((c.Ny, c.Nx), 2.0, device="cuda")
        with pytest.raises(cg.CGHError) as e:
            cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=out, handle=h)
        assert e.value.status == cg.CGH_ERR_NOMEM
        assert "injected" in str(e.value)
        torch.cuda.synchronize()
        assert torch.all(out == 2.0)
    finally:
        cg.cgh_destroy(h)
    h2 = cg.cgh_create(0)   # a handle made without the hook works
    try:
        cg.cgh_forward(pts, A, z, c.lam, c.p, c.Nx, c.Ny, out=out, handle=h2)
        torch.cuda.synchronize()
        assert not torch.all(out == 2.0)
    finally:
        cg.cgh_destroy(h2)
