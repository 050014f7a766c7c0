"""The pipe-rate diagnostic behind the ALU rooflines (cgh_debug_pipe_rates):
hardware cosines and packed FP32 FMAs per SM clock, within the range the
architecture allows (the nominal figures are 16 and 128)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1002_0916_gb300 as cg
    return cg


def test_pipe_rates_in_range(cg):
    h = cg.cgh_create(0)
    try:
        r = cg.cgh_debug_pipe_rates(h)
        r2 = cg.cgh_debug_pipe_rates(h)
    finally:
        cg.cgh_destroy(h)
    assert 8.0 <= r["mufu_cos_per_clk_per_sm"] <= 40.0, r
    assert 64.0 <= r["fma_per_clk_per_sm"] <= 136.0, r
    for k in r:  # a property of the hardware: repeatable
        assert abs(r[k] - r2[k]) <= 0.05 * r[k], (r, r2)


def test_pipe_rates_rejects_null(cg):
    import ctypes
    h = cg.cgh_create(0)
    try:
        d = ctypes.c_double()
        assert cg.lib.cgh_debug_pipe_rates(h, None, ctypes.byref(d), None) == \
            cg.CGH_ERR_INVALID_ARG
        assert cg.lib.cgh_debug_pipe_rates(None, ctypes.byref(d), ctypes.byref(d),
                                           None) == cg.CGH_ERR_INVALID_ARG
    finally:
        cg.cgh_destroy(h)
