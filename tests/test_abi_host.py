"""Host-side checks of the C ABI that need no GPU: the library loads, it
exports every function include/cgh.h declares, and the status strings and
tile registry answer without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(cgh_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def cg():
    from paper_1002_0916_gb300 import build
    build.build()
    import paper_1002_0916_gb300 as cg
    return cg


def test_header_declares_the_boundary():
    names = _declared("cgh.h")
    for required in ("cgh_create", "cgh_destroy", "cgh_forward",
                     "cgh_backward", "cgh_batch", "cgh_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(cg):
    lib = ctypes.CDLL(cg.library_path)
    for header in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if header.endswith(".h"):
            for name in _declared(header):
                assert hasattr(lib, name), f"{name} declared in {header} not exported"


def test_status_strings(cg):
    for code in range(6):
        s = cg.cgh_status_string(code)
        assert s.startswith("CGH_")
    assert "unknown" in cg.cgh_status_string(99)


def test_tile_registry(cg):
    tiles = cg.cgh_direct_tiles()
    assert len(tiles) >= 4
    for tx, ty, vx, vy, pt, np_, g, pk in tiles:
        assert tx % vx == 0 and ty % vy == 0 and pt % (4 * g) == 0
        assert g * (tx // vx) * (ty // vy) == 256 and 0 <= np_ <= vx * vy
        assert pk in range(9) and (pk == 0 or (vx % 2 == 0 and np_ % 2 == 0))
        if pk in (4, 5):   # one extra polynomial pair on every second or fourth point
            assert np_ + 2 <= vx * vy and (pt // g) % (2 if pk == 4 else 4) == 0
        if pk == 6:        # the row rotation form: rows of 4 pixels, no polynomial
            assert vx == 4 and np_ == 0 and (pt // g) % 4 == 0
        if pk in (7, 8):   # the two-axis rotation form: groups in fours along both axes
            assert vx % 4 == 0 and vy % 4 == 0 and np_ == 0 and (pt // g) % 4 == 0


def test_null_handle_is_rejected(cg):
    assert cg.lib.cgh_forward(None, None, None, None, 0, 1.0, 1.0, 1, 1, None,
                              0, None) == cg.CGH_ERR_INVALID_ARG
    assert cg.lib.cgh_last_device_status(None, None) == cg.CGH_ERR_INVALID_ARG
    assert cg.lib.cgh_destroy(None) == cg.CGH_OK
    assert cg.lib.cgh_create(None, 0) == cg.CGH_ERR_INVALID_ARG


def test_create_without_gpu_fails_cleanly(cg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = cg.lib.cgh_create(ctypes.byref(h), 0)
    assert st in (cg.CGH_ERR_CUDA, cg.CGH_ERR_INVALID_ARG)
    assert not h.value
