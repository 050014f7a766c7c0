"""Host logic of the parity tests' row sampling (no GPU): the rows checked on
the large frames reach the first and last row (the ragged tail) and spread
over the whole frame, so that a fault in an interior tile, a later wave or a
later K chunk cannot slip between them."""
import numpy as np

from oracle_cache import spread_rows


def test_spread_rows_cover_the_frame():
    rows = spread_rows(2160)
    assert rows.dtype == np.int32
    assert len(rows) == 72 and len(np.unique(rows)) == 72
    assert rows[0] == 0 and rows[-1] == 2159
    assert np.all(np.diff(rows) > 0)
    # every stretch of 2160 / 63 rows holds at least one checked row
    assert np.max(np.diff(rows)) <= int(np.ceil(2159 / 63))
    # every 256-row band (one CTA-pair tile of the tensor-core GEMM)
    # holds several checked rows
    counts = np.bincount(rows // 256)
    assert counts.min() >= 4


def test_spread_rows_small_frames():
    assert list(spread_rows(1)) == [0]
    assert list(spread_rows(5)) == [0, 1, 2, 3, 4]
    r = spread_rows(70)
    assert len(r) == 70 and r[0] == 0 and r[-1] == 69


def test_spread_rows_deterministic():
    assert np.array_equal(spread_rows(1080, 16, 4, seed=3),
                          spread_rows(1080, 16, 4, seed=3))
