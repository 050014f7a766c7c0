"""Host-side arithmetic of bench.py: the ALU rooflines it reports are the
best point of the two pipe limits of each kernel's recipe (FMA pipe: 128
FP32 operations per SM per clock; MUFU: 16 per SM per clock), found here by
a brute-force scan over the share s of updates on the FMA-pipe polynomial."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _best(fma_ops, mufu_ops, f=128.0, m=16.0):
    """max over s of min(FMA-pipe limit, MUFU limit) in updates/clk/SM."""
    s = np.linspace(0.0, 1.0, 200001)
    fma = f / fma_ops(s)
    with np.errstate(divide="ignore"):
        mufu = np.where(mufu_ops(s) > 0, m / np.maximum(mufu_ops(s), 1e-300), np.inf)
    return float(np.max(np.minimum(fma, mufu)))


def test_direct_forward_recipe():
    # MUFU path 3 FP32 ops + 1 MUFU, polynomial path 9 FP32 ops
    best = _best(lambda s: 3 * (1 - s) + 9 * s, lambda s: 1 - s)
    assert abs(best - bench.MIXED_PP_PER_CLK_PER_SM) < 1e-3
    assert abs(best - 24.89) < 0.01


def test_direct_adjoint_recipe():
    # hardware path 5 FP32 ops + 2 MUFU, polynomial path 17 FP32 ops
    best = _best(lambda s: 5 * (1 - s) + 17 * s, lambda s: 2 * (1 - s))
    assert abs(best - bench.ADJ_MIXED_PP_PER_CLK_PER_SM) < 1e-3


def test_measured_rate_forms_match_the_recipes():
    """The closed forms bench.py uses with measured pipe rates f, m are the
    same scans with f and m in place of 128 and 16."""
    f, m = 107.0, 15.97
    fwd = _best(lambda s: 3 * (1 - s) + 9 * s, lambda s: 1 - s, f, m)
    adj = _best(lambda s: 5 * (1 - s) + 17 * s, lambda s: 2 * (1 - s), f, m)
    assert abs(fwd - (f + 6 * m) / 9) < 1e-3
    assert abs(adj - (f + 6 * m) / 17) < 1e-3


def test_fma_only_recipes():
    assert bench.SIMT_PP_PER_CLK_PER_SM == 128 / 2
    assert bench.BWD_SIMT_PP_PER_CLK_PER_SM == 128 / 4
    assert bench.RECUR_PP_PER_CLK_PER_SM == 16


def _rotation_ops(vx, vy, packed):
    """FP32 operations of one point on one thread's vx x vy block in the
    two-axis rotation form, counted operation by operation."""
    ops = 1 + 1 + 2                    # angle add, sincos argument scale, A cos, A sin
    for i in range(vy):
        if i > 0:
            ops += 4                   # the row's (Re w, Im w) by angle addition
        for k in range(vx):
            if packed:
                ops += 2               # every pixel: two lanes of two packed FMAs
            else:
                ops += 1 if k == 0 else 2
    return ops


def test_rotation_recipes():
    for tile in [(64, 32, 16, 4, 64, 0, 8, 7), (64, 32, 8, 4, 32, 0, 4, 7),
                 (32, 32, 4, 4, 64, 0, 4, 8), (64, 64, 16, 4, 32, 0, 4, 8)]:
        vx, vy, pk = tile[2], tile[3], tile[7]
        per_clk, _, measured, mufu = bench.alu_recipe("direct", tile)
        f = _rotation_ops(vx, vy, pk == 8) / (vx * vy)
        assert abs(per_clk - 128.0 / f) < 1e-9
        assert abs(measured(16.0, 128.0) - per_clk) < 1e-9
        assert abs(mufu - 2.0 / (vx * vy)) < 1e-12
    # the row rotation form: a sincos per 4 pixels bounds it at 32
    per_clk, _, measured, _ = bench.alu_recipe("batch", (32, 32, 4, 4, 64, 0, 4, 6))
    assert per_clk == 32.0 and measured(16.0, 128.0) == 32.0
    # without a tile (or with a cosine-per-pixel tile) the mixed recipe stays
    assert bench.alu_recipe("direct")[0] == bench.MIXED_PP_PER_CLK_PER_SM
    assert bench.alu_recipe("direct", (32, 32, 4, 4, 64, 4, 4, 5))[0] == \
        bench.MIXED_PP_PER_CLK_PER_SM


def test_rotation_roofline_reports_the_old_bound():
    tile = (64, 64, 8, 8, 32, 0, 4, 8)
    r = bench.kernel_roofline("direct", 2.013e9, 0.0, 0.194, 152, {}, tile=tile)
    old = 152 * bench.MIXED_PP_PER_CLK_PER_SM * bench.NOMINAL_MAX_MHZ * 1e6 / 1e9
    assert abs(r["vs_cosine_per_pixel_bound"] - r["achieved"] / old) < 1e-12
    assert r["frac"] < 1.0 < r["vs_cosine_per_pixel_bound"]
    assert "vs_cosine_per_pixel_bound" not in bench.kernel_roofline(
        "direct", 2.013e9, 0.0, 0.33, 152, {}, tile=(32, 32, 4, 4, 64, 4, 4, 5))
