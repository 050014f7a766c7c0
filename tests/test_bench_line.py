"""bench.py's JSON line on the GPU: one short run of the default workload
carries every key of the benchmark contract with consistent values (the
roofline of the dominant kernel, the CPU oracle baseline, the end-to-end
pipeline through the host-buffer API, clocks sampled in the timed region,
the launch count, and the split of the step into its two methods)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def line():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3",
                        "--warmup", "3"], capture_output=True, text=True, timeout=400,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_contract_keys(line):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] >= 3
    assert line["higher_is_better"] is True and line["data"] == "synthetic"
    assert "workload" in line["config"] and "l2" in line["config"]


def test_value_is_the_step_rate(line):
    pp = 2 * 1920 * 1024 * 1024          # two holograms per step
    assert line["value"] == pytest.approx(pp / (line["ms_per_step"] / 1e3), rel=1e-6)
    # the methods are timed one by one (each call bracketed by events, L2
    # flushed before each), the step as a whole: their sum is close to it
    ms = sum(m["ms"] for m in line["methods"].values())
    assert ms == pytest.approx(line["ms_per_step"], rel=0.15)
    assert line["vs_baseline"] == pytest.approx(line["value"] / (pp / 2 / 31e-3), rel=1e-6)


def test_roofline_and_baselines(line):
    r = line["roofline"]
    assert r["kernel"] == "direct" and r["bound"] == "alu"
    assert 0.3 < r["frac"] < 1.2
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-6)
    assert r["traffic"] is None or r["traffic"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    e = line["e2e"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in e
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] == 2 * 1920 * 1024 * 4
    assert 0.5 * line["value"] < e["value"] < 2.0 * line["value"]


def test_extra_workloads(line):
    """The large frame, the 64-hologram batch and the adjoint, measured in
    the same run: per method its ms per call and its main kernel's roofline
    fraction; the dominant kernel of each workload."""
    ex = line["extra"]
    assert set(ex) >= {"large", "batch64", "adjoint", "clocks"}
    assert set(ex["large"]["methods"]) >= {"direct", "sep_fp16x3", "sep_bf16"}
    assert set(ex["batch64"]["methods"]) == {"batch_direct", "batch_sep_fp16x3"}
    assert set(ex["adjoint"]["methods"]) >= {"direct_bwd", "sep_fp16x3_bwd"}
    for w in ("large", "batch64", "adjoint"):
        d = ex[w]["dominant_kernel"]
        assert d["ms_per_call"] > 0 and 0.2 < d["frac"] < 1.3, (w, d)
        for m, e in ex[w]["methods"].items():
            assert e["ms"] > 0 and e["pp_per_s"] > 0, (w, m)


def test_launches_and_clocks(line):
    # four of the library's kernels per step: direct tables, direct,
    # separable tables (both tables kernels build their point records), GEMM
    assert line["gpu_launches"] == 4 * line["steps"]
    c = line["clocks"]
    assert c["sm_mhz"] > 0 and c["sm_max_mhz"] >= c["sm_mhz"] * 0.5
    assert isinstance(c["reasons"], list)
