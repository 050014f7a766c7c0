"""Shared helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np


def to_dev(cloud, device="cuda"):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(cloud.xy)).to(device),
            torch.from_numpy(np.ascontiguousarray(cloud.A)).to(device),
            torch.from_numpy(np.ascontiguousarray(cloud.z)).to(device))


def sum_abs_A(cloud):
    return float(np.abs(cloud.A.astype(np.float64)).sum())


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))))


def rel_rms(a, ref):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def sample_rows(Ny, k, seed=1234):
    """k distinct rows, always including the first and last (ragged tail)."""
    rng = np.random.default_rng(seed)
    inner = rng.choice(np.arange(1, Ny - 1), size=max(0, min(k, Ny) - 2),
                       replace=False) if Ny > 2 else np.array([], int)
    rows = sorted(set([0, Ny - 1] + [int(r) for r in inner]))
    return np.array(rows, dtype=np.int32)


def record(workload_name, method, got, ref, cloud):
    """max |got - ref| and relative RMS of a parity check; when the
    environment variable CGH_ACCURACY_LOG names a file, also appends one JSON
    line (workload, method, rows checked, max error / sum |A_j|, relative
    RMS) to it, from which the accuracy table of the design notes is made."""
    import json
    import os
    err, rel = max_abs(got, ref), rel_rms(got, ref)
    path = os.environ.get("CGH_ACCURACY_LOG")
    if path:
        rows = int(np.asarray(ref).shape[0]) if np.asarray(ref).ndim == 2 else 1
        with open(path, "a") as fh:
            fh.write(json.dumps({"workload": workload_name, "method": method,
                                 "rows": rows, "max_err_over_sumA": err / sum_abs_A(cloud),
                                 "rel_rms": rel}) + "\n")
    return err, rel
