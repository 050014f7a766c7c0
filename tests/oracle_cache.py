"""Oracle values shared by the parity tests: each (workload, rows) or
(workload, points) sample is computed once per test session and reused by
every method and tiling that checks against it.  Test infrastructure; no
method arithmetic here (the values come from ``oracle``)."""
import functools

import numpy as np

from workloads import batch_problems, workload


def spread_rows(Ny, n_even=64, n_random=8, seed=2024):
    """n_even evenly spaced rows from the first to the last (the ragged
    tail included), plus n_random further distinct rows drawn at random."""
    even = np.unique(np.linspace(0, Ny - 1, min(n_even, Ny)).round().astype(np.int64))
    rest = np.setdiff1d(np.arange(Ny), even)
    rng = np.random.default_rng(seed)
    extra = rng.choice(rest, size=min(n_random, rest.size), replace=False)
    return np.sort(np.concatenate([even, extra])).astype(np.int32)


@functools.lru_cache(maxsize=None)
def _rows_ref(name, n_even, n_random, seed):
    import oracle
    c = workload(name)
    rows = spread_rows(c.Ny, n_even, n_random, seed)
    return rows, oracle.forward(c, rows=rows)


def workload_rows(name, n_even=64, n_random=8, seed=2024):
    """(rows, oracle rows) of a named workload: Eq. 1 in FP64 on
    spread_rows(Ny, n_even, n_random, seed)."""
    return _rows_ref(name, n_even, n_random, seed)


@functools.lru_cache(maxsize=None)
def _batch_refs(n_rows):
    import oracle
    out = []
    for i, c in enumerate(batch_problems(seed=0)):
        rows = spread_rows(c.Ny, n_even=n_rows - 1, n_random=1, seed=100 + i)
        out.append((rows, oracle.forward(c, rows=rows)))
    return out


def batch_rows(n_rows=4):
    """Per problem of the 64-hologram batch: (rows, oracle rows) on n_rows
    rows (n_rows - 1 evenly spaced from first to last, one at random)."""
    return _batch_refs(n_rows)
