"""FP64 CPU oracle for the point-source Fresnel CGH (Eq. 1) and its adjoint.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_1002_0916_gb300``) and never imports it.

The arithmetic lives in ``cgh_oracle.c`` (plain C99 + OpenMP, FP64); this
module compiles it with gcc on first use and wraps it with ctypes.

Entry points (all return float64 numpy arrays):

* ``forward``            Eq. 1, FP64, phase reduced in turns; optional row
                         subset for large frames.
* ``forward_ld``         Eq. 1 in long double, unreduced (brute force; keep it
                         tiny).
* ``forward_recurrence`` Eq. 2 (Section 2.1) along rows, FP64 radians.
* ``grad``               adjoint of Eq. 1 for a given dL/dI field; optional
                         point subset.

Every function accepts either explicit arrays or any object with attributes
``xy, A, z, lam, p, Nx, Ny`` (e.g. ``workloads.Cloud``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgh_oracle.c")
_LIB = os.path.join(_HERE, "libcgh_oracle.so")
_lock = threading.Lock()
_lib = None

__all__ = ["build", "forward", "forward_ld", "forward_recurrence", "grad",
           "max_threads", "load", "use_library"]


def build(force: bool = False) -> str:
    """Compile cgh_oracle.c into libcgh_oracle.so (no fast-math, no FMA
    contraction, so x86 and aarch64 round the same way)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu99", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _bind(path):
    lib = ctypes.CDLL(path)
    f32p = ctypes.POINTER(ctypes.c_float)
    f64p = ctypes.POINTER(ctypes.c_double)
    i32p = ctypes.POINTER(ctypes.c_int)
    ci, cd = ctypes.c_int, ctypes.c_double
    lib.oracle_forward.argtypes = [f32p, f32p, f32p, ci, cd, cd, ci, ci, i32p,
                                   ci, f64p, ci]
    lib.oracle_forward_ld.argtypes = [f32p, f32p, f32p, ci, cd, cd, ci, ci, f64p]
    lib.oracle_forward_recurrence.argtypes = lib.oracle_forward.argtypes
    lib.oracle_grad.argtypes = [f32p, f32p, f32p, ci, cd, cd, ci, ci, f64p,
                                i32p, ci, f64p, f64p, f64p, ci]
    lib.oracle_max_threads.argtypes = [ci]
    for fn in (lib.oracle_forward, lib.oracle_forward_ld,
               lib.oracle_forward_recurrence, lib.oracle_grad,
               lib.oracle_max_threads):
        fn.restype = ci
    return lib


def load():
    """The oracle library, compiled on first use."""
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def use_library(path=None):
    """Point the wrappers at another build of cgh_oracle.c (``None``: the
    default one).  The mutation tests use this to check that the pins catch
    deliberately broken copies."""
    global _lib
    with _lock:
        _lib = _bind(path) if path is not None else None
    return load()


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _unpack(cloud, xy, A, z, lam, p, Nx, Ny):
    if cloud is not None:
        xy, A, z = cloud.xy, cloud.A, cloud.z
        lam, p, Nx, Ny = cloud.lam, cloud.p, cloud.Nx, cloud.Ny
    xy = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    A = np.ascontiguousarray(A, dtype=np.float32).reshape(-1)
    z = np.ascontiguousarray(z, dtype=np.float32).reshape(-1)
    if not (xy.shape[0] == A.shape[0] == z.shape[0]):
        raise ValueError("xy, A, z must describe the same number of points")
    return xy, A, z, float(lam), float(p), int(Nx), int(Ny)


def max_threads(nthreads: int = 0) -> int:
    """OpenMP threads the oracle uses (after optionally setting them)."""
    return int(load().oracle_max_threads(int(nthreads)))


def _rows_arg(rows, Ny):
    if rows is None:
        return None, Ny
    rows = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1)
    if rows.size and (rows.min() < 0 or rows.max() >= Ny):
        raise ValueError("row index out of range")
    return rows, int(rows.size)


def forward(cloud=None, *, xy=None, A=None, z=None, lam=None, p=None,
            Nx=None, Ny=None, rows=None, nthreads: int = 0) -> np.ndarray:
    """Eq. 1 in FP64.  Returns (Ny, Nx), or (len(rows), Nx) for a row subset."""
    xy, A, z, lam, p, Nx, Ny = _unpack(cloud, xy, A, z, lam, p, Nx, Ny)
    rows, R = _rows_arg(rows, Ny)
    out = np.empty((R, Nx), dtype=np.float64)
    rc = load().oracle_forward(_ptr(xy, ctypes.c_float), _ptr(A, ctypes.c_float),
                               _ptr(z, ctypes.c_float), A.shape[0], lam, p, Nx,
                               Ny, _ptr(rows, ctypes.c_int), R,
                               _ptr(out, ctypes.c_double), int(nthreads))
    if rc:
        raise ValueError(f"oracle_forward rejected its arguments ({rc})")
    return out


def forward_ld(cloud=None, *, xy=None, A=None, z=None, lam=None, p=None,
               Nx=None, Ny=None) -> np.ndarray:
    """Eq. 1 by long-double brute force (unreduced phase).  Tiny grids only."""
    xy, A, z, lam, p, Nx, Ny = _unpack(cloud, xy, A, z, lam, p, Nx, Ny)
    out = np.empty((Ny, Nx), dtype=np.float64)
    rc = load().oracle_forward_ld(_ptr(xy, ctypes.c_float), _ptr(A, ctypes.c_float),
                                  _ptr(z, ctypes.c_float), A.shape[0], lam, p,
                                  Nx, Ny, _ptr(out, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_forward_ld rejected its arguments ({rc})")
    return out


def forward_recurrence(cloud=None, *, xy=None, A=None, z=None, lam=None,
                       p=None, Nx=None, Ny=None, rows=None,
                       nthreads: int = 0) -> np.ndarray:
    """Eq. 2 recurrence along each row (the paper's CPU method), FP64."""
    xy, A, z, lam, p, Nx, Ny = _unpack(cloud, xy, A, z, lam, p, Nx, Ny)
    rows, R = _rows_arg(rows, Ny)
    out = np.empty((R, Nx), dtype=np.float64)
    rc = load().oracle_forward_recurrence(
        _ptr(xy, ctypes.c_float), _ptr(A, ctypes.c_float), _ptr(z, ctypes.c_float),
        A.shape[0], lam, p, Nx, Ny, _ptr(rows, ctypes.c_int), R,
        _ptr(out, ctypes.c_double), int(nthreads))
    if rc:
        raise ValueError(f"oracle_forward_recurrence rejected its arguments ({rc})")
    return out


def grad(cloud=None, G=None, *, xy=None, A=None, z=None, lam=None, p=None,
         Nx=None, Ny=None, pts=None, nthreads: int = 0):
    """Adjoint of Eq. 1: sums over pixels of G * dI/d(param).

    Returns (gxy (M, 2), gA (M,), gz (M,)) for all points or the subset
    ``pts``.
    """
    xy, A, z, lam, p, Nx, Ny = _unpack(cloud, xy, A, z, lam, p, Nx, Ny)
    G = np.ascontiguousarray(G, dtype=np.float64)
    if G.shape != (Ny, Nx):
        raise ValueError("G must have shape (Ny, Nx)")
    if pts is not None:
        pts = np.ascontiguousarray(pts, dtype=np.int32).reshape(-1)
        if pts.size and (pts.min() < 0 or pts.max() >= A.shape[0]):
            raise ValueError("point index out of range")
        M = int(pts.size)
    else:
        M = A.shape[0]
    gxy = np.empty((M, 2), dtype=np.float64)
    gA = np.empty(M, dtype=np.float64)
    gz = np.empty(M, dtype=np.float64)
    rc = load().oracle_grad(_ptr(xy, ctypes.c_float), _ptr(A, ctypes.c_float),
                            _ptr(z, ctypes.c_float), A.shape[0], lam, p, Nx, Ny,
                            _ptr(G, ctypes.c_double), _ptr(pts, ctypes.c_int),
                            M, _ptr(gxy, ctypes.c_double), _ptr(gA, ctypes.c_double),
                            _ptr(gz, ctypes.c_double), int(nthreads))
    if rc:
        raise ValueError(f"oracle_grad rejected its arguments ({rc})")
    return gxy, gA, gz
