"""Python binding of libcgh: point-source Fresnel CGH on one sm_103a GPU.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libcgh.so`` (built in-tree by ``paper_1002_0916_gb300.build``).
There is no CPU fallback: importing this package on a machine without the
built library, or calling it without a CUDA device, raises.

The functions mirror the C ABI in ``include/cgh.h`` and keep its names:
``cgh_create``, ``cgh_destroy``, ``cgh_forward``, ``cgh_forward_host``,
``cgh_forward_host_async``, ``cgh_host_wait``, ``cgh_backward``, ``cgh_batch``, ``cgh_tune``, ``cgh_last_device_status``,
``cgh_launch_count``, ``cgh_status_string``, plus the autograd wrapper
``CGHFunction``.  Tensors are PyTorch CUDA tensors (float32, contiguous);
PyTorch supplies device memory and the current stream, nothing else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

__all__ = [
    "CGH_OK", "CGH_ERR_INVALID_ARG", "CGH_ERR_CUDA", "CGH_ERR_NOMEM",
    "CGH_ERR_UNSUPPORTED", "CGH_ERR_TIMEOUT", "CGH_DIRECT_FP32", "CGH_SEP_BF16",
    "CGH_SEP_FP16", "CGH_SEP_FP16X3", "CGH_NAIVE_FP32", "CGH_RECUR_FP32",
    "CGH_SEP_FP32", "METHODS",
    "CGHError",
    "lib", "library_path", "cgh_create", "cgh_destroy", "cgh_forward",
    "cgh_forward_host", "cgh_backward", "cgh_batch", "cgh_tune",
    "cgh_set_direct_tile", "cgh_direct_tiles", "cgh_last_device_status",
    "cgh_launch_count", "cgh_status_string", "cgh_last_error",
    "cgh_debug_gemm", "CGHFunction", "default_handle", "KERNELS",
    "cgh_kernel_timing", "cgh_kernel_time", "cgh_tune_batch",
    "cgh_kernel_timing_mask", "cgh_set_gemm_tiles", "GEMM_TILES",
    "cgh_debug_pipe_rates", "cgh_direct_tile_for", "cgh_forward_host_async",
    "cgh_host_wait", "cgh_gemm_plan", "cgh_host_ticket", "cgh_host_wait_ticket",
    "cgh_gemm_plan_for", "cgh_batch_plan", "cgh_set_gemm_plan", "cgh_forward_rows",
]

CGH_OK, CGH_ERR_INVALID_ARG, CGH_ERR_CUDA = 0, 1, 2
CGH_ERR_NOMEM, CGH_ERR_UNSUPPORTED, CGH_ERR_TIMEOUT = 3, 4, 5
CGH_DIRECT_FP32, CGH_SEP_BF16, CGH_SEP_FP16 = 0, 1, 2
CGH_SEP_FP16X3, CGH_NAIVE_FP32, CGH_RECUR_FP32, CGH_SEP_FP32 = 3, 4, 5, 6
METHODS = {"direct": CGH_DIRECT_FP32, "sep_bf16": CGH_SEP_BF16,
           "sep_fp16": CGH_SEP_FP16, "sep_fp16x3": CGH_SEP_FP16X3,
           "naive": CGH_NAIVE_FP32, "recur": CGH_RECUR_FP32,
           "sep_fp32": CGH_SEP_FP32}

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "_lib", "libcgh.so")


class CGHError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


class _Tile(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("vec_x", ctypes.c_int), ("vec_y", ctypes.c_int),
                ("points_per_stage", ctypes.c_int), ("poly_pixels", ctypes.c_int),
                ("point_groups", ctypes.c_int), ("packed", ctypes.c_int)]


class _Problem(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("A", ctypes.c_void_p),
                ("z", ctypes.c_void_p), ("N", ctypes.c_int),
                ("lam", ctypes.c_double), ("p", ctypes.c_double),
                ("Nx", ctypes.c_int), ("Ny", ctypes.c_int),
                ("out", ctypes.c_void_p)]


def _load():
    if not os.path.exists(library_path):
        raise ImportError(
            f"libcgh.so is not built ({library_path} missing); run "
            "`python -m paper_1002_0916_gb300.build` or __graft_entry__.build()")
    L = ctypes.CDLL(library_path)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    fp = ctypes.c_void_p
    L.cgh_create.argtypes = [ctypes.POINTER(vp), ci]
    L.cgh_destroy.argtypes = [vp]
    L.cgh_forward.argtypes = [vp, fp, fp, fp, ci, cd, cd, ci, ci, fp, ci, vp]
    L.cgh_forward_host.argtypes = L.cgh_forward.argtypes
    L.cgh_forward_host_async.argtypes = L.cgh_forward.argtypes
    L.cgh_forward_rows.argtypes = [vp, fp, fp, fp, ci, cd, cd, ci, ci, ci, fp, ci, vp]
    L.cgh_forward_rows.restype = ci
    L.cgh_host_wait.argtypes = [vp, vp]
    L.cgh_host_ticket.argtypes = [vp]
    L.cgh_host_ticket.restype = ctypes.c_uint64
    L.cgh_host_wait_ticket.argtypes = [vp, ctypes.c_uint64]
    L.cgh_host_wait_ticket.restype = ci
    L.cgh_backward.argtypes = [vp, fp, fp, fp, ci, cd, cd, ci, ci, fp, fp, fp,
                               fp, ci, vp]
    L.cgh_batch.argtypes = [vp, ctypes.POINTER(_Problem), ci, ci, vp]
    L.cgh_direct_tile_count.argtypes = []
    L.cgh_direct_tile_get.argtypes = [ci, ctypes.POINTER(_Tile)]
    L.cgh_set_direct_tile.argtypes = [vp, ctypes.POINTER(_Tile)]
    L.cgh_set_direct_schedule.argtypes = [vp, ci]
    L.cgh_direct_tile_for.argtypes = [vp, ci, ci, ci, ctypes.POINTER(_Tile)]
    L.cgh_direct_tile_for.restype = ci
    L.cgh_set_gemm_tiles.argtypes = [vp, ci]
    L.cgh_set_gemm_tiles.restype = ci
    L.cgh_gemm_plan.argtypes = [vp, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    L.cgh_gemm_plan_for.argtypes = [vp, ci, ci, ci, ci, ctypes.POINTER(ci),
                                    ctypes.POINTER(ci), ctypes.POINTER(ci)]
    L.cgh_gemm_plan_for.restype = ci
    L.cgh_set_gemm_plan.argtypes = [vp, ci, ci]
    L.cgh_set_gemm_plan.restype = ci
    L.cgh_batch_plan.argtypes = [vp, ctypes.POINTER(_Problem), ci, ci,
                                 ctypes.POINTER(_Tile), ctypes.POINTER(ci),
                                 ctypes.POINTER(ci)]
    L.cgh_batch_plan.restype = ci
    L.cgh_gemm_plan.restype = ci
    L.cgh_debug_pipe_rates.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), vp]
    L.cgh_debug_pipe_rates.restype = ci
    L.cgh_tune.argtypes = [vp, ci, ci, ci, ci, vp, ctypes.POINTER(_Tile)]
    L.cgh_tune_batch.argtypes = [vp, ctypes.POINTER(_Problem), ci, ci, vp,
                                 ctypes.POINTER(_Tile)]
    L.cgh_tune_batch.restype = ci
    L.cgh_last_device_status.argtypes = [vp, vp]
    L.cgh_launch_count.argtypes = [vp]
    L.cgh_launch_count.restype = ctypes.c_uint64
    L.cgh_status_string.argtypes = [ci]
    L.cgh_status_string.restype = ctypes.c_char_p
    L.cgh_last_error.argtypes = [vp]
    L.cgh_last_error.restype = ctypes.c_char_p
    L.cgh_debug_gemm.argtypes = [vp, fp, fp, fp, ci, ci, ci, ci, vp]
    L.cgh_debug_stalled_wait.argtypes = [vp, ctypes.c_longlong, vp]
    L.cgh_debug_stalled_wait.restype = ci
    L.cgh_forward_noalloc.argtypes = [fp, fp, fp, ci, cd, cd, ci, ci, fp, vp]
    L.cgh_forward_noalloc.restype = ci
    L.cgh_kernel_timing.argtypes = [vp, ci]
    L.cgh_kernel_timing_mask.argtypes = [vp, ctypes.c_uint32]
    L.cgh_kernel_timing_mask.restype = ci
    L.cgh_kernel_time.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_uint64)]
    for name in ("cgh_create", "cgh_destroy", "cgh_forward", "cgh_forward_host",
                 "cgh_forward_host_async", "cgh_host_wait", "cgh_backward", "cgh_batch", "cgh_direct_tile_get",
                 "cgh_set_direct_tile", "cgh_tune", "cgh_last_device_status",
                 "cgh_debug_gemm", "cgh_kernel_timing", "cgh_kernel_time"):
        getattr(L, name).restype = ci
    L.cgh_direct_tile_count.restype = ci
    return L


_lib = None


def _L():
    """The loaded libcgh.so (loaded on first use; raises if it is not built)."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def __getattr__(name):
    if name == "lib":
        return _L()
    raise AttributeError(name)


def cgh_status_string(status: int) -> str:
    return _L().cgh_status_string(int(status)).decode()


def cgh_last_error(h) -> str:
    return _L().cgh_last_error(h).decode()


def _check(h, status: int, what: str):
    if status != CGH_OK:
        detail = cgh_last_error(h) if h else ""
        raise CGHError(status, f"{what}: {cgh_status_string(status)}"
                               + (f" ({detail})" if detail else ""))


def _method(m) -> int:
    if isinstance(m, str):
        if m not in METHODS:
            raise ValueError(f"unknown method {m!r}; one of {sorted(METHODS)}")
        return METHODS[m]
    return int(m)


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev_f32(t, name: str, numel: Optional[int] = None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float32")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return t.data_ptr() if t.numel() else None


# ------------------------------------------------------------- handles
def cgh_create(device: int = 0):
    h = ctypes.c_void_p()
    st = _L().cgh_create(ctypes.byref(h), int(device))
    _check(None, st, "cgh_create")
    return h


def cgh_destroy(h) -> None:
    _L().cgh_destroy(h)


_handles = {}


def default_handle(device: Optional[int] = None):
    """One lazily created handle per device for the convenience wrappers."""
    torch = _torch()
    if device is None:
        device = torch.cuda.current_device()
    if device not in _handles:
        _handles[device] = cgh_create(device)
    return _handles[device]


# ------------------------------------------------------------- forward
def cgh_forward(points, A, z, lam: float, p: float, Nx: int, Ny: int, *,
                out=None, method="direct", handle=None, stream=None):
    """Eq. 1 on the GPU.  points (N, 2), A (N,), z (N,) float32 CUDA tensors;
    returns (or fills) out (Ny, Nx) float32."""
    torch = _torch()
    N = int(A.numel())
    if out is None:
        out = torch.empty((Ny, Nx), dtype=torch.float32, device=A.device)
    h = handle if handle is not None else default_handle(A.device.index)
    st = _L().cgh_forward(h, _dev_f32(points, "points", 2 * N), _dev_f32(A, "A", N),
                         _dev_f32(z, "z", N), N, float(lam), float(p), int(Nx),
                         int(Ny), _dev_f32(out, "out", Nx * Ny), _method(method),
                         _stream_ptr(stream))
    _check(h, st, "cgh_forward")
    return out


def cgh_forward_rows(points, A, z, lam: float, p: float, Nx: int, y0: int, rows: int,
                     *, out=None, method="direct", handle=None, stream=None):
    """Rows y0 .. y0 + rows - 1 of the hologram of Eq. 1 (a slab of a row
    split over GPUs); returns (or fills) out (rows, Nx) float32."""
    torch = _torch()
    N = int(A.numel())
    if out is None:
        out = torch.empty((rows, Nx), dtype=torch.float32, device=A.device)
    h = handle if handle is not None else default_handle(A.device.index)
    st = _L().cgh_forward_rows(h, _dev_f32(points, "points", 2 * N), _dev_f32(A, "A", N),
                              _dev_f32(z, "z", N), N, float(lam), float(p), int(Nx),
                              int(y0), int(rows), _dev_f32(out, "out", Nx * rows),
                              _method(method), _stream_ptr(stream))
    _check(h, st, "cgh_forward_rows")
    return out


def _host_ptr(a, name, n):
    import numpy as np
    if hasattr(a, "data_ptr"):
        if a.is_cuda or str(a.dtype) != "torch.float32" or not a.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32 host tensor")
        if a.numel() != n:
            raise ValueError(f"{name} must have {n} elements")
        return a.data_ptr() if n else None
    a = np.asarray(a)
    if a.dtype != np.float32 or not a.flags.c_contiguous or a.size != n:
        raise TypeError(f"{name} must be contiguous float32 with {n} elements")
    return a.ctypes.data if n else None


def _forward_host(entry, points, A, z, lam, p, Nx, Ny, out, method, handle, stream):
    import numpy as np
    N = int(A.numel() if hasattr(A, "numel") else np.asarray(A).size)
    st = getattr(_L(), entry)(handle, _host_ptr(points, "points", 2 * N),
                              _host_ptr(A, "A", N), _host_ptr(z, "z", N), N,
                              float(lam), float(p), int(Nx), int(Ny),
                              _host_ptr(out, "out", Nx * Ny), _method(method),
                              _stream_ptr(stream))
    _check(handle, st, entry)
    return out


def cgh_forward_host(points, A, z, lam: float, p: float, Nx: int, Ny: int, *,
                     out, method="direct", handle, stream=None):
    """cgh_forward from host buffers (numpy arrays or CPU tensors, float32,
    contiguous; pinned memory is fastest).  Synchronises the stream."""
    return _forward_host("cgh_forward_host", points, A, z, lam, p, Nx, Ny, out,
                         method, handle, stream)


def cgh_forward_host_async(points, A, z, lam: float, p: float, Nx: int, Ny: int,
                           *, out, method="direct", handle, stream=None):
    """cgh_forward_host without the synchronisation: every buffer must be a
    pinned CPU tensor (or page-locked array); ``out`` is complete after
    ``cgh_host_wait(handle, stream)``.  Keep the inputs unchanged until then."""
    return _forward_host("cgh_forward_host_async", points, A, z, lam, p, Nx, Ny,
                         out, method, handle, stream)


def cgh_host_wait(handle, stream=None):
    """Wait for ``stream`` and for the host copies of earlier
    ``cgh_forward_host_async`` calls of ``handle``."""
    _check(handle, _L().cgh_host_wait(handle, _stream_ptr(stream)), "cgh_host_wait")


def cgh_host_ticket(handle) -> int:
    """Number of the last ``cgh_forward_host_async`` call of ``handle``."""
    return int(_L().cgh_host_ticket(handle))


def cgh_host_wait_ticket(handle, ticket: int) -> None:
    """Wait until every asynchronous host call up to ``ticket`` has finished
    (outputs complete, inputs free), leaving later calls running."""
    _check(handle, _L().cgh_host_wait_ticket(handle, int(ticket)), "cgh_host_wait_ticket")


# ------------------------------------------------------------ backward
def cgh_backward(points, A, z, lam: float, p: float, Nx: int, Ny: int,
                 grad_out, *, method="direct", handle=None, stream=None,
                 need=(True, True, True)):
    """Adjoint of Eq. 1 for dL/dI = grad_out (Ny, Nx).  Returns
    (grad_points (N, 2), grad_A (N,), grad_z (N,)); entries not in ``need``
    are None."""
    torch = _torch()
    N = int(A.numel())
    dev = A.device
    gp = torch.empty((N, 2), dtype=torch.float32, device=dev) if need[0] else None
    gA = torch.empty((N,), dtype=torch.float32, device=dev) if need[1] else None
    gz = torch.empty((N,), dtype=torch.float32, device=dev) if need[2] else None
    h = handle if handle is not None else default_handle(dev.index)
    go = grad_out.contiguous()
    st = _L().cgh_backward(
        h, _dev_f32(points, "points", 2 * N), _dev_f32(A, "A", N),
        _dev_f32(z, "z", N), N, float(lam), float(p), int(Nx), int(Ny),
        _dev_f32(go, "grad_out", Nx * Ny),
        _dev_f32(gp, "grad_points") if gp is not None else None,
        _dev_f32(gA, "grad_A") if gA is not None else None,
        _dev_f32(gz, "grad_z") if gz is not None else None,
        _method(method), _stream_ptr(stream))
    _check(h, st, "cgh_backward")
    return gp, gA, gz


# --------------------------------------------------------------- batch
def _problems(problems):
    n = len(problems)
    arr = (_Problem * max(n, 1))()
    for i, pr in enumerate(problems):
        N = int(pr["A"].numel())
        arr[i].points = _dev_f32(pr["points"], "points", 2 * N)
        arr[i].A = _dev_f32(pr["A"], "A", N)
        arr[i].z = _dev_f32(pr["z"], "z", N)
        arr[i].N = N
        arr[i].lam = float(pr["lam"])
        arr[i].p = float(pr["p"])
        arr[i].Nx = int(pr["Nx"])
        arr[i].Ny = int(pr["Ny"])
        arr[i].out = _dev_f32(pr["out"], "out", int(pr["Nx"]) * int(pr["Ny"]))
    return arr, n


def cgh_batch(problems: Sequence[dict], *, method="direct", handle=None,
              stream=None):
    """Many holograms in one persistent launch.  Each problem is a dict with
    points, A, z (CUDA tensors), lam, p, Nx, Ny and out (CUDA tensor)."""
    arr, n = _problems(problems)
    dev = problems[0]["A"].device.index if n else None
    h = handle if handle is not None else default_handle(dev)
    st = _L().cgh_batch(h, arr, n, _method(method), _stream_ptr(stream))
    _check(h, st, "cgh_batch")


def cgh_tune_batch(h, problems: Sequence[dict], method="direct", stream=None):
    """Tune this batch: "direct" times every direct tile shape and returns
    the fastest; "sep_fp16x3" times one-CTA and CTA-pair GEMM items and
    returns the faster tiling ("single" or "pairs")."""
    arr, n = _problems(problems)
    t = _Tile()
    st = _L().cgh_tune_batch(h, arr, n, _method(method), _stream_ptr(stream),
                             ctypes.byref(t))
    _check(h, st, "cgh_tune_batch")
    if _method(method) == METHODS["sep_fp16x3"]:
        return cgh_batch_plan(h, problems, method)["gemm_tiling"]
    return (t.tile_x, t.tile_y, t.vec_x, t.vec_y, t.points_per_stage, t.poly_pixels,
            t.point_groups, t.packed)


def cgh_batch_plan(h, problems: Sequence[dict], method="direct") -> dict:
    """What cgh_batch runs for this batch: {"tile": direct tile shape or
    None, "gemm_tiling": "single"/"pairs" or None, "tuned": bool}."""
    arr, n = _problems(problems)
    t, g, tu = _Tile(), ctypes.c_int(), ctypes.c_int()
    st = _L().cgh_batch_plan(h, arr, n, _method(method), ctypes.byref(t),
                             ctypes.byref(g), ctypes.byref(tu))
    _check(h, st, "cgh_batch_plan")
    direct = _method(method) == METHODS["direct"]
    return {"tile": (t.tile_x, t.tile_y, t.vec_x, t.vec_y, t.points_per_stage,
                     t.poly_pixels, t.point_groups, t.packed) if direct else None,
            "gemm_tiling": None if direct else
            {v: k for k, v in GEMM_TILES.items()}[g.value],
            "tuned": bool(tu.value)}


# ---------------------------------------------------------- tiles/tuning
def cgh_direct_tiles():
    out = []
    for i in range(_L().cgh_direct_tile_count()):
        t = _Tile()
        _L().cgh_direct_tile_get(i, ctypes.byref(t))
        out.append((t.tile_x, t.tile_y, t.vec_x, t.vec_y, t.points_per_stage,
                    t.poly_pixels, t.point_groups, t.packed))
    return out


def cgh_direct_tile_for(h, N: int, Nx: int, Ny: int):
    """The direct tile shape (as in cgh_direct_tiles()) the handle uses for
    this problem size."""
    t = _Tile()
    st = _L().cgh_direct_tile_for(h, int(N), int(Nx), int(Ny), ctypes.byref(t))
    _check(h, st, "cgh_direct_tile_for")
    return (t.tile_x, t.tile_y, t.vec_x, t.vec_y, t.points_per_stage,
            t.poly_pixels, t.point_groups, t.packed)


def cgh_set_direct_tile(h, tile=None):
    if tile is None:
        st = _L().cgh_set_direct_tile(h, None)
    else:
        t = _Tile(*tile)
        st = _L().cgh_set_direct_tile(h, ctypes.byref(t))
    _check(h, st, "cgh_set_direct_tile")


SCHEDULES = {"auto": 0, "grid": 1, "split": 2}


def cgh_set_direct_schedule(h, schedule="auto"):
    """How the direct kernel spreads pixel tiles over the SMs: "grid" (one
    CTA per tile), "split" (persistent CTAs with equal runs of (tile, point
    stage) units, split tiles summed in a fixed order) or "auto"."""
    st = _L().cgh_set_direct_schedule(h, SCHEDULES[schedule])
    _check(h, st, "cgh_set_direct_schedule")


def cgh_debug_pipe_rates(h, stream=None) -> dict:
    """Measured MUFU cosines and packed FP32 FMAs per SM clock on the
    handle's device (see include/cgh.h)."""
    mufu, fma = ctypes.c_double(), ctypes.c_double()
    st = _L().cgh_debug_pipe_rates(h, ctypes.byref(mufu), ctypes.byref(fma),
                                   _stream_ptr(stream))
    _check(h, st, "cgh_debug_pipe_rates")
    return {"mufu_cos_per_clk_per_sm": mufu.value, "fma_per_clk_per_sm": fma.value}


GEMM_TILES = {"auto": 0, "single": 1, "pairs": 2, "pairs_gen": 3}


def cgh_set_gemm_tiles(h, tiles="auto"):
    """Tiling of the separable methods' tensor-core GEMM: "single" (one CTA
    per 128-row tile), "pairs" (two CTAs of a cluster per 256-row tile,
    tcgen05 cta_group::2), "pairs_gen" (pairs that generate their operand
    tiles in shared memory, no U/V tables) or "auto" (tuned plan, else the
    heuristic)."""
    st = _L().cgh_set_gemm_tiles(h, GEMM_TILES[tiles])
    _check(h, st, "cgh_set_gemm_tiles")


def cgh_gemm_plan(h, Nx: int, Ny: int):
    """(tiling, width) the separable forward GEMM of an Nx x Ny hologram
    takes on this handle: tiling is "single" or "pairs"."""
    t, w = ctypes.c_int(), ctypes.c_int()
    _check(h, _L().cgh_gemm_plan(h, int(Nx), int(Ny), ctypes.byref(t), ctypes.byref(w)),
           "cgh_gemm_plan")
    return {v: k for k, v in GEMM_TILES.items()}[t.value], w.value


def cgh_set_gemm_plan(h, tiling="auto", width=0):
    """Force the separable GEMM's tiling ("single", "pairs", "pairs_gen")
    and tile width; "auto" returns to the tuned plan or the heuristic."""
    st = _L().cgh_set_gemm_plan(h, GEMM_TILES[tiling], int(width))
    _check(h, st, "cgh_set_gemm_plan")


def cgh_gemm_plan_for(h, N: int, Nx: int, Ny: int, method="sep_fp16x3"):
    """(tiling, width, tuned) of the separable forward GEMM of `method` for
    N points on an Nx x Ny frame on this handle."""
    t, w, tu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(h, _L().cgh_gemm_plan_for(h, _method(method), int(N), int(Nx), int(Ny),
                                     ctypes.byref(t), ctypes.byref(w), ctypes.byref(tu)),
           "cgh_gemm_plan_for")
    return {v: k for k, v in GEMM_TILES.items()}[t.value], w.value, bool(tu.value)


def cgh_tune(h, N: int, Nx: int, Ny: int, method="direct", stream=None):
    """Measure the tunable shapes of `method` for this size and keep the
    fastest on the handle: the direct tile (returned), or for the
    tensor-core methods the GEMM plan (returned as cgh_gemm_plan_for's
    (tiling, width, tuned))."""
    t = _Tile()
    st = _L().cgh_tune(h, int(N), int(Nx), int(Ny), _method(method),
                      _stream_ptr(stream), ctypes.byref(t))
    _check(h, st, "cgh_tune")
    if _method(method) != METHODS["direct"]:
        return cgh_gemm_plan_for(h, N, Nx, Ny, method)
    return (t.tile_x, t.tile_y, t.vec_x, t.vec_y, t.points_per_stage, t.poly_pixels,
            t.point_groups, t.packed)


def cgh_last_device_status(h, stream=None) -> int:
    """Synchronise and return (and clear) the device status as a cgh_status."""
    return int(_L().cgh_last_device_status(h, _stream_ptr(stream)))


def cgh_launch_count(h) -> int:
    return int(_L().cgh_launch_count(h))


KERNELS = {"prologue": 0, "direct_tables": 1, "direct": 2, "naive": 3,
           "sep_tables": 4, "gemm": 5, "bwd_direct": 6, "bwd_gemm": 7,
           "bwd_reduce": 8, "batch": 9, "aux": 10, "batch_sep": 11, "recur": 12,
           "simt": 13, "bwd_simt": 14}


def cgh_kernel_timing(h, enable: bool = True) -> None:
    """Bracket every kernel launch of ``h`` with CUDA events on its stream
    (resets the totals)."""
    _check(h, _L().cgh_kernel_timing(h, 1 if enable else 0), "cgh_kernel_timing")


def cgh_kernel_timing_mask(h, kernels) -> None:
    """Bracket only the named kernels (names or ids) with events."""
    mask = 0
    for k in kernels:
        mask |= 1 << (KERNELS[k] if isinstance(k, str) else int(k))
    _check(h, _L().cgh_kernel_timing_mask(h, mask), "cgh_kernel_timing_mask")


def cgh_kernel_time(h, kernel):
    """(total device ms, launches) of one kernel since timing was enabled."""
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(h, _L().cgh_kernel_time(h, k, ctypes.byref(ms), ctypes.byref(n)),
           "cgh_kernel_time")
    return float(ms.value), int(n.value)


def cgh_debug_gemm(A, B, *, handle=None, stream=None):
    """D = A B^T on the tcgen05 GEMM (A: M x K, B: N x K, fp16 or bf16)."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or A.dtype != B.dtype:
        raise ValueError("A and B must be M x K and N x K of one 16-bit dtype")
    is_bf16 = {torch.float16: 0, torch.bfloat16: 1}[A.dtype]
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    h = handle if handle is not None else default_handle(A.device.index)
    st = _L().cgh_debug_gemm(h, A.contiguous().data_ptr(),
                            B.contiguous().data_ptr(), D.data_ptr(), M, N, K,
                            is_bf16, _stream_ptr(stream))
    _check(h, st, "cgh_debug_gemm")
    return D


# ------------------------------------------------------------- autograd
def _make_function():
    torch = _torch()

    class CGHFunction(torch.autograd.Function):
        """I = CGHFunction.apply(points, A, z, lam, p, Nx, Ny, method,
        backward_method): Eq. 1 forward, hand-written adjoint backward."""

        @staticmethod
        def forward(ctx, points, A, z, lam, p, Nx, Ny, method="direct",
                    backward_method="direct"):
            pts, A_, z_ = points.contiguous(), A.contiguous(), z.contiguous()
            ctx.save_for_backward(pts, A_, z_)
            ctx.args = (lam, p, Nx, Ny, backward_method)
            return cgh_forward(pts, A_, z_, lam, p, Nx, Ny, method=method)

        @staticmethod
        def backward(ctx, grad_out):
            pts, A_, z_ = ctx.saved_tensors
            lam, p, Nx, Ny, bm = ctx.args
            need = ctx.needs_input_grad[:3]
            gp, gA, gz = cgh_backward(pts, A_, z_, lam, p, Nx, Ny,
                                      grad_out.contiguous(), method=bm,
                                      need=(need[0], need[1], need[2]))
            return gp, gA, gz, None, None, None, None, None, None

    return CGHFunction


class _LazyFunction:
    _fn = None

    def __getattr__(self, name):
        if _LazyFunction._fn is None:
            _LazyFunction._fn = _make_function()
        return getattr(_LazyFunction._fn, name)


CGHFunction = _LazyFunction()
