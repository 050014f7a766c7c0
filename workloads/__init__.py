"""Seeded synthetic point clouds for the Fresnel CGH workloads.

This module only draws random inputs.  It holds none of the hologram
arithmetic, so both the CUDA path and the CPU oracle may use it.

The paper (Section 3, Table 1) computes 1,920 x 1,024 holograms from N object
points but does not describe its 3D objects; uniform random clouds with the
stated extents stand in for them.

Recipe (shared by every workload):
  * ``numpy.random.default_rng(seed)`` (PCG64);
  * draw order per cloud: x, y, z, A;
  * integer coordinates: ``rng.integers(0, Nx, N)``, continuous coordinates:
    ``rng.uniform(0, Nx, N)`` (same for y with Ny);
  * z ~ U[zlo, zhi] metres, A ~ U[0, 1];
  * everything is cast to float32 before either side sees it.

Coordinates are in units of the pixel pitch p (Eq. 1: positions normalised
by p); lambda and p are in metres.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = ["Cloud", "make_cloud", "WORKLOADS", "workload", "batch_problems",
           "grad_field", "TABLE1_POINTS", "table1_cloud"]


@dataclass
class Cloud:
    """One hologram problem: N points plus the optical constants."""

    xy: np.ndarray      # float32 (N, 2), interleaved (x_j, y_j), pixel units
    A: np.ndarray       # float32 (N,), point amplitudes
    z: np.ndarray       # float32 (N,), metres, > 0
    lam: float          # wavelength, metres
    p: float            # pixel pitch, metres
    Nx: int
    Ny: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.A.shape[0])

    @property
    def pp(self) -> int:
        """Point-pixel updates of one hologram: N * Nx * Ny."""
        return self.N * self.Nx * self.Ny


def make_cloud(seed: int, N: int, Nx: int, Ny: int, *, integer: bool,
               zlo: float, zhi: float, lam: float, p: float,
               rng: Optional[np.random.Generator] = None,
               name: str = "") -> Cloud:
    """Draw one cloud (order x, y, z, A) from ``rng`` or a fresh PCG64(seed)."""
    if rng is None:
        rng = np.random.default_rng(seed)
    if integer:
        x = rng.integers(0, Nx, N)
        y = rng.integers(0, Ny, N)
    else:
        x = rng.uniform(0, Nx, N)
        y = rng.uniform(0, Ny, N)
    z = rng.uniform(zlo, zhi, N)
    A = rng.uniform(0.0, 1.0, N)
    xy = np.empty((N, 2), dtype=np.float32)
    xy[:, 0] = x
    xy[:, 1] = y
    return Cloud(xy=xy, A=A.astype(np.float32), z=z.astype(np.float32),
                 lam=float(lam), p=float(p), Nx=int(Nx), Ny=int(Ny), name=name)


# The five workloads.  Sizes, ranges and constants as specified for this
# build; the 1920x1024 shape is the paper's Table 1 frame.
WORKLOADS = {
    "cfg1_256x256_n64": dict(N=64, Nx=256, Ny=256, integer=True, zlo=0.5,
                             zhi=1.0, lam=532e-9, p=8e-6),
    "cfg2_1920x1024_n1024": dict(N=1024, Nx=1920, Ny=1024, integer=True,
                                 zlo=0.5, zhi=1.5, lam=633e-9, p=6.4e-6),
    "cfg3_3840x2160_n16384": dict(N=16384, Nx=3840, Ny=2160, integer=False,
                                  zlo=0.3, zhi=2.0, lam=532e-9, p=3.74e-6),
    "cfg5_1920x1080_n4096": dict(N=4096, Nx=1920, Ny=1080, integer=False,
                                 zlo=0.5, zhi=1.5, lam=532e-9, p=6.4e-6),
}


def workload(name: str, seed: int = 0) -> Cloud:
    """The named single-hologram workload drawn with ``seed`` (default 0)."""
    kw = dict(WORKLOADS[name])
    return make_cloud(seed, name=name, **kw)


# The point counts of the paper's Table 1 (1,920 x 1,024 pixels).
TABLE1_POINTS = (512, 1024, 1536, 2048, 2560, 3072, 3584)


def table1_cloud(N: int, seed: int = 0) -> Cloud:
    """A cloud of N points on the paper's Table 1 frame, with the 1920x1024
    workload's recipe (integer coordinates, z ~ U[0.5, 1.5] m, 633 nm,
    6.4 um) and only N changed."""
    kw = dict(WORKLOADS["cfg2_1920x1024_n1024"])
    kw["N"] = int(N)
    return make_cloud(seed, name=f"table1_n{N}", **kw)


BATCH_WAVELENGTHS = (633e-9, 532e-9, 473e-9)


def batch_problems(seed: int = 0, count: int = 64, *, nx_choices=None,
                   n_lo: int = 100, n_hi: int = 8192, p: float = 8e-6,
                   zlo: float = 0.5, zhi: float = 1.5) -> List[Cloud]:
    """The batched workload: ``count`` holograms of uneven size.

    Per problem, in order: Nx, Ny from {512, 640, ..., 2048}; N ~ U[n_lo, n_hi];
    a wavelength index into (633, 532, 473) nm; then the cloud (integer
    coordinates) from the same generator.
    """
    rng = np.random.default_rng(seed)
    if nx_choices is None:
        nx_choices = np.arange(512, 2048 + 1, 128)
    out = []
    for i in range(count):
        Nx = int(rng.choice(nx_choices))
        Ny = int(rng.choice(nx_choices))
        N = int(rng.integers(n_lo, n_hi + 1))
        li = int(rng.integers(0, len(BATCH_WAVELENGTHS)))
        c = make_cloud(seed, N, Nx, Ny, integer=True, zlo=zlo, zhi=zhi,
                       lam=BATCH_WAVELENGTHS[li], p=p, rng=rng,
                       name=f"batch{i}")
        c.meta["lambda_index"] = li
        out.append(c)
    return out


def grad_field(seed: int, Nx: int, Ny: int, scale: float = 1.0) -> np.ndarray:
    """A seeded float32 (Ny, Nx) field standing in for dL/dI."""
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal((Ny, Nx))).astype(np.float32)
