"""Pins for the FP64 oracle: facts fixed by the paper's Eq. 1 / Eq. 2 and by
mathematics, none of which re-types the oracle's own code.

* textbook Fresnel zone-plate radii for one point (constants, units, P_j);
* superposition and linearity in A_j (Eq. 1 is a weighted sum);
* integer-shift translation invariance (coordinate frame, x/y roles);
* 8-fold symmetry about an integer point (r^2 = dx^2 + dy^2);
* exact-rational phase reduction on a tiny grid (turn reduction);
* long-double brute force, unreduced (turn reduction, precision);
* Eq. 2 recurrence (Section 2.1) equals Eq. 1 along rows;
* separable identity I = Re(U diag(A) V^T) in complex128;
* adjoint against central finite differences (Richardson-checked).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from workloads import make_cloud, workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sumA(c):
    return float(np.abs(c.A.astype(np.float64)).sum())


def test_zone_plate_radii(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "zone_plate.json")))
    P, G = g["params"], g["grid"]
    xy = np.array([[G["x0"], G["y0"]]], np.float32)
    I = oracle_mod.forward(xy=xy, A=np.array([P["A"]], np.float32),
                           z=np.array([P["z"]], np.float32), lam=P["lambda"],
                           p=P["p"], Nx=G["Nx"], Ny=G["Ny"])
    for case in g["cases"]:
        v = I[G["y0"] + case["dy"], G["x0"] + case["dx"]]
        assert v == pytest.approx(P["A"] * case["I_over_A"], abs=1e-12), case


def test_zone_plate_long_double_agrees(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "zone_plate.json")))
    P, G = g["params"], g["grid"]
    xy = np.array([[G["x0"], G["y0"]]], np.float32)
    kw = dict(xy=xy, A=np.array([P["A"]], np.float32),
              z=np.array([P["z"]], np.float32), lam=P["lambda"], p=P["p"],
              Nx=G["Nx"], Ny=G["Ny"])
    ld = oracle_mod.forward_ld(**kw)
    for case in g["cases"]:
        v = ld[G["y0"] + case["dy"], G["x0"] + case["dx"]]
        assert v == pytest.approx(P["A"] * case["I_over_A"], abs=1e-12), case


@pytest.mark.parametrize("integer", [True, False])
def test_superposition_and_linearity(oracle_mod, integer):
    c1 = make_cloud(11, 20, 40, 30, integer=integer, zlo=0.05, zhi=0.2,
                    lam=532e-9, p=8e-6)
    c2 = make_cloud(12, 13, 40, 30, integer=integer, zlo=0.05, zhi=0.2,
                    lam=532e-9, p=8e-6)
    both = dict(xy=np.concatenate([c1.xy, c2.xy]),
                A=np.concatenate([c1.A, c2.A]), z=np.concatenate([c1.z, c2.z]),
                lam=c1.lam, p=c1.p, Nx=40, Ny=30)
    I12 = oracle_mod.forward(**both)
    I1, I2 = oracle_mod.forward(c1), oracle_mod.forward(c2)
    tol = 1e-12 * (_sumA(c1) + _sumA(c2))
    assert np.max(np.abs(I12 - (I1 + I2))) < tol
    # linearity in A: A -> alpha A, alpha a power of two (exact in float32)
    for alpha in (0.25, -2.0):
        I1s = oracle_mod.forward(xy=c1.xy, A=(alpha * c1.A).astype(np.float32),
                                 z=c1.z, lam=c1.lam, p=c1.p, Nx=40, Ny=30)
        assert np.max(np.abs(I1s - alpha * I1)) < 1e-12 * _sumA(c1)
    # an empty cloud is the zero hologram
    I0 = oracle_mod.forward(xy=np.zeros((0, 2), np.float32),
                            A=np.zeros(0, np.float32), z=np.zeros(0, np.float32),
                            lam=c1.lam, p=c1.p, Nx=40, Ny=30)
    assert np.all(I0 == 0.0)


@pytest.mark.parametrize("integer", [True, False])
def test_integer_shift_invariance(oracle_mod, integer):
    c = make_cloud(3, 9, 24, 20, integer=integer, zlo=0.1, zhi=0.3,
                   lam=633e-9, p=6.4e-6)
    a, b = 5, -3
    sh = c.xy.copy()
    sh[:, 0] += a
    sh[:, 1] += b
    I = oracle_mod.forward(c)
    Is = oracle_mod.forward(xy=sh, A=c.A, z=c.z, lam=c.lam, p=c.p, Nx=24, Ny=20)
    # Is[y + b, x + a] == I[y, x] wherever both are in the frame
    ys = np.arange(max(0, -b), min(20, 20 - b))
    xs = np.arange(max(0, -a), min(24, 24 - a))
    lhs = Is[np.ix_(ys + b, xs + a)]
    rhs = I[np.ix_(ys, xs)]
    # integer shifts of float32 coordinates are exact only for integers
    tol = 1e-12 * _sumA(c) if integer else 1e-6 * _sumA(c)
    assert np.max(np.abs(lhs - rhs)) < tol


def test_eightfold_symmetry(oracle_mod):
    x0, y0, R = 10, 10, 10
    I = oracle_mod.forward(xy=np.array([[x0, y0]], np.float32),
                           A=np.array([0.6], np.float32),
                           z=np.array([0.02], np.float32), lam=532e-9, p=8e-6,
                           Nx=2 * R + 1, Ny=2 * R + 1)
    for a in range(R + 1):
        for b in range(R + 1):
            ref = I[y0 + b, x0 + a]
            for sx in (1, -1):
                for sy in (1, -1):
                    assert I[y0 + sy * b, x0 + sx * a] == pytest.approx(ref, abs=1e-13)
                    assert I[y0 + sy * a, x0 + sx * b] == pytest.approx(ref, abs=1e-13)
    # and it is not constant: the pattern really varies with r
    assert np.ptp(I) > 0.5


def _exact_turn_fraction(Q: Fraction, r2: Fraction) -> float:
    t = Q * r2
    f = t - round(t)          # exact rational reduction to [-1/2, 1/2]
    return float(f)


def test_exact_rational_reduction(oracle_mod):
    """Phase reduced exactly in rationals, then one double cos: agrees with
    the FP64 oracle to rounding (independent of libm's large-argument path)."""
    c = make_cloud(5, 4, 7, 6, integer=False, zlo=0.01, zhi=0.02, lam=473e-9,
                   p=3.74e-6)
    # make the phase large (hundreds of turns) by a small z
    I = oracle_mod.forward(c)
    p, lam = Fraction(c.p), Fraction(c.lam)
    ref = np.zeros((c.Ny, c.Nx))
    for j in range(c.N):
        Q = p * p / (2 * lam * Fraction(float(c.z[j])))
        xj, yj = Fraction(float(c.xy[j, 0])), Fraction(float(c.xy[j, 1]))
        for y in range(c.Ny):
            for x in range(c.Nx):
                r2 = (x - xj) ** 2 + (y - yj) ** 2
                f = _exact_turn_fraction(Q, r2)
                ref[y, x] += float(c.A[j]) * math.cos(2 * math.pi * f)
    assert np.max(np.abs(I - ref)) < 1e-11 * _sumA(c)


def test_long_double_brute_force(oracle_mod):
    c = make_cloud(7, 8, 16, 12, integer=False, zlo=0.3, zhi=2.0, lam=532e-9,
                   p=3.74e-6)
    # stretch the cloud so the phases reach tens of turns on a tiny grid
    c.xy[:, 0] *= 20.0
    c.xy[:, 1] *= 20.0
    I = oracle_mod.forward(c)
    ld = oracle_mod.forward_ld(c)
    assert np.max(np.abs(I - ld)) < 1e-12 * _sumA(c)


def test_config1_long_double_rows(oracle_mod):
    """The 256x256 / 64-point workload itself, two rows, against long double."""
    c = workload("cfg1_256x256_n64")
    rows = [0, 200]
    I = oracle_mod.forward(c, rows=rows)
    small = dict(xy=c.xy, A=c.A, z=c.z, lam=c.lam, p=c.p, Nx=c.Nx, Ny=201)
    ld = oracle_mod.forward_ld(**small)
    assert np.max(np.abs(I - ld[rows])) < 1e-12 * _sumA(c)


@pytest.mark.parametrize("integer", [True, False])
def test_recurrence_equals_eq1(oracle_mod, integer):
    c = make_cloud(9, 16, 96, 40, integer=integer, zlo=0.5, zhi=1.5,
                   lam=633e-9, p=6.4e-6)
    c.xy[:, 0] *= 8.0    # points off the frame too: larger phases
    I = oracle_mod.forward(c)
    Ir = oracle_mod.forward_recurrence(c)
    assert np.max(np.abs(I - Ir)) < 1e-9 * _sumA(c)
    rows = [3, 17, 39]
    assert np.max(np.abs(oracle_mod.forward_recurrence(c, rows=rows) - I[rows])) \
        < 1e-9 * _sumA(c)


def _separable(c):
    """Re(U diag(A) V^T) with U[x, j] = exp(i P_j (x - x_j)^2), complex128."""
    xj = c.xy[:, 0].astype(np.float64)
    yj = c.xy[:, 1].astype(np.float64)
    P = np.pi * c.p ** 2 / (c.lam * c.z.astype(np.float64))
    x = np.arange(c.Nx, dtype=np.float64)[:, None]
    y = np.arange(c.Ny, dtype=np.float64)[:, None]
    U = np.exp(1j * P[None, :] * (x - xj[None, :]) ** 2)     # (Nx, N)
    V = np.exp(1j * P[None, :] * (y - yj[None, :]) ** 2)     # (Ny, N)
    return np.real(V @ np.diag(c.A.astype(np.float64)) @ U.T)  # (Ny, Nx)


@pytest.mark.parametrize("integer", [True, False])
def test_separable_identity(oracle_mod, integer):
    c = make_cloud(13, 37, 45, 33, integer=integer, zlo=0.5, zhi=1.5,
                   lam=532e-9, p=6.4e-6)
    assert np.max(np.abs(oracle_mod.forward(c) - _separable(c))) < 1e-10 * _sumA(c)


# ---------------------------------------------------------------- adjoint


def _eq1_fd(xy, A, z, lam, p, Nx, Ny):
    """Eq. 1 with FP64 parameters (finite-difference witness only)."""
    x = np.arange(Nx, dtype=np.float64)[None, :]
    y = np.arange(Ny, dtype=np.float64)[:, None]
    I = np.zeros((Ny, Nx))
    for j in range(len(A)):
        P = np.pi * p * p / (lam * z[j])
        I += A[j] * np.cos(P * ((x - xy[j, 0]) ** 2 + (y - xy[j, 1]) ** 2))
    return I


def _fd_grad(c, G, j, which, h):
    xy = c.xy.astype(np.float64)
    A = c.A.astype(np.float64)
    z = c.z.astype(np.float64)

    def L(delta):
        xy2, A2, z2 = xy.copy(), A.copy(), z.copy()
        if which == "x":
            xy2[j, 0] += delta
        elif which == "y":
            xy2[j, 1] += delta
        elif which == "A":
            A2[j] += delta
        else:
            z2[j] += delta
        return float(np.sum(G * _eq1_fd(xy2, A2, z2, c.lam, c.p, c.Nx, c.Ny)))

    d1 = (L(h) - L(-h)) / (2 * h)
    d2 = (L(h / 2) - L(-h / 2)) / h
    return (4 * d2 - d1) / 3, abs(d2 - d1)  # Richardson + its own error scale


@pytest.mark.parametrize("seed", [21, 22])
def test_grad_vs_finite_differences(oracle_mod, seed):
    c = make_cloud(seed, 5, 24, 20, integer=False, zlo=0.05, zhi=0.1,
                   lam=532e-9, p=8e-6)
    G = np.random.default_rng(seed + 100).standard_normal((c.Ny, c.Nx))
    gxy, gA, gz = oracle_mod.grad(c, G)
    for j in range(c.N):
        for which, h, got in (("A", 1e-4, gA[j]), ("x", 1e-4, gxy[j, 0]),
                              ("y", 1e-4, gxy[j, 1]),
                              ("z", 1e-6 * float(c.z[j]), gz[j])):
            fd, err = _fd_grad(c, G, j, which, h)
            scale = max(abs(fd), 1e-3)
            assert abs(got - fd) <= 1e-6 * scale + 10 * err, (j, which, got, fd)


def test_grad_point_subset_and_loss_form(oracle_mod):
    """Point subsets agree with the full call; L = sum (I - T)^2 gives
    G = 2 (I - T) and the gradient of that loss matches central FD."""
    c = make_cloud(31, 6, 20, 16, integer=True, zlo=0.05, zhi=0.1,
                   lam=633e-9, p=6.4e-6)
    t = make_cloud(32, 6, 20, 16, integer=True, zlo=0.05, zhi=0.1,
                   lam=633e-9, p=6.4e-6)
    I, T = oracle_mod.forward(c), oracle_mod.forward(t)
    G = 2.0 * (I - T)
    gxy, gA, gz = oracle_mod.grad(c, G)
    sxy, sA, sz = oracle_mod.grad(c, G, pts=[4, 1])
    assert np.array_equal(sxy, gxy[[4, 1]]) and np.array_equal(sA, gA[[4, 1]])
    assert np.array_equal(sz, gz[[4, 1]])

    xy = c.xy.astype(np.float64)
    A = c.A.astype(np.float64)
    z = c.z.astype(np.float64)

    def loss(Ad):
        I2 = _eq1_fd(xy, Ad, z, c.lam, c.p, c.Nx, c.Ny)
        return float(np.sum((I2 - T) ** 2))

    for j in range(c.N):
        h = 1e-5
        Ap, Am = A.copy(), A.copy()
        Ap[j] += h
        Am[j] -= h
        fd = (loss(Ap) - loss(Am)) / (2 * h)
        assert gA[j] == pytest.approx(fd, rel=1e-6, abs=1e-6)
