// point_rec.cuh -- construction of one per-point record (see prologue.cu
// for the mathematics).  Internal to libcgh.
#pragma once

#include <math.h>

#include "common.cuh"

namespace cgh {

// f in [0, 1) -> round-down 0.64 fixed point, floor(f 2^64) exactly, from
// the bits of f (integer operations only: FP64 is slow on this GPU):
// f = m 2^(e - 1075) with the 53-bit significand m and biased exponent e.
__device__ __forceinline__ uint64_t to_fix64(double f) {
    const uint64_t bits = (uint64_t)__double_as_longlong(f);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0) return 0;  // zero or subnormal: below 2^-1022
    const uint64_t m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = e - 1011;  // f 2^64 = m 2^sh; f < 1 gives sh <= 11
    if (sh >= 0) return m << sh;
    return sh > -64 ? m >> -sh : 0;
}

// |x| = m 2^-s exactly, with m a 24-bit integer (frexpf) and s an integer
// shift (negative for |x| >= 2^24).
__device__ __forceinline__ void float_mant_shift(float x, uint64_t &m, int &s) {
    const float ax = fabsf(x);
    if (ax == 0.0f) {
        m = 0;
        s = 0;
        return;
    }
    int e;
    const float f = frexpf(ax, &e);          // ax = f 2^e, f in [1/2, 1)
    m = (uint64_t)(f * 16777216.0f);         // exact: 24 significant bits
    s = 24 - e;
}

// (c v) 2^-s modulo 2^64 from the 128-bit product (bits below 2^0 dropped).
__device__ __forceinline__ uint64_t mul_shift(uint64_t c, uint64_t v, int s) {
    const uint64_t lo = c * v, hi = __umul64hi(c, v);
    if (s <= 0) return s > -64 ? lo << (-s) : 0;
    if (s < 64) return (hi << (64 - s)) | (lo >> s);
    if (s < 128) return hi >> (s - 64);
    return 0;
}

// Record of point j (all zero for padding points j >= N and for rejected
// points, which also raise DEV_BAD_POINT: z <= 0, a non-finite value, or
// z_j <= p^2 / (2 lambda), i.e. Q_j >= 1 turn per pixel^2, far inside the
// distance where the Fresnel form of Eq. 1 holds).
//
// Only Q_j itself is computed in FP64.  With c = Q_j in 0.64 fixed point
// and u_j = m 2^-s exactly, the axis coefficients are exact integer
// arithmetic on c: b = 2 c u_j and a = c u_j^2 (mod 1 turn).
//
// y0 != 0 moves the y origin: the record then gives the phase of pixel row
// y0 + v at row index v, i.e. c (v + y0)^2 - b (v + y0) + a
//   = c v^2 - (b - 2 c y0) v + (a - b y0 + c y0^2),
// again exact modulo one turn (a slab of rows of a larger hologram).
__device__ __forceinline__ PointRec make_point_rec(const float *points,
                                                   const float *A,
                                                   const float *z, int N, int j,
                                                   double K, unsigned *status,
                                                   int y0 = 0) {
    PointRec r;
    r.c = r.bx = r.ax = r.by = r.ay = 0;
    r.A = 0.0f;
    r.Q32 = 0.0f;
    if (j < N) {
        const float xj = points[2 * j], yj = points[2 * j + 1];
        const float aj = A[j], zj = z[j];
        // Q_j = K / z_j with K = p^2 / (2 lambda) from the host: 1 / z_j from
        // the FP32 reciprocal and two Newton steps in FP64 (relative error
        // 2^-23 -> 2^-46 -> FP64 rounding), no FP64 division
        const double zd = (double)zj;
        double rz = (double)__frcp_rn(zj);
        rz = fma(fma(-zd, rz, 1.0), rz, rz);
        rz = fma(fma(-zd, rz, 1.0), rz, rz);
        const double Q = K * rz;
        const bool ok = isfinite(xj) && isfinite(yj) && isfinite(aj) &&
                        isfinite(zj) && zj > 0.0f && Q < 1.0;
        if (ok) {
            r.c = to_fix64(Q);
            uint64_t m;
            int s;
            float_mant_shift(xj, m, s);
            uint64_t b = mul_shift(r.c, m, s) << 1;
            r.bx = xj < 0.0f ? (uint64_t)0 - b : b;
            r.ax = mul_shift(r.c, m * m, 2 * s);
            float_mant_shift(yj, m, s);
            b = mul_shift(r.c, m, s) << 1;
            r.by = yj < 0.0f ? (uint64_t)0 - b : b;
            r.ay = mul_shift(r.c, m * m, 2 * s);
            if (y0 != 0) {
                const uint64_t Y = (uint64_t)(int64_t)y0;
                r.ay = r.ay - r.by * Y + r.c * (Y * Y);
                r.by = r.by - 2 * r.c * Y;
            }
            r.A = aj;
            r.Q32 = (float)Q;
        } else {
            set_status(status, DEV_BAD_POINT);
        }
    }
    return r;
}

}  // namespace cgh
