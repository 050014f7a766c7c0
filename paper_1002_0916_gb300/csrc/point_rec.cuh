// point_rec.cuh -- construction of one per-point record (see prologue.cu
// for the mathematics).  Internal to libcgh.
#pragma once

#include <math.h>

#include "common.cuh"

namespace cgh {

// f in [0, 1) -> round-down 0.64 fixed point (error < 2^-64 turns).
__device__ __forceinline__ uint64_t to_fix64(double f) {
    double u = f * 4294967296.0;          // exact scaling
    double hi = floor(u);                 // < 2^32
    double lo = floor((u - hi) * 4294967296.0);
    return ((uint64_t)hi << 32) | (uint64_t)lo;
}

__device__ __forceinline__ double frac(double v) { return v - floor(v); }

// Record of point j (all zero for padding points j >= N and for rejected
// points: z <= 0 or a non-finite value, which also raise DEV_BAD_POINT).
__device__ __forceinline__ PointRec make_point_rec(const float *points,
                                                   const float *A,
                                                   const float *z, int N, int j,
                                                   double lambda, double p,
                                                   unsigned *status) {
    PointRec r;
    r.c = r.bx = r.ax = r.by = r.ay = 0;
    r.A = 0.0f;
    r.Q32 = 0.0f;
    if (j < N) {
        float xj = points[2 * j], yj = points[2 * j + 1];
        float aj = A[j], zj = z[j];
        bool ok = isfinite(xj) && isfinite(yj) && isfinite(aj) &&
                  isfinite(zj) && zj > 0.0f;
        if (ok) {
            double Q = (p * p) / (2.0 * lambda * (double)zj);
            double x = (double)xj, y = (double)yj;
            r.c = to_fix64(frac(Q));
            r.bx = to_fix64(frac(2.0 * Q * x));
            r.ax = to_fix64(frac(Q * x * x));
            r.by = to_fix64(frac(2.0 * Q * y));
            r.ay = to_fix64(frac(Q * y * y));
            r.A = aj;
            r.Q32 = (float)Q;
        } else {
            set_status(status, DEV_BAD_POINT);
        }
    }
    return r;
}

}  // namespace cgh
