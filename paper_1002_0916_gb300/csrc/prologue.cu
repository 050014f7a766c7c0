// prologue.cu -- per-point records (step A1 of the hot path).
//
// For each object point j (Section 1, Eq. 1; P_j = pi p^2 / (lambda z_j)):
//   Q_j = P_j / (2 pi) = p^2 / (2 lambda z_j)     [turns per pixel^2]
//   c   = frac(Q_j),  b = frac(2 Q_j u_j),  a = frac(Q_j u_j^2)  per axis u
// in FP64, each converted to unsigned 0.64 fixed-point turns.  Then the axis
// phase c u^2 - b u + a (mod 1) equals Q_j (u - u_j)^2 (mod 1) for integer u,
// evaluated without rounding in 64-bit integer arithmetic.  The only
// rounding left is FP64's in Q_j, b and a (relative 2^-53 of Q_j u_j^2,
// about 1e-13 turns at 3840 x 2160).
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

__global__ void prologue_kernel(const float *__restrict__ points,
                                const float *__restrict__ A,
                                const float *__restrict__ z, int N, int Npad,
                                double lambda, double p,
                                PointRec *__restrict__ rec,
                                unsigned *status) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Npad) return;
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
    rec[j] = r;
}

cudaError_t launch_prologue(const float *points, const float *A,
                            const float *z, int N, int Npad, double lambda,
                            double p, PointRec *rec, unsigned *status,
                            cudaStream_t s) {
    if (Npad <= 0) return cudaSuccess;
    int threads = 128;
    int blocks = (Npad + threads - 1) / threads;
    prologue_kernel<<<blocks, threads, 0, s>>>(points, A, z, N, Npad, lambda,
                                                p, rec, status);
    return cudaGetLastError();
}

}  // namespace cgh
