// prologue.cu -- per-point records (step A1 of the hot path).
//
// For each object point j (Section 1, Eq. 1; P_j = pi p^2 / (lambda z_j)):
//   Q_j = P_j / (2 pi) = p^2 / (2 lambda z_j)     [turns per pixel^2]
// in FP64, stored as c = Q_j in unsigned 0.64 fixed-point turns; then per
// axis u the coefficients b = 2 Q_j u_j and a = Q_j u_j^2 (mod 1) in exact
// integer arithmetic on c (u_j is a float, i.e. an integer times a power of
// two).  The axis phase c u^2 - b u + a (mod 1) equals Q_j (u - u_j)^2
// (mod 1) for integer u, evaluated without rounding in 64-bit integer
// arithmetic; the only rounding is Q_j's own (FP64, then 2^-64).
#include <math.h>

#include "common.cuh"
#include "point_rec.cuh"

namespace cgh {

__global__ void prologue_kernel(const float *__restrict__ points,
                                const float *__restrict__ A,
                                const float *__restrict__ z, int N, int Npad,
                                double K, PointRec *__restrict__ rec,
                                unsigned *status, int y0) {
    pdl_wait();  // the inputs may come from the kernel before
    pdl_trigger();
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Npad) return;
    rec[j] = make_point_rec(points, A, z, N, j, K, status, y0);
}

cudaError_t launch_prologue(const float *points, const float *A,
                            const float *z, int N, int Npad, double lambda,
                            double p, PointRec *rec, unsigned *status,
                            cudaStream_t s, int y0) {
    if (Npad <= 0) return cudaSuccess;
    // FP64 runs at a few operations per clock per SM on this GPU, so spread
    // the points thinly over many SMs
    int threads = 32;
    int blocks = (Npad + threads - 1) / threads;
    // (the first kernel of its call: an ordinary launch)
    return launch_kernel(false, prologue_kernel, dim3(blocks), dim3(threads), 0, s, points,
                         A, z, N, Npad, fresnel_scale(lambda, p), rec, status, y0);
}

}  // namespace cgh
