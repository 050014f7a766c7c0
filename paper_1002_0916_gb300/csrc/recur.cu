// recur.cu -- the paper's optimised kernel design restated for sm_103a: the
// phase advanced pixel by pixel along a row by the two recurrences of Eq. 2
// (Section 2.1), as a comparison point for the per-axis angle tables of
// direct.cu.
//
// What the paper's kernel does (Section 2.1, optimisations (1)-(5)):
//  * groups of 16 x 16 items; each item computes eight consecutive pixels
//    along x (the float8 vector);
//  * object points are copied to shared memory 256 at a time, with a barrier
//    after each copy;
//  * the point loop is unrolled by four;
//  * along the item's eight pixels the phase follows Eq. 2:
//        Gamma_n = Gamma_{n-1} + delta_{n-1},  delta_n = delta_{n-1} + Delta,
//        Gamma_0 = P_j r^2 at the first pixel, delta_0 = P_j (2 (x_h - x_j) + 1),
//        Delta = 2 P_j;
//  * the cosine is the hardware ("native") one.
//
// Here the recurrence runs in 32-bit fixed-point turns (mod 1 turn, so it
// never loses precision with the size of the phase): Gamma_0 and delta_0
// are the exact 0.64 fixed-point values of the point record rounded to
// 0.32, Delta = 2 Q_j rounded to 0.32.  After n steps the phase error is at
// most (1 + n + n (n - 1) / 2) 2^-33 turns (3.4e-9 turns at n = 7).
//
// Per point-pixel update: two integer adds (the recurrences), shift + or to
// turn the phase into a float in [1, 2) (the top 23 bits of the turn), one
// FMA to radians in [-pi, pi), the hardware cosine (argument scale + MUFU),
// one FMA to accumulate: 7 issue slots and 1 MUFU operation.
#include <math.h>

#include "common.cuh"

namespace cgh {

constexpr int RC_ITEMS_X = 16;       // items per group along x
constexpr int RC_ITEMS_Y = 16;       // items per group along y
constexpr int RC_VEC = 8;            // pixels per item along x
constexpr int RC_POINTS = 256;       // points per shared-memory stage
constexpr int RC_THREADS = RC_ITEMS_X * RC_ITEMS_Y;
static_assert(RC_THREADS == RC_POINTS, "one record per thread per stage");

constexpr float RC_TWO_PI = 6.28318530717958647692f;
constexpr float RC_THREE_PI = 9.42477796076937971538f;

__global__ void __launch_bounds__(RC_THREADS)
recur_fwd_kernel(const PointRec *__restrict__ rec, int Npad, int Nx, int Ny,
                 float *__restrict__ out, int vec_store) {
    // one stage of points, structure of arrays (every lane of a warp reads
    // the same point: broadcast)
    __shared__ uint64_t s_c[RC_POINTS], s_bx[RC_POINTS], s_by[RC_POINTS],
        s_a[RC_POINTS];
    __shared__ uint32_t s_D[RC_POINTS];
    __shared__ float s_A[RC_POINTS];

    const int ix = threadIdx.x % RC_ITEMS_X, iy = threadIdx.x / RC_ITEMS_X;
    const int x0 = blockIdx.x * (RC_ITEMS_X * RC_VEC) + ix * RC_VEC;
    const int y = blockIdx.y * RC_ITEMS_Y + iy;
    // per-thread constants of the phase at (x0, y):
    //   Gamma_0 = c (x0^2 + y^2) - bx x0 - by y + (ax + ay)   (0.64 turns)
    //   delta_0 = c (2 x0 + 1) - bx
    const uint64_t sq = (uint64_t)((int64_t)x0 * x0 + (int64_t)y * y);
    const uint64_t ux = (uint64_t)(int64_t)x0, uy = (uint64_t)(int64_t)y;
    const uint64_t u2x1 = (uint64_t)(2 * (int64_t)x0 + 1);

    float acc[RC_VEC];
#pragma unroll
    for (int n = 0; n < RC_VEC; ++n) acc[n] = 0.0f;

    for (int j0 = 0; j0 < Npad; j0 += RC_POINTS) {
        __syncthreads();  // the previous stage is no longer read
        {
            const PointRec r = rec[j0 + threadIdx.x];
            s_c[threadIdx.x] = r.c;
            s_bx[threadIdx.x] = r.bx;
            s_by[threadIdx.x] = r.by;
            s_a[threadIdx.x] = r.ax + r.ay;
            // Delta = 2 Q_j, rounded to 0.32
            s_D[threadIdx.x] = (uint32_t)(((r.c << 1) + 0x80000000ull) >> 32);
            s_A[threadIdx.x] = r.A;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < RC_POINTS; ++k) {
            const uint64_t c = s_c[k];
            const uint64_t ph = c * sq - s_bx[k] * ux - s_by[k] * uy + s_a[k];
            const uint64_t dl = c * u2x1 - s_bx[k];
            // Gamma in 0.32 turns, offset by half a turn (so that the float
            // below is centred) and by half a unit of its 23-bit truncation
            // (so that truncation rounds to nearest)
            uint32_t G = (uint32_t)((ph + 0x80000000ull) >> 32) + 0x80000100u;
            uint32_t d = (uint32_t)((dl + 0x80000000ull) >> 32);
            const uint32_t D = s_D[k];
            const float a = s_A[k];
#pragma unroll
            for (int n = 0; n < RC_VEC; ++n) {
                // 1 + (turn + 1/2) in [1, 2), then 2 pi (v - 3/2) in [-pi, pi)
                const float v = __uint_as_float((G >> 9) | 0x3F800000u);
                const float th = fmaf(v, RC_TWO_PI, -RC_THREE_PI);
                acc[n] = fmaf(a, __cosf(th), acc[n]);
                G += d;   // Gamma_{n+1} = Gamma_n + delta_n
                d += D;   // delta_{n+1} = delta_n + Delta
            }
        }
    }
    if (y >= Ny) return;
    float *row = out + (size_t)y * Nx;
    // vec_store: Nx a multiple of 4 and out 16-byte aligned (x0 is a
    // multiple of 8, so every row's vectors are aligned too)
    if (vec_store && x0 + RC_VEC <= Nx) {
        float4 *dst = reinterpret_cast<float4 *>(row + x0);
        dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    } else {
#pragma unroll
        for (int n = 0; n < RC_VEC; ++n)
            if (x0 + n < Nx) row[x0 + n] = acc[n];
    }
}

int recur_points_per_stage() { return RC_POINTS; }

cudaError_t launch_recur_forward(const PointRec *rec, int Npad, int Nx, int Ny,
                                 float *out, cudaStream_t s) {
    if (Npad % RC_POINTS) return cudaErrorInvalidValue;
    dim3 grid((Nx + RC_ITEMS_X * RC_VEC - 1) / (RC_ITEMS_X * RC_VEC),
              (Ny + RC_ITEMS_Y - 1) / RC_ITEMS_Y);
    const int vec_store = (Nx % 4 == 0) && (((uintptr_t)out & 15) == 0);
    recur_fwd_kernel<<<grid, RC_THREADS, 0, s>>>(rec, Npad, Nx, Ny, out, vec_store);
    return cudaGetLastError();
}

}  // namespace cgh
