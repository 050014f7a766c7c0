// separable.cu -- the separable form of Eq. 1 on the tensor cores (steps
// A6-A7).
//
// The phase of Eq. 1 is a sum of an x part and a y part, so
//     I(x, y) = sum_j A_j cos(th_x(x, j) + th_y(y, j))
//             = sum_j [A_j cos th_x][cos th_y] - [A_j sin th_x][sin th_y]
//             = Re(U diag(A) V^T)[x, y],  U = e^{i th_x}, V = e^{i th_y},
// with th_u(u, j) = P_j (u - u_j)^2 (exact: no approximation).  Written with
// interleaved real pairs along K = 2N,
//     L[x][2j] = A_j cos th_x,  L[x][2j+1] = -A_j sin th_x   (Nx x K)
//     R[y][2j] =     cos th_y,  R[y][2j+1] =      sin th_y   (Ny x K)
// the hologram is the plain product I = R L^T (Ny x Nx, row-major), a dense
// contraction of depth 2N run by the tcgen05 GEMM of umma.cu.
//
// Tables: the axis phase is evaluated exactly in 64-bit fixed-point turns
// from the point records (prologue.cu) -- directly for a thread's first row,
// then by the exact integer recurrence of Eq. 2 -- its top 32 bits give the
// angle, and the hardware sincos gives the pair (absolute error about 2^-21,
// below FP16's 2^-11 and the split pair's 2^-22 rounding).  Entries for
// padding points (j >= N) are 0.
// Precision variants:
//   kind 0  BF16 single pass   (one plane per table)
//   kind 1  FP16 single pass
//   kind 2  FP16 split: hi = fp16(v), lo = fp16((v - hi) * 2^12); the GEMM
//           forms hi*hi + 2^-12 (hi*lo + lo*hi) with FP32 accumulation.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "api_internal.h"
#include "common.cuh"
#include "sep_table.cuh"

namespace cgh {

// Grid: x over pairs of points (128 pairs per block), y over groups of
// ST_ROWS consecutive table rows from row0.  Each thread loads its two
// records once, evaluates the axis phase of its first row directly and then
// steps it row by row with the exact fixed-point form of Eq. 2 (the phase
// difference c (2u + 1) - b and its constant second difference 2c, all
// modulo one turn), and writes the four interleaved entries of the pair as
// one 8-byte store per plane.
constexpr int ST_ROWS = 16;
constexpr int ST_PAIRS = 128;

template <int KIND>
__device__ __forceinline__ void sep_value(float A, bool valid, bool is_x,
                                          uint64_t ph, float &re, float &im) {
    float s, c;
    __sincosf((float)phase_hi(ph) * RAD_PER_U32, &s, &c);
    re = valid ? (is_x ? A * c : c) : 0.0f;
    im = valid ? (is_x ? -A * s : s) : 0.0f;
}

template <int KIND>
__device__ __forceinline__ void sep_store(void *hi, void *lo, size_t off, float re0,
                                          float im0, float re1, float im1) {
    if (KIND == 0) {
        __nv_bfloat162 v[2] = {__floats2bfloat162_rn(re0, im0),
                               __floats2bfloat162_rn(re1, im1)};
        *reinterpret_cast<uint2 *>((__nv_bfloat16 *)hi + off) =
            *reinterpret_cast<const uint2 *>(v);
    } else {
        __half2 v[2] = {__floats2half2_rn(re0, im0), __floats2half2_rn(re1, im1)};
        *reinterpret_cast<uint2 *>((__half *)hi + off) = *reinterpret_cast<const uint2 *>(v);
        if (KIND == 2) {
            const float2 h0 = __half22float2(v[0]), h1 = __half22float2(v[1]);
            __half2 w[2] = {__floats2half2_rn((re0 - h0.x) * LO_SCALE, (im0 - h0.y) * LO_SCALE),
                            __floats2half2_rn((re1 - h1.x) * LO_SCALE, (im1 - h1.y) * LO_SCALE)};
            *reinterpret_cast<uint2 *>((__half *)lo + off) =
                *reinterpret_cast<const uint2 *>(w);
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(ST_PAIRS)
sep_tables_kernel(const PointRec *__restrict__ rec, int N, int Nx, int Ny, int Kp,
                  int row0, void *__restrict__ Lhi, void *__restrict__ Llo,
                  void *__restrict__ Rhi, void *__restrict__ Rlo) {
    pdl_wait();  // the records come from the kernel before
    pdl_trigger();
    const int j0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j0 >= Kp / 2) return;  // Kp / 2 is even: j0 + 1 is in range too
    const int r0 = row0 + (int)blockIdx.y * ST_ROWS;
    const int r1 = r0 + ST_ROWS < Nx + Ny ? r0 + ST_ROWS : Nx + Ny;
    const bool v0 = j0 < N, v1 = j0 + 1 < N;
    const PointRec p0 = v0 ? rec[j0] : PointRec{};
    const PointRec p1 = v1 ? rec[j0 + 1] : PointRec{};
#pragma unroll
    for (int seg = 0; seg < 2; ++seg) {  // the x rows, then the y rows
        const bool is_x = seg == 0;
        const int a = is_x ? r0 : (r0 > Nx ? r0 : Nx);
        const int b = is_x ? (r1 < Nx ? r1 : Nx) : r1;
        if (a >= b) continue;
        int u = is_x ? a : a - Nx;
        const uint64_t b0 = is_x ? p0.bx : p0.by, b1 = is_x ? p1.bx : p1.by;
        uint64_t ph0 = axis_phase(p0.c, b0, is_x ? p0.ax : p0.ay, u);
        uint64_t ph1 = axis_phase(p1.c, b1, is_x ? p1.ax : p1.ay, u);
        const uint64_t step = (uint64_t)(2 * (int64_t)u + 1);
        uint64_t d0 = p0.c * step - b0, d1 = p1.c * step - b1;
        const uint64_t dd0 = 2 * p0.c, dd1 = 2 * p1.c;
        void *hi = is_x ? Lhi : Rhi;
        void *lo = is_x ? Llo : Rlo;
        size_t off = (size_t)u * Kp + 2 * (size_t)j0;
        for (int r = a; r < b; ++r, off += Kp) {
            float re0, im0, re1, im1;
            sep_value<KIND>(p0.A, v0, is_x, ph0, re0, im0);
            sep_value<KIND>(p1.A, v1, is_x, ph1, re1, im1);
            sep_store<KIND>(hi, lo, off, re0, im0, re1, im1);
            ph0 += d0;
            d0 += dd0;
            ph1 += d1;
            d1 += dd1;
        }
    }
}

cudaError_t launch_sep_tables(const PointRec *rec, int N, int Npad, int Nx,
                              int Ny, int Kp, int kind, void *Lhi, void *Llo,
                              void *Rhi, void *Rlo, cudaStream_t s) {
    (void)Npad;
    // row groups in launches of at most 65535 (the grid's y limit)
    const int rows = Nx + Ny;
    const int pairs = Kp / 4;
    for (int row0 = 0; row0 < rows; row0 += 65535 * ST_ROWS) {
        const int n = rows - row0 < 65535 * ST_ROWS ? rows - row0 : 65535 * ST_ROWS;
        dim3 grid((pairs + ST_PAIRS - 1) / ST_PAIRS, (n + ST_ROWS - 1) / ST_ROWS);
        cudaError_t e;
        if (kind == 0)
            e = launch_dependent(sep_tables_kernel<0>, grid, dim3(ST_PAIRS), 0, s, rec,
                                 N, Nx, Ny, Kp, row0, Lhi, Llo, Rhi, Rlo);
        else if (kind == 1)
            e = launch_dependent(sep_tables_kernel<1>, grid, dim3(ST_PAIRS), 0, s, rec,
                                 N, Nx, Ny, Kp, row0, Lhi, Llo, Rhi, Rlo);
        else
            e = launch_dependent(sep_tables_kernel<2>, grid, dim3(ST_PAIRS), 0, s, rec,
                                 N, Nx, Ny, Kp, row0, Lhi, Llo, Rhi, Rlo);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace cgh

using namespace cgh;

cgh_status cgh_ctx::forward_separable(const float *points, const float *A,
                                      const float *z, int N, double lambda,
                                      double p, int Nx, int Ny, float *out,
                                      int method, cudaStream_t s) {
    const int kind = method == CGH_SEP_BF16 ? 0 : method == CGH_SEP_FP16 ? 1 : 2;
    const bool split = kind == 2;
    const int Kp = pad_to(2 * N, 64);
    const int Npad = Kp / 2;
    const size_t rec_b = align256((size_t)Npad * sizeof(PointRec));
    const size_t l_b = align256((size_t)Nx * Kp * 2);
    const size_t r_b = align256((size_t)Ny * Kp * 2);
    const size_t planes = split ? 2 : 1;
    cgh_status st = ensure(ws, rec_b + planes * (l_b + r_b), s, "separable workspace");
    if (st) return st;
    char *base = (char *)ws.ptr;
    PointRec *rec = (PointRec *)base;
    void *Lhi = base + rec_b;
    void *Rhi = base + rec_b + l_b;
    void *Llo = split ? base + rec_b + l_b + r_b : nullptr;
    void *Rlo = split ? base + rec_b + 2 * l_b + r_b : nullptr;
    {
        TimedLaunch tl(this, CGH_K_PROLOGUE, s);
        cudaError_t e = launch_prologue(points, A, z, N, Npad, lambda, p, rec,
                                        d_status, s);
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        tl.done();
    }
    {
        TimedLaunch tl(this, CGH_K_SEP_TABLES, s);
        cudaError_t e = launch_sep_tables(rec, N, Npad, Nx, Ny, Kp, kind, Lhi, Llo,
                                          Rhi, Rlo, s);
        if (e != cudaSuccess) return cuda_fail(e, "separable tables launch");
        tl.done();
    }
    GemmOperands op{};
    op.A_hi = Rhi;
    op.A_lo = Rlo;
    op.B_hi = Lhi;
    op.B_lo = Llo;
    op.M = Ny;
    op.N = Nx;
    op.K = Kp;
    op.lda = Kp;
    op.ldb = Kp;
    op.bf16 = kind == 0;
    op.split = split;
    op.lo_scale = 1.0f / LO_SCALE;
    op.D = out;
    op.ldd = Nx;
    {
        TimedLaunch tl(this, CGH_K_GEMM, s);
        cudaError_t e = launch_umma_gemm(op, d_status, s);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core GEMM launch");
        tl.done();
    }
    return CGH_OK;
}

extern "C" cgh_status cgh_debug_gemm(cgh_handle h, const void *A, const void *B,
                                     float *D, int M, int N, int K, int is_bf16,
                                     void *stream) {
    if (!h) return CGH_ERR_INVALID_ARG;
    GemmOperands op{};
    op.A_hi = A;
    op.B_hi = B;
    op.M = M;
    op.N = N;
    op.K = K;
    op.lda = K;
    op.ldb = K;
    op.bf16 = is_bf16 != 0;
    op.split = false;
    op.lo_scale = 0.0f;
    op.D = D;
    op.ldd = N;
    if (!A || !B || !D || K % 64 != 0 || !gemm_operands_ok(op))
        return h->fail(CGH_ERR_INVALID_ARG,
                       "debug GEMM: need M, N >= 1, K a positive multiple of 64, "
                       "16-byte aligned A and B");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cgh_status st = CGH_OK;
    {
        TimedLaunch tl(h, CGH_K_GEMM, (cudaStream_t)stream);
        cudaError_t e = launch_umma_gemm(op, h->d_status, (cudaStream_t)stream);
        if (e != cudaSuccess)
            st = h->cuda_fail(e, "tensor-core GEMM launch");
        else
            tl.done();
    }
    cudaSetDevice(prev);
    return st;
}
