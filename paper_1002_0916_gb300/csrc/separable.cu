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
// ST_ROWS consecutive table rows from row0 (sep_table_rows, sep_table.cuh).
constexpr int ST_PAIRS = 128;

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
    sep_table_rows<KIND>(p0, p1, v0, v1, Nx, Kp, j0, r0, r1, Lhi, Llo, Rhi, Rlo);
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
    op.tiles = gemm_tiles;
    {
        TimedLaunch tl(this, CGH_K_GEMM, s);
        cudaError_t e = launch_umma_gemm(op, d_status, s);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core GEMM launch");
        launches += gemm_k_chunks(Kp, split) - 1;  // K chunks beyond the first
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
    op.tiles = h->gemm_tiles;
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
