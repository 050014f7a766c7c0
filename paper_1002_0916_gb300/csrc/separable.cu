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
// from the point records (built by the tables kernel itself, as prologue.cu
// builds them for the other methods) -- directly for a thread's first row,
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
#include "point_rec.cuh"
#include "sep_table.cuh"

namespace cgh {

// Grid: x over blocks of ST_POINTS points, y over runs of ST_BLOCK_ROWS
// consecutive table rows (x rows, then y rows).  The block first builds the
// records of its points in shared memory (step A1 in FP64, as prologue.cu;
// each record is built once per row block, which costs less than a
// separate prologue launch in the chain), then each warp writes one run of
// ST_ROWS rows for 32 point pairs (sep_table_rows): a warp's stores are
// contiguous 256-byte pieces of a table row.
constexpr int ST_POINTS = 64;
constexpr int ST_BLOCK_ROWS = 8 * ST_ROWS;

template <int KIND>
__global__ void __launch_bounds__(256)
sep_tables_kernel(PointSource src, int Npad, int Nx, int Ny, int Kp,
                  void *__restrict__ Lhi, void *__restrict__ Llo,
                  void *__restrict__ Rhi, void *__restrict__ Rlo) {
    __shared__ PointRec srec[ST_POINTS];
    pdl_wait();  // the caller's points may come from the kernel before
    pdl_trigger();
    const int j0 = blockIdx.x * ST_POINTS;
    if (threadIdx.x < ST_POINTS && j0 + (int)threadIdx.x < Npad)
        srec[threadIdx.x] = make_point_rec(src.points, src.A, src.z, src.N,
                                           j0 + threadIdx.x, src.K,
                                           src.status, src.y0);
    __syncthreads();
    const int pair = threadIdx.x & 31, run = threadIdx.x >> 5;
    const int jj = j0 + 2 * pair;  // even; Npad is even, so jj + 1 < Npad too
    if (jj >= Npad) return;
    const int r0 = blockIdx.y * ST_BLOCK_ROWS + run * ST_ROWS;
    const int rows = Nx + Ny;
    if (r0 >= rows) return;
    const int r1 = r0 + ST_ROWS < rows ? r0 + ST_ROWS : rows;
    const bool v0 = jj < src.N, v1 = jj + 1 < src.N;
    sep_table_rows<KIND>(srec[2 * pair], srec[2 * pair + 1], v0, v1, Nx, Kp, jj, r0,
                         r1, Lhi, Llo, Rhi, Rlo);
}

cudaError_t launch_sep_tables(const PointSource &src, int Npad, int Nx, int Ny, int Kp,
                              int kind, void *Lhi, void *Llo, void *Rhi, void *Rlo,
                              cudaStream_t s) {
    const int rows = Nx + Ny;  // <= 65536: grid y stays below its limit
    dim3 grid((Npad + ST_POINTS - 1) / ST_POINTS, (rows + ST_BLOCK_ROWS - 1) / ST_BLOCK_ROWS);
    // (builds the records itself: the call's first kernel, an ordinary launch)
    if (kind == 0)
        return launch_kernel(false, sep_tables_kernel<0>, grid, dim3(256), 0, s, src, Npad,
                             Nx, Ny, Kp, Lhi, Llo, Rhi, Rlo);
    if (kind == 1)
        return launch_kernel(false, sep_tables_kernel<1>, grid, dim3(256), 0, s, src, Npad,
                             Nx, Ny, Kp, Lhi, Llo, Rhi, Rlo);
    return launch_kernel(false, sep_tables_kernel<2>, grid, dim3(256), 0, s, src, Npad, Nx,
                         Ny, Kp, Lhi, Llo, Rhi, Rlo);
}

}  // namespace cgh

using namespace cgh;

cgh_ctx::GemmPlanChoice cgh_ctx::sep_plan(int method, int N, int Nx, int Ny) {
    const int kind = method == CGH_SEP_BF16 ? 0 : method == CGH_SEP_FP16 ? 1 : 2;
    if (forced_plan >= 0) {
        const GemmPlan p = gemm_plan(Ny, Nx, forced_plan / 1000, sm_count, kind,
                                     forced_plan % 1000);
        return GemmPlanChoice{p.tiling, p.bn, false};
    }
    if (gemm_tiles == CGH_GEMM_AUTO) {
        auto it = tuned_gemm.find(size_bucket(method, N, Nx, Ny));
        if (it != tuned_gemm.end()) {
            const GemmPlan p = gemm_plan(Ny, Nx, it->second / 1000, sm_count, kind,
                                         it->second % 1000);
            return GemmPlanChoice{p.tiling, p.bn, true};
        }
    }
    const GemmPlan p = gemm_plan(Ny, Nx, gemm_tiles, sm_count, kind, gemm_bn);
    return GemmPlanChoice{p.tiling, p.bn, false};
}

cgh_status cgh_ctx::forward_separable(const float *points, const float *A,
                                      const float *z, int N, double lambda,
                                      double p, int Nx, int Ny, float *out,
                                      int method, cudaStream_t s) {
    const int kind = method == CGH_SEP_BF16 ? 0 : method == CGH_SEP_FP16 ? 1 : 2;
    const bool split = kind == 2;
    const int Kp = pad_to(2 * N, 64);
    const int Npad = Kp / 2;
    const size_t rec_b = align256((size_t)Npad * sizeof(PointRec));
    const GemmPlanChoice plan = sep_plan(method, N, Nx, Ny);
    if (plan.tiling == CGH_GEMM_PAIRS_GEN) {
        // the GEMM generates its operand tiles from the point records
        cgh_status st = ensure(ws, rec_b, s, "separable workspace");
        if (st) return st;
        PointRec *rec = (PointRec *)ws.ptr;
        {
            TimedLaunch tl(this, CGH_K_PROLOGUE, s);
            cudaError_t e = launch_prologue(points, A, z, N, Npad, lambda, p, rec,
                                            d_status, s, row_origin);
            if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
            tl.done();
        }
        TimedLaunch tl(this, CGH_K_GEMM, s);
        cudaError_t e = launch_umma_gen(rec, N, Npad, kind, plan.bn, out, Ny, Nx, Nx,
                                        1.0f / LO_SCALE, d_status, s);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core GEMM launch");
        launches += gemm_k_chunks(Kp, split) - 1;  // K chunks beyond the first
        tl.done();
        return CGH_OK;
    }
    const size_t l_b = align256((size_t)Nx * Kp * 2);
    const size_t r_b = align256((size_t)Ny * Kp * 2);
    const size_t planes = split ? 2 : 1;
    cgh_status st = ensure(ws, planes * (l_b + r_b), s, "separable workspace");
    if (st) return st;
    char *base = (char *)ws.ptr;
    void *Lhi = base;
    void *Rhi = base + l_b;
    void *Llo = split ? base + l_b + r_b : nullptr;
    void *Rlo = split ? base + 2 * l_b + r_b : nullptr;
    {
        // the tables kernel builds the point records itself (no prologue)
        TimedLaunch tl(this, CGH_K_SEP_TABLES, s);
        cudaError_t e = launch_sep_tables(
            PointSource{points, A, z, N, fresnel_scale(lambda, p), d_status, row_origin}, Npad, Nx, Ny,
            Kp, kind, Lhi, Llo, Rhi, Rlo, s);
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
    op.tiles = plan.tiling;
    op.bn = plan.bn;
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
    op.tiles = h->gemm_tiles == CGH_GEMM_PAIRS_GEN ? CGH_GEMM_PAIRS : h->gemm_tiles;
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
