// common.cuh -- internal declarations and PTX helpers shared by the CUDA
// translation units of libcgh (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "cgh.h"

namespace cgh {

// Bits of the device status word.
enum : unsigned {
    DEV_BAD_POINT = 1u,   // a point had z <= 0 or a non-finite coordinate
    DEV_TIMEOUT = 2u,     // a bounded wait gave up
    DEV_BOUNDS = 4u       // an internal bounds check failed
};

// Per-point record built by the prologue (Section 1, Eq. 1).  The phase of
// point j at pixel (x, y), in turns, is
//     Q_j ((x - x_j)^2 + (y - y_j)^2),   Q_j = P_j / (2 pi) = p^2 / (2 lambda z_j),
// and each axis part expands to c x^2 - b x + a (mod 1) with
//     c = frac(Q_j), b = frac(2 Q_j x_j), a = frac(Q_j x_j^2).
// All three are stored as unsigned 0.64 fixed-point turns, so that the
// per-pixel evaluation is exact integer arithmetic modulo 1 turn.
struct PointRec {
    uint64_t c;
    uint64_t bx, ax;
    uint64_t by, ay;
    float A;       // amplitude (0 for rejected points)
    float Q32;     // Q_j rounded to FP32 (diagnostics)
};
static_assert(sizeof(PointRec) == 48, "PointRec layout");

// Axis phase in 0.64 turns at integer coordinate u: c u^2 - b u + a (mod 1).
__device__ __forceinline__ uint64_t axis_phase(uint64_t c, uint64_t b,
                                               uint64_t a, int u) {
    uint64_t uu = (uint64_t)((int64_t)u * (int64_t)u);
    return c * uu - b * (uint64_t)(int64_t)u + a;
}

// Top 32 bits of a 0.64 phase as a signed turn count in [-1/2, 1/2).
__device__ __forceinline__ int phase_hi(uint64_t ph) { return (int)(ph >> 32); }

// 2 pi / 2^32: radians per unit of a signed 0.32 phase.
constexpr float RAD_PER_U32 = 1.4629180792671596e-9f;
// 1 / 2^32: turns per unit of a signed 0.32 phase.
constexpr float TURN_PER_U32 = 2.3283064365386963e-10f;

// ---------------------------------------------------------------- PTX
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar,
                                                      uint32_t bytes) {
    asm volatile(
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// About one second at the GB300's clocks.
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;

// Wait for phase `parity` of `bar` to complete, giving up after
// WAIT_LIMIT_CYCLES.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar,
                                                  uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
    }
    return true;
}

// 1-D bulk copy global -> shared, completing `bytes` on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void set_status(unsigned *status, unsigned bits) {
    if (status) atomicOr(status, bits);
}

// Programmatic dependent launch: a kernel launched with
// launch_dependent() may start while the previous kernel of the stream is
// still running; it must call pdl_wait() before touching global memory that
// kernel writes (a no-op for an ordinary launch).  pdl_trigger() lets the
// next such kernel launch early.
__device__ __forceinline__ void pdl_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace cgh

// ------------------------------------------------ launch helper (host side)
namespace cgh {

// Launch `kern` on stream s as a programmatic dependent of the kernel
// before it in the stream (see pdl_wait), or, with dependent = false, as an
// ordinary launch that starts only after everything before it in the stream
// has finished.  The first kernel of every call is launched the ordinary
// way: calls never overlap one another, whatever ran before them.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(bool dependent, void (*kern)(KArgs...), dim3 grid, dim3 block,
                          size_t smem, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dependent ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block,
                             size_t smem, cudaStream_t s, Args &&...args) {
    return launch_kernel(true, kern, grid, block, smem, s, std::forward<Args>(args)...);
}

}  // namespace cgh

// ------------------------------------------------ launchers (host side)
namespace cgh {

struct DirectTile {
    int tx, ty, vx, vy, pt, np, g, pk;
};

// x-table floats per pixel column of a direct tile with packing pk: 1 (the
// angle), or 2 for the rotation forms (pk 6 - 8: per group of a thread's
// columns, the first column's angle, the cosines and the sines of the
// columns' phase offsets from it); the same for the y table and rows (pk 7,
// 8).
__host__ __device__ constexpr int direct_xf(int pk) { return pk >= 6 ? 2 : 1; }
__host__ __device__ constexpr int direct_yf(int pk) { return pk >= 7 ? 2 : 1; }
// Rotation group sizes of a tile's x and y tables (0: one angle per
// coordinate).
inline int direct_xg(const DirectTile &t) { return direct_xf(t.pk) == 2 ? t.vx : 0; }
inline int direct_yg(const DirectTile &t) { return direct_yf(t.pk) == 2 ? t.vy : 0; }
// Floats of a tile's x table and y table for Npad points.
inline size_t direct_x_floats(const DirectTile &t, int nxt, int Npad) {
    return (size_t)nxt * Npad * t.tx * direct_xf(t.pk);
}
inline size_t direct_y_floats(const DirectTile &t, int nyt, int Npad) {
    return (size_t)nyt * Npad * t.ty * direct_yf(t.pk);
}

// Number of points after padding to a multiple of `pt`.
inline int pad_to(int n, int m) { return (n + m - 1) / m * m; }

// prologue.cu; y0: origin of the pixel rows (see make_point_rec)
cudaError_t launch_prologue(const float *points, const float *A,
                            const float *z, int N, int Npad, double lambda,
                            double p, PointRec *rec, unsigned *status,
                            cudaStream_t s, int y0 = 0);

// direct.cu
int direct_tile_count();
DirectTile direct_tile_get(int i);
int direct_tile_index(const DirectTile &t);
size_t direct_phase_table_floats(const DirectTile &t, int Npad, int Nx, int Ny);
// (zero, nzero): words the tables kernel sets to zero (the split
// schedule's arrival counters), or (nullptr, 0)
cudaError_t launch_direct_tables(const PointRec *rec, int Npad, int Nx, int Ny,
                                 const DirectTile &t, float *phx, float *phy,
                                 float *amp, unsigned *zero, int nzero,
                                 cudaStream_t s);
// The caller's point arrays, for kernels that build the records themselves.
// p^2 / (2 lambda): Q_j = P_j / (2 pi) = this / z_j turns per pixel^2 (the
// definition of P_j under Eq. 1), the part of Q_j shared by every point.
inline double fresnel_scale(double lambda, double p) { return p * p / (2.0 * lambda); }

struct PointSource {
    const float *points, *A, *z;
    int N;
    double K;  // fresnel_scale(lambda, p)
    unsigned *status;
    int y0 = 0;  // origin of the pixel rows (see make_point_rec)
};
// The same tables with the records built inside the kernel (no prologue).
cudaError_t launch_direct_tables_fused(const PointSource &src, int Npad, int Nx,
                                       int Ny, const DirectTile &t, float *phx,
                                       float *phy, float *amp, unsigned *zero,
                                       int nzero, cudaStream_t s);
// Tail split of the direct kernel: `tiles` pixel tiles, those from `tail`
// on each cut into m chunks of point stages (tail == tiles: none).
struct DirectSplit {
    int tiles, tail, m;
    int chunks() const { return (tiles - tail) * m; }
};
DirectSplit direct_split_plan(int tile_index, int sm_count, int Npad, int Nx,
                              int Ny, bool split);
// part: chunks() partial tiles; count: tiles - tail words, zero at launch
cudaError_t launch_direct_forward(int tile_index, const float *phx,
                                  const float *phy, const float *amp, int Npad,
                                  int Nx, int Ny, float *out,
                                  const DirectSplit &d, float *part,
                                  unsigned *count, unsigned *status,
                                  cudaStream_t s);
cudaError_t launch_naive_forward(const PointRec *rec, int N, int Nx, int Ny,
                                 float *out, cudaStream_t s);

// recur.cu: the Eq. 2 recurrence kernel; Npad a multiple of
// recur_points_per_stage() (records padded with zero amplitude)
int recur_points_per_stage();
cudaError_t launch_recur_forward(const PointRec *rec, int Npad, int Nx, int Ny,
                                 float *out, cudaStream_t s);

// umma.cu: D = A B^T (single pass) or Ahi Bhi^T + lo_scale (Ahi Blo^T +
// Alo Bhi^T) (split) on the tensor cores.  A: M x K, B: N x K, 16-bit,
// K-major with row strides lda, ldb (elements); D: FP32, row stride ldd.
struct GemmOperands {
    const void *A_hi, *A_lo, *B_hi, *B_lo;
    int M, N, K;
    long long lda, ldb;
    bool bf16, split;
    float lo_scale;
    float *D;
    long long ldd;
    int tiles = CGH_GEMM_AUTO;  // a cgh_gemm_tiles value
    int accumulate = 0;         // 1: D += product instead of D = product
    int bn = 0;                 // tile width of a tuned plan (0: the heuristic's)
};
bool gemm_operands_ok(const GemmOperands &op);
// Longest K one launch accumulates in tensor memory.  The tensor cores' FP32
// accumulation drops the low bits of every add; over a long run of
// same-sign terms (points whose phases agree at a pixel) that bias grows
// in proportion to K: measured 1.3e-4 relative (100,000 coincident
// points) for runs of 32,768, about 4e-9 per value of k.  Products of
// larger K therefore run as consecutive launches of at most this many
// values of k, each adding its partial product into D in FP32 with round
// to nearest: 16,384 for split FP16 (bound 1e-4: about 6e-5 at worst),
// 131,072 for the single-pass forms (bound 1e-2: about 5e-4 at worst).
constexpr int GEMM_K_CHUNK = 16384;
constexpr int GEMM_K_CHUNK_SINGLE = 131072;
inline int gemm_k_chunk(bool split) { return split ? GEMM_K_CHUNK : GEMM_K_CHUNK_SINGLE; }
inline int gemm_k_chunks(int K, bool split) {
    return (K + gemm_k_chunk(split) - 1) / gemm_k_chunk(split);
}
// umma2.cu: the same product on CTA pairs (256-row tiles over two SMs);
// bnp = columns of a pair tile (one of the compiled widths)
// The pair tile width for an M x N product and its cost (SM waves x width).
int pick_pair_n(int M, int N, int sms, double *cost = nullptr);
bool pair_width_ok(int bnp);
// How launch_umma_gemm tiles an M x N forward product under a cgh_gemm_tiles
// setting: CGH_GEMM_SINGLE or CGH_GEMM_PAIRS, and the tile width.
struct GemmPlan {
    int tiling, bn;
};
// kind: 0 BF16, 1 FP16, 2 split FP16 (the widths compiled for the
// generating kernel depend on it); bn: a width to use instead of the
// heuristic's (0: none)
GemmPlan gemm_plan(int M, int N, int tiles, int sms, int kind = 2, int bn = 0);
// Cost of a pair width: SM waves x columns per CTA (umma2.cu).
double pair_cost(int M, int N, int bnp, int sms);
// umma_gen.cu: the pair GEMM with its operand tiles generated in shared
// memory from the point records (no U / V tables): D = R L^T over the Npad
// records at rec (N real), K chunks as launch_umma_gemm.
bool gen_pair_width_ok(int kind, int bnp);
int pick_gen_n(int M, int N, int sms, int kind);
cudaError_t launch_umma_gen(const PointRec *rec, int N, int Npad, int kind, int bnp,
                            float *D, int M, int Ncols, long long ldd, float lo_scale,
                            unsigned *status, cudaStream_t s);
cudaError_t launch_umma_pair(const GemmOperands &op, int bnp, unsigned *status,
                             cudaStream_t s);
struct AdjEpiArgs;
cudaError_t launch_umma_pair_adjoint(const GemmOperands &op, const AdjEpiArgs &ea,
                                     int sms, unsigned *status, cudaStream_t s,
                                     int *tile_n);
cudaError_t launch_umma_gemm(const GemmOperands &op, unsigned *status,
                             cudaStream_t s);
// Split GEMM whose epilogue reduces the adjoint sums over its columns into
// part[n_tile][npad][3] (see umma_epi.cuh); rows are k = 2j + {0: cos, 1:
// sin}.  *tile_n receives the column width of one n_tile (128, or a CTA-pair
// width >= 160), so part needs ceil(N / 128) tiles at most.
cudaError_t launch_umma_adjoint(const GemmOperands &op, const PointRec *rec,
                                const float *points, int npoints, int npad,
                                int axis, float *part, unsigned *status,
                                cudaStream_t s, int *tile_n);
int umma_tile_n();

// separable.cu: U / V tables of the separable form, the point records
// built inside the kernel from the caller's points.
cudaError_t launch_sep_tables(const PointSource &src, int Npad, int Nx, int Ny, int Kp,
                              int kind, void *Lhi, void *Llo, void *Rhi, void *Rlo,
                              cudaStream_t s);

}  // namespace cgh
