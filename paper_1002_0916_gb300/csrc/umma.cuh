// umma.cuh -- inline-PTX helpers for the sm_100-family tensor cores
// (tcgen05.* with accumulators in tensor memory) and tiled TMA loads.
// Internal to libcgh.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the driver is reached at run time)

#include "common.cuh"

namespace cgh {
namespace umma {

// ------------------------------------------------------------------ TMA
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

// 2-D tiled load of box (c0 = innermost element index, c1 = row) into dst,
// completing on `bar`.  c0 * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map,
                                            int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::"
        "bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// ----------------------------------------------------------------- TMEM
// Allocation and release are executed by one whole warp, joined first (the
// instructions are .sync.aligned).
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    __syncwarp();
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_u32(dst_smem)),
        "r"(ncols)
        : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
    __syncwarp();
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::
                     : "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ------------------------------------------------------------------ MMA
// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzle: rows of 64 16-bit elements (128 B), groups of 8 rows
// 1024 B apart.  The tile must start on a 1024-byte boundary.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused)
    d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8 rows
    d |= (uint64_t)1 << 46;                        // descriptor version
    d |= (uint64_t)2 << 61;                        // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, A and B both FP16
// (bf16 = false) or both BF16, both K-major, tile M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16) {
    return (1u << 4)                         // D format: F32
           | ((bf16 ? 1u : 0u) << 7)         // A format
           | ((bf16 ? 1u : 0u) << 10)        // B format
           | ((uint32_t)(N >> 3) << 17)      // N / 8
           | ((uint32_t)(M >> 4) << 24);     // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T, one 128 x N x 16 step, issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc,
                                        uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on `bar` when every tcgen05.mma issued so far by this thread
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
        "[%0];" ::"r"(smem_u32(bar))
        : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp-wide).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]),
          "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-wide).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]),
          "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace umma

// One problem of a grouped split GEMM: its four tensor maps (A hi, B hi,
// A lo, B lo) live in global memory and are read by TMA, which wants them
// 64-byte aligned; the struct keeps CUtensorMap's own 128-byte alignment.
struct alignas(alignof(CUtensorMap)) GroupProb {
    CUtensorMap tA, tB, tA2, tB2;
    float *D;
    long long ldd;
    int M, N, K;
    float lo_scale;
};

// Fill gp (tensor maps and sizes) for the split GEMM `op`; false if a
// tensor map cannot be encoded.
// Tensor map of a rows x inner FP32 matrix (row stride `ld` elements), box =
// box_inner x box_rows, no swizzle, zero fill out of bounds.  inner * 4 and
// ld * 4 must be multiples of 16 bytes, base 16-byte aligned.
bool make_f32_map(CUtensorMap *m, const void *base, long long inner, long long rows,
                  long long ld, int box_inner, int box_rows);

// b_box_rows: rows of B per TMA box (the tile's columns for one-CTA items,
// half of them for CTA-pair items)
bool encode_group_prob(GroupProb *gp, const GemmOperands &op, int b_box_rows);
cudaError_t launch_umma_grouped(const GroupProb *probs, const uint2 *items,
                                int nitems, unsigned *status, int sm_count,
                                cudaStream_t s);
cudaError_t prepare_umma_grouped();
int group_tile_n();
// umma2.cu: the same on CTA pairs; items are (problem, 256-row tile,
// group_pair_tile_n()-column tile)
cudaError_t launch_umma_grouped_pair(const GroupProb *probs, const uint2 *items,
                                     int nitems, unsigned *status, int sm_count,
                                     cudaStream_t s);
cudaError_t prepare_umma_grouped_pair();
int group_pair_tile_m();
int group_pair_tile_n();
int group_pair_box_b();

}  // namespace cgh
