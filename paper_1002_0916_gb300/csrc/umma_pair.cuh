// umma_pair.cuh -- inline-PTX helpers for tensor-core work on CTA pairs
// (tcgen05 cta_group::2 within a cluster of two CTAs) and the shape of a
// pair tile, shared by the pair GEMMs (umma2.cu, umma_gen.cu).  Internal to
// libcgh.
#pragma once

#include "common.cuh"
#include "umma.cuh"

namespace cgh {
namespace umma2 {

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared-memory address of `p` in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(const void *p, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(out)
                 : "r"(smem_u32(p)), "r"(rank));
    return out;
}

// Every thread of both CTAs.  The .aligned barrier wants each warp
// converged: role branches (one lane producing, one issuing MMAs) may leave
// a warp split, so it is joined first.
__device__ __forceinline__ void cluster_sync() {
    __syncwarp();
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}

// A wait whose phase may be completed by the other CTA's arrive: acquire at
// cluster scope.  Bounded like mbar_wait_bounded.
__device__ __forceinline__ bool try_wait_cluster(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool wait_cluster_bounded(uint64_t *bar, uint32_t parity) {
    if (try_wait_cluster(bar, parity)) return true;
    const long long t0 = clock64();
    while (!try_wait_cluster(bar, parity))
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
    return true;
}

// Tensor memory of a CTA pair: one warp of each CTA, collectively (each
// helper joins the warp first: the instructions are .sync.aligned).
__device__ __forceinline__ void tmem_alloc2(uint32_t *dst_smem, uint32_t ncols) {
    __syncwarp();
    asm volatile(
        "tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_u32(dst_smem)),
        "r"(ncols)
        : "memory");
}

__device__ __forceinline__ void tmem_relinquish2() {
    __syncwarp();
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::
                     : "memory");
}

__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(ncols)
                 : "memory");
}

// One 256 x N x 16 step of the pair, issued by one thread of the even CTA.
__device__ __forceinline__ void mma2_f16(uint32_t d_tmem, uint64_t adesc,
                                         uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on `bar` (same offset) in every CTA of `mask` when the MMAs
// issued so far by this thread have completed.
__device__ __forceinline__ void commit2(uint64_t *bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster."
        "multicast::cluster.b64 [%0], %1;" ::"r"(smem_u32(bar)),
        "h"(mask)
        : "memory");
}

// 2-D tiled load into this CTA's shared memory whose completion (bytes) is
// signalled on the mbarrier at cluster address `bar`, which may lie in the
// other CTA of the pair.  c0 * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map,
                                                 int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes."
        "cta_group::2 [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Arrive (release, cluster scope) on the mbarrier at cluster address
// `cluster_addr`, which may lie in the other CTA of the pair.
__device__ __forceinline__ void remote_arrive(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                     cluster_addr)
                 : "memory");
}

}  // namespace umma2

template <int BNP, bool SPLIT, int STAGES>
struct PairShape {
    static constexpr int BM = 128, BK = 64, BNH = BNP / 2;
    static constexpr uint32_t A_BYTES = BM * BK * 2;
    static constexpr uint32_t B_BYTES = BNH * BK * 2;
    static constexpr uint32_t STAGE_BYTES =
        SPLIT ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
    static constexpr uint32_t ACC1 = BNP <= 128 ? 128 : 256;
    static constexpr uint32_t ACC_COLS = SPLIT ? ACC1 + BNP : BNP;
    static constexpr uint32_t TMEM_COLS =
        ACC_COLS <= 32 ? 32 : ACC_COLS <= 64 ? 64 : ACC_COLS <= 128 ? 128
        : ACC_COLS <= 256 ? 256 : 512;
    static constexpr int CH = BNP % 32 == 0 ? 32 : 16;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
    static_assert(BNH % 8 == 0, "each B half is whole 8-row swizzle atoms");
    static_assert(BNP % 16 == 0 && BNP >= 32 && BNP <= 256, "UMMA N at M = 256");
    static_assert(ACC_COLS <= 512, "TMEM");
    static_assert(SMEM <= 232448, "shared memory");
};

}  // namespace cgh
