// umma2.cu -- the forward GEMM of the separable methods on CTA pairs
// (tcgen05 cta_group::2): the same product as umma.cu,
//
//     D[m][n] = sum_k A[m][k] B[n][k]                      (single pass)
//     D[m][n] = sum_k Ahi Bhi + s * (Ahi Blo + Alo Bhi)    (split, s = 2^-12)
//
// but each MMA covers a 256 x BNP tile computed by two SMs together.  The
// two CTAs of a cluster each stage their own 128 rows of A and their own
// half (BNP / 2 rows) of B; one thread of the even CTA issues the MMAs, which
// read both CTAs' shared memory and write each CTA's 128 rows of D into that
// CTA's tensor memory.  Per SM this moves half the operand bytes per
// multiply-add of the one-CTA kernel at the same shared-memory footprint
// (the one-CTA 128 x BN kernel loads 128 + BN rows per 128 BN outputs; a
// pair loads 128 + BNP / 2 per SM for 128 BNP).
//
// Synchronisation (every wait bounded, as in umma.cu):
//   * both CTAs' TMA loads of a stage complete on the even CTA's `full`
//     barrier (the odd CTA's loads signal it across the pair, cta_group::2),
//     whose expected byte count covers both halves; the MMA issuer waits on
//     it alone;
//   * the MMA issuer's commits arrive on the `empty` barriers and, at the
//     end, the accumulator barrier of both CTAs (multicast commit);
//   * cluster barriers after set-up (all barriers initialised, tensor memory
//     allocated in both CTAs) and before the tensor memory is released.
#include <cudaTypedefs.h>
#include <stdlib.h>

#include "api_internal.h"
#include "common.cuh"
#include "umma.cuh"
#include "umma_epi.cuh"
#include "umma_pair.cuh"

namespace cgh {

// Grid: x = 2 x (column blocks of BNP), y = row blocks of 256; clusters of
// two CTAs along x.  MODE 0: store D; MODE 1: the fused adjoint epilogue of
// umma_epi.cuh over the pair's BNP columns (column tile blockIdx.x / 2).
template <int BNP, bool SPLIT, int STAGES, int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(192, 1)
umma_pair_kernel(const __grid_constant__ CUtensorMap tA,
                 const __grid_constant__ CUtensorMap tB,
                 const __grid_constant__ CUtensorMap tA2,
                 const __grid_constant__ CUtensorMap tB2, GemmArgs g,
                 AdjEpiArgs ea, uint32_t idesc) {
    using S = PairShape<BNP, SPLIT, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES];   // (even CTA) both halves landed
    __shared__ __align__(8) uint64_t empty[STAGES];
    __shared__ __align__(8) uint64_t accum_bar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t rank = umma2::cluster_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * 2 * S::BM + (int)rank * S::BM;  // this CTA's rows
    const int np0 = (blockIdx.x >> 1) * BNP;                     // the pair's columns
    const int nb = np0 + (int)rank * S::BNH;                     // this CTA's B rows
    const int KB = (g.K + S::BK - 1) / S::BK;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accum_bar, 1);
        mbar_fence_init();
        umma::prefetch_tmap(&tA);
        umma::prefetch_tmap(&tB);
        if (SPLIT) {
            umma::prefetch_tmap(&tA2);
            umma::prefetch_tmap(&tB2);
        }
    }
    if (warp == 1) {
        umma2::tmem_alloc2(&tmem_base, S::TMEM_COLS);
        umma2::tmem_relinquish2();
    }
    umma::fence_before_sync();
    umma2::cluster_sync();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_base;
    pdl_wait();  // operands come from (and D may be read by) the kernel before

    if (warp == 0 && lane == 0) {
        // ------------------------------------------ producer (both CTAs)
        int issued = 0;
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES &&
                !mbar_wait_bounded(&empty[s], (uint32_t)(((kb / STAGES) - 1) & 1))) {
                abort_flag = 1;
                set_status(g.status, DEV_TIMEOUT);
            }
            if (abort_flag) break;
            uint8_t *st = smem + (size_t)s * S::STAGE_BYTES;
            // the even CTA's barrier counts the bytes of both CTAs' loads
            if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * S::STAGE_BYTES);
            const uint32_t bar = umma2::map_to_rank(&full[s], 0);
            umma2::tma_load_2d_pair(st, &tA, kb * S::BK, m0, bar);
            umma2::tma_load_2d_pair(st + S::A_BYTES, &tB, kb * S::BK, nb, bar);
            if (SPLIT) {
                umma2::tma_load_2d_pair(st + S::A_BYTES + S::B_BYTES, &tA2, kb * S::BK,
                                        m0, bar);
                umma2::tma_load_2d_pair(st + 2 * S::A_BYTES + S::B_BYTES, &tB2,
                                        kb * S::BK, nb, bar);
            }
            ++issued;
        }
        if (abort_flag && rank == 0) {
            // let the stages' copies land before shared memory goes: their
            // barriers are here (the odd CTA cannot see its own loads'
            // completion; it leaves only after the closing cluster barrier)
            for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb)
                mbar_wait_bounded(&full[kb % STAGES], (uint32_t)((kb / STAGES) & 1));
        } else if (!abort_flag) {
            // The MMA issuer's commits of the last stages arrive on this
            // CTA's empty barriers asynchronously (multicast to both CTAs),
            // and nothing else waits for them: wait here (bounded), so that
            // no arrive is still in flight when the CTA exits and its shared
            // memory passes to the next CTA on the SM.
            for (int kb = KB - STAGES < 0 ? 0 : KB - STAGES; kb < KB; ++kb)
                mbar_wait_bounded(&empty[kb % STAGES], (uint32_t)((kb / STAGES) & 1));
        }
    } else if (warp == 1 && lane == 0) {
        if (rank == 0) {
            // ---------------------------------------- MMA issuer (even CTA)
            int done = 0;
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % STAGES;
                const uint32_t par = (uint32_t)((kb / STAGES) & 1);
                if (!umma2::wait_cluster_bounded(&full[s], par)) {
                    abort_flag = 1;
                    set_status(g.status, DEV_TIMEOUT);
                }
                if (abort_flag) break;
                umma::fence_after_sync();
                const uint32_t a = smem_u32(smem + (size_t)s * S::STAGE_BYTES);
                const uint32_t b = a + S::A_BYTES;
                const uint64_t ad = umma::sw128_kmajor_desc(a);
                const uint64_t bd = umma::sw128_kmajor_desc(b);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma2::mma2_f16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0);
                if (SPLIT) {
                    const uint32_t a2 = b + S::B_BYTES, b2 = a2 + S::A_BYTES;
                    const uint64_t ad2 = umma::sw128_kmajor_desc(a2);
                    const uint64_t bd2 = umma::sw128_kmajor_desc(b2);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma2::mma2_f16(tmem + S::ACC1, ad + 2 * kk, bd2 + 2 * kk, idesc,
                                        (kb | kk) != 0);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma2::mma2_f16(tmem + S::ACC1, ad2 + 2 * kk, bd + 2 * kk, idesc, 1);
                }
                umma2::commit2(&empty[s], 0x3);
                ++done;
            }
            // both CTAs' accumulators are complete -- or, after a timeout,
            // only this CTA learns that its MMAs in flight have finished (the
            // odd CTA's epilogue wait then runs out and skips its store)
            umma2::commit2(&accum_bar, done == KB ? 0x3 : 0x1);
        }
    } else if (warp >= 2) {
        // --------------------------------------- epilogue (both CTAs)
        const int q = warp & 3;  // the 32-lane quarter of TMEM this warp reads
        const int row = m0 + q * 32 + lane;
        const bool ok = __all_sync(0xffffffffu, umma2::wait_cluster_bounded(&accum_bar, 0));
        umma::fence_after_sync();
        pdl_trigger();  // only the epilogue is left
        if (!ok) set_status(g.status, DEV_TIMEOUT);
        if (MODE == 1 && ok && !abort_flag) {
            adjoint_epilogue<BNP, SPLIT, S::ACC1>(tmem + ((uint32_t)(q * 32) << 16), row,
                                                  np0, g, ea, lane, blockIdx.x >> 1);
        } else if (ok && !abort_flag) {
            const uint32_t t_row = tmem + ((uint32_t)(q * 32) << 16);
            float *drow = g.D + (long long)row * g.ldd;
            const bool vec = ((g.ldd & 3) == 0) && ((((uintptr_t)g.D) & 15) == 0);
            constexpr int CH = S::CH;
#pragma unroll 1
            for (int c = 0; c < BNP; c += CH) {
                uint32_t r[CH];
                float v[CH];
                if constexpr (CH == 32) umma::tmem_ld32(t_row + c, r);
                else umma::tmem_ld16(t_row + c, r);
                if (SPLIT) {
                    uint32_t r2[CH];
                    if constexpr (CH == 32) umma::tmem_ld32(t_row + S::ACC1 + c, r2);
                    else umma::tmem_ld16(t_row + S::ACC1 + c, r2);
                    umma::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        v[i] = fmaf(g.lo_scale, __uint_as_float(r2[i]),
                                    __uint_as_float(r[i]));
                } else {
                    umma::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < CH; ++i) v[i] = __uint_as_float(r[i]);
                }
                if (row < g.M) epilogue_store_row<CH>(drow, np0 + c, v, g, vec);
            }
        }
    }
    umma::fence_before_sync();
    umma2::cluster_sync();  // no MMA, commit or relayed arrive still aims at either CTA
    if (warp == 1) {
        umma::fence_after_sync();
        umma2::tmem_dealloc2(tmem, S::TMEM_COLS);
    }
}

// ------------------------------------------------------------- host side
bool make_gemm_map(CUtensorMap *m, const void *base, long long inner, long long rows,
                   long long ld, int box_rows, bool bf16);

template <int BNP, bool SPLIT, int STAGES, int MODE = 0>
static cudaError_t launch_pair_t(const GemmOperands &op, unsigned *status,
                                 cudaStream_t s, const AdjEpiArgs &ea = AdjEpiArgs{}) {
    using S = PairShape<BNP, SPLIT, STAGES>;
    CUtensorMap tA, tB, tA2, tB2;
    if (!make_gemm_map(&tA, op.A_hi, op.K, op.M, op.lda, S::BM, op.bf16) ||
        !make_gemm_map(&tB, op.B_hi, op.K, op.N, op.ldb, S::BNH, op.bf16))
        return cudaErrorInvalidValue;
    if (SPLIT) {
        if (!make_gemm_map(&tA2, op.A_lo, op.K, op.M, op.lda, S::BM, op.bf16) ||
            !make_gemm_map(&tB2, op.B_lo, op.K, op.N, op.ldb, S::BNH, op.bf16))
            return cudaErrorInvalidValue;
    } else {
        tA2 = tA;
        tB2 = tB;
    }
    auto kern = umma_pair_kernel<BNP, SPLIT, STAGES, MODE>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    GemmArgs g{op.M, op.N, op.K, op.D, op.ldd, op.lo_scale, status, op.accumulate};
    dim3 grid(2 * ((op.N + BNP - 1) / BNP), (op.M + 2 * S::BM - 1) / (2 * S::BM));
    const uint32_t idesc = umma::idesc_f16(2 * S::BM, BNP, op.bf16);
    return launch_dependent(kern, grid, dim3(192), S::SMEM, s, tA, tB, tA2, tB2, g, ea,
                            idesc);
}

// The pair widths compiled in (columns of one 256-row pair tile).
static const int kPairBN[] = {112, 144, 160, 224, 256};

// Cost of a pair width: SM waves x columns per CTA (the work of one CTA is
// proportional to its columns), with a small preference for wide tiles.
double pair_cost(int M, int N, int bnp, int sms) {
    const long long ctas = 2LL * ((M + 255) / 256) * ((N + bnp - 1) / bnp);
    return (double)((ctas + sms - 1) / sms) * bnp / (1.0 + 0.002 * bnp);
}

bool pair_width_ok(int bnp) {
    for (int w : kPairBN)
        if (w == bnp) return true;
    return false;
}

int pick_pair_n(int M, int N, int sms, double *cost) {
    int best = kPairBN[0];
    double best_cost = 1e300;
    for (int bnp : kPairBN) {
        const double c = pair_cost(M, N, bnp, sms);
        if (c < best_cost) {
            best_cost = c;
            best = bnp;
        }
    }
    if (cost) *cost = best_cost;
    return best;
}

// Stages: as many as fit in shared memory (the loads' latency is hidden by
// the bytes in flight).
cudaError_t launch_umma_pair(const GemmOperands &op, int bnp, unsigned *status,
                             cudaStream_t s) {
    static const int forced = [] {
        const char *f = getenv("CGH_PAIR_BN");
        return f ? atoi(f) : 0;
    }();
    if (forced) bnp = forced;
    if (op.split) {
        switch (bnp) {
        case 112: return launch_pair_t<112, true, 4>(op, status, s);
        case 144: return launch_pair_t<144, true, 4>(op, status, s);
        case 160: return launch_pair_t<160, true, 4>(op, status, s);
        case 224: return launch_pair_t<224, true, 3>(op, status, s);
        case 256: return launch_pair_t<256, true, 3>(op, status, s);
        }
    } else {
        switch (bnp) {
        case 112: return launch_pair_t<112, false, 9>(op, status, s);
        case 144: return launch_pair_t<144, false, 8>(op, status, s);
        case 160: return launch_pair_t<160, false, 8>(op, status, s);
        case 224: return launch_pair_t<224, false, 7>(op, status, s);
        case 256: return launch_pair_t<256, false, 7>(op, status, s);
        }
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------ grouped (batch), pairs
// The persistent grouped split GEMM of the batch on CTA pairs: clusters of
// two CTAs take work items (problem, 256-row tile, 128-column tile) round
// robin; per SM 128 rows of A and 64 rows of B per stage.  Two TMEM
// accumulator buffers (hi*hi and cross terms, 256 columns each) let the
// epilogue of one item overlap the MMAs of the next.  The even CTA's
// `acc_empty` barrier collects one arrival from each of the 8 epilogue warps
// of the pair (the odd CTA's arrive remotely) before that buffer is reused.
constexpr int GP_BN = 128, GP_STAGES = 4;

template <int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(192, 1)
umma_grouped_pair_kernel(const GroupProb *__restrict__ probs,
                         const uint2 *__restrict__ items, int nitems,
                         unsigned *status) {
    using S = PairShape<GP_BN, true, STAGES>;
    constexpr uint32_t ACC_COLS = 2 * GP_BN;        // hi*hi and cross terms
    constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;    // two buffers
    static_assert(TMEM_COLS <= 512, "TMEM");
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES];
    __shared__ __align__(8) uint64_t empty[STAGES];
    __shared__ __align__(8) uint64_t acc_full[2];
    __shared__ __align__(8) uint64_t acc_empty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t rank = umma2::cluster_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 8);  // 4 epilogue warps in each CTA
        }
        mbar_fence_init();
    }
    if (warp == 1) {
        umma2::tmem_alloc2(&tmem_base, TMEM_COLS);
        umma2::tmem_relinquish2();
    }
    umma::fence_before_sync();
    umma2::cluster_sync();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------ producer (both CTAs)
        unsigned g = 0, issued_from = 0;
        for (int it = cl; it < nitems && !abort_flag; it += ncl) {
            const uint2 w = items[it];
            const GroupProb *gp = probs + w.x;
            const int m0 = (int)(w.y & 0xffffu) * 2 * S::BM + (int)rank * S::BM;
            const int nb = (int)(w.y >> 16) * GP_BN + (int)rank * S::BNH;
            const int KB = (gp->K + S::BK - 1) / S::BK;
            for (int kb = 0; kb < KB; ++kb, ++g) {
                const int s = (int)(g % STAGES);
                if (g >= STAGES &&
                    !mbar_wait_bounded(&empty[s], (uint32_t)(((g / STAGES) - 1) & 1))) {
                    abort_flag = 1;
                    set_status(status, DEV_TIMEOUT);
                }
                if (abort_flag) break;
                uint8_t *st = smem + (size_t)s * S::STAGE_BYTES;
                if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * S::STAGE_BYTES);
                const uint32_t bar = umma2::map_to_rank(&full[s], 0);
                umma2::tma_load_2d_pair(st, &gp->tA, kb * S::BK, m0, bar);
                umma2::tma_load_2d_pair(st + S::A_BYTES, &gp->tB, kb * S::BK, nb, bar);
                umma2::tma_load_2d_pair(st + S::A_BYTES + S::B_BYTES, &gp->tA2,
                                        kb * S::BK, m0, bar);
                umma2::tma_load_2d_pair(st + 2 * S::A_BYTES + S::B_BYTES, &gp->tB2,
                                        kb * S::BK, nb, bar);
                issued_from = g + 1;
            }
        }
        if (abort_flag && rank == 0) {
            const unsigned lo = issued_from > STAGES ? issued_from - STAGES : 0;
            for (unsigned u = lo; u < issued_from; ++u)
                mbar_wait_bounded(&full[u % STAGES], (uint32_t)((u / STAGES) & 1));
        } else if (!abort_flag) {
            // The MMA issuer's commits of the last stages arrive on this
            // CTA's empty barriers asynchronously (multicast to both CTAs),
            // and nothing else waits for them: wait here (bounded), so that
            // no arrive is still in flight when the CTA exits and its shared
            // memory passes to the next CTA on the SM.
            const unsigned lo = g > STAGES ? g - STAGES : 0;
            for (unsigned u = lo; u < g; ++u)
                mbar_wait_bounded(&empty[u % STAGES], (uint32_t)((u / STAGES) & 1));
        }
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // ---------------------------------------- MMA issuer (even CTA)
        const uint32_t idesc = umma::idesc_f16(2 * S::BM, GP_BN, false);
        unsigned g = 0;
        int n = 0;
        for (int it = cl; it < nitems && !abort_flag; it += ncl, ++n) {
            const int b = n & 1;
            if (!umma2::wait_cluster_bounded(&acc_empty[b],
                                             (uint32_t)(((n >> 1) & 1) ^ 1))) {
                abort_flag = 1;
                set_status(status, DEV_TIMEOUT);
                break;
            }
            umma::fence_after_sync();
            const uint32_t d0 = tmem + (uint32_t)b * ACC_COLS, d1 = d0 + GP_BN;
            const GroupProb *gp = probs + items[it].x;
            const int KB = (gp->K + S::BK - 1) / S::BK;
            bool ok = true;
            for (int kb = 0; kb < KB; ++kb, ++g) {
                const int s = (int)(g % STAGES);
                if (!umma2::wait_cluster_bounded(&full[s], (uint32_t)((g / STAGES) & 1))) {
                    abort_flag = 1;
                    set_status(status, DEV_TIMEOUT);
                    ok = false;
                    break;
                }
                umma::fence_after_sync();
                const uint32_t a = smem_u32(smem + (size_t)s * S::STAGE_BYTES);
                const uint32_t bb = a + S::A_BYTES;
                const uint32_t a2 = bb + S::B_BYTES, b2 = a2 + S::A_BYTES;
                const uint64_t ad = umma::sw128_kmajor_desc(a);
                const uint64_t bd = umma::sw128_kmajor_desc(bb);
                const uint64_t ad2 = umma::sw128_kmajor_desc(a2);
                const uint64_t bd2 = umma::sw128_kmajor_desc(b2);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma2::mma2_f16(d0, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma2::mma2_f16(d1, ad + 2 * kk, bd2 + 2 * kk, idesc, (kb | kk) != 0);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma2::mma2_f16(d1, ad2 + 2 * kk, bd + 2 * kk, idesc, 1);
                umma2::commit2(&empty[s], 0x3);
            }
            // a timed-out item is not handed to the odd CTA's epilogue (its
            // wait runs out); this CTA's epilogue learns that its MMAs ended
            umma2::commit2(&acc_full[b], ok ? 0x3 : 0x1);
        }
    } else if (warp >= 2) {
        // --------------------------------------- epilogue (both CTAs)
        const int q = warp & 3;
        const uint32_t lead_empty0 = umma2::map_to_rank(&acc_empty[0], 0);
        int n = 0;
        for (int it = cl; it < nitems; it += ncl, ++n) {
            const int b = n & 1;
            const bool ok = __all_sync(
                0xffffffffu,
                umma2::wait_cluster_bounded(&acc_full[b], (uint32_t)((n >> 1) & 1)));
            umma::fence_after_sync();
            if (!ok || abort_flag) {
                if (!ok) set_status(status, DEV_TIMEOUT);
                break;
            }
            const uint2 w = items[it];
            const GroupProb *gp = probs + w.x;
            const int m0 = (int)(w.y & 0xffffu) * 2 * S::BM + (int)rank * S::BM;
            const int n0 = (int)(w.y >> 16) * GP_BN;
            const int row = m0 + q * 32 + lane;
            const int M = gp->M, Ncols = gp->N;
            const long long ldd = gp->ldd;
            const float los = gp->lo_scale;
            float *drow = gp->D + (long long)row * ldd;
            const bool vec = ((ldd & 3) == 0) && ((((uintptr_t)gp->D) & 15) == 0);
            const uint32_t t_row =
                tmem + (uint32_t)b * ACC_COLS + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
            for (int c = 0; c < GP_BN; c += 32) {
                uint32_t r[32], r2[32];
                umma::tmem_ld32(t_row + c, r);
                umma::tmem_ld32(t_row + GP_BN + c, r2);
                umma::tmem_ld_wait();
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    v[i] = fmaf(los, __uint_as_float(r2[i]), __uint_as_float(r[i]));
                if (row < M) {
                    const int col = n0 + c;
                    if (vec && col + 32 <= Ncols) {
#pragma unroll
                        for (int i = 0; i < 32; i += 4)
                            *reinterpret_cast<float4 *>(drow + col + i) =
                                make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (col + i < Ncols) drow[col + i] = v[i];
                    }
                }
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) umma2::remote_arrive(lead_empty0 + (uint32_t)b * 8u);
        }
    }
    umma::fence_before_sync();
    umma2::cluster_sync();
    if (warp == 1) {
        umma::fence_after_sync();
        umma2::tmem_dealloc2(tmem, TMEM_COLS);
    }
}

cudaError_t prepare_umma_grouped_pair() {
    using S = PairShape<GP_BN, true, GP_STAGES>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(umma_grouped_pair_kernel<GP_STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::SMEM);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

cudaError_t launch_umma_grouped_pair(const GroupProb *probs, const uint2 *items,
                                     int nitems, unsigned *status, int sm_count,
                                     cudaStream_t s) {
    using S = PairShape<GP_BN, true, GP_STAGES>;
    if (nitems <= 0) return cudaSuccess;
    const int clusters = nitems < sm_count / 2 ? nitems : sm_count / 2;
    umma_grouped_pair_kernel<GP_STAGES><<<2 * (clusters > 0 ? clusters : 1), 192,
                                          S::SMEM, s>>>(probs, items, nitems, status);
    return cudaGetLastError();
}

int group_pair_tile_m() { return 2 * 128; }
int group_pair_tile_n() { return GP_BN; }
int group_pair_box_b() { return GP_BN / 2; }

// The adjoint GEMMs (split, fused epilogue) on CTA pairs: width from
// {160, 224, 256} (the epilogue walks its columns 32 at a time); the column
// tile width is returned in *tile_n (partial sums per tile of that width).
cudaError_t launch_umma_pair_adjoint(const GemmOperands &op, const AdjEpiArgs &ea,
                                     int sms, unsigned *status, cudaStream_t s,
                                     int *tile_n) {
    int best = 256;
    double best_cost = 1e300;
    for (int bnp : {160, 224, 256}) {
        const double c = pair_cost(op.M, op.N, bnp, sms) / (1.0 + 0.002 * bnp);
        if (c < best_cost) {
            best_cost = c;
            best = bnp;
        }
    }
    *tile_n = best;
    switch (best) {
    case 160: return launch_pair_t<160, true, 4, 1>(op, status, s, ea);
    case 224: return launch_pair_t<224, true, 3, 1>(op, status, s, ea);
    default: return launch_pair_t<256, true, 3, 1>(op, status, s, ea);
    }
}

}  // namespace cgh
