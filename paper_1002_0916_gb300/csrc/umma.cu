// umma.cu -- the tensor-core GEMM of the separable methods (step A7):
//
//     D[m][n] = sum_k A[m][k] B[n][k]                      (single pass)
//     D[m][n] = sum_k Ahi Bhi + s * (Ahi Blo + Alo Bhi)    (split, s = 2^-12)
//
// A, B: 16-bit (FP16 or BF16), K-major; D: FP32 row-major.
//
// One CTA computes a 128 x BN tile of D with tcgen05.mma (kind::f16,
// cta_group::1) accumulating in tensor memory (TMEM).  Warp roles:
//   warp 0      TMA producer: 2-D tiled loads (128-byte swizzle) of the
//               K-blocks of A and B into a STAGES-deep shared-memory ring,
//               completing on `full` mbarriers;
//   warp 1      allocates TMEM; its lane 0 issues the MMAs (4 per 64-wide
//               K-block per product) and releases ring slots through
//               tcgen05.commit -> `empty` mbarriers;
//   warps 2..5  epilogue: tcgen05.ld of the accumulator(s), combine, store.
// The split form keeps two accumulators (hi*hi and the two cross terms),
// so the lo planes can be stored pre-scaled by 2^12 and stay normal FP16
// numbers; the epilogue adds them back with the factor 2^-12.
// Every mbarrier wait is bounded; a timeout raises DEV_TIMEOUT, the CTA
// skips its store, waits (bounded) for its own copies, frees TMEM and exits.
#include <cudaTypedefs.h>

#include <mutex>

#include "api_internal.h"
#include "common.cuh"
#include "umma.cuh"
#include "umma_epi.cuh"

namespace cgh {

template <int BN, bool SPLIT, int STAGES>
struct GemmShape {
    static constexpr int BM = 128, BK = 64;
    static constexpr uint32_t A_BYTES = BM * BK * 2;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
    static constexpr uint32_t STAGE_BYTES =
        SPLIT ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
    // second accumulator (split form) on a 128-column boundary
    static constexpr uint32_t ACC1 = BN <= 128 ? 128 : BN;
    static constexpr uint32_t ACC_COLS = SPLIT ? ACC1 + BN : BN;
    // TMEM allocations are powers of two of at least 32 columns
    static constexpr uint32_t TMEM_COLS =
        ACC_COLS <= 32 ? 32 : ACC_COLS <= 64 ? 64 : ACC_COLS <= 128 ? 128
        : ACC_COLS <= 256 ? 256 : 512;
    // epilogue column chunk: 32 columns, or 16 when BN is not a multiple of 32
    static constexpr int CH = BN % 32 == 0 ? 32 : 16;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "UMMA N");
    static_assert(ACC_COLS <= 512, "TMEM");
    static_assert(TMEM_COLS == 64 || TMEM_COLS == 128 || TMEM_COLS == 256 ||
                      TMEM_COLS == 512,
                  "TMEM allocation must be a power of two >= 32 columns");
    static_assert(SMEM <= 232448, "shared memory");
};

template <int BN, bool SPLIT, int STAGES, int MODE>
__global__ void __launch_bounds__(192, 1)
umma_gemm_kernel(const __grid_constant__ CUtensorMap tA,
                 const __grid_constant__ CUtensorMap tB,
                 const __grid_constant__ CUtensorMap tA2,
                 const __grid_constant__ CUtensorMap tB2, GemmArgs g,
                 AdjEpiArgs ea, uint32_t idesc) {
    using S = GemmShape<BN, SPLIT, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES];
    __shared__ __align__(8) uint64_t empty[STAGES];
    __shared__ __align__(8) uint64_t accum_bar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * S::BM;
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
        umma::tmem_alloc(&tmem_base, S::TMEM_COLS);
        umma::tmem_relinquish();
    }
    pdl_wait();  // operands come from the kernel before
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------- producer
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
            mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
            umma::tma_load_2d(st, &tA, kb * S::BK, m0, &full[s]);
            umma::tma_load_2d(st + S::A_BYTES, &tB, kb * S::BK, n0, &full[s]);
            if (SPLIT) {
                umma::tma_load_2d(st + S::A_BYTES + S::B_BYTES, &tA2, kb * S::BK,
                                  m0, &full[s]);
                umma::tma_load_2d(st + 2 * S::A_BYTES + S::B_BYTES, &tB2,
                                  kb * S::BK, n0, &full[s]);
            }
            ++issued;
        }
        if (abort_flag) {
            // let this CTA's own copies land before its shared memory goes
            for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb)
                mbar_wait_bounded(&full[kb % STAGES], (uint32_t)((kb / STAGES) & 1));
        } else {
            // The MMA issuer's commits of the last stages arrive on this
            // CTA's empty barriers asynchronously, and nothing else waits for
            // them: wait here (bounded), so that no arrive is still in flight
            // when the CTA exits and its shared memory passes to the next CTA
            // on the SM.
            for (int kb = KB - STAGES < 0 ? 0 : KB - STAGES; kb < KB; ++kb)
                mbar_wait_bounded(&empty[kb % STAGES], (uint32_t)((kb / STAGES) & 1));
        }
    } else if (warp == 1 && lane == 0) {
        // --------------------------------------------------- MMA issuer
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait_bounded(&full[s], (uint32_t)((kb / STAGES) & 1))) {
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
                umma::mma_f16(tmem, ad + 2 * kk, bd + 2 * kk, idesc,
                              (kb | kk) != 0);
            if (SPLIT) {
                const uint32_t a2 = b + S::B_BYTES, b2 = a2 + S::A_BYTES;
                const uint64_t ad2 = umma::sw128_kmajor_desc(a2);
                const uint64_t bd2 = umma::sw128_kmajor_desc(b2);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma::mma_f16(tmem + S::ACC1, ad + 2 * kk, bd2 + 2 * kk, idesc,
                                  (kb | kk) != 0);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma::mma_f16(tmem + S::ACC1, ad2 + 2 * kk, bd + 2 * kk, idesc, 1);
            }
            umma::mma_commit(&empty[s]);
        }
        umma::mma_commit(&accum_bar);  // fires once every issued MMA is done
    } else if (warp >= 2) {
        // ----------------------------------------------------- epilogue
        const int q = warp & 3;  // the 32-lane quarter of TMEM this warp reads
        const int row = m0 + q * 32 + lane;
        // warp-uniform, so the .sync.aligned TMEM loads and the shuffles
        // below are executed by whole warps
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&accum_bar, 0));
        umma::fence_after_sync();
        pdl_trigger();  // only the epilogue is left
        if (!ok) set_status(g.status, DEV_TIMEOUT);
        if (MODE == 1 && ok && !abort_flag) {
            adjoint_epilogue<BN, SPLIT, S::ACC1>(tmem + ((uint32_t)(q * 32) << 16),
                                                 row, n0, g, ea, lane, blockIdx.x);
        } else if (ok && !abort_flag) {
            const uint32_t t_row = tmem + ((uint32_t)(q * 32) << 16);
            float *drow = g.D + (long long)row * g.ldd;
            const bool vec = ((g.ldd & 3) == 0) && ((((uintptr_t)g.D) & 15) == 0);
            constexpr int CH = S::CH;
#pragma unroll 1
            for (int c = 0; c < BN; c += CH) {
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
                if (row < g.M) epilogue_store_row<CH>(drow, n0 + c, v, g, vec);
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, S::TMEM_COLS);
    }
}

// ------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a rows x inner matrix of 16-bit elements (row stride `ld`
// elements), box = 64 elements x box_rows rows, 128-byte swizzle, zero fill.
static bool make_map(CUtensorMap *m, const void *base, long long inner,
                     long long rows, long long ld, int box_rows, bool bf16) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                    2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_gemm_map(CUtensorMap *m, const void *base, long long inner, long long rows,
                   long long ld, int box_rows, bool bf16) {
    return make_map(m, base, inner, rows, ld, box_rows, bf16);
}

bool make_f32_map(CUtensorMap *m, const void *base, long long inner, long long rows,
                  long long ld, int box_inner, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, bool SPLIT, int STAGES, int MODE>
static cudaError_t launch_gemm_t(const GemmOperands &op, const AdjEpiArgs &ea,
                                 unsigned *status, cudaStream_t s) {
    using S = GemmShape<BN, SPLIT, STAGES>;
    CUtensorMap tA, tB, tA2, tB2;
    if (!make_map(&tA, op.A_hi, op.K, op.M, op.lda, S::BM, op.bf16) ||
        !make_map(&tB, op.B_hi, op.K, op.N, op.ldb, BN, op.bf16))
        return cudaErrorInvalidValue;
    if (SPLIT) {
        if (!make_map(&tA2, op.A_lo, op.K, op.M, op.lda, S::BM, op.bf16) ||
            !make_map(&tB2, op.B_lo, op.K, op.N, op.ldb, BN, op.bf16))
            return cudaErrorInvalidValue;
    } else {
        tA2 = tA;
        tB2 = tB;
    }
    auto kern = umma_gemm_kernel<BN, SPLIT, STAGES, MODE>;
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
    dim3 grid((op.N + BN - 1) / BN, (op.M + S::BM - 1) / S::BM);
    const uint32_t idesc = umma::idesc_f16(S::BM, BN, op.bf16);
    return launch_dependent(kern, grid, dim3(192), S::SMEM, s, tA, tB, tA2, tB2, g,
                            ea, idesc);
}

bool gemm_operands_ok(const GemmOperands &op) {
    if (op.M < 1 || op.N < 1 || op.K < 1) return false;
    if (op.lda < op.K || op.ldb < op.K || op.lda % 8 || op.ldb % 8) return false;
    if (op.ldd < op.N) return false;
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (!al16(op.A_hi) || !al16(op.B_hi)) return false;
    if (op.split && (!al16(op.A_lo) || !al16(op.B_lo))) return false;
    if (((uintptr_t)op.D & 3) != 0) return false;
    if (op.M > (1 << 30) || op.N > (1 << 30)) return false;
    return true;
}

static int sm_count_of_current_device() {
    static int cache[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        n = 148;
    }
    if (dev >= 0 && dev < 64) cache[dev] = n;
    return n;
}

// One CTA per tile, one tile per SM at a time: the GEMM takes about
// ceil(tiles / SMs) x (work of one tile).  A 112-column tile does 7/8 of the
// work of a 128-column one and can fill the SMs better (1920 columns x 1024
// rows: 144 tiles of 112 on 152 SMs instead of 120 of 128).
static int pick_tile_n(int M, int N, int sms) {
    auto cost = [&](int bn) {
        long long tiles = (long long)((M + 127) / 128) * ((N + bn - 1) / bn);
        return (double)((tiles + sms - 1) / sms) * bn;
    };
    return cost(112) < cost(128) ? 112 : 128;
}

GemmPlan gemm_plan(int M, int N, int tiles, int sms, int kind, int bn) {
    // CTA pairs halve each SM's operand bytes per multiply-add; measured on
    // the 3840 x 2160 x 16384 product 1.9x (single pass) and 1.3x (split)
    // faster than one-CTA tiles, equal at 1920 x 1024 x 1024.  A frame of
    // at most 128 rows would leave half of every pair tile empty.
    if (tiles == CGH_GEMM_PAIRS_GEN)
        return GemmPlan{CGH_GEMM_PAIRS_GEN,
                        gen_pair_width_ok(kind, bn) ? bn : pick_gen_n(M, N, sms, kind)};
    const bool pairs = tiles == CGH_GEMM_PAIRS || (tiles == CGH_GEMM_AUTO && M > 128);
    if (!pairs)
        return GemmPlan{CGH_GEMM_SINGLE, (bn == 112 || bn == 128) ? bn : pick_tile_n(M, N, sms)};
    return GemmPlan{CGH_GEMM_PAIRS, pair_width_ok(bn) ? bn : pick_pair_n(M, N, sms)};
}

cudaError_t launch_umma_gemm(const GemmOperands &op, unsigned *status,
                             cudaStream_t s) {
    if (!gemm_operands_ok(op)) return cudaErrorInvalidValue;
    const int chunk = gemm_k_chunk(op.split);
    if (op.K > chunk) {
        // consecutive launches over K chunks, the later ones adding into D
        for (int k0 = 0; k0 < op.K; k0 += chunk) {
            GemmOperands c = op;
            const size_t off = (size_t)k0 * 2;  // bytes of 16-bit elements
            c.K = op.K - k0 < chunk ? op.K - k0 : chunk;
            c.A_hi = (const char *)op.A_hi + off;
            c.B_hi = (const char *)op.B_hi + off;
            if (op.split) {
                c.A_lo = (const char *)op.A_lo + off;
                c.B_lo = (const char *)op.B_lo + off;
            }
            c.accumulate = op.accumulate || k0 > 0;
            cudaError_t e = launch_umma_gemm(c, status, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    AdjEpiArgs ea{};
    const GemmPlan plan = gemm_plan(op.M, op.N, op.tiles, sm_count_of_current_device(),
                                    op.bf16 ? 0 : op.split ? 2 : 1, op.bn);
    if (plan.tiling == CGH_GEMM_PAIRS) return launch_umma_pair(op, plan.bn, status, s);
    const int bn = plan.bn;
    if (op.split)
        return bn == 112 ? launch_gemm_t<112, true, 3, 0>(op, ea, status, s)
                         : launch_gemm_t<128, true, 3, 0>(op, ea, status, s);
    return bn == 112 ? launch_gemm_t<112, false, 6, 0>(op, ea, status, s)
                     : launch_gemm_t<128, false, 6, 0>(op, ea, status, s);
}

cudaError_t launch_umma_adjoint(const GemmOperands &op, const PointRec *rec,
                                const float *points, int npoints, int npad,
                                int axis, float *part, unsigned *status,
                                cudaStream_t s, int *tile_n) {
    if (!gemm_operands_ok(op) || !op.split || (op.M & 1)) return cudaErrorInvalidValue;
    AdjEpiArgs ea{rec, points, npoints, npad, axis, part};
    const bool pairs = op.tiles == CGH_GEMM_PAIRS ||
                       (op.tiles == CGH_GEMM_AUTO && op.M > 128);
    if (pairs)
        return launch_umma_pair_adjoint(op, ea, sm_count_of_current_device(), status, s,
                                        tile_n);
    *tile_n = 128;
    return launch_gemm_t<128, true, 3, 1>(op, ea, status, s);
}

int umma_tile_n() { return 128; }

// ------------------------------------------------------ grouped (batch)
// Persistent grouped split GEMM: work items (problem, m tile, n tile) are
// taken round-robin by the CTAs (one per SM) in the order of a host list
// sorted longest-K first.  The producer and MMA roles run ahead across
// items; two TMEM accumulator buffers let the epilogue of item i overlap
// the main loop of item i + 1 (acc_full / acc_empty mbarriers).
template <int BN, int STAGES>
__global__ void __launch_bounds__(192, 1)
umma_grouped_kernel(const GroupProb *__restrict__ probs,
                    const uint2 *__restrict__ items, int nitems,
                    unsigned *status) {
    using S = GemmShape<BN, true, STAGES>;
    constexpr uint32_t ACC_COLS = 2 * BN;          // hi*hi and cross terms
    constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;   // two buffers
    static_assert(TMEM_COLS <= 512, "TMEM");
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES];
    __shared__ __align__(8) uint64_t empty[STAGES];
    __shared__ __align__(8) uint64_t acc_full[2];
    __shared__ __align__(8) uint64_t acc_empty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
        }
        mbar_fence_init();
    }
    if (warp == 1) {
        umma::tmem_alloc(&tmem_base, TMEM_COLS);
        umma::tmem_relinquish();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------- producer
        unsigned g = 0, issued_from = 0;
        for (int it = blockIdx.x; it < nitems && !abort_flag; it += gridDim.x) {
            const uint2 w = items[it];
            const GroupProb *gp = probs + w.x;
            const int m0 = (int)(w.y & 0xffffu) * S::BM, n0 = (int)(w.y >> 16) * BN;
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
                mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
                umma::tma_load_2d(st, &gp->tA, kb * S::BK, m0, &full[s]);
                umma::tma_load_2d(st + S::A_BYTES, &gp->tB, kb * S::BK, n0, &full[s]);
                umma::tma_load_2d(st + S::A_BYTES + S::B_BYTES, &gp->tA2, kb * S::BK,
                                  m0, &full[s]);
                umma::tma_load_2d(st + 2 * S::A_BYTES + S::B_BYTES, &gp->tB2,
                                  kb * S::BK, n0, &full[s]);
                issued_from = g + 1;
            }
        }
        if (abort_flag) {
            unsigned lo = issued_from > STAGES ? issued_from - STAGES : 0;
            for (unsigned u = lo; u < issued_from; ++u)
                mbar_wait_bounded(&full[u % STAGES], (uint32_t)((u / STAGES) & 1));
        } else {
            // The MMA issuer's commits of the last stages arrive on this
            // CTA's empty barriers asynchronously, and nothing else waits for
            // them: wait here (bounded), so that no arrive is still in flight
            // when the CTA exits and its shared memory passes to the next CTA
            // on the SM.
            const unsigned lo = g > STAGES ? g - STAGES : 0;
            for (unsigned u = lo; u < g; ++u)
                mbar_wait_bounded(&empty[u % STAGES], (uint32_t)((u / STAGES) & 1));
        }
    } else if (warp == 1 && lane == 0) {
        // --------------------------------------------------- MMA issuer
        const uint32_t idesc = umma::idesc_f16(S::BM, BN, false);
        unsigned g = 0;
        int n = 0;
        for (int it = blockIdx.x; it < nitems && !abort_flag; it += gridDim.x, ++n) {
            const int b = n & 1;
            if (!mbar_wait_bounded(&acc_empty[b], (uint32_t)(((n >> 1) & 1) ^ 1))) {
                abort_flag = 1;
                set_status(status, DEV_TIMEOUT);
                break;
            }
            umma::fence_after_sync();
            const uint32_t d0 = tmem + (uint32_t)b * ACC_COLS, d1 = d0 + BN;
            const GroupProb *gp = probs + items[it].x;
            const int KB = (gp->K + S::BK - 1) / S::BK;
            for (int kb = 0; kb < KB; ++kb, ++g) {
                const int s = (int)(g % STAGES);
                if (!mbar_wait_bounded(&full[s], (uint32_t)((g / STAGES) & 1))) {
                    abort_flag = 1;
                    set_status(status, DEV_TIMEOUT);
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
                    umma::mma_f16(d0, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma::mma_f16(d1, ad + 2 * kk, bd2 + 2 * kk, idesc, (kb | kk) != 0);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma::mma_f16(d1, ad2 + 2 * kk, bd + 2 * kk, idesc, 1);
                umma::mma_commit(&empty[s]);
            }
            umma::mma_commit(&acc_full[b]);
        }
    } else if (warp >= 2) {
        // ----------------------------------------------------- epilogue
        const int q = warp & 3;
        int n = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++n) {
            const int b = n & 1;
            const bool ok = __all_sync(
                0xffffffffu, mbar_wait_bounded(&acc_full[b], (uint32_t)((n >> 1) & 1)));
            umma::fence_after_sync();
            if (!ok || abort_flag) {
                if (!ok) set_status(status, DEV_TIMEOUT);
                break;
            }
            const uint2 w = items[it];
            const GroupProb *gp = probs + w.x;
            const int m0 = (int)(w.y & 0xffffu) * S::BM, n0 = (int)(w.y >> 16) * BN;
            const int row = m0 + q * 32 + lane;
            const int M = gp->M, Ncols = gp->N;
            const long long ldd = gp->ldd;
            const float los = gp->lo_scale;
            float *drow = gp->D + (long long)row * ldd;
            const bool vec = ((ldd & 3) == 0) && ((((uintptr_t)gp->D) & 15) == 0);
            const uint32_t t_row =
                tmem + (uint32_t)b * ACC_COLS + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t r[32], r2[32];
                umma::tmem_ld32(t_row + c, r);
                umma::tmem_ld32(t_row + BN + c, r2);
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
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, TMEM_COLS);
    }
}

constexpr int GROUP_BN = 128, GROUP_STAGES = 3;

bool encode_group_prob(GroupProb *gp, const GemmOperands &op, int b_box_rows) {
    if (!gemm_operands_ok(op) || !op.split) return false;
    if (!make_map(&gp->tA, op.A_hi, op.K, op.M, op.lda, 128, op.bf16) ||
        !make_map(&gp->tB, op.B_hi, op.K, op.N, op.ldb, b_box_rows, op.bf16) ||
        !make_map(&gp->tA2, op.A_lo, op.K, op.M, op.lda, 128, op.bf16) ||
        !make_map(&gp->tB2, op.B_lo, op.K, op.N, op.ldb, b_box_rows, op.bf16))
        return false;
    gp->D = op.D;
    gp->ldd = op.ldd;
    gp->M = op.M;
    gp->N = op.N;
    gp->K = op.K;
    gp->lo_scale = op.lo_scale;
    return true;
}

cudaError_t prepare_umma_grouped() {
    using S = GemmShape<GROUP_BN, true, GROUP_STAGES>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(umma_grouped_kernel<GROUP_BN, GROUP_STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::SMEM);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

cudaError_t launch_umma_grouped(const GroupProb *probs, const uint2 *items,
                                int nitems, unsigned *status, int sm_count,
                                cudaStream_t s) {
    using S = GemmShape<GROUP_BN, true, GROUP_STAGES>;
    if (nitems <= 0) return cudaSuccess;
    int grid = nitems < sm_count ? nitems : sm_count;
    umma_grouped_kernel<GROUP_BN, GROUP_STAGES><<<grid, 192, S::SMEM, s>>>(
        probs, items, nitems, status);
    return cudaGetLastError();
}

int group_tile_n() { return GROUP_BN; }

}  // namespace cgh
