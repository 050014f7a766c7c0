// umma_gen.cu -- the separable forward GEMM on CTA pairs with its operand
// tiles generated in shared memory instead of read from U / V tables.
//
// The separable form of Eq. 1 (Section 1: the phase is an x part plus a y
// part) is the product I = R L^T with, per point j,
//     R[y][2j] = cos th_y,     R[y][2j+1] = sin th_y        (A operand, Ny rows)
//     L[x][2j] = A_j cos th_x, L[x][2j+1] = -A_j sin th_x   (B operand, Nx rows)
// (separable.cu).  There the tables are written to global memory by one
// kernel and read back by the GEMM's TMA loads.  Here eight producer warps
// of each CTA compute the tile of every K block (32 points) straight into
// the stage ring, in the 128-byte-swizzled K-major layout the tensor-core
// descriptors read: this CTA's 128 rows of R and its half (BNP / 2 rows) of
// the pair's L columns.  The tables never touch global memory
// ("recompute rather than store").
//
// Entry values are those of the table kernel, bit for bit: the axis phase
// in exact 0.64 fixed-point turns -- evaluated directly at the first row of
// a warp's run and stepped row by row with the exact fixed-point form of
// Eq. 2 (first difference c (2 u + 1) - b, second difference 2 c, all
// modulo one turn) -- its top 32 bits as an FP32 angle, the hardware
// sincos, then BF16 / FP16 / split hi + lo FP16 (sep_table.cuh).
// The MMAs, their order and the epilogue are those of umma2.cu, so the
// hologram equals the table path's bit for bit.
//
// Roles (544 threads): warp 0 allocates tensor memory and, in the even CTA,
// issues the MMAs (one thread); warps 1-16 produce the tiles -- each warp
// one run of rows for all 32 points of a K block, lane = point -- then
// warps 1-4 read the accumulators back (warp w reads TMEM lanes
// 32 (w % 4) ..).
// Synchronisation (every wait bounded):
//   * full[s] of the even CTA counts 32 arrivals per stage, one per producer
//     warp of both CTAs (the odd CTA's arrive remotely, release at cluster
//     scope, after a proxy fence that makes their shared-memory stores
//     visible to the tensor cores);
//   * the MMA issuer's commits arrive on empty[s] of both CTAs (multicast),
//     which the producers wait on before rewriting stage s;
//   * the accumulator barrier as in umma2.cu.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdlib.h>

#include "api_internal.h"
#include "common.cuh"
#include "sep_table.cuh"
#include "umma.cuh"
#include "umma_epi.cuh"
#include "umma_pair.cuh"

namespace cgh {

constexpr int GEN_PRODUCER_WARPS = 16;
constexpr int GEN_THREADS = 32 * (1 + GEN_PRODUCER_WARPS);

struct GenArgs {
    const PointRec *rec;  // records of this launch's points (K / 2 of them)
    int nvalid;           // points with j < nvalid are real; the rest padding
};

// The entry of point j at one tile row as a packed (re, im) pair: BF16
// (KIND 0), FP16 (1) or split FP16 (2: hi, and lo scaled by LO_SCALE).
template <int KIND>
__device__ __forceinline__ void gen_pack(float re, float im, uint32_t &hi, uint32_t &lo) {
    if (KIND == 0) {
        __nv_bfloat162 v = __floats2bfloat162_rn(re, im);
        hi = *reinterpret_cast<uint32_t *>(&v);
        lo = 0u;
    } else {
        __half2 v = __floats2half2_rn(re, im);
        hi = *reinterpret_cast<uint32_t *>(&v);
        lo = 0u;
        if (KIND == 2) {
            const float2 f = __half22float2(v);
            __half2 w = __floats2half2_rn((re - f.x) * LO_SCALE, (im - f.y) * LO_SCALE);
            lo = *reinterpret_cast<uint32_t *>(&w);
        }
    }
}

// Rows [r0, r1) of one operand tile for point p (the warp's lane) of K
// block kb: global axis coordinate u0 + r; rows at or beyond `umax`
// (outside the matrix) and padding points are zero.  IS_X: the L operand
// (x axis, amplitude-weighted (cos, -sin)); else R (y axis, (cos, sin)).
// The phase is evaluated once, at row r0, then stepped row by row with the
// exact fixed-point form of Eq. 2 (as sep_table.cuh).  A warp writes one
// whole 128-byte tile row per step (lane p: bytes 4p .. 4p + 3 of the row
// before the swizzle), so its stores hit 32 distinct banks.
template <int KIND, bool IS_X>
__device__ __forceinline__ void gen_run(const GenArgs &ga, int kb, int p, int r0, int r1,
                                        int u0, int umax, uint8_t *hi_tile,
                                        uint8_t *lo_tile) {
    const int j = kb * 32 + p;
    const PointRec *pr = ga.rec + j;
    const bool valid = j < ga.nvalid;
    const uint64_t c = pr->c;
    const uint64_t b = IS_X ? pr->bx : pr->by;
    const uint64_t a = IS_X ? pr->ax : pr->ay;
    const float amp = pr->A;
    const int u_first = u0 + r0;
    uint64_t ph = axis_phase(c, b, a, u_first);
    uint64_t d = c * (uint64_t)(2 * (int64_t)u_first + 1) - b;
    const uint64_t dd = 2 * c;
    // 128-byte swizzle: 16-byte chunk p / 4 of row r sits at chunk
    // (p / 4) ^ (r mod 8)
    const uint32_t chunk = (uint32_t)(p >> 2), within = (uint32_t)(p & 3) * 4u;
#pragma unroll 4
    for (int r = r0; r < r1; ++r) {
        float s, co;
        __sincosf((float)phase_hi(ph) * RAD_PER_U32, &s, &co);
        const bool ok = valid && u0 + r < umax;
        const float re = ok ? (IS_X ? amp * co : co) : 0.0f;
        const float im = ok ? (IS_X ? -amp * s : s) : 0.0f;
        uint32_t h, l;
        gen_pack<KIND>(re, im, h, l);
        const uint32_t off = (uint32_t)r * 128u + ((chunk ^ (uint32_t)(r & 7)) << 4) + within;
        *reinterpret_cast<uint32_t *>(hi_tile + off) = h;
        if (KIND == 2) *reinterpret_cast<uint32_t *>(lo_tile + off) = l;
        ph += d;
        d += dd;
    }
}

// Grid: x = 2 x (column blocks of BNP), y = row blocks of 256; clusters of
// two CTAs along x.  D = R L^T (M = Ny rows, N = Nx columns) for the K / 2
// points of ga.rec.
template <int BNP, int KIND, int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(GEN_THREADS, 1)
umma_gen_pair_kernel(GenArgs ga, GemmArgs g, uint32_t idesc) {
    constexpr bool SPLIT = KIND == 2;
    using S = PairShape<BNP, SPLIT, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES];   // (even CTA) both CTAs' tiles written
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
            mbar_init(&full[s], 2 * GEN_PRODUCER_WARPS);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accum_bar, 1);
        mbar_fence_init();
    }
    if (warp == 0) {
        umma2::tmem_alloc2(&tmem_base, S::TMEM_COLS);
        umma2::tmem_relinquish2();
    }
    umma::fence_before_sync();
    umma2::cluster_sync();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_base;
    pdl_wait();  // the point records come from (and D may be read by) the kernel before

    if (warp == 0) {
        if (lane == 0 && rank == 0) {
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
            // only this CTA learns that its MMAs in flight have finished
            umma2::commit2(&accum_bar, done == KB ? 0x3 : 0x1);
        }
    } else {
        // ------------------------------------------ producers (both CTAs)
        // producer warp pw: pw < 8 writes rows [16 pw, 16 pw + 16) of this
        // CTA's 128 R rows, pw >= 8 its share of the BNH L rows (8 runs)
        const int pw = warp - 1;
        constexpr int BRUN = (S::BNH + 7) / 8;
        const bool on_a = pw < 8;
        const int r0 = on_a ? 16 * pw : BRUN * (pw - 8);
        const int r1 = on_a ? r0 + 16 : (r0 + BRUN < S::BNH ? r0 + BRUN : S::BNH);
        const uint32_t full_even0 = umma2::map_to_rank(&full[0], 0);
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES) {
                bool ok = true;
                if (lane == 0)
                    ok = mbar_wait_bounded(&empty[s], (uint32_t)(((kb / STAGES) - 1) & 1));
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) {
                    abort_flag = 1;
                    set_status(g.status, DEV_TIMEOUT);
                }
            }
            if (abort_flag) break;
            uint8_t *st = smem + (size_t)s * S::STAGE_BYTES;
            if (on_a)
                gen_run<KIND, false>(ga, kb, lane, r0, r1, m0, g.M, st,
                                     st + S::A_BYTES + S::B_BYTES);
            else if (r0 < r1)
                gen_run<KIND, true>(ga, kb, lane, r0, r1, nb, g.N, st + S::A_BYTES,
                                    st + 2 * S::A_BYTES + S::B_BYTES);
            // make the stores visible to the tensor cores, then count this
            // warp in on the even CTA's barrier
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) umma2::remote_arrive(full_even0 + (uint32_t)s * 8u);
        }
        if (warp == GEN_PRODUCER_WARPS && lane == 0 && !abort_flag) {
            // The MMA issuer's commits of the last stages arrive on this
            // CTA's empty barriers asynchronously (multicast to both CTAs),
            // and nothing else waits for them: wait here (bounded), so that
            // no arrive is still in flight when the CTA exits and its shared
            // memory passes to the next CTA on the SM.
            for (int kb = KB - STAGES < 0 ? 0 : KB - STAGES; kb < KB; ++kb)
                mbar_wait_bounded(&empty[kb % STAGES], (uint32_t)((kb / STAGES) & 1));
        }
        // ------------------------------------ epilogue (warps 1-4, both CTAs)
        if (warp <= 4) {
            const int qq = warp & 3;  // the 32-lane quarter of TMEM this warp reads
            const int row = m0 + qq * 32 + lane;
            const bool ok =
                __all_sync(0xffffffffu, umma2::wait_cluster_bounded(&accum_bar, 0));
            umma::fence_after_sync();
            pdl_trigger();  // only the epilogue is left
            if (!ok) set_status(g.status, DEV_TIMEOUT);
            if (ok && !abort_flag) {
                const uint32_t t_row = tmem + ((uint32_t)(qq * 32) << 16);
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
    }
    umma::fence_before_sync();
    umma2::cluster_sync();  // no MMA, commit or remote arrive still aims at either CTA
    if (warp == 0) {
        umma::fence_after_sync();
        umma2::tmem_dealloc2(tmem, S::TMEM_COLS);
    }
}

// ------------------------------------------------------------- host side
template <int BNP, int KIND, int STAGES>
static cudaError_t launch_gen_t(const GenArgs &ga, const GemmArgs &g, cudaStream_t s) {
    constexpr bool SPLIT = KIND == 2;
    using S = PairShape<BNP, SPLIT, STAGES>;
    auto kern = umma_gen_pair_kernel<BNP, KIND, STAGES>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid(2 * ((g.N + BNP - 1) / BNP), (g.M + 2 * S::BM - 1) / (2 * S::BM));
    const uint32_t idesc = umma::idesc_f16(2 * S::BM, BNP, KIND == 0);
    return launch_dependent(kern, grid, dim3(GEN_THREADS), S::SMEM, s, ga, g, idesc);
}

static cudaError_t launch_gen_one(const GenArgs &ga, const GemmArgs &g, int kind, int bnp,
                                  cudaStream_t s) {
    if (kind == 2) {
        switch (bnp) {
        case 112: return launch_gen_t<112, 2, 4>(ga, g, s);
        case 144: return launch_gen_t<144, 2, 4>(ga, g, s);
        case 160: return launch_gen_t<160, 2, 4>(ga, g, s);
        case 224: return launch_gen_t<224, 2, 3>(ga, g, s);
        case 256: return launch_gen_t<256, 2, 3>(ga, g, s);
        }
    } else if (kind == 1) {
        switch (bnp) {
        case 112: return launch_gen_t<112, 1, 8>(ga, g, s);
        case 256: return launch_gen_t<256, 1, 6>(ga, g, s);
        }
    } else {
        switch (bnp) {
        case 112: return launch_gen_t<112, 0, 8>(ga, g, s);
        case 256: return launch_gen_t<256, 0, 6>(ga, g, s);
        }
    }
    return cudaErrorInvalidValue;
}

bool gen_pair_width_ok(int kind, int bnp) {
    if (kind == 2) return bnp == 112 || bnp == 144 || bnp == 160 || bnp == 224 || bnp == 256;
    return bnp == 112 || bnp == 256;
}

// The width the generating kernel takes for an M x N product: the split form
// compiles the table GEMM's widths (same choice), the single-pass forms 112
// and 256 (the cheaper by SM waves x width).
int pick_gen_n(int M, int N, int sms, int kind) {
    if (kind == 2) return pick_pair_n(M, N, sms);
    return pair_cost(M, N, 112, sms) <= pair_cost(M, N, 256, sms) ? 112 : 256;
}

// D (M x N, FP32, row stride ldd) = R L^T over the Npad points of `rec`
// (N of them real), the operand tiles generated in the kernel; K = 2 Npad
// (a multiple of 64).  Longer products than one K chunk run as consecutive
// launches over consecutive point ranges, the later ones adding into D.
cudaError_t launch_umma_gen(const PointRec *rec, int N, int Npad, int kind, int bnp,
                            float *D, int M, int Ncols, long long ldd, float lo_scale,
                            unsigned *status, cudaStream_t s) {
    const int K = 2 * Npad;
    if (K % 64 != 0 || M < 1 || Ncols < 1 || !gen_pair_width_ok(kind, bnp) ||
        (((uintptr_t)rec) & 7))
        return cudaErrorInvalidValue;
    const int chunk = gemm_k_chunk(kind == 2);
    for (int k0 = 0; k0 < K; k0 += chunk) {
        const int Kc = K - k0 < chunk ? K - k0 : chunk;
        const int j0 = k0 / 2;
        GenArgs ga{rec + j0, N - j0};
        GemmArgs g{M, Ncols, Kc, D, ldd, lo_scale, status, k0 > 0 ? 1 : 0};
        cudaError_t e = launch_gen_one(ga, g, kind, bnp, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cgh
