// sep_simt.cu -- the separable form of Eq. 1 in FP32 on the FMA pipe:
// cos(theta_x + theta_y) = cos theta_x cos theta_y - sin theta_x sin theta_y,
// so that each point-pixel update is two FP32 multiply-adds and no
// special-function operation.
//
// The phase of Eq. 1 is a sum of an x part and a y part (Q_j (x - x_j)^2 +
// Q_j (y - y_j)^2), so with
//     L[x][2j] = A_j cos theta_x,  L[x][2j+1] = -A_j sin theta_x,
//     R[y][2j] =     cos theta_y,  R[y][2j+1] =      sin theta_y,
// I[y][x] = sum_k R[y][k] L[x][k]: an FP32 matrix product of depth K = 2N.
// The angles come from the exact fixed-point axis phase (mod 1 turn) and an
// accurate sincospi, so the tables are good to FP32 rounding; the products
// and the FP32 accumulation keep the result at the direct kernel's accuracy
// (max |I - I_ref| <= 1e-4 sum|A_j|).
//
// Kernel (sm_103a, FP32 SIMT):
//  * CTA tile 128 (y) x 128 (x), 256 threads, 8 x 8 outputs per thread kept
//    as packed FP32x2 pairs along x (fma.rn.f32x2: two multiply-adds per
//    issue slot);
//  * operands staged in shared memory by 1-D bulk copies (cp.async.bulk with
//    mbarrier completion), NST stages of BK values of k: the tables are
//    laid out tile by tile ([tile][k][pixel in tile]) so that one stage of
//    one operand is one contiguous block;
//  * R entries are stored twice in a row (each value next to itself, in the
//    order the threads read them), so that one 16-byte shared-memory load
//    gives two ready (r, r) pairs for the packed multiply-adds and every
//    warp-wide load touches 128 contiguous bytes;
//  * small frames are cut along k into S slices (split-K) so that the units
//    fill the SMs; the last slice of a tile to finish adds the S partial
//    tiles in slice order (deterministic) and writes the tile.
#include <math.h>

#include "api_internal.h"
#include "common.cuh"

namespace cgh {

constexpr int SS_BM = 128;          // y rows per CTA tile
constexpr int SS_BN = 128;          // x columns per CTA tile
constexpr int SS_THREADS = 256;
constexpr int SS_MAX_SPLIT = 16;
constexpr int SS_KPAD = 32;         // K (= 2 Npad) is padded to this multiple

// Stage geometry: BK values of k per stage, NST stages in flight.
template <int BK, int NST>
struct SimtStage {
    static constexpr int L = BK * SS_BN;          // floats of L per stage
    static constexpr int R = BK * 2 * SS_BM;      // floats of R per stage (doubled)
    static constexpr int ALL = L + R;
    static constexpr size_t SMEM = (size_t)NST * ALL * sizeof(float);
    static_assert((L * 4) % 16 == 0 && (R * 4) % 16 == 0, "bulk sizes");
    static_assert(SS_KPAD % BK == 0, "K padding covers the stage");
};
// The shapes compiled in: (BK, NST, PK): PK 1 = fma.rn.f32x2 pairs, two
// CTAs per SM (128 registers); 0 = scalar FMAs; 2 = pairs, one CTA per SM
// (up to 255 registers, room to load the next k's operands early).
// Measured on the 1920x1024x1024 and 3840x2160x16384 frames, (32, 2, 1)
// was fastest (fewest barriers per multiply-add at two CTAs per SM);
// (16, 4, 1) within 3%; (8, 8, 1), (32, 3, 1) (one CTA per SM), scalar FMAs
// (32, 2, 0: 5-7%) and (32, 4, 2) (8-16%) slower.  The last two are not
// compiled in.
#define CGH_SIMT_STAGES(X) X(16, 4, 1) X(32, 2, 1) X(8, 8, 1) X(32, 3, 1)

// Position of R value (row i of the tile, copy d) in a doubled R row of
// 2 * SS_BM floats.  Row i = wy 64 + h 32 + ty 4 + q (warp row wy, half h,
// lane row ty, q = 0..3); the thread (wy, ty) reads four 16-byte vectors
// (h, q / 2) = (r_q, r_q, r_{q+1}, r_{q+1}), each at 32 (4 (2 wy + h) ... )
// so that the 8 lane rows of a warp read 128 contiguous bytes.
__host__ __device__ constexpr int ss_rpos(int i, int d) {
    return ((((i >> 6) * 2 + ((i >> 5) & 1)) * 2 + ((i & 3) >> 1)) * 32) +
           ((i >> 2) & 7) * 4 + (i & 1) * 2 + d;
}

// ---------------------------------------------------------------- tables
// Grid: x = groups of SS_TP points, y = runs of 256 coordinates of the
// concatenated (padded) x and y ranges.  Block (0, *) also zeroes the split
// schedule's arrival counters.
constexpr int SS_TP = 16;

__global__ void simt_tables_kernel(const PointRec *__restrict__ rec, int Npad,
                                   int nxt, int nyt, float *__restrict__ Lt,
                                   float *__restrict__ Rt,
                                   unsigned *__restrict__ zero, int nzero) {
    __shared__ PointRec srec[SS_TP];
    if (blockIdx.x == 0)
        for (int k = blockIdx.y * blockDim.x + threadIdx.x; k < nzero;
             k += gridDim.y * blockDim.x)
            zero[k] = 0u;
    const int j0 = blockIdx.x * SS_TP;
    if (threadIdx.x < SS_TP && j0 + (int)threadIdx.x < Npad)
        srec[threadIdx.x] = rec[j0 + threadIdx.x];
    __syncthreads();
    const int npts = Npad - j0 < SS_TP ? Npad - j0 : SS_TP;
    const size_t K = 2 * (size_t)Npad;
    const int u = blockIdx.y * blockDim.x + threadIdx.x;
    const int nx = nxt * SS_BN, ny = nyt * SS_BM;
    if (u < nx) {
        const int t = u / SS_BN, i = u - t * SS_BN;
        float *dst = Lt + ((size_t)t * K + 2 * (size_t)j0) * SS_BN + i;
        for (int q = 0; q < npts; ++q) {
            const PointRec &r = srec[q];
            float s, c;
            sincospif(2.0f * ((float)phase_hi(axis_phase(r.c, r.bx, r.ax, u)) *
                              TURN_PER_U32),
                      &s, &c);
            dst[(size_t)(2 * q) * SS_BN] = r.A * c;
            dst[(size_t)(2 * q + 1) * SS_BN] = -r.A * s;
        }
    } else if (u < nx + ny) {
        const int v = u - nx;
        const int t = v / SS_BM, i = v - t * SS_BM;
        const int p0 = ss_rpos(i, 0), p1 = ss_rpos(i, 1);
        float *dst = Rt + ((size_t)t * K + 2 * (size_t)j0) * (2 * SS_BM);
        for (int q = 0; q < npts; ++q) {
            const PointRec &r = srec[q];
            float s, c;
            sincospif(2.0f * ((float)phase_hi(axis_phase(r.c, r.by, r.ay, v)) *
                              TURN_PER_U32),
                      &s, &c);
            float *rc = dst + (size_t)(2 * q) * (2 * SS_BM);
            float *rs = rc + 2 * SS_BM;
            rc[p0] = c;
            rc[p1] = c;
            rs[p0] = s;
            rs[p1] = s;
        }
    }
}

// ------------------------------------------------------------------ GEMM
template <int BK, int NST>
__device__ __forceinline__ void ss_issue(float *smem, uint64_t *full,
                                         const float *Lb, const float *Rb,
                                         int stage, int slot) {
    using G = SimtStage<BK, NST>;
    float *st = smem + (size_t)slot * G::ALL;
    mbar_arrive_expect_tx(&full[slot], G::ALL * 4);
    bulk_g2s(st, Lb + (size_t)stage * G::L, G::L * 4, &full[slot]);
    bulk_g2s(st + G::L, Rb + (size_t)stage * G::R, G::R * 4, &full[slot]);
}

// One unit = (tile, k slice).  Units are numbered tile-major: unit =
// tile * S + slice.  Tiles are row-major over (x tile, y tile).
template <int BK, int NST, int PK>
__global__ void __launch_bounds__(SS_THREADS, PK == 2 ? 1 : 2)
simt_gemm_kernel(const float *__restrict__ Lt, const float *__restrict__ Rt,
                 int Npad, int Nx, int Ny, int nxt, int S,
                 float *__restrict__ out, int vec_store,
                 float *__restrict__ part, unsigned *__restrict__ count,
                 unsigned *status) {
    extern __shared__ __align__(128) float smem[];
    using G = SimtStage<BK, NST>;
    __shared__ __align__(8) uint64_t full[NST];
    __shared__ volatile int abort_flag;
    __shared__ int s_last;

    const int unit = blockIdx.x;
    const int tile = unit / S, slice = unit - tile * S;
    const int xt = tile % nxt, yt = tile / nxt;
    const int nst = 2 * Npad / BK;
    const int s0 = (int)((long long)nst * slice / S);
    const int s1 = (int)((long long)nst * (slice + 1) / S);
    const int ntile = s1 - s0;
    const size_t K = 2 * (size_t)Npad;
    const float *Lb = Lt + ((size_t)xt * K + (size_t)s0 * BK) * SS_BN;
    const float *Rb = Rt + ((size_t)yt * K + (size_t)s0 * BK) * (2 * SS_BM);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int issued = 0;  // thread 0 only
    if (threadIdx.x == 0)
        for (int s = 0; s < NST && s < ntile; ++s) {
            ss_issue<BK, NST>(smem, full, Lb, Rb, s, s);
            ++issued;
        }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wx = warp & 3, wy = warp >> 2;
    const int tx = lane & 3, ty = lane >> 2;
    // this thread's columns: cx + {0..3} and cx + 16 + {0..3}; rows: ry +
    // {0..3} and ry + 32 + {0..3}
    const int cx = wx * 32 + tx * 4;
    const int ry = wy * 64 + ty * 4;
    // offsets of this thread's four doubled-R vectors within an R row
    const int rq0 = ((wy * 2 + 0) * 2 + 0) * 32 + ty * 4;
    const int rq1 = ((wy * 2 + 0) * 2 + 1) * 32 + ty * 4;
    const int rq2 = ((wy * 2 + 1) * 2 + 0) * 32 + ty * 4;
    const int rq3 = ((wy * 2 + 1) * 2 + 1) * 32 + ty * 4;

    float2 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = make_float2(0.0f, 0.0f);

    int t = 0;
    for (; t < ntile; ++t) {
        const int s = t % NST;
        const uint32_t par = (uint32_t)((t / NST) & 1);
        if (!mbar_wait_bounded(&full[s], par)) {
            abort_flag = 1;
            set_status(status, DEV_TIMEOUT);
        } else {
            const float *Ls = smem + (size_t)s * G::ALL;
            const float *Rs = Ls + G::L;
#pragma unroll 2
            for (int k = 0; k < BK; ++k) {
                const float4 la = *reinterpret_cast<const float4 *>(Ls + k * SS_BN + cx);
                const float4 lb =
                    *reinterpret_cast<const float4 *>(Ls + k * SS_BN + cx + 16);
                const float *rr = Rs + k * (2 * SS_BM);
                const float4 r0 = *reinterpret_cast<const float4 *>(rr + rq0);
                const float4 r1 = *reinterpret_cast<const float4 *>(rr + rq1);
                const float4 r2 = *reinterpret_cast<const float4 *>(rr + rq2);
                const float4 r3 = *reinterpret_cast<const float4 *>(rr + rq3);
                const float2 l[4] = {make_float2(la.x, la.y), make_float2(la.z, la.w),
                                     make_float2(lb.x, lb.y), make_float2(lb.z, lb.w)};
                const float2 r[8] = {make_float2(r0.x, r0.y), make_float2(r0.z, r0.w),
                                     make_float2(r1.x, r1.y), make_float2(r1.z, r1.w),
                                     make_float2(r2.x, r2.y), make_float2(r2.z, r2.w),
                                     make_float2(r3.x, r3.y), make_float2(r3.z, r3.w)};
                if constexpr (PK) {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            acc[i][c] = __ffma2_rn(r[i], l[c], acc[i][c]);
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            acc[i][c].x = fmaf(r[i].x, l[c].x, acc[i][c].x);
                            acc[i][c].y = fmaf(r[i].x, l[c].y, acc[i][c].y);
                        }
                }
            }
        }
        __syncthreads();  // every thread is done with slot s
        if (abort_flag) break;
        if (threadIdx.x == 0 && t + NST < ntile) {
            fence_proxy_async_smem();
            ss_issue<BK, NST>(smem, full, Lb, Rb, t + NST, s);
            ++issued;
        }
    }
    if (abort_flag) {
        // let this CTA's copies still in flight land (each wait bounded)
        if (threadIdx.x == 0)
            for (int u = t; u < issued; ++u)
                mbar_wait_bounded(&full[u % NST], (uint32_t)((u / NST) & 1));
        return;
    }

    const int x0 = xt * SS_BN, y0 = yt * SS_BM;
    if (S > 1) {
        // publish this slice's partial tile ([row][col], 128 x 128), count in
        float *dst = part + (size_t)unit * SS_BM * SS_BN;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float *row = dst + (size_t)(ry + (i & 3) + (i >> 2) * 32) * SS_BN + cx;
            *reinterpret_cast<float4 *>(row) =
                make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
            *reinterpret_cast<float4 *>(row + 16) =
                make_float4(acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(&count[tile], 1u) == (unsigned)(S - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        // the last slice adds the S partials in slice order (each thread
        // reads back exactly the positions it owns)
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][c] = make_float2(0.0f, 0.0f);
        for (int q = 0; q < S; ++q) {
            const float *src = part + ((size_t)tile * S + q) * SS_BM * SS_BN;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float *row =
                    src + (size_t)(ry + (i & 3) + (i >> 2) * 32) * SS_BN + cx;
                const float4 a = __ldcg(reinterpret_cast<const float4 *>(row));
                const float4 b = __ldcg(reinterpret_cast<const float4 *>(row + 16));
                acc[i][0] = __fadd2_rn(acc[i][0], make_float2(a.x, a.y));
                acc[i][1] = __fadd2_rn(acc[i][1], make_float2(a.z, a.w));
                acc[i][2] = __fadd2_rn(acc[i][2], make_float2(b.x, b.y));
                acc[i][3] = __fadd2_rn(acc[i][3], make_float2(b.z, b.w));
            }
        }
    }
    // write the tile, clipped to the frame
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int y = y0 + ry + (i & 3) + (i >> 2) * 32;
        if (y >= Ny) continue;
        float *orow = out + (size_t)y * Nx;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = x0 + cx + 16 * h;
            const float v[4] = {acc[i][2 * h].x, acc[i][2 * h].y, acc[i][2 * h + 1].x,
                                acc[i][2 * h + 1].y};
            if (vec_store && x + 4 <= Nx) {
                *reinterpret_cast<float4 *>(orow + x) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (x + e < Nx) orow[x + e] = v[e];
            }
        }
    }
}

// Number of k slices for `tiles` output tiles of `nst` stages each: the
// fewest slices whose units fill the SMs' CTA slots (`per_sm` per SM) in
// nearly whole waves, counting about four stages of work per unit for its
// epilogue.
static int simt_split(int tiles, int nst, int sm_count, int per_sm) {
    const int slots = per_sm * (sm_count > 0 ? sm_count : 1);
    int best = 1;
    double best_cost = 1e300;
    for (int S = 1; S <= SS_MAX_SPLIT && S <= nst; ++S) {
        const long long units = (long long)tiles * S;
        const long long waves = (units + slots - 1) / slots;
        const double per_unit = (double)((nst + S - 1) / S) + (S > 1 ? 4.0 : 0.0);
        const double cost = (double)waves * per_unit;
        if (cost < best_cost * 0.97) {  // a split must pay for itself
            best_cost = cost;
            best = S;
        }
    }
    return best;
}

struct SimtPlan {
    int bk, nst_ring, per_sm;
};

static SimtPlan simt_plan(int index) {
    int i = 0;
#define X(bk, ns, pk)                                                           \
    if (index == i)                                                             \
        return SimtPlan{bk, ns,                                                 \
                        SimtStage<bk, ns>::SMEM <= 110 * 1024 ? 2 : 1};         \
    ++i;
    CGH_SIMT_STAGES(X)
#undef X
    return SimtPlan{16, 4, 2};
}

int simt_stage_count() {
    int n = 0;
#define X(bk, ns, pk) ++n;
    CGH_SIMT_STAGES(X)
#undef X
    return n;
}

template <int BK, int NST, int PK>
static cudaError_t launch_simt_gemm(int device, unsigned grid, cudaStream_t s,
                                    const float *Lt, const float *Rt, int Npad,
                                    int Nx, int Ny, int nxt, int S, float *out,
                                    int vec_store, float *part, unsigned *count,
                                    unsigned *status) {
    using G = SimtStage<BK, NST>;
    static bool attr_set[64] = {};
    if (device < 0 || device >= 64 || !attr_set[device]) {
        cudaError_t e = cudaFuncSetAttribute(simt_gemm_kernel<BK, NST, PK>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::SMEM);
        if (e != cudaSuccess) return e;
        if (device >= 0 && device < 64) attr_set[device] = true;
    }
    simt_gemm_kernel<BK, NST, PK><<<grid, SS_THREADS, G::SMEM, s>>>(
        Lt, Rt, Npad, Nx, Ny, nxt, S, out, vec_store, part, count, status);
    return cudaGetLastError();
}

static cudaError_t launch_simt_index(int index, int device, unsigned grid,
                                     cudaStream_t s, const float *Lt,
                                     const float *Rt, int Npad, int Nx, int Ny,
                                     int nxt, int S, float *out, int vec_store,
                                     float *part, unsigned *count,
                                     unsigned *status) {
    int i = 0;
#define X(bk, ns, pk)                                                           \
    if (index == i)                                                             \
        return launch_simt_gemm<bk, ns, pk>(device, grid, s, Lt, Rt, Npad, Nx,  \
                                            Ny, nxt, S, out, vec_store, part,   \
                                            count, status);                     \
    ++i;
    CGH_SIMT_STAGES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace cgh

using namespace cgh;

cgh_status cgh_ctx::forward_simt(const float *points, const float *A,
                                 const float *z, int N, double lambda,
                                 double p, int Nx, int Ny, float *out,
                                 cudaStream_t s) {
    const int index = simt_stage >= 0 && simt_stage < simt_stage_count() ? simt_stage : 1;
    const SimtPlan plan = simt_plan(index);
    const int Npad = pad_to(N, SS_KPAD / 2);
    const int nxt = (Nx + SS_BN - 1) / SS_BN, nyt = (Ny + SS_BM - 1) / SS_BM;
    const int tiles = nxt * nyt;
    const int nst = 2 * Npad / plan.bk;
    const int S = simt_split(tiles, nst, sm_count, plan.per_sm);
    const size_t K = 2 * (size_t)Npad;
    const size_t rec_b = align256((size_t)Npad * sizeof(PointRec));
    const size_t l_b = align256((size_t)nxt * K * SS_BN * sizeof(float));
    const size_t r_b = align256((size_t)nyt * K * 2 * SS_BM * sizeof(float));
    const size_t part_b =
        S > 1 ? align256((size_t)tiles * S * SS_BM * SS_BN * sizeof(float)) : 0;
    const size_t cnt_b = S > 1 ? align256((size_t)tiles * sizeof(unsigned)) : 0;
    cgh_status st = ensure(ws, rec_b + l_b + r_b + part_b + cnt_b, s,
                           "FP32 separable workspace");
    if (st) return st;
    char *base = (char *)ws.ptr;
    PointRec *rec = (PointRec *)base;
    float *Lt = (float *)(base + rec_b);
    float *Rt = (float *)(base + rec_b + l_b);
    float *part = S > 1 ? (float *)(base + rec_b + l_b + r_b) : nullptr;
    unsigned *count = S > 1 ? (unsigned *)(base + rec_b + l_b + r_b + part_b) : nullptr;
    {
        TimedLaunch tl(this, CGH_K_PROLOGUE, s);
        cudaError_t e = launch_prologue(points, A, z, N, Npad, lambda, p, rec,
                                        d_status, s, row_origin);
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        tl.done();
    }
    {
        TimedLaunch tl(this, CGH_K_SEP_TABLES, s);
        const int span = nxt * SS_BN + nyt * SS_BM;
        dim3 grid((Npad + SS_TP - 1) / SS_TP, (span + 255) / 256);
        simt_tables_kernel<<<grid, 256, 0, s>>>(rec, Npad, nxt, nyt, Lt, Rt, count,
                                                S > 1 ? tiles : 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "FP32 separable tables launch");
        tl.done();
    }
    {
        TimedLaunch tl(this, CGH_K_SIMT, s);
        const int vec_store = (Nx % 4 == 0) && (((uintptr_t)out & 15) == 0);
        cudaError_t e = launch_simt_index(index, device, (unsigned)(tiles * S), s, Lt,
                                          Rt, Npad, Nx, Ny, nxt, S, out, vec_store,
                                          part, count, d_status);
        if (e != cudaSuccess) return cuda_fail(e, "FP32 GEMM launch");
        tl.done();
    }
    return CGH_OK;
}
