// backward.cu -- the hand-written adjoint of Eq. 1 (step A8).
//
// For a loss L with G = dL/dI (Ny x Nx) and phi = P_j r^2 (Section 1,
// Eq. 1; P_j = 2 pi Q_j, dx = x - x_j, dy = y - y_j, dP_j/dz_j = -P_j/z_j):
//     dL/dA_j = sum G cos(phi)
//     dL/dx_j = 2 P_j A_j sum G sin(phi) dx
//     dL/dy_j = 2 P_j A_j sum G sin(phi) dy
//     dL/dz_j = (P_j A_j / z_j) sum G sin(phi) (dx^2 + dy^2)
// Both methods produce per-tile partial sums
//     part_x[t][j] = (sum G cos phi, sum G sin phi dx, sum G sin phi dx^2)
//     part_y[t][j] = (-, sum G sin phi dy, sum G sin phi dy^2)
// and one reduction kernel adds the tiles in a fixed order (deterministic)
// and applies the per-point factors.
//
// Direct (FP32): each thread owns one point and walks a 16-pixel-wide
// column strip of G top to bottom; G rows are read with uniform (broadcast)
// loads; the x angles of the strip stay in registers and the y angle follows
// the exact fixed-point form of the paper's Eq. 2 recurrence.  A quarter of
// the columns take sin and cos from FMA-pipe polynomials, the rest from the
// hardware sincos (two MUFU operations per point-pixel update).
//
// Separable (split FP16 on the tensor cores): with U = e^{i th_x},
// V = e^{i th_y},
//     sum_{x,y} G e^{i(th_x + th_y)} w(x) = sum_x w(x) U[x] (sum_y G[y][x] V[y])
// so two GEMMs give the inner transforms -- D1[2j+c][x] = sum_y V'[2j+c][y] G[y][x]
// and D2[2j+c][y] = sum_x U'[2j+c][x] G[y][x], with U', V' the cos/sin
// rows -- and their epilogues (umma.cu) multiply by the recomputed U or V
// and reduce over the GEMM columns with weights 1, d, d^2.  U and V are
// recomputed from the point records here, not kept from the forward pass.
// G is scaled by a power of two (from max |G|) before the FP16 split and
// the scale is removed in the reduction.
#include <cuda_fp16.h>
#include <math.h>

#include "api_internal.h"
#include "common.cuh"
#include "cos_poly.h"
#include "umma.cuh"

namespace cgh {

constexpr float PI_F = 3.14159265358979323846f;
constexpr float ADJ_LO_SCALE = 4096.0f;

// ------------------------------------------------------------- G prep
__global__ void g_absmax_kernel(const float *__restrict__ G, long long n,
                                unsigned *word) {
    float m = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v = fabsf(G[i]);
        m = v > m ? v : (v != v ? v : m);  // keep NaN
    }
    for (int o = 16; o > 0; o >>= 1) {
        float t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : (t != t ? t : m);
    }
    if ((threadIdx.x & 31) == 0) atomicMax(word, __float_as_uint(m));
}

// 2^-e with e the exponent that maps max |G| into [1/2, 1); 1 if max is 0
// or not finite.
__device__ __forceinline__ float g_scale(unsigned word) {
    const float m = __uint_as_float(word);
    if (!(m > 0.0f) || !isfinite(m)) return 1.0f;
    return ldexpf(1.0f, -(ilogbf(m) + 1));
}

// G (FP32, Ny x Nx) -> scaled FP16 hi/lo planes in both orientations:
// Gr[y][x] (row stride ldx) and Gt[x][y] (row stride ldy).
__global__ void g_convert_kernel(const float *__restrict__ G, int Nx, int Ny,
                                 const unsigned *word, __half *Gr_hi,
                                 __half *Gr_lo, int ldx, __half *Gt_hi,
                                 __half *Gt_lo, int ldy) {
    __shared__ float tile[32][33];
    const float s = g_scale(*word);
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int y = by + r, x = bx + tx;
        float v = 0.0f;
        if (y < Ny && x < Nx) v = G[(size_t)y * Nx + x] * s;
        tile[r][tx] = v;
        if (y < Ny && x < Nx) {
            const __half h = __float2half_rn(v);
            Gr_hi[(size_t)y * ldx + x] = h;
            Gr_lo[(size_t)y * ldx + x] =
                __float2half_rn((v - __half2float(h)) * ADJ_LO_SCALE);
        }
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int x = bx + r, y = by + tx;
        if (x < Nx && y < Ny) {
            const float v = tile[tx][r];
            const __half h = __float2half_rn(v);
            Gt_hi[(size_t)x * ldy + y] = h;
            Gt_lo[(size_t)x * ldy + y] =
                __float2half_rn((v - __half2float(h)) * ADJ_LO_SCALE);
        }
    }
}

// ---------------------------------------------------------- U', V' rows
// Row 2j: cos th(u, j), row 2j+1: sin th(u, j), along u = 0..n-1, for the
// x axis (U', n = Nx, row stride ldx) and the y axis (V', n = Ny, ldy).
// FP16 hi and lo (scaled by 2^12) planes; rows of padding points are 0.
// Grid: x over u in [0, Nx + Ny) (x coordinates, then y), y over groups of
// AT_POINTS points from j0, whose records are staged in shared memory.
constexpr int AT_POINTS = 16;

__global__ void adj_tables_kernel(const PointRec *__restrict__ rec, int N,
                                  int Npad, int j0, int Nx, int Ny, int ldx,
                                  int ldy, __half *Uhi, __half *Ulo, __half *Vhi,
                                  __half *Vlo) {
    __shared__ PointRec srec[AT_POINTS];
    const int jb = j0 + (int)blockIdx.y * AT_POINTS;
    if (threadIdx.x < AT_POINTS) {
        const int j = jb + threadIdx.x;
        srec[threadIdx.x] = j < N ? rec[j] : PointRec{};
    }
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Nx + Ny) return;
    const bool is_x = r < Nx;
    const int u = is_x ? r : r - Nx;
    __half *hi = is_x ? Uhi : Vhi;
    __half *lo = is_x ? Ulo : Vlo;
    const int ld = is_x ? ldx : ldy;
    const int npts = Npad - jb < AT_POINTS ? Npad - jb : AT_POINTS;
    for (int q = 0; q < npts; ++q) {
        const int j = jb + q;
        float s = 0.0f, c = 0.0f;
        if (j < N) {
            const PointRec &pr = srec[q];
            const uint64_t ph = is_x ? axis_phase(pr.c, pr.bx, pr.ax, u)
                                     : axis_phase(pr.c, pr.by, pr.ay, u);
            __sincosf((float)phase_hi(ph) * RAD_PER_U32, &s, &c);
        }
        const __half hc = __float2half_rn(c), hs = __float2half_rn(s);
        const size_t oc = (size_t)(2 * j) * ld + u, os = oc + ld;
        hi[oc] = hc;
        hi[os] = hs;
        lo[oc] = __float2half_rn((c - __half2float(hc)) * ADJ_LO_SCALE);
        lo[os] = __float2half_rn((s - __half2float(hs)) * ADJ_LO_SCALE);
    }
}

// ------------------------------------------------------ direct adjoint
// Each thread owns one point and a BWD_STRIP-column strip; the arithmetic
// runs on column pairs in packed FP32x2.  NPOLY columns (pairs spread evenly
// over the strip) take sin and cos from FMA-pipe polynomials (u = |theta| - pi: cos theta = -C(u^2),
// sin theta = -sign(theta) u S(u^2); cos_poly.h), the others from the
// hardware sincos (two MUFU operations).  The offset dx = x - x_j is
// constant down a column, so the x sums of G sin(phi) dx and G sin(phi) dx^2
// are taken as dx and dx^2 times each column's sum of G sin(phi), formed once
// at the end: per update 5 FP32 operations and 2 MUFU on the hardware path
// (angle add, argument scale, and the cos, column and row sums), 17 on the
// polynomial path.  The polynomial columns accumulate negated sums, whose
// sign is restored at the end.
constexpr int BWD_STRIP = 16;    // pixels per column strip
// points per CTA: 256 with G staged through shared memory (each staged row
// serves more points), 128 reading G rows from global memory (measured on
// the direct adjoint at 1920x1080x4096, before the per-column sums: 3.34
// against 3.44 ms staged, 3.59 against 4.10 ms unstaged); points are padded
// to the larger
constexpr int BWD_THREADS_STAGED = 256;
constexpr int BWD_THREADS_GLOBAL = 128;
constexpr int BWD_PAD = 256;
constexpr int BWD_NP2 = BWD_STRIP / 2;
// G staged through shared memory (bwd_staged_walk): BWD_RB rows of the
// CTA's strip per stage, BWD_NST stages in flight
constexpr int BWD_RB = 32;
constexpr int BWD_NST = 4;

// One thread's sums over its strip: G cos(phi) of the hardware columns (+)
// and of the polynomial columns (negated), G sin(phi) per column pair (the
// polynomial pairs negated), and the y sums.
struct BwdAcc {
    float2 sC, nC;
    float2 S[BWD_NP2];
    float sY, sYY;
};

// The x angles of the thread's strip, and the start of its exact
// fixed-point y recurrence.
struct BwdPoint {
    float2 tx[BWD_NP2];
    uint64_t th, dth, d2;
    float xj, yj;
    bool valid;
};

// Polynomial column pairs, spread evenly among the hardware ones.
template <int NPOLY>
__device__ __forceinline__ constexpr bool bwd_poly_pair(int k) {
    return NPOLY > 0 && k % (BWD_STRIP / (NPOLY > 0 ? NPOLY : 1)) == 0 &&
           k / (BWD_STRIP / (NPOLY > 0 ? NPOLY : 1)) < NPOLY / 2;
}

__device__ __forceinline__ void bwd_point(const PointRec *__restrict__ rec,
                                          const float *__restrict__ points, int N,
                                          int j, int x0, BwdPoint &P, BwdAcc &acc) {
    P.valid = j < N;
    PointRec pr{};
    P.xj = 0.0f;
    P.yj = 0.0f;
    if (P.valid) {
        pr = rec[j];
        P.xj = points[2 * j];
        P.yj = points[2 * j + 1];
    }
#pragma unroll
    for (int k = 0; k < BWD_NP2; ++k)
        P.tx[k] = make_float2(
            (float)phase_hi(axis_phase(pr.c, pr.bx, pr.ax, x0 + 2 * k)) * RAD_PER_U32,
            (float)phase_hi(axis_phase(pr.c, pr.bx, pr.ax, x0 + 2 * k + 1)) * RAD_PER_U32);
    // y angle by the fixed-point recurrence: th(y+1) = th(y) + d(y),
    // d(y+1) = d(y) + 2c (exact modulo one turn)
    P.th = pr.ay;
    P.dth = pr.c - pr.by;
    P.d2 = 2 * pr.c;
    const float2 z2 = make_float2(0.0f, 0.0f);
    acc.sC = acc.nC = z2;
#pragma unroll
    for (int k = 0; k < BWD_NP2; ++k) acc.S[k] = z2;
    acc.sY = acc.sYY = 0.0f;
}

// One row y of the strip with G values g.
template <int NPOLY>
__device__ __forceinline__ void bwd_row(BwdPoint &P, int y, const float2 (&g)[BWD_NP2],
                                        BwdAcc &acc) {
    const float ty = (float)phase_hi(P.th) * RAD_PER_U32;
    P.th += P.dth;
    P.dth += P.d2;
    const float dy = (float)y - P.yj;
    const float2 ty2 = make_float2(ty, ty);
    const float2 z2 = make_float2(0.0f, 0.0f);
    float2 rs = z2, nrs = z2;
#pragma unroll
    for (int k = 0; k < BWD_NP2; ++k) {
        const float2 a = __fadd2_rn(P.tx[k], ty2);
        if (bwd_poly_pair<NPOLY>(k)) {
            const float2 u = make_float2(fabsf(a.x) - PI_F, fabsf(a.y) - PI_F);
            const float2 w = __fmul2_rn(u, u);
            float2 c = make_float2(COS5_C5, COS5_C5);
            c = __ffma2_rn(c, w, make_float2(COS5_C4, COS5_C4));
            c = __ffma2_rn(c, w, make_float2(COS5_C3, COS5_C3));
            c = __ffma2_rn(c, w, make_float2(COS5_C2, COS5_C2));
            c = __ffma2_rn(c, w, make_float2(COS5_C1, COS5_C1));
            c = __ffma2_rn(c, w, make_float2(COS5_C0, COS5_C0));  // -cos a
            float2 sn = make_float2(SIN5_C5, SIN5_C5);
            sn = __ffma2_rn(sn, w, make_float2(SIN5_C4, SIN5_C4));
            sn = __ffma2_rn(sn, w, make_float2(SIN5_C3, SIN5_C3));
            sn = __ffma2_rn(sn, w, make_float2(SIN5_C2, SIN5_C2));
            sn = __ffma2_rn(sn, w, make_float2(SIN5_C1, SIN5_C1));
            sn = __ffma2_rn(sn, w, make_float2(SIN5_C0, SIN5_C0));
            float2 v = __fmul2_rn(sn, u);  // sin u
            // -sin a = sign(a) sin u: flip the sign bit where a < 0
            v = make_float2(
                __int_as_float(__float_as_int(v.x) ^ (__float_as_int(a.x) & 0x80000000)),
                __int_as_float(__float_as_int(v.y) ^ (__float_as_int(a.y) & 0x80000000)));
            acc.nC = __ffma2_rn(g[k], c, acc.nC);
            acc.S[k] = __ffma2_rn(g[k], v, acc.S[k]);
            nrs = __ffma2_rn(g[k], v, nrs);
        } else {
            float2 sv, cv;
            __sincosf(a.x, &sv.x, &cv.x);
            __sincosf(a.y, &sv.y, &cv.y);
            acc.sC = __ffma2_rn(g[k], cv, acc.sC);
            acc.S[k] = __ffma2_rn(g[k], sv, acc.S[k]);
            rs = __ffma2_rn(g[k], sv, rs);
        }
    }
    const float r = (rs.x + rs.y) - (nrs.x + nrs.y);
    acc.sY = fmaf(r, dy, acc.sY);
    acc.sYY = fmaf(r * dy, dy, acc.sYY);
}

template <int NPOLY>
__device__ __forceinline__ void bwd_store(const BwdPoint &P, const BwdAcc &acc, int strip,
                                          int j, int Npad, float *__restrict__ part_x,
                                          float *__restrict__ part_y) {
    if (!P.valid) return;
    float *px = part_x + ((size_t)strip * Npad + j) * 3;
    float *py = part_y + ((size_t)strip * Npad + j) * 3;
    const int x0 = strip * BWD_STRIP;
    // the x sums: dx and dx^2 times each column's sum of G sin(phi)
    float sX = 0.0f, sXX = 0.0f;
#pragma unroll
    for (int k = 0; k < BWD_NP2; ++k) {
        const float sgn = bwd_poly_pair<NPOLY>(k) ? -1.0f : 1.0f;
        const float dx0 = (float)(x0 + 2 * k) - P.xj, dx1 = (float)(x0 + 2 * k + 1) - P.xj;
        const float t0 = sgn * acc.S[k].x * dx0, t1 = sgn * acc.S[k].y * dx1;
        sX += t0 + t1;
        sXX = fmaf(t0, dx0, fmaf(t1, dx1, sXX));
    }
    px[0] = (acc.sC.x + acc.sC.y) - (acc.nC.x + acc.nC.y);
    px[1] = sX;
    px[2] = sXX;
    py[0] = 0.0f;
    py[1] = acc.sY;
    py[2] = acc.sYY;
}

// ------------------------------------------------ walks down a strip
// G read from global memory row by row (any alignment, any Nx): calls
// row(y, g) for y = 0 .. Ny-1 with the strip's 16 values as 8 column pairs
// (zero beyond the frame).
template <class ROW>
__device__ __forceinline__ void bwd_global_walk(const float *__restrict__ G, int Nx,
                                                int Ny, int x0, ROW &&row) {
    const int ncols = Nx - x0 < BWD_STRIP ? Nx - x0 : BWD_STRIP;
    // whole 16-byte vectors: a full strip of a 16-byte aligned G whose rows
    // start 16-byte aligned (Nx a multiple of 4)
    const bool vec = (ncols == BWD_STRIP) && ((Nx & 3) == 0) && (((uintptr_t)G & 15) == 0);
#pragma unroll 1
    for (int y = 0; y < Ny; ++y) {
        const float *grow = G + (size_t)y * Nx + x0;
        float2 g[BWD_NP2];
        if (vec) {
#pragma unroll
            for (int k = 0; k < BWD_NP2; k += 2) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(grow + 2 * k));
                g[k] = make_float2(v.x, v.y);
                g[k + 1] = make_float2(v.z, v.w);
            }
        } else {
#pragma unroll
            for (int k = 0; k < BWD_NP2; ++k)
                g[k] = make_float2(2 * k < ncols ? __ldg(grow + 2 * k) : 0.0f,
                                   2 * k + 1 < ncols ? __ldg(grow + 2 * k + 1) : 0.0f);
        }
        row(y, g);
    }
}

// G staged through shared memory: the CTA's 16-column strip arrives BWD_RB
// rows at a time by 2-D TMA loads (zero fill beyond the frame), BWD_NST
// stages in flight, so the row loads do not wait on L2 in the loop.  The
// rows are read from shared memory by every thread at the same address
// (broadcast).  Calls row(y, g) for y = 0 .. Ny-1.  Waits are bounded; after
// a timeout (DEV_TIMEOUT recorded) the CTA's own copies are let land and the
// walk returns false.  Needs G 16-byte aligned and Nx a multiple of 4; every
// thread of the CTA must call it.
template <class ROW>
__device__ __forceinline__ bool bwd_staged_walk(const CUtensorMap &tG, int Ny, int x0,
                                                unsigned *status, ROW &&row) {
    constexpr uint32_t STAGE_BYTES = BWD_RB * BWD_STRIP * sizeof(float);
    __shared__ __align__(128) float sgrow[BWD_NST][BWD_RB][BWD_STRIP];
    __shared__ __align__(8) uint64_t full[BWD_NST];
    __shared__ volatile int abort_flag;
    const int nstage = (Ny + BWD_RB - 1) / BWD_RB;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < BWD_NST; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
        umma::prefetch_tmap(&tG);
    }
    __syncthreads();
    int issued = 0;  // thread 0 only
    if (threadIdx.x == 0)
        for (int s = 0; s < BWD_NST && s < nstage; ++s) {
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            umma::tma_load_2d(&sgrow[s][0][0], &tG, x0, s * BWD_RB, &full[s]);
            ++issued;
        }
    int t = 0;
    for (; t < nstage; ++t) {
        const int s = t % BWD_NST;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((t / BWD_NST) & 1))) {
            abort_flag = 1;
            set_status(status, DEV_TIMEOUT);
        } else {
            const int y0 = t * BWD_RB;
            const int rows = Ny - y0 < BWD_RB ? Ny - y0 : BWD_RB;
#pragma unroll 1
            for (int r = 0; r < rows; ++r) {
                const float4 *src = reinterpret_cast<const float4 *>(&sgrow[s][r][0]);
                float2 g[BWD_NP2];
#pragma unroll
                for (int k = 0; k < BWD_NP2; k += 2) {
                    const float4 v = src[k >> 1];
                    g[k] = make_float2(v.x, v.y);
                    g[k + 1] = make_float2(v.z, v.w);
                }
                row(y0 + r, g);
            }
        }
        __syncthreads();  // every thread is done with slot s
        if (abort_flag) break;
        if (threadIdx.x == 0 && t + BWD_NST < nstage) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            umma::tma_load_2d(&sgrow[s][0][0], &tG, x0, (t + BWD_NST) * BWD_RB, &full[s]);
            ++issued;
        }
    }
    if (abort_flag) {
        if (threadIdx.x == 0)
            for (int u = t; u < issued; ++u)
                mbar_wait_bounded(&full[u % BWD_NST], (uint32_t)((u / BWD_NST) & 1));
        return false;
    }
    return true;
}

// --------------------------------------------------- direct adjoint
template <int NPOLY>
__global__ void __launch_bounds__(BWD_THREADS_GLOBAL)
direct_bwd_kernel(const PointRec *__restrict__ rec, const float *__restrict__ points,
                  int N, int Npad, int Nx, int Ny, const float *__restrict__ G,
                  float *__restrict__ part_x, float *__restrict__ part_y) {
    static_assert(NPOLY % 2 == 0 && NPOLY <= BWD_STRIP, "polynomial column pairs");
    const int strip = blockIdx.x;
    const int j = blockIdx.y * BWD_THREADS_GLOBAL + threadIdx.x;
    const int x0 = strip * BWD_STRIP;
    BwdPoint P;
    BwdAcc acc;
    bwd_point(rec, points, N, j, x0, P, acc);
    bwd_global_walk(G, Nx, Ny, x0, [&](int y, const float2 (&g)[BWD_NP2]) {
        bwd_row<NPOLY>(P, y, g, acc);
    });
    bwd_store<NPOLY>(P, acc, strip, j, Npad, part_x, part_y);
}

template <int NPOLY>
__global__ void __launch_bounds__(BWD_THREADS_STAGED)
direct_bwd_staged_kernel(const __grid_constant__ CUtensorMap tG,
                         const PointRec *__restrict__ rec,
                         const float *__restrict__ points, int N, int Npad, int Ny,
                         float *__restrict__ part_x, float *__restrict__ part_y,
                         unsigned *status) {
    static_assert(NPOLY % 2 == 0 && NPOLY <= BWD_STRIP, "polynomial column pairs");
    const int strip = blockIdx.x;
    const int j = blockIdx.y * BWD_THREADS_STAGED + threadIdx.x;
    const int x0 = strip * BWD_STRIP;
    BwdPoint P;
    BwdAcc acc;
    bwd_point(rec, points, N, j, x0, P, acc);
    if (bwd_staged_walk(tG, Ny, x0, status, [&](int y, const float2 (&g)[BWD_NP2]) {
            bwd_row<NPOLY>(P, y, g, acc);
        }))
        bwd_store<NPOLY>(P, acc, strip, j, Npad, part_x, part_y);
}

// ------------------------------------ FP32 separable adjoint (angle addition)
// The same sums with cos and sin of theta_x + theta_y expanded by angle
// addition: with (cx, sx) of each column's angle and (cy, sy) of each row's,
//     sum_y G cos(phi) = cx U - sx V,   sum_y G sin(phi) = sx U + cx V,
//     U = sum_y G cy,   V = sum_y G sy           (per column, down the strip)
//     sum_x G sin(phi) = cy P + sy Q,
//     P = sum_x G sx,   Q = sum_x G cx           (per row, across the strip)
// Per update: 4 FP32 multiply-adds (U, V, P, Q) and no MUFU operation; the
// row's sincos (2 MUFU) and the column's (once per strip) are shared by 16
// updates.  FP32 throughout, like the FP32 separable forward.
struct Sep32Point {
    float2 cx[BWD_NP2], sx[BWD_NP2];
    uint64_t th, dth, d2;
    float xj, yj;
    bool valid;
};

struct Sep32Acc {
    float2 U[BWD_NP2], V[BWD_NP2];
    float sY, sYY;
};

__device__ __forceinline__ void sep32_point(const PointRec *__restrict__ rec,
                                            const float *__restrict__ points, int N,
                                            int j, int x0, Sep32Point &P, Sep32Acc &acc) {
    P.valid = j < N;
    PointRec pr{};
    P.xj = 0.0f;
    P.yj = 0.0f;
    if (P.valid) {
        pr = rec[j];
        P.xj = points[2 * j];
        P.yj = points[2 * j + 1];
    }
    const float2 z2 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < BWD_NP2; ++k) {
        const float a0 =
            (float)phase_hi(axis_phase(pr.c, pr.bx, pr.ax, x0 + 2 * k)) * RAD_PER_U32;
        const float a1 =
            (float)phase_hi(axis_phase(pr.c, pr.bx, pr.ax, x0 + 2 * k + 1)) * RAD_PER_U32;
        __sincosf(a0, &P.sx[k].x, &P.cx[k].x);
        __sincosf(a1, &P.sx[k].y, &P.cx[k].y);
        acc.U[k] = acc.V[k] = z2;
    }
    // y angle by the fixed-point recurrence (as bwd_point)
    P.th = pr.ay;
    P.dth = pr.c - pr.by;
    P.d2 = 2 * pr.c;
    acc.sY = acc.sYY = 0.0f;
}

__device__ __forceinline__ void sep32_row(Sep32Point &P, int y, const float2 (&g)[BWD_NP2],
                                          Sep32Acc &acc) {
    const float ty = (float)phase_hi(P.th) * RAD_PER_U32;
    P.th += P.dth;
    P.dth += P.d2;
    float sy, cy;
    __sincosf(ty, &sy, &cy);
    const float dy = (float)y - P.yj;
    const float2 cy2 = make_float2(cy, cy), sy2 = make_float2(sy, sy);
    float2 p2 = make_float2(0.0f, 0.0f), q2 = p2;
#pragma unroll
    for (int k = 0; k < BWD_NP2; ++k) {
        acc.U[k] = __ffma2_rn(g[k], cy2, acc.U[k]);
        acc.V[k] = __ffma2_rn(g[k], sy2, acc.V[k]);
        p2 = __ffma2_rn(g[k], P.sx[k], p2);
        q2 = __ffma2_rn(g[k], P.cx[k], q2);
    }
    const float r = fmaf(cy, p2.x + p2.y, sy * (q2.x + q2.y));
    acc.sY = fmaf(r, dy, acc.sY);
    acc.sYY = fmaf(r * dy, dy, acc.sYY);
}

__device__ __forceinline__ void sep32_store(const Sep32Point &P, const Sep32Acc &acc,
                                            int strip, int j, int Npad,
                                            float *__restrict__ part_x,
                                            float *__restrict__ part_y) {
    if (!P.valid) return;
    float *px = part_x + ((size_t)strip * Npad + j) * 3;
    float *py = part_y + ((size_t)strip * Npad + j) * 3;
    const int x0 = strip * BWD_STRIP;
    float C = 0.0f, sX = 0.0f, sXX = 0.0f;
#pragma unroll
    for (int k = 0; k < BWD_NP2; ++k) {
        const float2 cx = P.cx[k], sx = P.sx[k], U = acc.U[k], V = acc.V[k];
        C += fmaf(cx.x, U.x, -sx.x * V.x) + fmaf(cx.y, U.y, -sx.y * V.y);
        const float s0 = fmaf(sx.x, U.x, cx.x * V.x), s1 = fmaf(sx.y, U.y, cx.y * V.y);
        const float dx0 = (float)(x0 + 2 * k) - P.xj, dx1 = (float)(x0 + 2 * k + 1) - P.xj;
        const float t0 = s0 * dx0, t1 = s1 * dx1;
        sX += t0 + t1;
        sXX = fmaf(t0, dx0, fmaf(t1, dx1, sXX));
    }
    px[0] = C;
    px[1] = sX;
    px[2] = sXX;
    py[0] = 0.0f;
    py[1] = acc.sY;
    py[2] = acc.sYY;
}

__global__ void __launch_bounds__(BWD_THREADS_GLOBAL)
sep32_bwd_kernel(const PointRec *__restrict__ rec, const float *__restrict__ points,
                 int N, int Npad, int Nx, int Ny, const float *__restrict__ G,
                 float *__restrict__ part_x, float *__restrict__ part_y) {
    const int strip = blockIdx.x;
    const int j = blockIdx.y * BWD_THREADS_GLOBAL + threadIdx.x;
    const int x0 = strip * BWD_STRIP;
    Sep32Point P;
    Sep32Acc acc;
    sep32_point(rec, points, N, j, x0, P, acc);
    bwd_global_walk(G, Nx, Ny, x0, [&](int y, const float2 (&g)[BWD_NP2]) {
        sep32_row(P, y, g, acc);
    });
    sep32_store(P, acc, strip, j, Npad, part_x, part_y);
}

__global__ void __launch_bounds__(BWD_THREADS_STAGED)
sep32_bwd_staged_kernel(const __grid_constant__ CUtensorMap tG,
                        const PointRec *__restrict__ rec,
                        const float *__restrict__ points, int N, int Npad, int Ny,
                        float *__restrict__ part_x, float *__restrict__ part_y,
                        unsigned *status) {
    const int strip = blockIdx.x;
    const int j = blockIdx.y * BWD_THREADS_STAGED + threadIdx.x;
    const int x0 = strip * BWD_STRIP;
    Sep32Point P;
    Sep32Acc acc;
    sep32_point(rec, points, N, j, x0, P, acc);
    if (bwd_staged_walk(tG, Ny, x0, status, [&](int y, const float2 (&g)[BWD_NP2]) {
            sep32_row(P, y, g, acc);
        }))
        sep32_store(P, acc, strip, j, Npad, part_x, part_y);
}

// ------------------------------------------------------------ reduce
// One block per RD_PTS points; its RD_SL slices of threads take every
// RD_SL-th partial-sum tile of their point (FP64), then slice 0 adds the
// slices' sums in slice order: deterministic, and enough threads in flight
// to cover the loads' latency (one thread per point walking ~100 tiles
// left the SMs nearly empty).
constexpr int RD_PTS = 32, RD_SL = 8;

__global__ void __launch_bounds__(RD_PTS * RD_SL)
adjoint_reduce_kernel(const PointRec *__restrict__ rec, const float *__restrict__ z,
                      int N, int Npad, const float *__restrict__ part_x, int Tx,
                      const float *__restrict__ part_y, int Ty, const unsigned *gword,
                      float *gpts, float *gA, float *gz) {
    __shared__ double part[RD_SL][5][RD_PTS];
    const int lj = threadIdx.x % RD_PTS, sl = threadIdx.x / RD_PTS;
    const int j = blockIdx.x * RD_PTS + lj;
    double sC = 0, sX = 0, sXX = 0, sY = 0, sYY = 0;
    if (j < N) {
        for (int t = sl; t < Tx; t += RD_SL) {
            const float *p = part_x + ((size_t)t * Npad + j) * 3;
            sC += p[0];
            sX += p[1];
            sXX += p[2];
        }
        for (int t = sl; t < Ty; t += RD_SL) {
            const float *p = part_y + ((size_t)t * Npad + j) * 3;
            sY += p[1];
            sYY += p[2];
        }
    }
    part[sl][0][lj] = sC;
    part[sl][1][lj] = sX;
    part[sl][2][lj] = sXX;
    part[sl][3][lj] = sY;
    part[sl][4][lj] = sYY;
    __syncthreads();
    if (sl != 0 || j >= N) return;
    sC = sX = sXX = sY = sYY = 0;
#pragma unroll
    for (int q = 0; q < RD_SL; ++q) {
        sC += part[q][0][lj];
        sX += part[q][1][lj];
        sXX += part[q][2][lj];
        sY += part[q][3][lj];
        sYY += part[q][4][lj];
    }
    const PointRec r = rec[j];
    const bool ok = r.Q32 > 0.0f;
    const double inv = gword ? 1.0 / (double)g_scale(*gword) : 1.0;
    const double P = 6.283185307179586 * (double)r.Q32;
    const double a = (double)r.A;
    if (gA) gA[j] = ok ? (float)(sC * inv) : 0.0f;
    if (gpts) {
        gpts[2 * j] = ok ? (float)(2.0 * P * a * sX * inv) : 0.0f;
        gpts[2 * j + 1] = ok ? (float)(2.0 * P * a * sY * inv) : 0.0f;
    }
    if (gz) gz[j] = ok ? (float)(P * a / (double)z[j] * (sXX + sYY) * inv) : 0.0f;
}

}  // namespace cgh

using namespace cgh;

static cgh_status run_backward(cgh_ctx *h, const float *points, const float *A,
                               const float *z, int N, double lambda, double p,
                               int Nx, int Ny, const float *G, float *gpts,
                               float *gA, float *gz, int method, cudaStream_t s) {
    const bool sep = method == CGH_SEP_FP16X3;
    const bool sep32 = method == CGH_SEP_FP32;  // strip kernels like the direct one
    const int Kp = pad_to(2 * N, 128);   // GEMM rows: whole 128-row tiles
    const int Npad = sep ? Kp / 2 : pad_to(N, BWD_PAD);
    const int ldx = pad_to(Nx, 8), ldy = pad_to(Ny, 8);
    // partial-sum tiles: allocated for the narrowest GEMM column tile (128);
    // the GEMM launches report the width they used
    int Tx = sep ? (Nx + umma_tile_n() - 1) / umma_tile_n()
                 : (Nx + BWD_STRIP - 1) / BWD_STRIP;
    int Ty = sep ? (Ny + umma_tile_n() - 1) / umma_tile_n() : Tx;
    const size_t word_b = 256;
    const size_t rec_b = align256((size_t)Npad * sizeof(PointRec));
    const size_t px_b = align256((size_t)Tx * Npad * 3 * sizeof(float));
    const size_t py_b = align256((size_t)Ty * Npad * 3 * sizeof(float));
    size_t total = word_b + rec_b + px_b + py_b;
    size_t u_b = 0, v_b = 0, gr_b = 0, gt_b = 0;
    if (sep) {
        u_b = align256((size_t)Kp * ldx * 2);
        v_b = align256((size_t)Kp * ldy * 2);
        gr_b = align256((size_t)Ny * ldx * 2);
        gt_b = align256((size_t)Nx * ldy * 2);
        total += 2 * (u_b + v_b + gr_b + gt_b);
    }
    cgh_status st = h->ensure(h->ws2, total, s, "adjoint workspace");
    if (st) return st;
    char *b = (char *)h->ws2.ptr;
    unsigned *gword = (unsigned *)b;
    PointRec *rec = (PointRec *)(b + word_b);
    float *part_x = (float *)(b + word_b + rec_b);
    float *part_y = (float *)(b + word_b + rec_b + px_b);
    char *q = b + word_b + rec_b + px_b + py_b;

    {
        TimedLaunch tl(h, CGH_K_PROLOGUE, s);
        cudaError_t e = launch_prologue(points, A, z, N, Npad, lambda, p, rec,
                                        h->d_status, s);
        if (e != cudaSuccess) return h->cuda_fail(e, "prologue launch");
        tl.done();
    }
    if (!sep) {
        TimedLaunch tl(h, sep32 ? CGH_K_BWD_SIMT : CGH_K_BWD_DIRECT, s);
        const dim3 grid_st(Tx, Npad / BWD_THREADS_STAGED);
        const dim3 grid_gl(Tx, Npad / BWD_THREADS_GLOBAL);
        // G through shared memory by TMA when its layout allows (16-byte
        // aligned rows), else row loads from global memory
        CUtensorMap tG;
        const bool staged = h->bwd_staged && (((uintptr_t)G & 15) == 0) && (Nx % 4 == 0) &&
                            make_f32_map(&tG, G, Nx, Ny, Nx, BWD_STRIP, BWD_RB);
        if (sep32 && staged) {
            sep32_bwd_staged_kernel<<<grid_st, BWD_THREADS_STAGED, 0, s>>>(
                tG, rec, points, N, Npad, Ny, part_x, part_y, h->d_status);
        } else if (sep32) {
            sep32_bwd_kernel<<<grid_gl, BWD_THREADS_GLOBAL, 0, s>>>(rec, points, N, Npad, Nx,
                                                                   Ny, G, part_x, part_y);
        } else if (staged) {
            if (h->bwd_poly == 0)
                direct_bwd_staged_kernel<0><<<grid_st, BWD_THREADS_STAGED, 0, s>>>(
                    tG, rec, points, N, Npad, Ny, part_x, part_y, h->d_status);
            else if (h->bwd_poly == 6)
                direct_bwd_staged_kernel<6><<<grid_st, BWD_THREADS_STAGED, 0, s>>>(
                    tG, rec, points, N, Npad, Ny, part_x, part_y, h->d_status);
            else
                direct_bwd_staged_kernel<4><<<grid_st, BWD_THREADS_STAGED, 0, s>>>(
                    tG, rec, points, N, Npad, Ny, part_x, part_y, h->d_status);
        } else if (h->bwd_poly == 0) {
            direct_bwd_kernel<0><<<grid_gl, BWD_THREADS_GLOBAL, 0, s>>>(rec, points, N, Npad, Nx,
                                                               Ny, G, part_x, part_y);
        } else if (h->bwd_poly == 6) {
            direct_bwd_kernel<6><<<grid_gl, BWD_THREADS_GLOBAL, 0, s>>>(rec, points, N, Npad, Nx,
                                                               Ny, G, part_x, part_y);
        } else {
            direct_bwd_kernel<4><<<grid_gl, BWD_THREADS_GLOBAL, 0, s>>>(rec, points, N, Npad, Nx,
                                                               Ny, G, part_x, part_y);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return h->cuda_fail(e, "direct adjoint launch");
        tl.done();
    } else {
        __half *Uhi = (__half *)q, *Ulo = (__half *)(q + u_b);
        __half *Vhi = (__half *)(q + 2 * u_b), *Vlo = (__half *)(q + 2 * u_b + v_b);
        char *q2 = q + 2 * (u_b + v_b);
        __half *Grh = (__half *)q2, *Grl = (__half *)(q2 + gr_b);
        __half *Gth = (__half *)(q2 + 2 * gr_b), *Gtl = (__half *)(q2 + 2 * gr_b + gt_b);
        cudaError_t e = cudaMemsetAsync(gword, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return h->cuda_fail(e, "cudaMemsetAsync");
        {
            TimedLaunch tl(h, CGH_K_AUX, s);
            const long long n = (long long)Nx * Ny;
            long long blocks = (n + 255) / 256;
            if (blocks > 152 * 8) blocks = 152 * 8;
            g_absmax_kernel<<<(int)blocks, 256, 0, s>>>(G, n, gword);
            e = cudaGetLastError();
            if (e != cudaSuccess) return h->cuda_fail(e, "G max launch");
            tl.done();
        }
        {
            TimedLaunch tl(h, CGH_K_AUX, s);
            dim3 grid((Nx + 31) / 32, (Ny + 31) / 32);
            g_convert_kernel<<<grid, dim3(32, 8), 0, s>>>(G, Nx, Ny, gword, Grh, Grl,
                                                          ldx, Gth, Gtl, ldy);
            e = cudaGetLastError();
            if (e != cudaSuccess) return h->cuda_fail(e, "G convert launch");
            tl.done();
        }
        {
            TimedLaunch tl(h, CGH_K_SEP_TABLES, s);
            e = cudaSuccess;
            const int span = 65535 * AT_POINTS;
            for (int j0 = 0; j0 < Npad && e == cudaSuccess; j0 += span) {
                const int nj = Npad - j0 < span ? Npad - j0 : span;
                dim3 grid((Nx + Ny + 255) / 256, (nj + AT_POINTS - 1) / AT_POINTS);
                adj_tables_kernel<<<grid, 256, 0, s>>>(rec, N, Npad, j0, Nx, Ny, ldx,
                                                       ldy, Uhi, Ulo, Vhi, Vlo);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) return h->cuda_fail(e, "adjoint tables launch");
            tl.done();
        }
        // D1[k][x] = sum_y V'[k][y] G[y][x]: A = V' (Kp x Ny), B = G^T (Nx x Ny)
        GemmOperands o1{};
        o1.A_hi = Vhi; o1.A_lo = Vlo; o1.B_hi = Gth; o1.B_lo = Gtl;
        o1.M = Kp; o1.N = Nx; o1.K = Ny; o1.lda = ldy; o1.ldb = ldy;
        o1.bf16 = false; o1.split = true; o1.lo_scale = 1.0f / ADJ_LO_SCALE;
        o1.D = nullptr; o1.ldd = Nx;
        // D2[k][y] = sum_x U'[k][x] G[y][x]: A = U' (Kp x Nx), B = G (Ny x Nx)
        GemmOperands o2 = o1;
        o2.A_hi = Uhi; o2.A_lo = Ulo; o2.B_hi = Grh; o2.B_lo = Grl;
        o2.M = Kp; o2.N = Ny; o2.K = Nx; o2.lda = ldx; o2.ldb = ldx; o2.ldd = Ny;
        // (the generating GEMM is a forward kernel: the adjoint's GEMMs
        // take CTA pairs then)
        o1.tiles = o2.tiles =
            h->gemm_tiles == CGH_GEMM_PAIRS_GEN ? CGH_GEMM_PAIRS : h->gemm_tiles;
        int wx = 128, wy = 128;  // column width of one partial-sum tile
        {
            TimedLaunch tl(h, CGH_K_BWD_GEMM, s);
            e = launch_umma_adjoint(o1, rec, points, N, Npad, 0, part_x, h->d_status, s,
                                    &wx);
            if (e != cudaSuccess) return h->cuda_fail(e, "adjoint GEMM (x) launch");
            tl.done();
        }
        {
            TimedLaunch tl(h, CGH_K_BWD_GEMM, s);
            e = launch_umma_adjoint(o2, rec, points, N, Npad, 1, part_y, h->d_status, s,
                                    &wy);
            if (e != cudaSuccess) return h->cuda_fail(e, "adjoint GEMM (y) launch");
            tl.done();
        }
        Tx = (Nx + wx - 1) / wx;
        Ty = (Ny + wy - 1) / wy;
    }
    {
        TimedLaunch tl(h, CGH_K_BWD_REDUCE, s);
        adjoint_reduce_kernel<<<(N + RD_PTS - 1) / RD_PTS, RD_PTS * RD_SL, 0, s>>>(
            rec, z, N, Npad, part_x, Tx, part_y, Ty, sep ? gword : nullptr, gpts, gA,
            gz);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return h->cuda_fail(e, "adjoint reduce launch");
        tl.done();
    }
    return CGH_OK;
}

extern "C" cgh_status cgh_backward(cgh_handle h, const float *points,
                                   const float *A, const float *z, int N,
                                   double lambda, double p, int Nx, int Ny,
                                   const float *grad_out, float *grad_points,
                                   float *grad_A, float *grad_z, int method,
                                   void *stream) {
    NvtxRange range("cgh_backward");
    if (!h) return CGH_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    h->err[0] = 0;
    cgh_status st = h->check_problem(points, A, z, N, lambda, p, Nx, Ny, grad_out);
    if (st == CGH_OK && method != CGH_DIRECT_FP32 && method != CGH_SEP_FP16X3 &&
        method != CGH_SEP_FP32)
        st = h->fail(CGH_ERR_INVALID_ARG,
                     "adjoint method must be CGH_DIRECT_FP32, CGH_SEP_FP32 or CGH_SEP_FP16X3");
    if (st == CGH_OK &&
        ((((uintptr_t)grad_points) | ((uintptr_t)grad_A) | ((uintptr_t)grad_z)) & 3))
        st = h->fail(CGH_ERR_INVALID_ARG, "gradient arrays must be 4-byte aligned");
    if (st == CGH_OK && N > 0 && (grad_points || grad_A || grad_z))
        st = run_backward(h, points, A, z, N, lambda, p, Nx, Ny, grad_out,
                          grad_points, grad_A, grad_z, method, (cudaStream_t)stream);
    if (prev != h->device) cudaSetDevice(prev);
    return st;
}
