// direct_tile.cuh -- the staged point loop of the direct kernel for one
// pixel tile, shared by the single-hologram kernel (direct.cu) and the
// persistent batch kernel (batch.cu).  Internal to libcgh.
#pragma once

#include "common.cuh"
#include "cos_poly.h"

namespace cgh {

// The tile shapes compiled in: X(TX, TY, VX, VY, PT, NST, NP, G) = pixels
// per CTA along x and y, pixels per thread along x and y, points per
// shared-memory stage, stages, how many of each thread's VX * VY pixels take
// the FMA-pipe cosine polynomial instead of the MUFU cosine (about a quarter
// balances the two pipes), G, the number of thread groups that split
// each stage's points between them (their partial sums are added in a fixed
// order at the end), and PK: 0 scalar, 1 packed FP32x2 arithmetic on pixel
// pairs along x (half the issue slots for the adds and FMAs), 2 packed with
// the degree-5 polynomial, 3 as 2 with the polynomial pixel pairs spread over
// the thread's block instead of leading it, 4 and 5 as 3 with one pixel pair
// more on the polynomial for every second point (4) or every fourth point
// (5) -- average shares between NP and NP + 2 pixels -- and 6, the rotation
// form: the first pixel of each of a thread's rows takes the hardware sincos
// of its phase, and the row's other three pixels follow by angle addition
// with the tabulated cosine and sine of their exact phase offsets along x
// (the complex form of the paper's Eq. 2 step along a row: one MUFU
// operation per two pixels, no polynomial; VX = 4); and 7, the rotation form
// along both axes: only the thread's first pixel takes the hardware sincos,
// its first-column pixels follow by angle addition with the tabulated row
// offsets, and every row then as in 6 (one sincos per thread and point, two
// FMAs per pixel); 8 as 7 on packed FP32x2 pixel pairs.  Every shape has 256
// threads per CTA.
#define CGH_DIRECT_TILES(X)                \
    X(64, 64, 4, 4, 32, 3, 4, 1, 0)        \
    X(64, 64, 4, 4, 32, 3, 0, 1, 0)        \
    X(64, 32, 4, 2, 32, 3, 2, 1, 0)        \
    X(128, 32, 4, 4, 32, 3, 4, 1, 0)       \
    X(32, 32, 2, 2, 64, 3, 1, 1, 0)        \
    X(32, 32, 2, 2, 64, 3, 0, 1, 0)        \
    X(128, 64, 8, 4, 16, 3, 8, 1, 0)       \
    X(64, 16, 4, 1, 64, 3, 1, 1, 0)        \
    X(32, 32, 4, 4, 64, 3, 4, 4, 0)        \
    X(32, 32, 4, 4, 64, 3, 0, 4, 0)        \
    X(64, 32, 4, 4, 64, 3, 4, 2, 0)        \
    X(64, 64, 8, 4, 64, 3, 8, 2, 0)        \
    X(32, 32, 4, 4, 64, 3, 4, 4, 1)        \
    X(32, 32, 4, 4, 64, 3, 6, 4, 1)        \
    X(64, 32, 4, 4, 64, 3, 6, 2, 1)        \
    X(64, 64, 8, 4, 64, 3, 10, 2, 1)       \
    X(32, 32, 4, 4, 64, 3, 4, 4, 2)        \
    X(32, 32, 4, 4, 64, 3, 6, 4, 2)        \
    X(32, 32, 4, 4, 32, 3, 4, 4, 2)        \
    X(32, 32, 4, 4, 64, 3, 4, 4, 3)        \
    X(32, 32, 4, 4, 64, 3, 6, 4, 3)        \
    X(32, 32, 4, 4, 64, 3, 4, 4, 4)        \
    X(32, 32, 4, 4, 64, 3, 4, 4, 5)        \
    X(32, 32, 4, 4, 64, 3, 0, 4, 6)        \
    X(32, 32, 4, 4, 64, 3, 0, 4, 7)        \
    X(32, 32, 8, 4, 64, 3, 0, 8, 7)        \
    X(64, 32, 8, 4, 32, 3, 0, 4, 7)        \
    X(64, 64, 8, 4, 32, 3, 0, 2, 7)        \
    X(64, 32, 8, 4, 64, 2, 0, 4, 7)        \
    X(64, 64, 16, 4, 32, 3, 0, 4, 7)       \
    X(64, 32, 16, 4, 64, 2, 0, 8, 7)       \
    X(64, 64, 8, 8, 32, 3, 0, 4, 7)        \
    X(64, 32, 8, 8, 64, 2, 0, 8, 7)        \
    X(64, 32, 8, 4, 32, 3, 0, 4, 8)        \
    X(64, 64, 8, 4, 32, 3, 0, 2, 8)        \
    X(32, 32, 4, 4, 64, 3, 0, 4, 8)        \
    X(64, 64, 8, 8, 32, 3, 0, 4, 8)

// ------------------------------------------------------------- tables
// The rotation tables.  Along an axis with rotation group size gs (the
// thread's pixels along that axis), the coordinates g0 .. g0 + gs - 1 of a
// group share 2 gs slots: 0: the angle at g0; k = 1 .. gs - 1: cos of the
// exact phase offset of coordinate g0 + k from g0; gs: 0 (the sine of
// coordinate g0's zero offset); gs + k: sin of the offset of g0 + k.  The
// offsets are exact in fixed point; their sines and cosines are accurate
// (sincospi of the offset in turns).
__device__ __forceinline__ float rotation_entry(uint64_t c, uint64_t b, uint64_t a, int g0,
                                                int gs, int slot) {
    if (slot == 0) return (float)phase_hi(axis_phase(c, b, a, g0)) * RAD_PER_U32;
    if (slot == gs) return 0.0f;
    const int k = slot < gs ? slot : slot - gs;
    const uint64_t d = axis_phase(c, b, a, g0 + k) - axis_phase(c, b, a, g0);
    float s, co;
    sincospif(2.0f * ((float)phase_hi(d) * TURN_PER_U32), &s, &co);
    return slot < gs ? co : s;
}

// Position of slot `slot` of group g within one point's row of a tile's
// rotation table with ng groups: the slots go in fours, and the k-th four
// of every group sit side by side (so a warp's 16-byte loads of the same
// four of neighbouring groups hit distinct banks).
__host__ __device__ constexpr int rotation_pos(int g, int slot, int ng) {
    return (slot >> 2) * ng * 4 + g * 4 + (slot & 3);
}

// The inverse: the (group, slot) of position pos of a row with ng groups.
__device__ __forceinline__ void rotation_slot(int pos, int ng, int &g, int &slot) {
    const int j = pos / (ng * 4), r = pos - j * ng * 4;
    g = r >> 2;
    slot = j * 4 + (r & 3);
}

// Entries of the per-axis tables of one problem: x values laid out
// [x tile][point][x in tile] (xg ? 2 : 1 floats per column, rotation groups
// of xg columns), then y values [y tile][point][y in tile] (likewise with
// yg), then the amplitudes [point].
__device__ __forceinline__ long long direct_table_entries(int Npad, int TX, int TY, int nxt,
                                                          int nyt, int xg, int yg) {
    return (long long)nxt * Npad * TX * (xg ? 2 : 1) +
           (long long)nyt * Npad * TY * (yg ? 2 : 1) + Npad;
}

__device__ __forceinline__ float axis_table_entry(uint64_t c, uint64_t b, uint64_t a,
                                                  int T, int gs, int t, int i) {
    if (gs) {
        int g, slot;
        rotation_slot(i, T / gs, g, slot);
        return rotation_entry(c, b, a, t * T + g * gs, gs, slot);
    }
    return (float)phase_hi(axis_phase(c, b, a, t * T + i)) * RAD_PER_U32;
}

__device__ __forceinline__ void direct_table_entry(
    const PointRec *__restrict__ rec, int Npad, int TX, int TY, int nxt,
    int nyt, int xg, int yg, long long e, float *__restrict__ phx,
    float *__restrict__ phy, float *__restrict__ amp) {
    const int rx = TX * (xg ? 2 : 1), ry = TY * (yg ? 2 : 1);
    const long long nx_e = (long long)nxt * Npad * rx;
    const long long ny_e = (long long)nyt * Npad * ry;
    if (e < nx_e) {
        const long long per = (long long)Npad * rx;
        const int t = (int)(e / per);
        const long long rem = e - (long long)t * per;
        const int j = (int)(rem / rx);
        const int i = (int)(rem - (long long)j * rx);
        const PointRec &r = rec[j];
        phx[e] = axis_table_entry(r.c, r.bx, r.ax, TX, xg, t, i);
    } else if (e < nx_e + ny_e) {
        const long long f = e - nx_e;
        const long long per = (long long)Npad * ry;
        const int t = (int)(f / per);
        const long long rem = f - (long long)t * per;
        const int j = (int)(rem / ry);
        const int i = (int)(rem - (long long)j * ry);
        const PointRec &r = rec[j];
        phy[f] = axis_table_entry(r.c, r.by, r.ay, TY, yg, t, i);
    } else {
        const int j = (int)(e - nx_e - ny_e);
        amp[j] = rec[j].A;
    }
}

template <int N>
struct VecLoad;
template <>
struct VecLoad<1> {
    __device__ static void ld(float *v, const float *p) { v[0] = p[0]; }
};
template <>
struct VecLoad<2> {
    __device__ static void ld(float *v, const float *p) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x;
        v[1] = t.y;
    }
};
template <>
struct VecLoad<4> {
    __device__ static void ld(float *v, const float *p) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
};
template <>
struct VecLoad<8> {
    __device__ static void ld(float *v, const float *p) {
        VecLoad<4>::ld(v, p);
        VecLoad<4>::ld(v + 4, p + 4);
    }
};

// cos(theta) for |theta| < 2 pi on the FMA pipe: with u = |theta| - pi in
// [-pi, pi), cos(theta) = cos(|theta|) = -cos(u), and cos(u) is the degree-6
// polynomial in u^2 of cos_poly.h (max error about 6e-7, like the hardware
// cosine's 2^-21.4 on [-pi, pi]).  The caller folds the sign into A.
constexpr float PI_F = 3.14159265358979323846f;

__device__ __forceinline__ float neg_cos_poly(float th) {
    const float u = fabsf(th) - PI_F;
    const float s = u * u;
    float p = COS_C6;
    p = fmaf(p, s, COS_C5);
    p = fmaf(p, s, COS_C4);
    p = fmaf(p, s, COS_C3);
    p = fmaf(p, s, COS_C2);
    p = fmaf(p, s, COS_C1);
    p = fmaf(p, s, COS_C0);
    return p;  // = -cos(th)
}

// The same for two angles at once with packed FP32x2 arithmetic; DEG 6 (the
// table above) or 5 (COS5_C, max error about 1.3e-6, one FMA fewer).
template <int DEG>
__device__ __forceinline__ float2 neg_cos_poly2(float2 th) {
    const float2 u = make_float2(fabsf(th.x) - PI_F, fabsf(th.y) - PI_F);
    const float2 s = __fmul2_rn(u, u);
    float2 p;
    if constexpr (DEG == 6) {
        p = make_float2(COS_C6, COS_C6);
        p = __ffma2_rn(p, s, make_float2(COS_C5, COS_C5));
        p = __ffma2_rn(p, s, make_float2(COS_C4, COS_C4));
        p = __ffma2_rn(p, s, make_float2(COS_C3, COS_C3));
        p = __ffma2_rn(p, s, make_float2(COS_C2, COS_C2));
        p = __ffma2_rn(p, s, make_float2(COS_C1, COS_C1));
        p = __ffma2_rn(p, s, make_float2(COS_C0, COS_C0));
    } else {
        p = make_float2(COS5_C5, COS5_C5);
        p = __ffma2_rn(p, s, make_float2(COS5_C4, COS5_C4));
        p = __ffma2_rn(p, s, make_float2(COS5_C3, COS5_C3));
        p = __ffma2_rn(p, s, make_float2(COS5_C2, COS5_C2));
        p = __ffma2_rn(p, s, make_float2(COS5_C1, COS5_C1));
        p = __ffma2_rn(p, s, make_float2(COS5_C0, COS5_C0));
    }
    return p;  // = (-cos(th.x), -cos(th.y))
}

// Per-thread accumulators: VY x VX floats, or VY x VX/2 packed pairs.
template <int VY, int VX, bool PK>
struct DirectAcc {
    float v[VY][VX];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < VY; ++i)
#pragma unroll
            for (int k = 0; k < VX; ++k) v[i][k] = 0.0f;
    }
    __device__ __forceinline__ float get(int i, int k) const { return v[i][k]; }
    __device__ __forceinline__ void add(int i, int k, float x) { v[i][k] += x; }
};

template <int VY, int VX>
struct DirectAcc<VY, VX, true> {
    static_assert(VX % 2 == 0, "packed pairs along x");
    float2 v[VY][VX / 2];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < VY; ++i)
#pragma unroll
            for (int k = 0; k < VX / 2; ++k) v[i][k] = make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ float get(int i, int k) const {
        return (k & 1) ? v[i][k >> 1].y : v[i][k >> 1].x;
    }
    __device__ __forceinline__ void add(int i, int k, float x) {
        if (k & 1)
            v[i][k >> 1].y += x;
        else
            v[i][k >> 1].x += x;
    }
};

template <int TX, int TY, int VX, int VY, int PT, int NST, int G = 1, int XF = 1,
          int YF = 1>
struct DirectShape {
    static constexpr int NTX = TX / VX;
    static constexpr int NTY = TY / VY;
    static constexpr int GT = NTX * NTY;        // threads of one point group
    static constexpr int THREADS = G * GT;
    static constexpr int PG = PT / G;           // points per group per stage
    static constexpr int SX = PT * TX * XF;     // floats of x values per stage
    static constexpr int SY = PT * TY * YF;     // floats of y values per stage
    static constexpr int SA = PT;               // amplitudes per stage
    static constexpr int STAGE = SX + SY + SA;
    static constexpr size_t SMEM = (size_t)NST * STAGE * sizeof(float);
    static_assert(TX % VX == 0 && TY % VY == 0, "tile not divisible");
    static_assert(PT % 4 == 0, "bulk copies need 16-byte multiples");
    static_assert(PT % G == 0, "points of a stage split evenly over groups");
    static_assert((STAGE * 4) % 16 == 0, "stage alignment");
    static_assert((size_t)(G - 1) * TX * TY <= (size_t)NST * STAGE,
                  "partial sums of the extra groups fit in the stage ring");
};

// Per-CTA driver of the staged loop.  Point tile t of a pixel tile is the
// (g0 + t)-th stage load of the CTA, so a persistent CTA can run many pixel
// tiles back to back on the same NST-slot ring and mbarriers: slot
// (g0 + t) % NST, barrier parity ((g0 + t) / NST) & 1.
template <int TX, int TY, int VX, int VY, int PT, int NST, int NP, int G,
          int PKV>
struct DirectTileLoop {
    // PKV: 0 scalar arithmetic, 1 packed FP32x2 with the degree-6 polynomial,
    // 2 packed with the degree-5 polynomial, 3 as 2 with the polynomial pairs
    // interleaved, 4 and 5 as 3 with one extra polynomial pair on every
    // second (4) or fourth (5) point; 6-8 the rotation forms (one sincos per
    // thread row (6) or per thread (7 scalar, 8 packed) and point)
    static constexpr bool PK = PKV != 0;
    static constexpr int NPAIRS = VX * VY / 2;
    // points per period of the polynomial pattern
    // (the rotation forms take their amplitudes four at a time too)
    static constexpr int PERIOD = PKV == 4 ? 2 : (PKV == 5 || PKV >= 6) ? 4 : 1;
    static_assert(NP >= 0 && NP <= VX * VY, "polynomial pixels per thread");
    static_assert(!PK || NP % 2 == 0, "packed pairs take the polynomial together");
    static_assert(PKV < 4 || PKV >= 6 || (NP / 2 + 1 <= NPAIRS && (PT / G) % PERIOD == 0),
                  "the extra polynomial pair fits and the periods tile a stage");
    static_assert(PKV < 6 || (VX % 4 == 0 && NP == 0 && (PT / G) % 4 == 0),
                  "the rotation forms: columns in fours, no polynomial, points in fours");
    static_assert(PKV != 6 || VX == 4, "the row rotation form: 4 columns");
    static_assert(PKV < 7 || VY % 4 == 0, "the two-axis rotation form: rows in fours");
    static constexpr int XF = direct_xf(PKV);
    static constexpr int YF = direct_yf(PKV);
    using S = DirectShape<TX, TY, VX, VY, PT, NST, G, XF, YF>;
    // CTAs per SM the register allocation must leave room for: for the
    // rotation forms, two with 64-pixel blocks (at most 128 registers a
    // thread), three with 32-pixel blocks (at most 85)
    static constexpr int MIN_CTAS = PKV < 7 ? 1 : VX * VY >= 64 ? 2 : 3;
    // (the two-axis rotation form updates its pixels one by one)
    using Acc = DirectAcc<VY, VX, PK && PKV != 7>;
    static_assert(PKV != 8 || VX % 4 == 0, "the packed two-axis form: column groups of 4 or 8");

    // `npoly` pairs of the thread's NPAIRS spread evenly over its pixels
    static constexpr bool spread_pair(int pair, int npoly) {
        if (npoly <= 0) return false;
        const int spread = NPAIRS / npoly;
        return pair % spread == 0 && pair / spread < npoly;
    }

    // Packed tiles: which pixel pairs take the polynomial for the point at
    // position r of the pattern's period -- the first NP / 2 (PKV 1, 2), or
    // NP / 2 pairs spread evenly over the thread's pixels so that polynomial
    // and MUFU work alternate in the instruction stream (3), one more on the
    // odd points (4) or on the last point of four (5).
    static constexpr bool is_poly_pair(int pair, int r) {
        if (PKV == 1 || PKV == 2) return pair < NP / 2;
        const bool extra = (PKV == 4 && (r & 1)) || (PKV == 5 && r == 3);
        return spread_pair(pair, NP / 2 + (extra ? 1 : 0));
    }

    // acc += A_q cos(theta_x + theta_y) over the thread's pixels for point q
    // of the stage (pattern position R).
    template <int R>
    __device__ __forceinline__ static void point_step(Acc &acc, const float *sx,
                                                      const float *sy, float a,
                                                      int q) {
        if constexpr (PKV == 6) {
            // the rotation form: per thread row i, the row's first pixel has
            // phase theta_0 = theta_x0 + theta_y[i]; its sine and cosine come
            // from the MUFU, and pixel k = 1..3 of the row is
            //     cos(theta_0 + d_k) = cos theta_0 cos d_k - sin theta_0 sin d_k
            // with (cos d_k, sin d_k) of the exact x-phase offset d_k from the
            // table: one packed multiply and one packed multiply-add per two
            // pixels (pixel 0 rides along as cos theta_0 * 1 - sin * 0)
            const float4 xa = *reinterpret_cast<const float4 *>(sx + q * TX * XF);
            const float4 xb =
                *reinterpret_cast<const float4 *>(sx + q * TX * XF + S::NTX * 4);
            float vy[VY];
            VecLoad<VY>::ld(vy, sy + q * TY);
            const float2 a2 = make_float2(a, a);
            const float2 c01 = make_float2(1.0f, xa.y), s01 = make_float2(xb.x, xb.y);
            const float2 c23 = make_float2(xa.z, xa.w), s23 = make_float2(xb.z, xb.w);
#pragma unroll
            for (int i = 0; i < VY; i += 2) {
                const float2 th = __fadd2_rn(make_float2(xa.x, xa.x),
                                             make_float2(vy[i], vy[i + 1]));
                float s0, co0, s1, co1;
                __sincosf(th.x, &s0, &co0);
                __sincosf(th.y, &s1, &co1);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float c = h ? co1 : co0, s = h ? s1 : s0;
                    const float2 cc = make_float2(c, c), ns = make_float2(-s, -s);
                    const float2 v01 = __ffma2_rn(ns, s01, __fmul2_rn(cc, c01));
                    const float2 v23 = __ffma2_rn(ns, s23, __fmul2_rn(cc, c23));
                    acc.v[i + h][0] = __ffma2_rn(a2, v01, acc.v[i + h][0]);
                    acc.v[i + h][1] = __ffma2_rn(a2, v23, acc.v[i + h][1]);
                }
            }
            return;
        }
        if constexpr (PKV == 7) {
            // the rotation form along both axes: the thread's first pixel
            // has phase theta_00 = theta_x0 + theta_y0, and the MUFU gives
            // w_0 = A_q e^(i theta_00); the first pixel of row i has
            // w_i = w_0 e^(i e_i), with (cos e_i, sin e_i) of the row's exact
            // y-phase offset e_i from the y table, and pixel k of row i adds
            //     Re(w_i e^(i d_k)) = Re w_i cos d_k - Im w_i sin d_k
            // with the x table's (cos d_k, sin d_k): two FMAs per pixel
            float xv[2 * VX], yv[2 * VY];
            const float *px = sx + q * TX * XF, *py = sy + q * TY * YF;
#pragma unroll
            for (int j = 0; j < VX / 2; ++j) VecLoad<4>::ld(xv + 4 * j, px + j * S::NTX * 4);
#pragma unroll
            for (int j = 0; j < VY / 2; ++j) VecLoad<4>::ld(yv + 4 * j, py + j * S::NTY * 4);
            float s0, c0;
            __sincosf(xv[0] + yv[0], &s0, &c0);
            const float wr0 = a * c0, wi0 = a * s0;
#pragma unroll
            for (int i = 0; i < VY; ++i) {
                float wr = wr0, wi = wi0;
                if (i > 0) {
                    const float ce = yv[i], se = yv[VY + i];
                    wr = fmaf(-wi0, se, wr0 * ce);
                    wi = fmaf(wr0, se, wi0 * ce);
                }
                acc.v[i][0] += wr;
#pragma unroll
                for (int k = 1; k < VX; ++k)
                    acc.v[i][k] = fmaf(-wi, xv[VX + k], fmaf(wr, xv[k], acc.v[i][k]));
            }
            return;
        }
        if constexpr (PKV == 8) {
            // as 7, with the pixels of a row taken in packed pairs along x:
            // the pair (k, k + 1) adds Re w_i (cos d_k, cos d_k+1) -
            // Im w_i (sin d_k, sin d_k+1) in two packed FMAs (pixel 0 rides
            // along with cos 0 = 1 and sin 0 = 0)
            float4 xq[VX / 2];
            float yv[2 * VY];
            const float *px = sx + q * TX * XF, *py = sy + q * TY * YF;
#pragma unroll
            for (int j = 0; j < VX / 2; ++j)
                xq[j] = *reinterpret_cast<const float4 *>(px + j * S::NTX * 4);
#pragma unroll
            for (int j = 0; j < VY / 2; ++j) VecLoad<4>::ld(yv + 4 * j, py + j * S::NTY * 4);
            float2 cx[VX / 2], sxp[VX / 2];
#pragma unroll
            for (int j = 0; j < VX / 4; ++j) {
                cx[2 * j] = make_float2(j == 0 ? 1.0f : xq[j].x, xq[j].y);
                cx[2 * j + 1] = make_float2(xq[j].z, xq[j].w);
                sxp[2 * j] = make_float2(xq[VX / 4 + j].x, xq[VX / 4 + j].y);
                sxp[2 * j + 1] = make_float2(xq[VX / 4 + j].z, xq[VX / 4 + j].w);
            }
            float s0, c0;
            __sincosf(xq[0].x + yv[0], &s0, &c0);
            const float wr0 = a * c0, wi0 = a * s0;
#pragma unroll
            for (int i = 0; i < VY; ++i) {
                float wr = wr0, nwi = -wi0;
                if (i > 0) {
                    const float ce = yv[i], se = yv[VY + i];
                    wr = fmaf(-wi0, se, wr0 * ce);
                    nwi = fmaf(-wr0, se, -wi0 * ce);
                }
                const float2 w2 = make_float2(wr, wr), n2 = make_float2(nwi, nwi);
#pragma unroll
                for (int k = 0; k < VX / 2; ++k)
                    acc.v[i][k] = __ffma2_rn(n2, sxp[k], __ffma2_rn(w2, cx[k], acc.v[i][k]));
            }
            return;
        }
        if constexpr (PKV < 6) {
            float vx[VX], vy[VY];
            VecLoad<VX>::ld(vx, sx + q * TX);
            VecLoad<VY>::ld(vy, sy + q * TY);
            if constexpr (PK) {
                const float2 a2 = make_float2(a, a), na2 = make_float2(-a, -a);
#pragma unroll
                for (int i = 0; i < VY; ++i) {
                    const float2 y2 = make_float2(vy[i], vy[i]);
#pragma unroll
                    for (int k = 0; k < VX; k += 2) {
                        const float2 th = __fadd2_rn(make_float2(vx[k], vx[k + 1]), y2);
                        float2 &ac = acc.v[i][k >> 1];
                        if (is_poly_pair((i * VX + k) / 2, R))
                            ac = __ffma2_rn(na2, neg_cos_poly2<PKV == 1 ? 6 : 5>(th), ac);
                        else
                            ac = __ffma2_rn(a2, make_float2(__cosf(th.x), __cosf(th.y)), ac);
                    }
                }
            } else {
                // the first NP pixels of the thread take the FMA-pipe polynomial,
                // the rest the MUFU cosine (compile-time split)
#pragma unroll
                for (int i = 0; i < VY; ++i)
#pragma unroll
                    for (int k = 0; k < VX; ++k) {
                        const float th = vx[k] + vy[i];
                        float &ac = acc.v[i][k];
                        if (i * VX + k < NP)
                            ac = fmaf(-a, neg_cos_poly(th), ac);
                        else
                            ac = fmaf(a, __cosf(th), ac);
                    }
            }
    
        }
    }

    __device__ static void issue(float *smem, uint64_t *full, const float *gx,
                                 const float *gy, const float *amp, int t,
                                 int slot) {
        float *st = smem + slot * S::STAGE;
        mbar_arrive_expect_tx(&full[slot], S::STAGE * 4);
        bulk_g2s(st, gx + (size_t)t * S::SX, S::SX * 4, &full[slot]);
        bulk_g2s(st + S::SX, gy + (size_t)t * S::SY, S::SY * 4, &full[slot]);
        bulk_g2s(st + S::SX + S::SY, amp + (size_t)t * S::SA, S::SA * 4,
                 &full[slot]);
    }

    // acc += the point tiles [0, ntile) for this thread's VX x VY pixels.
    // Returns false (after letting its own copies land) if a wait timed out.
    __device__ static bool accumulate(float *smem, uint64_t *full,
                                      volatile int *abort_flag, const float *gx,
                                      const float *gy, const float *amp,
                                      int ntile, unsigned g0, Acc &acc,
                                      unsigned *status) {
        int issued = 0;  // meaningful in thread 0 only
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();  // the ring may hold partial sums
            for (int s = 0; s < NST && s < ntile; ++s) {
                issue(smem, full, gx, gy, amp, s, (int)((g0 + s) % NST));
                ++issued;
            }
        }
        const int lt = threadIdx.x % S::GT, grp = threadIdx.x / S::GT;
        const int tx = lt % S::NTX, ty = lt / S::NTX;
        int t = 0;
        for (; t < ntile; ++t) {
            const unsigned g = g0 + (unsigned)t;
            const int s = (int)(g % NST);
            const uint32_t par = (uint32_t)((g / NST) & 1);
            bool ok = mbar_wait_bounded(&full[s], par);
            if (!ok) {
                *abort_flag = 1;
                set_status(status, DEV_TIMEOUT);
            } else {
                const float *st = smem + s * S::STAGE;
                // (the rotation tables interleave their groups' fours)
                const float *sx = st + (PKV >= 6 ? tx * 4 : tx * VX * XF);
                const float *sy = st + S::SX + (PKV >= 7 ? ty * 4 : ty * VY);
                const float *sa = st + S::SX + S::SY;
                const int q0 = grp * S::PG;
                // (the amplitudes of a period's points: one broadcast load;
                // q0 and the stage offsets are multiples of 4 floats)
                if constexpr (PERIOD == 1) {
#pragma unroll 2
                    for (int q = q0; q < q0 + S::PG; ++q)
                        point_step<0>(acc, sx, sy, sa[q], q);
                } else if constexpr (PERIOD == 2) {
                    for (int q = q0; q < q0 + S::PG; q += 2) {
                        const float2 a = *reinterpret_cast<const float2 *>(sa + q);
                        point_step<0>(acc, sx, sy, a.x, q);
                        point_step<1>(acc, sx, sy, a.y, q + 1);
                    }
                } else {
                    for (int q = q0; q < q0 + S::PG; q += 4) {
                        const float4 a = *reinterpret_cast<const float4 *>(sa + q);
                        point_step<0>(acc, sx, sy, a.x, q);
                        point_step<1>(acc, sx, sy, a.y, q + 1);
                        point_step<2>(acc, sx, sy, a.z, q + 2);
                        point_step<3>(acc, sx, sy, a.w, q + 3);
                    }
                }
            }
            __syncthreads();  // every thread is done with slot s
            if (*abort_flag) break;
            if (threadIdx.x == 0 && t + NST < ntile) {
                fence_proxy_async_smem();
                issue(smem, full, gx, gy, amp, t + NST, s);
                ++issued;
            }
        }
        if (*abort_flag) {
            // let the copies still in flight land before the shared memory
            // goes away (each wait bounded again)
            if (threadIdx.x == 0) {
                for (int u = t; u < issued; ++u) {
                    const unsigned g = g0 + (unsigned)u;
                    mbar_wait_bounded(&full[g % NST], (uint32_t)((g / NST) & 1));
                }
            }
            return false;
        }
        return true;
    }

    // Add the G groups' partial sums into the first group's accumulators:
    // the other groups leave theirs in the (now idle) stage ring and the
    // first group adds them in group order (deterministic).  The ring is in
    // use until the caller's next __syncthreads.
    __device__ static void reduce_groups(Acc &acc, float *smem) {
        if (G == 1) return;
        const int lt = threadIdx.x % S::GT, grp = threadIdx.x / S::GT;
        const int tx = lt % S::NTX, ty = lt / S::NTX;
        if (grp > 0) {
            float *part = smem + (size_t)(grp - 1) * TX * TY;
#pragma unroll
            for (int i = 0; i < VY; ++i)
#pragma unroll
                for (int k = 0; k < VX; ++k)
                    part[(ty * VY + i) * TX + tx * VX + k] = acc.get(i, k);
        }
        __syncthreads();
        if (grp == 0) {
#pragma unroll
            for (int g = 1; g < G; ++g) {
                const float *part = smem + (size_t)(g - 1) * TX * TY;
#pragma unroll
                for (int i = 0; i < VY; ++i)
#pragma unroll
                    for (int k = 0; k < VX; ++k)
                        acc.add(i, k, part[(ty * VY + i) * TX + tx * VX + k]);
            }
        }
    }

    // The first group writes its pixels of pixel tile (xt, yt) to the frame
    // (clipped to Nx x Ny).
    __device__ static void write_out(const Acc &acc, int xt, int yt, int Nx,
                                     int Ny, float *out, int vec_store) {
        const int lt = threadIdx.x % S::GT, grp = threadIdx.x / S::GT;
        const int tx = lt % S::NTX, ty = lt / S::NTX;
        if (grp != 0) return;
        const int x0 = xt * TX + tx * VX, y0 = yt * TY + ty * VY;
#pragma unroll
        for (int i = 0; i < VY; ++i) {
            const int y = y0 + i;
            if (y >= Ny) break;
            float *orow = out + (size_t)y * Nx;
            if (VX % 4 == 0 && vec_store && x0 + VX <= Nx) {
#pragma unroll
                for (int k = 0; k < VX; k += 4)
                    *reinterpret_cast<float4 *>(orow + x0 + k) =
                        make_float4(acc.get(i, k), acc.get(i, k + 1),
                                    acc.get(i, k + 2), acc.get(i, k + 3));
            } else {
#pragma unroll
                for (int k = 0; k < VX; ++k)
                    if (x0 + k < Nx) orow[x0 + k] = acc.get(i, k);
            }
        }
    }

    // Store the pixels of pixel tile (xt, yt).  Ends with the ring free for
    // the next copies of a persistent CTA.
    __device__ static void store(Acc &acc, float *smem, int xt, int yt, int Nx,
                                 int Ny, float *out, int vec_store) {
        reduce_groups(acc, smem);
        write_out(acc, xt, yt, Nx, Ny, out, vec_store);
        if (G > 1) __syncthreads();
    }
};

}  // namespace cgh
