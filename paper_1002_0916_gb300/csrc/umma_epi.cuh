// umma_epi.cuh -- arguments and the fused adjoint epilogue shared by the
// one-CTA (umma.cu) and CTA-pair (umma2.cu) tensor-core GEMMs.  Internal to
// libcgh.
#pragma once

#include "common.cuh"
#include "umma.cuh"

namespace cgh {

struct GemmArgs {
    int M, N, K;
    float *D;
    long long ldd;
    float lo_scale;
    unsigned *status;
    int accumulate;  // 0: D = product; 1: D += product (a later K chunk)
};

// Store CH consecutive FP32 values of one output row (row < M checked by the
// caller), clipped to N columns; with g.accumulate the row's current values
// are added first (FP32, round to nearest).
template <int CH>
__device__ __forceinline__ void epilogue_store_row(float *drow, int col, float (&v)[CH],
                                                   const GemmArgs &g, bool vec) {
    if (vec && col + CH <= g.N) {
        if (g.accumulate) {
            // all of the chunk's loads before any of its stores: one memory
            // latency per chunk instead of one per vector
            float4 d[CH / 4];
#pragma unroll
            for (int i = 0; i < CH; i += 4)
                d[i / 4] = *reinterpret_cast<const float4 *>(drow + col + i);
#pragma unroll
            for (int i = 0; i < CH; i += 4) {
                d[i / 4].x += v[i];
                d[i / 4].y += v[i + 1];
                d[i / 4].z += v[i + 2];
                d[i / 4].w += v[i + 3];
            }
#pragma unroll
            for (int i = 0; i < CH; i += 4)
                *reinterpret_cast<float4 *>(drow + col + i) = d[i / 4];
            return;
        }
#pragma unroll
        for (int i = 0; i < CH; i += 4)
            *reinterpret_cast<float4 *>(drow + col + i) =
                make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < CH; ++i)
            if (col + i < g.N) drow[col + i] = g.accumulate ? drow[col + i] + v[i] : v[i];
    }
}

// Fused adjoint epilogue (MODE 1).  The GEMM rows are k = 2j + c (c = 0:
// cos row, 1: sin row of point j) and its columns are pixel coordinates u
// along one image axis; D[2j][u] = W_c, D[2j+1][u] = W_s are the partial
// transforms of dL/dI over the other axis.  With (cu, su) = (cos, sin) of
// th_axis(u, j) and d = u - u_j the epilogue accumulates over its columns
//     C = cu W_c - su W_s,   S = su W_c + cu W_s,
//     part[tile][j] += (C, S d, S d^2)
// (the pixel sums of G cos(phi), G sin(phi) d, G sin(phi) d^2).
struct AdjEpiArgs {
    const PointRec *rec;
    const float *points;  // N x 2 (x_j, y_j)
    int npoints;          // N
    int npad;             // partial-sum stride (points)
    int axis;             // 0: columns are x, 1: columns are y
    float *part;          // [column tile][npad][3]
};

// The fused adjoint epilogue for one TMEM lane (= GEMM row `row`).
template <int BN, bool SPLIT, uint32_t ACC1>
__device__ __forceinline__ void adjoint_epilogue(uint32_t t_row, int row, int n0,
                                                 const GemmArgs &g,
                                                 const AdjEpiArgs &ea, int lane,
                                                 int tile) {
    const int j = row >> 1;
    const bool cos_row = (row & 1) == 0;
    const bool valid = j < ea.npoints;
    PointRec pr{};
    float uj = 0.0f;
    if (valid) {
        pr = ea.rec[j];
        uj = ea.points[2 * j + ea.axis];
    }
    const uint64_t b = ea.axis == 0 ? pr.bx : pr.by;
    const uint64_t a = ea.axis == 0 ? pr.ax : pr.ay;
    // exact fixed-point phase at column n0 and its first difference
    // (the paper's Eq. 2 recurrence, modulo one turn)
    uint64_t th = axis_phase(pr.c, b, a, n0);
    uint64_t dth = pr.c * (uint64_t)(2 * (long long)n0 + 1) - b;
    const uint64_t d2 = 2 * pr.c;
    float accC = 0.0f, accS1 = 0.0f, accS2 = 0.0f;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        umma::tmem_ld32(t_row + c, r);
        float v[32];
        if (SPLIT) {
            uint32_t r2[32];
            umma::tmem_ld32(t_row + ACC1 + c, r2);
            umma::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i)
                v[i] = fmaf(g.lo_scale, __uint_as_float(r2[i]), __uint_as_float(r[i]));
        } else {
            umma::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
        }
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
            const float other = __shfl_xor_sync(0xffffffffu, v[i], 1);
            const float wc = cos_row ? v[i] : other;
            const float ws = cos_row ? other : v[i];
            const float ang = (float)phase_hi(th) * RAD_PER_U32;
            th += dth;
            dth += d2;
            float su, cu;
            __sincosf(ang, &su, &cu);
            const int u = n0 + c + i;
            const float d = (float)u - uj;
            const float C = cu * wc - su * ws;
            const float Sv = su * wc + cu * ws;
            if (u < g.N) {
                accC += C;
                const float t = Sv * d;
                accS1 += t;
                accS2 = fmaf(t, d, accS2);
            }
        }
    }
    if (valid && cos_row) {
        float *p = ea.part + ((size_t)tile * ea.npad + j) * 3;
        p[0] = accC;
        p[1] = accS1;
        p[2] = accS2;
    }
    (void)lane;
}

}  // namespace cgh
