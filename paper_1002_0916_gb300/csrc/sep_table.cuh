// sep_table.cuh -- rows of the U / V tables of the separable form (one
// point pair, a run of pixel rows or columns); see separable.cu.  Internal
// to libcgh.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace cgh {

constexpr float LO_SCALE = 4096.0f;  // 2^12: lo planes stored scaled up

// Entry values: x rows L = A_j (cos, -sin), y rows R = (cos, sin) of the
// angle, zeros for padding points.  The angle (exact fixed point, then FP32
// radians in [-pi, pi)) goes through the hardware sincos: absolute error
// about 2^-21, far below FP16's 2^-11 and the 2^-22 of the split hi+lo
// pair's own rounding, and the same in BF16.
template <int KIND>
__device__ __forceinline__ void sep_value(float A, bool valid, bool is_x,
                                          uint64_t ph, float &re, float &im) {
    float s, c;
    __sincosf((float)phase_hi(ph) * RAD_PER_U32, &s, &c);
    re = valid ? (is_x ? A * c : c) : 0.0f;
    im = valid ? (is_x ? -A * s : s) : 0.0f;
}

template <int KIND>
__device__ __forceinline__ void sep_store(void *hi, void *lo, size_t off, float re0,
                                          float im0, float re1, float im1) {
    if (KIND == 0) {
        __nv_bfloat162 v[2] = {__floats2bfloat162_rn(re0, im0),
                               __floats2bfloat162_rn(re1, im1)};
        *reinterpret_cast<uint2 *>((__nv_bfloat16 *)hi + off) =
            *reinterpret_cast<const uint2 *>(v);
    } else {
        __half2 v[2] = {__floats2half2_rn(re0, im0), __floats2half2_rn(re1, im1)};
        *reinterpret_cast<uint2 *>((__half *)hi + off) = *reinterpret_cast<const uint2 *>(v);
        if (KIND == 2) {
            const float2 h0 = __half22float2(v[0]), h1 = __half22float2(v[1]);
            __half2 w[2] = {__floats2half2_rn((re0 - h0.x) * LO_SCALE, (im0 - h0.y) * LO_SCALE),
                            __floats2half2_rn((re1 - h1.x) * LO_SCALE, (im1 - h1.y) * LO_SCALE)};
            *reinterpret_cast<uint2 *>((__half *)lo + off) =
                *reinterpret_cast<const uint2 *>(w);
        }
    }
}

// Table rows [r0, r1) of the (Nx + Ny) x Kp tables for the point pair
// (j0, j0 + 1), j0 even (x rows first, then y rows).  The axis phase of the
// first row of each part is evaluated directly, then stepped row by row with
// the exact fixed-point form of Eq. 2: the phase difference c (2u + 1) - b
// and its constant second difference 2c, all modulo one turn.  The four
// interleaved entries of the pair go out as one 8-byte store per plane.
constexpr int ST_ROWS = 16;

template <int KIND>
__device__ __forceinline__ void sep_table_rows(const PointRec &p0, const PointRec &p1,
                                               bool v0, bool v1, int Nx, int Kp,
                                               int j0, int r0, int r1,
                                               void *__restrict__ Lhi,
                                               void *__restrict__ Llo,
                                               void *__restrict__ Rhi,
                                               void *__restrict__ Rlo) {
#pragma unroll
    for (int seg = 0; seg < 2; ++seg) {  // the x rows, then the y rows
        const bool is_x = seg == 0;
        const int a = is_x ? r0 : (r0 > Nx ? r0 : Nx);
        const int b = is_x ? (r1 < Nx ? r1 : Nx) : r1;
        if (a >= b) continue;
        int u = is_x ? a : a - Nx;
        const uint64_t b0 = is_x ? p0.bx : p0.by, b1 = is_x ? p1.bx : p1.by;
        uint64_t ph0 = axis_phase(p0.c, b0, is_x ? p0.ax : p0.ay, u);
        uint64_t ph1 = axis_phase(p1.c, b1, is_x ? p1.ax : p1.ay, u);
        const uint64_t step = (uint64_t)(2 * (int64_t)u + 1);
        uint64_t d0 = p0.c * step - b0, d1 = p1.c * step - b1;
        const uint64_t dd0 = 2 * p0.c, dd1 = 2 * p1.c;
        void *hi = is_x ? Lhi : Rhi;
        void *lo = is_x ? Llo : Rlo;
        size_t off = (size_t)u * Kp + 2 * (size_t)j0;
        for (int r = a; r < b; ++r, off += Kp) {
            float re0, im0, re1, im1;
            sep_value<KIND>(p0.A, v0, is_x, ph0, re0, im0);
            sep_value<KIND>(p1.A, v1, is_x, ph1, re1, im1);
            sep_store<KIND>(hi, lo, off, re0, im0, re1, im1);
            ph0 += d0;
            d0 += dd0;
            ph1 += d1;
            d1 += dd1;
        }
    }
}

}  // namespace cgh
