// sep_table.cuh -- one entry (one point, one pixel row or column) of the
// U / V tables of the separable form; see separable.cu.  Internal to libcgh.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace cgh {

constexpr float LO_SCALE = 4096.0f;  // 2^12: lo planes stored scaled up

// Entry (row r, point j) of the (Nx + Ny) x (Kp / 2) table entries: x rows
// first, then y rows.  Writes the interleaved pair at [row][2j] of L (x rows:
// A_j (cos, -sin)) or R (y rows: (cos, sin)); zeros for padding points.  The
// angle (exact fixed point, then FP32 radians in [-pi, pi)) goes through the
// hardware sincos: absolute error about 2^-21, far below FP16's 2^-11 and the
// 2^-22 of the split hi+lo pair's own rounding, and the same in BF16.
template <int KIND>
__device__ __forceinline__ void sep_table_entry_rj(const PointRec &pr, bool valid,
                                                   int Nx, int Kp, int r, int j,
                                                   void *__restrict__ Lhi,
                                                   void *__restrict__ Llo,
                                                   void *__restrict__ Rhi,
                                                   void *__restrict__ Rlo) {
    const bool is_x = r < Nx;
    const int u = is_x ? r : r - Nx;
    float re = 0.0f, im = 0.0f;
    if (valid) {
        const uint64_t ph = is_x ? axis_phase(pr.c, pr.bx, pr.ax, u)
                                 : axis_phase(pr.c, pr.by, pr.ay, u);
        float s, c;
        __sincosf((float)phase_hi(ph) * RAD_PER_U32, &s, &c);
        if (is_x) {
            re = pr.A * c;
            im = -pr.A * s;
        } else {
            re = c;
            im = s;
        }
    }
    const size_t off = (size_t)u * Kp + 2 * (size_t)j;
    void *hi_base = is_x ? Lhi : Rhi;
    if (KIND == 0) {
        *reinterpret_cast<__nv_bfloat162 *>((__nv_bfloat16 *)hi_base + off) =
            __floats2bfloat162_rn(re, im);
    } else {
        const __half2 h = __floats2half2_rn(re, im);
        *reinterpret_cast<__half2 *>((__half *)hi_base + off) = h;
        if (KIND == 2) {
            const float2 hf = __half22float2(h);
            void *lo_base = is_x ? Llo : Rlo;
            *reinterpret_cast<__half2 *>((__half *)lo_base + off) =
                __floats2half2_rn((re - hf.x) * LO_SCALE, (im - hf.y) * LO_SCALE);
        }
    }
}

// The same by linear entry index e = r * (Kp / 2) + j.
template <int KIND>
__device__ __forceinline__ void sep_table_entry(const PointRec *__restrict__ rec,
                                                int N, int Nx, int Kp, long long e,
                                                void *__restrict__ Lhi,
                                                void *__restrict__ Llo,
                                                void *__restrict__ Rhi,
                                                void *__restrict__ Rlo) {
    const int half = Kp / 2;
    const int r = (int)(e / half);
    const int j = (int)(e - (long long)r * half);
    const PointRec pr = j < N ? rec[j] : PointRec{};
    sep_table_entry_rj<KIND>(pr, j < N, Nx, Kp, r, j, Lhi, Llo, Rhi, Rlo);
}

}  // namespace cgh
