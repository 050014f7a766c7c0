// sep_table.cuh -- one entry (one point, one pixel row or column) of the
// U / V tables of the separable form; see separable.cu.  Internal to libcgh.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace cgh {

constexpr float LO_SCALE = 4096.0f;  // 2^12: lo planes stored scaled up

// Entry e of (Nx + Ny) x (Kp / 2): row r = e / (Kp / 2) (x rows first, then
// y rows), point j = e % (Kp / 2).  Writes the interleaved pair at
// [row][2j] of L (x rows: A_j (cos, -sin)) or R (y rows: (cos, sin)).
template <int KIND>
__device__ __forceinline__ void sep_table_entry(const PointRec *__restrict__ rec,
                                                int N, int Nx, int Kp, long long e,
                                                void *__restrict__ Lhi,
                                                void *__restrict__ Llo,
                                                void *__restrict__ Rhi,
                                                void *__restrict__ Rlo) {
    const int r = (int)(e / (Kp / 2));
    const int j = (int)(e - (long long)r * (Kp / 2));
    const bool is_x = r < Nx;
    const int u = is_x ? r : r - Nx;
    float re = 0.0f, im = 0.0f;
    if (j < N) {
        const PointRec pr = rec[j];
        const uint64_t ph = is_x ? axis_phase(pr.c, pr.bx, pr.ax, u)
                                 : axis_phase(pr.c, pr.by, pr.ay, u);
        const float turns = (float)phase_hi(ph) * TURN_PER_U32;
        float s, c;
        sincospif(2.0f * turns, &s, &c);
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

}  // namespace cgh
