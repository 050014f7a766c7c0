// direct.cu -- the direct FP32 evaluation of Eq. 1 (steps A2-A5).
//
// Design (sm_103a):
//  * Phase.  The phase of Eq. 1 in turns splits exactly into an x part and a
//    y part, Q_j (x - x_j)^2 + Q_j (y - y_j)^2.  Each part is evaluated once
//    per (point, pixel column) and (point, pixel row) -- not per pixel -- in
//    64-bit fixed-point turns (exact modulo one turn; this is the exact
//    integer form of the paper's Eq. 2 recurrence, Section 2.1, which also
//    avoids recomputing the full phase per pixel), then rounded to an FP32
//    angle in [-pi, pi).  Per pixel only theta_x + theta_y remains: one add.
//  * Tables.  These per-axis angles are written once per call into tables
//    laid out tile by tile, so that the slice a CTA needs for one stage of
//    points is one contiguous block: [x tile][point][x in tile].
//  * Staging.  Point tiles are staged in shared memory by 1-D bulk copies
//    (cp.async.bulk, mbarrier completion), NST stages deep -- the paper's
//    shared-memory staging of 256 points per barrier (Section 2.1).
//  * Work per thread.  Each thread owns a VX x VY block of pixels (the
//    paper's float8 "eight pixels per item", Section 2.1); per point it reads
//    VX x-angles, VY y-angles and A_j (broadcast) from shared memory and does
//    VX*VY of: add, hardware cosine (the paper's native cos), FMA.
//  * Bound.  One MUFU cosine per point-pixel update; everything else is
//    2 FP32 ops, so the kernel is bound by the MUFU issue rate.
//
// Accuracy: angle rounding about 2^-22 rad per axis, __cosf absolute error
// about 2^-21 on |x| <= pi, FP32 accumulation: far inside
// max |I - I_ref| <= 1e-4 sum |A_j|.
#include <math.h>

#include "common.cuh"

namespace cgh {

// ------------------------------------------------------------ tables
__global__ void direct_tables_kernel(const PointRec *__restrict__ rec,
                                     int Npad, int TX, int TY, int nxt,
                                     int nyt, float *__restrict__ phx,
                                     float *__restrict__ phy,
                                     float *__restrict__ amp) {
    const long long nx_e = (long long)nxt * Npad * TX;
    const long long ny_e = (long long)nyt * Npad * TY;
    const long long total = nx_e + ny_e + Npad;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
         e < total; e += (long long)gridDim.x * blockDim.x) {
        if (e < nx_e) {
            long long per = (long long)Npad * TX;
            int t = (int)(e / per);
            long long rem = e - (long long)t * per;
            int j = (int)(rem / TX);
            int i = (int)(rem - (long long)j * TX);
            const PointRec &r = rec[j];
            uint64_t ph = axis_phase(r.c, r.bx, r.ax, t * TX + i);
            phx[e] = (float)phase_hi(ph) * RAD_PER_U32;
        } else if (e < nx_e + ny_e) {
            long long f = e - nx_e;
            long long per = (long long)Npad * TY;
            int t = (int)(f / per);
            long long rem = f - (long long)t * per;
            int j = (int)(rem / TY);
            int i = (int)(rem - (long long)j * TY);
            const PointRec &r = rec[j];
            uint64_t ph = axis_phase(r.c, r.by, r.ay, t * TY + i);
            phy[f] = (float)phase_hi(ph) * RAD_PER_U32;
        } else {
            int j = (int)(e - nx_e - ny_e);
            amp[j] = rec[j].A;
        }
    }
}

// ------------------------------------------------------- direct kernel
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

template <int TX, int TY, int VX, int VY, int PT, int NST>
struct DirectShape {
    static constexpr int NTX = TX / VX;
    static constexpr int THREADS = NTX * (TY / VY);
    static constexpr int SX = PT * TX;        // floats of x-angles per stage
    static constexpr int SY = PT * TY;        // floats of y-angles per stage
    static constexpr int SA = PT;             // amplitudes per stage
    static constexpr int STAGE = SX + SY + SA;
    static constexpr size_t SMEM = (size_t)NST * STAGE * sizeof(float);
    static_assert(TX % VX == 0 && TY % VY == 0, "tile not divisible");
    static_assert(PT % 4 == 0, "bulk copies need 16-byte multiples");
    static_assert((STAGE * 4) % 16 == 0, "stage alignment");
};

template <int TX, int TY, int VX, int VY, int PT, int NST>
__global__ void __launch_bounds__(DirectShape<TX, TY, VX, VY, PT, NST>::THREADS)
direct_fwd_kernel(const float *__restrict__ phx, const float *__restrict__ phy,
                  const float *__restrict__ amp, int Npad, int Nx, int Ny,
                  float *__restrict__ out, int vec_store, unsigned *status) {
    using S = DirectShape<TX, TY, VX, VY, PT, NST>;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t full[NST];
    __shared__ int abort_flag;

    const int xt = blockIdx.x, yt = blockIdx.y;
    const int ntile = Npad / PT;
    const float *gx = phx + (size_t)xt * Npad * TX;
    const float *gy = phy + (size_t)yt * Npad * TY;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    int issued = 0;  // meaningful in thread 0 only
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST && s < ntile; ++s) {
            float *st = smem + s * S::STAGE;
            mbar_arrive_expect_tx(&full[s], S::STAGE * 4);
            bulk_g2s(st, gx + (size_t)s * S::SX, S::SX * 4, &full[s]);
            bulk_g2s(st + S::SX, gy + (size_t)s * S::SY, S::SY * 4, &full[s]);
            bulk_g2s(st + S::SX + S::SY, amp + (size_t)s * S::SA, S::SA * 4,
                     &full[s]);
            ++issued;
        }
    }

    const int tx = threadIdx.x % S::NTX, ty = threadIdx.x / S::NTX;
    float acc[VY][VX];
#pragma unroll
    for (int i = 0; i < VY; ++i)
#pragma unroll
        for (int k = 0; k < VX; ++k) acc[i][k] = 0.0f;

    int t = 0;
    for (; t < ntile; ++t) {
        const int s = t % NST;
        const uint32_t par = (uint32_t)((t / NST) & 1);
        bool ok = mbar_wait_bounded(&full[s], par);
        if (!ok) {
            abort_flag = 1;
            set_status(status, DEV_TIMEOUT);
        } else {
            const float *st = smem + s * S::STAGE;
            const float *sx = st + tx * VX;
            const float *sy = st + S::SX + ty * VY;
            const float *sa = st + S::SX + S::SY;
#pragma unroll 2
            for (int q = 0; q < PT; ++q) {
                const float a = sa[q];
                float vx[VX], vy[VY];
                VecLoad<VX>::ld(vx, sx + q * TX);
                VecLoad<VY>::ld(vy, sy + q * TY);
#pragma unroll
                for (int i = 0; i < VY; ++i)
#pragma unroll
                    for (int k = 0; k < VX; ++k)
                        acc[i][k] = fmaf(a, __cosf(vx[k] + vy[i]), acc[i][k]);
            }
        }
        __syncthreads();  // every thread is done with stage s
        if (abort_flag) break;
        if (threadIdx.x == 0 && t + NST < ntile) {
            fence_proxy_async_smem();
            float *st = smem + s * S::STAGE;
            const int tn = t + NST;
            mbar_arrive_expect_tx(&full[s], S::STAGE * 4);
            bulk_g2s(st, gx + (size_t)tn * S::SX, S::SX * 4, &full[s]);
            bulk_g2s(st + S::SX, gy + (size_t)tn * S::SY, S::SY * 4, &full[s]);
            bulk_g2s(st + S::SX + S::SY, amp + (size_t)tn * S::SA, S::SA * 4,
                     &full[s]);
            ++issued;
        }
    }

    if (abort_flag) {
        // Let the copies still in flight land before the CTA's shared memory
        // goes away (each wait bounded again).
        if (threadIdx.x == 0) {
            for (int u = t; u < issued; ++u)
                mbar_wait_bounded(&full[u % NST], (uint32_t)((u / NST) & 1));
        }
        return;
    }

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
                    make_float4(acc[i][k], acc[i][k + 1], acc[i][k + 2],
                                acc[i][k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < VX; ++k)
                if (x0 + k < Nx) orow[x0 + k] = acc[i][k];
        }
    }
}

// ------------------------------------------------------- naive kernel
// One thread per pixel, plain loop over points (the paper's unoptimised
// kernel, Fig. 2b, restated): exact 64-bit fixed-point phase, cospif.
__global__ void naive_fwd_kernel(const PointRec *__restrict__ rec, int N,
                                 int Nx, int Ny, float *__restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= Nx || y >= Ny) return;
    float acc = 0.0f;
    for (int j = 0; j < N; ++j) {
        const PointRec r = rec[j];
        uint64_t ph = axis_phase(r.c, r.bx, r.ax, x) + axis_phase(r.c, r.by, r.ay, y);
        float turns = (float)phase_hi(ph) * TURN_PER_U32;
        acc = fmaf(r.A, cospif(2.0f * turns), acc);
    }
    out[(size_t)y * Nx + x] = acc;
}

// ------------------------------------------------------------ registry
#define CGH_DIRECT_TILES(X)          \
    X(64, 64, 4, 4, 32, 3)           \
    X(64, 32, 4, 2, 32, 3)           \
    X(128, 32, 4, 4, 32, 3)          \
    X(32, 32, 2, 2, 64, 3)           \
    X(128, 64, 8, 4, 16, 3)          \
    X(64, 16, 4, 1, 64, 3)

static const DirectTile kTiles[] = {
#define X(tx, ty, vx, vy, pt, ns) {tx, ty, vx, vy, pt},
    CGH_DIRECT_TILES(X)
#undef X
};
static constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

int direct_tile_count() { return kNumTiles; }
DirectTile direct_tile_get(int i) { return kTiles[i]; }
int direct_tile_index(const DirectTile &t) {
    for (int i = 0; i < kNumTiles; ++i)
        if (kTiles[i].tx == t.tx && kTiles[i].ty == t.ty && kTiles[i].vx == t.vx &&
            kTiles[i].vy == t.vy && kTiles[i].pt == t.pt)
            return i;
    return -1;
}

size_t direct_phase_table_floats(const DirectTile &t, int Npad, int Nx,
                                 int Ny) {
    size_t nxt = (Nx + t.tx - 1) / t.tx, nyt = (Ny + t.ty - 1) / t.ty;
    return nxt * Npad * t.tx + nyt * Npad * t.ty;
}

cudaError_t launch_direct_tables(const PointRec *rec, int Npad, int Nx, int Ny,
                                 const DirectTile &t, float *phx, float *phy,
                                 float *amp, cudaStream_t s) {
    int nxt = (Nx + t.tx - 1) / t.tx, nyt = (Ny + t.ty - 1) / t.ty;
    long long total = (long long)nxt * Npad * t.tx + (long long)nyt * Npad * t.ty + Npad;
    int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    direct_tables_kernel<<<(int)blocks, threads, 0, s>>>(rec, Npad, t.tx, t.ty,
                                                          nxt, nyt, phx, phy,
                                                          amp);
    return cudaGetLastError();
}

template <int TX, int TY, int VX, int VY, int PT, int NST>
static cudaError_t launch_one(const float *phx, const float *phy,
                              const float *amp, int Npad, int Nx, int Ny,
                              float *out, unsigned *status, cudaStream_t s) {
    using S = DirectShape<TX, TY, VX, VY, PT, NST>;
    auto kern = direct_fwd_kernel<TX, TY, VX, VY, PT, NST>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((Nx + TX - 1) / TX, (Ny + TY - 1) / TY);
    int vec_store = (Nx % 4 == 0) && (((uintptr_t)out & 15) == 0);
    kern<<<grid, S::THREADS, S::SMEM, s>>>(phx, phy, amp, Npad, Nx, Ny, out,
                                          vec_store, status);
    return cudaGetLastError();
}

cudaError_t launch_direct_forward(int tile_index, const float *phx,
                                  const float *phy, const float *amp, int Npad,
                                  int Nx, int Ny, float *out, unsigned *status,
                                  cudaStream_t s) {
    int i = 0;
#define X(tx, ty, vx, vy, pt, ns)                                              \
    if (tile_index == i)                                                       \
        return launch_one<tx, ty, vx, vy, pt, ns>(phx, phy, amp, Npad, Nx, Ny, \
                                                  out, status, s);             \
    ++i;
    CGH_DIRECT_TILES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_naive_forward(const PointRec *rec, int N, int Nx, int Ny,
                                 float *out, cudaStream_t s) {
    dim3 grid((Nx + 127) / 128, Ny);
    naive_fwd_kernel<<<grid, 128, 0, s>>>(rec, N, Nx, Ny, out);
    return cudaGetLastError();
}

}  // namespace cgh
