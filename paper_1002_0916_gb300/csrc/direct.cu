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
#include "direct_tile.cuh"
#include "point_rec.cuh"

namespace cgh {

// ------------------------------------------------------------ tables
// One block per DT_POINTS points (grid x) and 256 pixel columns or rows
// (grid y: the x range, then the y range): the records are staged in shared
// memory once; each thread then writes its coordinate for every point, or,
// in a rotation table, four coordinates of a group for one point at a time.
// FUSE: the block builds its DT_POINTS records itself from the caller's
// points (step A1, as in prologue.cu) instead of reading them from `rec`;
// each record is then built once per block row of grid y, a few FP64
// operations each, which costs less than a separate kernel in the chain.
constexpr int DT_POINTS = 16;

// One coordinate w (column or row, axis 0 = x, 1 = y) of a tile's angle
// table for the npts points of srec: dst[q * stride] = its angle for point q.
__device__ __forceinline__ void angle_column(const PointRec *srec, int npts, int w, int axis,
                                             float *dst, int stride) {
    for (int q = 0; q < npts; ++q) {
        const PointRec &r = srec[q];
        const uint64_t b = axis ? r.by : r.bx, a = axis ? r.ay : r.ax;
        dst[(size_t)q * stride] = (float)phase_hi(axis_phase(r.c, b, a, w)) * RAD_PER_U32;
    }
}

// Four coordinates g0 + k0 .. g0 + k0 + 3 (k0 = 4 h) of one rotation group
// of gs coordinates along an axis (0 = x, 1 = y), for one point: slots k0 ..
// k0 + 3 (cosines of the offsets; slot 0 is the angle at g0) and gs + k0 ..
// gs + k0 + 3 (sines; slot gs is 0), one 16-byte store each into the
// point's row of the table (ng groups per tile).  The offsets are exact in
// fixed point: Phi(g0 + k) - Phi(g0) = k (c (2 g0 + k) - b) for the first,
// then each next one adds the first difference c (2 u + 1) - b, which grows
// by 2 c per coordinate (Eq. 2 on the axis).
__device__ __forceinline__ void rotation_quarter(const PointRec &r, int axis, int g0, int g,
                                                 int h, int gs, int ng, float *row) {
    const uint64_t c = r.c, b = axis ? r.by : r.bx, a = axis ? r.ay : r.ax;
    const int k0 = 4 * h;
    uint64_t d = (uint64_t)k0 * (c * (uint64_t)(2 * g0 + k0) - b);
    uint64_t step = c * (uint64_t)(2 * (g0 + k0) + 1) - b;
    float co[4], si[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (k0 + i == 0) {
            co[i] = (float)phase_hi(axis_phase(c, b, a, g0)) * RAD_PER_U32;
            si[i] = 0.0f;
        } else {
            sincospif(2.0f * ((float)phase_hi(d) * TURN_PER_U32), &si[i], &co[i]);
        }
        d += step;
        step += 2 * c;
    }
    *reinterpret_cast<float4 *>(row + rotation_pos(g, k0, ng)) =
        make_float4(co[0], co[1], co[2], co[3]);
    *reinterpret_cast<float4 *>(row + rotation_pos(g, gs + k0, ng)) =
        make_float4(si[0], si[1], si[2], si[3]);
}

template <bool FUSE>
__global__ void direct_tables_kernel(const PointRec *__restrict__ rec,
                                     PointSource src, int Npad, int TX, int TY, int XG,
                                     int YG, int nxt, int nyt, float *__restrict__ phx,
                                     float *__restrict__ phy,
                                     float *__restrict__ amp,
                                     unsigned *__restrict__ zero, int nzero) {
    __shared__ PointRec srec[DT_POINTS];
    pdl_wait();  // the records (or the caller's points) come from the kernel before
    pdl_trigger();
    // the split schedule's per-tile arrival counters start at zero (every
    // earlier kernel on the stream has finished: pdl_wait above)
    if (blockIdx.x == 0)
        for (int k = blockIdx.y * blockDim.x + threadIdx.x; k < nzero;
             k += gridDim.y * blockDim.x)
            zero[k] = 0u;
    const int j0 = blockIdx.x * DT_POINTS;
    if (threadIdx.x < DT_POINTS && j0 + (int)threadIdx.x < Npad) {
        if constexpr (FUSE)
            srec[threadIdx.x] =
                make_point_rec(src.points, src.A, src.z, src.N, j0 + threadIdx.x,
                               src.K, src.status, src.y0);
        else
            srec[threadIdx.x] = rec[j0 + threadIdx.x];
    }
    __syncthreads();
    // grid y: the x coordinates in blocks of 256, then the y coordinates
    const int nx = nxt * TX, ny = nyt * TY, nbx = (nx + 255) / 256;
    const int axis = (int)blockIdx.y >= nbx ? 1 : 0;
    const int w0 = ((int)blockIdx.y - axis * nbx) * 256;  // the block's first coordinate
    const int n = axis ? ny : nx, T = axis ? TY : TX, gs = axis ? YG : XG;
    float *tab = axis ? phy : phx;
    const int npts = Npad - j0 < DT_POINTS ? Npad - j0 : DT_POINTS;
    if (gs) {
        // a rotation table: one thread per four coordinates and point
        for (int it = threadIdx.x; it < 64 * npts; it += blockDim.x) {
            const int w = w0 + 4 * (it & 63), q = it >> 6;
            if (w >= n) continue;
            const int t = w / T, i = w - t * T, g = i / gs, h = (i - g * gs) >> 2;
            rotation_quarter(srec[q], axis, w - 4 * h, g, h, gs, T / gs,
                             tab + ((size_t)t * Npad + j0 + q) * T * 2);
        }
    } else {
        const int u = w0 + threadIdx.x;
        if (u < n) {
            const int t = u / T, i = u - t * T;
            angle_column(srec, npts, u, axis, tab + ((size_t)t * Npad + j0) * T + i, T);
        }
    }
    if (blockIdx.y == 0 && threadIdx.x < npts) amp[j0 + threadIdx.x] = srec[threadIdx.x].A;
}

// ------------------------------------------------------- direct kernel
// One CTA per pixel tile (1-D grid, tiles in row-major order), except for
// the last tiles when their count does not spread evenly over the SMs: the
// tiles from `tail` on are each cut into `m` chunks of point stages, one CTA
// per chunk, placed after the whole tiles in the grid so that they fill the
// SMs that finish first.  Each chunk CTA writes its partial tile to `part`
// (slot = chunk index) and counts itself in count[tile - tail]; the last to
// arrive adds the m partials in chunk order -- the same order whoever is
// last, so the result is deterministic -- and writes the tile.  No CTA waits
// for another.
template <int TX, int TY, int VX, int VY, int PT, int NST, int NP, int G, int PK>
__global__ void __launch_bounds__(DirectTileLoop<TX, TY, VX, VY, PT, NST, NP, G, PK>::S::THREADS,
                                    DirectTileLoop<TX, TY, VX, VY, PT, NST, NP, G, PK>::MIN_CTAS)
direct_fwd_kernel(const float *__restrict__ phx, const float *__restrict__ phy,
                  const float *__restrict__ amp, int Npad, int Nx, int Ny,
                  int nxt, int tail, int m, float *__restrict__ out,
                  int vec_store, float *__restrict__ part,
                  unsigned *__restrict__ count, unsigned *status) {
    using L = DirectTileLoop<TX, TY, VX, VY, PT, NST, NP, G, PK>;
    using S = typename L::S;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t full[NST];
    __shared__ volatile int abort_flag;
    __shared__ int s_last;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    pdl_wait();  // the tables (and zeroed counters) come from the kernel before
    __syncthreads();

    const int nst = Npad / PT;  // point stages per tile
    int tile = (int)blockIdx.x, s0 = 0, s1 = nst, q = -1;
    if (tile >= tail) {  // a chunk of a split tile
        q = tile - tail;
        tile = tail + q / m;
        const int k = q % m;
        s0 = (int)((long long)nst * k / m);
        s1 = (int)((long long)nst * (k + 1) / m);
    }
    const int xt = tile % nxt, yt = tile / nxt;
    typename L::Acc acc;
    acc.zero();
    if (!L::accumulate(smem, full, &abort_flag,
                       phx + (size_t)xt * Npad * TX * L::XF + (size_t)s0 * S::SX,
                       phy + (size_t)yt * Npad * TY * L::YF + (size_t)s0 * S::SY,
                       amp + (size_t)s0 * PT, s1 - s0, 0u, acc, status))
        return;
    // only the stores are left: the next kernel of the stream may launch
    pdl_trigger();
    if (q < 0) {
        L::store(acc, smem, xt, yt, Nx, Ny, out, vec_store);
        return;
    }
    // publish this chunk's partial tile, then count in
    L::reduce_groups(acc, smem);
    const int lt = threadIdx.x % S::GT, grp = threadIdx.x / S::GT;
    const int tx = lt % S::NTX, ty = lt / S::NTX;
    const int off = (ty * VY) * TX + tx * VX;
    if (grp == 0) {
        float *dst = part + (size_t)q * TX * TY + off;
#pragma unroll
        for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int k = 0; k < VX; ++k) dst[r * TX + k] = acc.get(r, k);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = atomicAdd(&count[tile - tail], 1u) == (unsigned)(m - 1);
    __syncthreads();
    if (s_last && grp == 0) {
        __threadfence();
        acc.zero();
        const float *src = part + (size_t)(tile - tail) * m * TX * TY + off;
        for (int k = 0; k < m; ++k, src += TX * TY)
#pragma unroll
            for (int r = 0; r < VY; ++r)
#pragma unroll
                for (int c = 0; c < VX; ++c) acc.add(r, c, __ldcg(src + r * TX + c));
        L::write_out(acc, xt, yt, Nx, Ny, out, vec_store);
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

static const DirectTile kTiles[] = {
#define X(tx, ty, vx, vy, pt, ns, np, g, pk) {tx, ty, vx, vy, pt, np, g, pk},
    CGH_DIRECT_TILES(X)
#undef X
};
static constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

int direct_tile_count() { return kNumTiles; }
DirectTile direct_tile_get(int i) { return kTiles[i]; }
int direct_tile_index(const DirectTile &t) {
    for (int i = 0; i < kNumTiles; ++i)
        if (kTiles[i].tx == t.tx && kTiles[i].ty == t.ty && kTiles[i].vx == t.vx &&
            kTiles[i].vy == t.vy && kTiles[i].pt == t.pt && kTiles[i].np == t.np &&
            kTiles[i].g == t.g && kTiles[i].pk == t.pk)
            return i;
    return -1;
}

size_t direct_phase_table_floats(const DirectTile &t, int Npad, int Nx,
                                 int Ny) {
    const int nxt = (Nx + t.tx - 1) / t.tx, nyt = (Ny + t.ty - 1) / t.ty;
    return direct_x_floats(t, nxt, Npad) + direct_y_floats(t, nyt, Npad);
}

static cudaError_t launch_tables(const PointRec *rec, const PointSource *src,
                                 int Npad, int Nx, int Ny, const DirectTile &t,
                                 float *phx, float *phy, float *amp,
                                 unsigned *zero, int nzero, cudaStream_t s) {
    int nxt = (Nx + t.tx - 1) / t.tx, nyt = (Ny + t.ty - 1) / t.ty;
    // grid y: the x coordinates, then the y coordinates, in blocks of 256
    const int nby = (nxt * t.tx + 255) / 256 + (nyt * t.ty + 255) / 256;
    dim3 grid((Npad + DT_POINTS - 1) / DT_POINTS, nby);
    const int xg = direct_xg(t), yg = direct_yg(t);
    if (src)  // (builds the records itself: the call's first kernel)
        return launch_kernel(false, direct_tables_kernel<true>, grid, dim3(256), 0, s,
                             (const PointRec *)nullptr, *src, Npad, t.tx, t.ty, xg, yg, nxt,
                             nyt, phx, phy, amp, zero, nzero);
    return launch_dependent(direct_tables_kernel<false>, grid, dim3(256), 0, s, rec,
                            PointSource{}, Npad, t.tx, t.ty, xg, yg, nxt, nyt, phx, phy,
                            amp, zero, nzero);
}

cudaError_t launch_direct_tables(const PointRec *rec, int Npad, int Nx, int Ny,
                                 const DirectTile &t, float *phx, float *phy,
                                 float *amp, unsigned *zero, int nzero,
                                 cudaStream_t s) {
    return launch_tables(rec, nullptr, Npad, Nx, Ny, t, phx, phy, amp, zero, nzero, s);
}

cudaError_t launch_direct_tables_fused(const PointSource &src, int Npad, int Nx,
                                       int Ny, const DirectTile &t, float *phx,
                                       float *phy, float *amp, unsigned *zero,
                                       int nzero, cudaStream_t s) {
    return launch_tables(nullptr, &src, Npad, Nx, Ny, t, phx, phy, amp, zero, nzero, s);
}

DirectSplit direct_split_plan(int tile_index, int sm_count, int Npad, int Nx,
                              int Ny, bool split) {
    const DirectTile &t = kTiles[tile_index];
    DirectSplit d;
    d.tiles = ((Nx + t.tx - 1) / t.tx) * ((Ny + t.ty - 1) / t.ty);
    d.tail = d.tiles;
    d.m = 1;
    const int nst = Npad / t.pt;
    const int rem = sm_count > 0 ? d.tiles % sm_count : 0;
    if (!split || rem == 0 || nst < 2) return d;
    // the last `rem` tiles, each cut into about 2 SMs' worth / rem chunks
    d.tail = d.tiles - rem;
    d.m = (2 * sm_count + rem - 1) / rem;
    if (d.m > nst) d.m = nst;
    if (d.m < 2) {
        d.tail = d.tiles;
        d.m = 1;
    }
    return d;
}

template <int TX, int TY, int VX, int VY, int PT, int NST, int NP, int G, int PK>
static cudaError_t launch_one(const float *phx, const float *phy,
                              const float *amp, int Npad, int Nx, int Ny,
                              float *out, const DirectSplit &d, float *part,
                              unsigned *count, unsigned *status, cudaStream_t s) {
    using S = typename DirectTileLoop<TX, TY, VX, VY, PT, NST, NP, G, PK>::S;
    auto kern = direct_fwd_kernel<TX, TY, VX, VY, PT, NST, NP, G, PK>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const int nxt = (Nx + TX - 1) / TX;
    const unsigned grid = (unsigned)d.tail + (unsigned)(d.tiles - d.tail) * d.m;
    int vec_store = (Nx % 4 == 0) && (((uintptr_t)out & 15) == 0);
    return launch_dependent(kern, dim3(grid), dim3(S::THREADS), S::SMEM, s, phx, phy,
                            amp, Npad, Nx, Ny, nxt, d.tail, d.m, out, vec_store, part,
                            count, status);
}

cudaError_t launch_direct_forward(int tile_index, const float *phx,
                                  const float *phy, const float *amp, int Npad,
                                  int Nx, int Ny, float *out,
                                  const DirectSplit &d, float *part,
                                  unsigned *count, unsigned *status,
                                  cudaStream_t s) {
    if (d.tail < d.tiles && (!part || !count)) return cudaErrorInvalidValue;
    int i = 0;
#define X(tx, ty, vx, vy, pt, ns, np, g, pk)                                   \
    if (tile_index == i)                                                       \
        return launch_one<tx, ty, vx, vy, pt, ns, np, g, pk>(                   \
            phx, phy, amp, Npad, Nx, Ny, out, d, part, count, status, s);      \
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
