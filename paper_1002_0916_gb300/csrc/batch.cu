// batch.cu -- many holograms of uneven size, point count and wavelength in
// one persistent launch (step A9).
//
// Direct FP32 batch:
//   1. one prologue launch builds the point records of every problem
//      (grid y = problem);
//   2. one launch writes every problem's per-axis angle tables;
//   3. one persistent launch (as many CTAs as fit on the SMs at once) pulls
//      work items -- (problem, pixel tile) -- from an atomic counter, in the
//      order of a host-built list sorted longest-first (by point count); each
//      item runs the same staged point loop as the single-hologram kernel,
//      with the shared-memory ring and its mbarriers carried from item to
//      item.
// The counter reset, the zero-fill of problems without points and the three
// launches are captured once per batch geometry into a CUDA graph on a
// private stream and replayed on the caller's stream.  If the caller's
// stream is itself being captured, the same nodes are enqueued on it instead.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "api_internal.h"
#include "common.cuh"
#include "direct_tile.cuh"
#include "point_rec.cuh"
#include "sep_table.cuh"
#include "umma.cuh"

namespace cgh {

struct BatchPrep {  // per problem: inputs and where its tables go
    const float *points, *A, *z;
    double K;  // fresnel_scale(lambda, p)
    int N, Npad, Nx, Ny, nxt, nyt, TX, TY, XG, YG;  // XG, YG: rotation groups (0: none)
    PointRec *rec;
    float *phx, *phy, *amp;
};

struct BatchTile {  // per problem: what the persistent kernel reads
    const float *phx, *phy, *amp;
    float *out;
    int Npad, Nx, Ny, vec_store;
};

__global__ void batch_prologue_kernel(const BatchPrep *__restrict__ prep,
                                      unsigned *status) {
    const BatchPrep &b = prep[blockIdx.y];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < b.Npad;
         j += gridDim.x * blockDim.x)
        b.rec[j] = make_point_rec(b.points, b.A, b.z, b.N, j, b.K, status);
}

__global__ void batch_tables_kernel(const BatchPrep *__restrict__ prep) {
    const BatchPrep &b = prep[blockIdx.y];
    const long long total =
        direct_table_entries(b.Npad, b.TX, b.TY, b.nxt, b.nyt, b.XG, b.YG);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        direct_table_entry(b.rec, b.Npad, b.TX, b.TY, b.nxt, b.nyt, b.XG, b.YG, e, b.phx,
                           b.phy, b.amp);
}

template <int TX, int TY, int VX, int VY, int PT, int NST, int NP, int G, int PK>
__global__ void __launch_bounds__(DirectTileLoop<TX, TY, VX, VY, PT, NST, NP, G, PK>::S::THREADS,
                                    DirectTileLoop<TX, TY, VX, VY, PT, NST, NP, G, PK>::MIN_CTAS)
direct_batch_kernel(const BatchTile *__restrict__ probs,
                    const uint2 *__restrict__ items, int nitems,
                    unsigned *counter, unsigned *status) {
    using L = DirectTileLoop<TX, TY, VX, VY, PT, NST, NP, G, PK>;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t full[NST];
    __shared__ volatile int abort_flag;
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    unsigned g = 0;  // stage loads this CTA has issued so far
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const uint2 w = items[it];
        const BatchTile bt = probs[w.x];
        const int xt = (int)(w.y & 0xffffu), yt = (int)(w.y >> 16);
        const int ntile = bt.Npad / PT;
        typename L::Acc acc;
        acc.zero();
        if (!L::accumulate(smem, full, &abort_flag,
                           bt.phx + (size_t)xt * bt.Npad * TX * L::XF,
                           bt.phy + (size_t)yt * bt.Npad * TY * L::YF, bt.amp, ntile, g,
                           acc,
                           status))
            return;
        g += (unsigned)ntile;
        L::store(acc, smem, xt, yt, bt.Nx, bt.Ny, bt.out, bt.vec_store);
    }
}

template <int TX, int TY, int VX, int VY, int PT, int NST, int NP, int G, int PK>
static cudaError_t launch_batch_t(const BatchTile *probs, const uint2 *items,
                                  int nitems, unsigned *counter, unsigned *status,
                                  int sm_count, cudaStream_t s) {
    // probs == nullptr: only set the kernel's attributes and cache its
    // occupancy (done before any capture)
    using S = typename DirectTileLoop<TX, TY, VX, VY, PT, NST, NP, G, PK>::S;
    auto kern = direct_batch_kernel<TX, TY, VX, VY, PT, NST, NP, G, PK>;
    // attribute and occupancy once per device (no such calls inside a capture
    // of a geometry that has run before)
    static int per_sm_cache[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = (dev >= 0 && dev < 64) ? per_sm_cache[dev] : 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::THREADS,
                                                          S::SMEM);
        if (e != cudaSuccess) return e;
        per_sm = std::max(1, per_sm);
        if (dev >= 0 && dev < 64) per_sm_cache[dev] = per_sm;
    }
    if (!probs) return cudaSuccess;
    int grid = per_sm * sm_count;
    if (grid > nitems) grid = nitems;
    kern<<<grid, S::THREADS, S::SMEM, s>>>(probs, items, nitems, counter, status);
    return cudaGetLastError();
}

static cudaError_t launch_batch(int tile_index, const BatchTile *probs,
                                const uint2 *items, int nitems, unsigned *counter,
                                unsigned *status, int sm_count, cudaStream_t s) {
    int i = 0;
#define X(tx, ty, vx, vy, pt, ns, np, g, pk)                                    \
    if (tile_index == i)                                                        \
        return launch_batch_t<tx, ty, vx, vy, pt, ns, np, g, pk>(                \
            probs, items, nitems, counter, status, sm_count, s);                \
    ++i;
    CGH_DIRECT_TILES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace cgh

using namespace cgh;

namespace {

uint64_t fnv1a(uint64_t h, const void *data, size_t n) {
    const unsigned char *p = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

cgh_status cgh_ctx::ensure_host_stage(size_t bytes) {
    if (bytes <= host_stage_bytes) return CGH_OK;
    if (stage_done) cudaEventSynchronize(stage_done);
    if (host_stage) cudaFreeHost(host_stage);
    host_stage = nullptr;
    host_stage_bytes = 0;
    size_t want = (bytes + bytes / 4 + 4095) & ~(size_t)4095;
    cudaError_t e = cudaMallocHost(&host_stage, want);
    if (e != cudaSuccess) {
        host_stage = nullptr;
        return cuda_fail(e, "cudaMallocHost (batch staging)");
    }
    host_stage_bytes = want;
    return CGH_OK;
}

// Stage `meta_b` bytes from host_stage to meta (only when the geometry key
// changed), then run `enqueue` -- through the cached graph of this key, or
// straight onto `s` when the caller is capturing `s`.
cgh_status cgh_ctx::run_batch_graph(uint64_t key, size_t meta_b, int nkernels,
                                    const std::function<void(char *)> &fill_stage,
                                    const std::function<cudaError_t(cudaStream_t)> &enqueue,
                                    cudaStream_t s, int timer) {
    void *ptrs[4] = {bws.ptr, meta.ptr, host_stage, (void *)d_status};
    key = fnv1a(key, ptrs, sizeof(ptrs));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    const bool outer_capture = cs != cudaStreamCaptureStatusNone;
    // Inside a caller's capture nothing may synchronise, so that case needs
    // the geometry to have been run once before (its work list is then
    // already on the device).
    if (outer_capture && key != batch_key)
        return fail(CGH_ERR_UNSUPPORTED,
                    "capture of a batch geometry this handle has not run yet; "
                    "run one uncaptured call of this batch first");
    if (key != batch_key) {
        // the previous copy out of the staging buffer must have happened
        if (stage_done) {
            e = cudaEventSynchronize(stage_done);
            if (e != cudaSuccess) return cuda_fail(e, "staging event");
        } else {
            e = cudaEventCreateWithFlags(&stage_done, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "staging event");
        }
        memset(host_stage, 0, meta_b);
        fill_stage((char *)host_stage);
        e = cudaMemcpyAsync(meta.ptr, host_stage, meta_b, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch metadata copy");
        e = cudaEventRecord(stage_done, s);
        if (e != cudaSuccess) return cuda_fail(e, "staging event");
    }
    if (outer_capture) {
        e = enqueue(s);
        if (e != cudaSuccess) return cuda_fail(e, "batch enqueue");
        launches += nkernels;
        return CGH_OK;
    }
    if (key != batch_key) {
        if (batch_exec) cudaGraphExecDestroy(batch_exec);
        batch_exec = nullptr;
        batch_key = 0;
        if (!cap_stream) {
            e = cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "capture stream");
        }
        e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        cudaError_t le = enqueue(cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap_stream, &graph);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(le != cudaSuccess ? le : e, "batch graph capture");
        }
        e = cudaGraphInstantiate(&batch_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            batch_exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        batch_key = key;
    }
    TimedLaunch tl(this, timer, s);
    e = cudaGraphLaunch(batch_exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    tl.done();
    launches += nkernels > 0 ? nkernels - 1 : 0;
    return CGH_OK;
}

cgh_status cgh_ctx::batch_direct(const cgh_problem *probs, int count,
                                 cudaStream_t s, int tile_index) {
    const DirectTile t = direct_tile_get(tile_index);
    // ---- per-problem layout
    std::vector<BatchPrep> prep;
    std::vector<BatchTile> tiles;
    std::vector<int> pidx;  // problem index of each prep entry
    size_t ws_bytes = 0;
    std::vector<size_t> off_rec, off_tab, off_amp;
    for (int i = 0; i < count; ++i) {
        const cgh_problem &pr = probs[i];
        if (pr.N == 0) continue;
        const int Npad = pad_to(pr.N, t.pt);
        off_rec.push_back(ws_bytes);
        ws_bytes += align256((size_t)Npad * sizeof(PointRec));
        off_tab.push_back(ws_bytes);
        ws_bytes += align256(direct_phase_table_floats(t, Npad, pr.Nx, pr.Ny) * 4);
        off_amp.push_back(ws_bytes);
        ws_bytes += align256((size_t)Npad * 4);
        pidx.push_back(i);
    }
    cgh_status st = ensure(bws, ws_bytes > 0 ? ws_bytes : 256, s, "batch workspace");
    if (st) return st;
    char *wb = (char *)bws.ptr;
    for (size_t k = 0; k < pidx.size(); ++k) {
        const cgh_problem &pr = probs[pidx[k]];
        BatchPrep b;
        b.points = pr.points;
        b.A = pr.A;
        b.z = pr.z;
        b.K = fresnel_scale(pr.lambda, pr.p);
        b.N = pr.N;
        b.Npad = pad_to(pr.N, t.pt);
        b.Nx = pr.Nx;
        b.Ny = pr.Ny;
        b.nxt = (pr.Nx + t.tx - 1) / t.tx;
        b.nyt = (pr.Ny + t.ty - 1) / t.ty;
        b.TX = t.tx;
        b.XG = direct_xg(t);
        b.YG = direct_yg(t);
        b.TY = t.ty;
        b.rec = (PointRec *)(wb + off_rec[k]);
        b.phx = (float *)(wb + off_tab[k]);
        b.phy = b.phx + direct_x_floats(t, b.nxt, b.Npad);
        b.amp = (float *)(wb + off_amp[k]);
        prep.push_back(b);
        BatchTile bt;
        bt.phx = b.phx;
        bt.phy = b.phy;
        bt.amp = b.amp;
        bt.out = pr.out;
        bt.Npad = b.Npad;
        bt.Nx = pr.Nx;
        bt.Ny = pr.Ny;
        bt.vec_store = (pr.Nx % 4 == 0) && (((uintptr_t)pr.out & 15) == 0);
        tiles.push_back(bt);
    }
    // ---- work list: (problem, tile), longest (most points) first
    std::vector<uint2> items;
    std::vector<int> order(prep.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return prep[a].N > prep[b].N; });
    for (int k : order)
        for (int yt = 0; yt < prep[k].nyt; ++yt)
            for (int xt = 0; xt < prep[k].nxt; ++xt)
                items.push_back(make_uint2((unsigned)k, (unsigned)xt | ((unsigned)yt << 16)));
    const int nitems = (int)items.size();
    // ---- metadata: counter | prep | tiles | items
    const size_t c_b = 256;
    const size_t prep_b = align256(prep.size() * sizeof(BatchPrep));
    const size_t tile_b = align256(tiles.size() * sizeof(BatchTile));
    const size_t item_b = align256(items.size() * sizeof(uint2));
    const size_t meta_b = c_b + prep_b + tile_b + item_b;
    st = ensure(meta, meta_b, s, "batch metadata");
    if (st) return st;
    st = ensure_host_stage(meta_b);
    if (st) return st;
    char *mb = (char *)meta.ptr;
    unsigned *counter = (unsigned *)mb;
    BatchPrep *d_prep = (BatchPrep *)(mb + c_b);
    BatchTile *d_tiles = (BatchTile *)(mb + c_b + prep_b);
    uint2 *d_items = (uint2 *)(mb + c_b + prep_b + tile_b);

    uint64_t key = 1469598103934665603ull;
    const int method = CGH_DIRECT_FP32;
    key = fnv1a(key, &method, sizeof(method));
    key = fnv1a(key, &tile_index, sizeof(tile_index));
    key = fnv1a(key, &count, sizeof(count));
    key = fnv1a(key, probs, sizeof(cgh_problem) * (size_t)count);

    int maxNpad = 1;
    for (auto &bp : prep) maxNpad = std::max(maxNpad, bp.Npad);
    int max_entries_blocks = 1;
    for (auto &bp : prep) {
        long long n = (long long)bp.nxt * bp.Npad * bp.TX * (bp.XG ? 2 : 1) +
                      (long long)bp.nyt * bp.Npad * bp.TY * (bp.YG ? 2 : 1) + bp.Npad;
        max_entries_blocks = (int)std::max<long long>(max_entries_blocks, (n + 255) / 256);
    }
    const int np = (int)prep.size();
    cudaError_t e = launch_batch(tile_index, nullptr, nullptr, 0, nullptr, nullptr,
                                 sm_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel set-up");
    auto fill = [&](char *hb) {
        memcpy(hb + c_b, prep.data(), prep.size() * sizeof(BatchPrep));
        memcpy(hb + c_b + prep_b, tiles.data(), tiles.size() * sizeof(BatchTile));
        memcpy(hb + c_b + prep_b + tile_b, items.data(), items.size() * sizeof(uint2));
    };
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t r = cudaMemsetAsync(counter, 0, sizeof(unsigned), q);
        for (int i = 0; i < count && r == cudaSuccess; ++i)
            if (probs[i].N == 0)
                r = cudaMemsetAsync(probs[i].out, 0,
                                    (size_t)probs[i].Nx * probs[i].Ny * sizeof(float), q);
        if (r != cudaSuccess || np == 0) return r;
        dim3 g1((maxNpad + 127) / 128, np);
        batch_prologue_kernel<<<g1, 128, 0, q>>>(d_prep, d_status);
        r = cudaGetLastError();
        if (r != cudaSuccess) return r;
        dim3 g2(std::min(max_entries_blocks, 1024), np);
        batch_tables_kernel<<<g2, 256, 0, q>>>(d_prep);
        r = cudaGetLastError();
        if (r != cudaSuccess) return r;
        return launch_batch(tile_index, d_tiles, d_items, nitems, counter, d_status,
                            sm_count, q);
    };
    return run_batch_graph(key, meta_b, np ? 3 : 0, fill, enqueue, s, CGH_K_BATCH);
}

cgh_status cgh_ctx::batch(const cgh_problem *probs, int count, int method,
                          cudaStream_t s, int forced_tile_index, int forced_pairs) {
    if (count < 1 || count > 4096 || !probs)
        return fail(CGH_ERR_INVALID_ARG, "batch count %d outside [1, 4096]", count);
    for (int i = 0; i < count; ++i) {
        const cgh_problem &p = probs[i];
        cgh_status st = check_problem(p.points, p.A, p.z, p.N, p.lambda, p.p, p.Nx,
                                      p.Ny, p.out);
        if (st) {
            // (the message names the problem; a long one is cut to fit)
            char msg[sizeof(err) + 32];
            snprintf(msg, sizeof(msg), "problem %d: %s", i, err);
            snprintf(err, sizeof(err), "%.*s", (int)sizeof(err) - 1, msg);
            return st;
        }
    }
    if (method == CGH_DIRECT_FP32) {
        int ti = forced_tile_index >= 0 ? forced_tile_index : forced_tile;
        if (ti < 0) {
            auto it = tuned.find(batch_bucket(probs, count));
            if (it != tuned.end()) {
                ti = it->second;
            } else {
                ti = default_batch_tile(probs, count);
            }
        }
        return batch_direct(probs, count, s, ti);
    }
    if (method == CGH_SEP_FP16X3) return batch_separable(probs, count, s, forced_pairs);
    return fail(CGH_ERR_INVALID_ARG,
                "batch method must be CGH_DIRECT_FP32 or CGH_SEP_FP16X3");
}

// Untuned: the heuristic's shape for the problem with the most work
// (persistent CTAs balance the rest).
int cgh_ctx::default_batch_tile(const cgh_problem *probs, int count) {
    int big = 0;
    for (int i = 1; i < count; ++i)
        if ((double)probs[i].N * probs[i].Nx * probs[i].Ny >
            (double)probs[big].N * probs[big].Nx * probs[big].Ny)
            big = i;
    return default_direct_tile(probs[big].N, probs[big].Nx, probs[big].Ny, sm_count);
}

std::string batch_bucket(const cgh_problem *probs, int count) {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < count; ++i) {
        int v[3] = {probs[i].N, probs[i].Nx, probs[i].Ny};
        h = fnv1a(h, v, sizeof(v));
    }
    char buf[64];
    snprintf(buf, sizeof(buf), "batch_%d_%016llx", count, (unsigned long long)h);
    return buf;
}

extern "C" cgh_status cgh_batch(cgh_handle h, const cgh_problem *probs, int count,
                                int method, void *stream) {
    NvtxRange range("cgh_batch");
    if (!h) return CGH_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    h->err[0] = 0;
    cgh_status st = h->batch(probs, count, method, (cudaStream_t)stream, -1);
    if (prev != h->device) cudaSetDevice(prev);
    return st;
}

extern "C" cgh_status cgh_batch_plan(cgh_handle h, const cgh_problem *probs, int count,
                                     int method, cgh_direct_tile *tile, int *gemm_tiling,
                                     int *tuned) {
    if (!h || !probs || count < 1 || count > 4096) return CGH_ERR_INVALID_ARG;
    if (tuned) *tuned = 0;
    if (method == CGH_DIRECT_FP32) {
        int ti = h->forced_tile;
        if (ti < 0) {
            auto it = h->tuned.find(batch_bucket(probs, count));
            if (it != h->tuned.end()) {
                ti = it->second;
                if (tuned) *tuned = 1;
            } else {
                ti = h->default_batch_tile(probs, count);
            }
        }
        if (gemm_tiling) *gemm_tiling = 0;
        return tile ? cgh_direct_tile_get(ti, tile) : CGH_OK;
    }
    if (method == CGH_SEP_FP16X3) {
        bool tu = false;
        const bool pairs = h->batch_sep_pairs(probs, count, &tu);
        if (gemm_tiling) *gemm_tiling = pairs ? CGH_GEMM_PAIRS : CGH_GEMM_SINGLE;
        if (tuned) *tuned = tu ? 1 : 0;
        if (tile) memset(tile, 0, sizeof(*tile));
        return CGH_OK;
    }
    return CGH_ERR_INVALID_ARG;
}

extern "C" cgh_status cgh_tune_batch(cgh_handle h, const cgh_problem *probs,
                                     int count, int method, void *stream,
                                     cgh_direct_tile *chosen) {
    NvtxRange range("cgh_tune_batch");
    if (!h) return CGH_ERR_INVALID_ARG;
    if (method != CGH_DIRECT_FP32 && method != CGH_SEP_FP16X3)
        return h->fail(CGH_ERR_INVALID_ARG,
                       "batch method must be CGH_DIRECT_FP32 or CGH_SEP_FP16X3");
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (method == CGH_SEP_FP16X3) {
        // the grouped split-FP16 GEMM's two item shapes: one-CTA items (the
        // default) and CTA-pair items, each timed on its captured graph
        int best_pairs = -1;
        cgh_status st = tune_pick(h, 2, 0, TUNE_KEEP, s,
                                  [&](int pairs) {
                                      return h->batch(probs, count, method, s, -1, pairs);
                                  },
                                  &best_pairs, nullptr);
        if (st == CGH_OK && best_pairs >= 0)
            h->tuned_gemm[batch_bucket(probs, count) + "_sep"] =
                (best_pairs ? CGH_GEMM_PAIRS : CGH_GEMM_SINGLE) * 1000 +
                (best_pairs ? group_pair_tile_n() : group_tile_n());
        if (chosen) memset(chosen, 0, sizeof(*chosen));
        if (prev != h->device) cudaSetDevice(prev);
        return st;
    }
    int best_i = -1;
    cgh_status st = tune_pick(h, direct_tile_count(), h->default_batch_tile(probs, count),
                              TUNE_KEEP, s,
                              [&](int i) {
                                  return h->batch(probs, count, CGH_DIRECT_FP32, s, i);
                              },
                              &best_i, nullptr, 1, 2);  // (each call is a whole batch)
    if (st == CGH_OK && best_i >= 0) {
        h->tuned[batch_bucket(probs, count)] = best_i;
        if (chosen) {
            DirectTile t = direct_tile_get(best_i);
            chosen->tile_x = t.tx;
            chosen->tile_y = t.ty;
            chosen->vec_x = t.vx;
            chosen->vec_y = t.vy;
            chosen->points_per_stage = t.pt;
            chosen->poly_pixels = t.np;
            chosen->point_groups = t.g;
            chosen->packed = t.pk;
        }
    }
    if (prev != h->device) cudaSetDevice(prev);
    return st;
}

struct SepPrep {  // per problem: inputs and where its U/V tables go
    const float *points, *A, *z;
    double K;  // fresnel_scale(lambda, p)
    int N, Npad, Nx, Ny, Kp;
    PointRec *rec;
    void *Lhi, *Llo, *Rhi, *Rlo;
};

__global__ void sep_batch_prologue_kernel(const SepPrep *__restrict__ prep,
                                          unsigned *status) {
    const SepPrep &b = prep[blockIdx.y];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < b.Npad;
         j += gridDim.x * blockDim.x)
        b.rec[j] = make_point_rec(b.points, b.A, b.z, b.N, j, b.K, status);
}

// Work items of one problem: (point pair, group of ST_ROWS table rows),
// pairs fastest so that a warp writes contiguous 256-byte rows.
__global__ void sep_batch_tables_kernel(const SepPrep *__restrict__ prep) {
    const SepPrep &b = prep[blockIdx.y];
    const int pairs = b.Kp / 4;
    const int groups = (b.Nx + b.Ny + ST_ROWS - 1) / ST_ROWS;
    const long long total = (long long)pairs * groups;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(w / pairs);
        const int j0 = 2 * (int)(w - (long long)g * pairs);
        const int r0 = g * ST_ROWS;
        const int r1 = r0 + ST_ROWS < b.Nx + b.Ny ? r0 + ST_ROWS : b.Nx + b.Ny;
        const bool v0 = j0 < b.N, v1 = j0 + 1 < b.N;
        const PointRec p0 = v0 ? b.rec[j0] : PointRec{};
        const PointRec p1 = v1 ? b.rec[j0 + 1] : PointRec{};
        sep_table_rows<2>(p0, p1, v0, v1, b.Nx, b.Kp, j0, r0, r1, b.Lhi, b.Llo,
                          b.Rhi, b.Rlo);
    }
}

// Split-FP16 batch: one prologue launch, one table launch, one persistent
// grouped tensor-core GEMM (umma.cu) over (problem, m tile, n tile) items.
bool cgh_ctx::batch_sep_pairs(const cgh_problem *probs, int count, bool *tuned_out) {
    if (tuned_out) *tuned_out = false;
    if (gemm_tiles == CGH_GEMM_PAIRS || gemm_tiles == CGH_GEMM_PAIRS_GEN) return true;
    if (gemm_tiles == CGH_GEMM_SINGLE) return false;
    auto it = tuned_gemm.find(batch_bucket(probs, count) + "_sep");
    if (it != tuned_gemm.end()) {
        if (tuned_out) *tuned_out = true;
        return it->second / 1000 == CGH_GEMM_PAIRS;
    }
    // one-CTA items (128 x 128) unless CTA pairs were asked for: pair items
    // (256 x 128) halve the number of work items, and on the 64-hologram
    // batch the coarser balance cost more (4.55 ms) than the halved operand
    // bytes per SM saved (one-CTA items: 4.24 ms)
    return false;
}

cgh_status cgh_ctx::batch_separable(const cgh_problem *probs, int count,
                                    cudaStream_t s, int pairs_override) {
    std::vector<SepPrep> prep;
    std::vector<size_t> offs;
    size_t ws_bytes = 0;
    for (int i = 0; i < count; ++i) {
        const cgh_problem &pr = probs[i];
        if (pr.N == 0) continue;
        const int Kp = pad_to(2 * pr.N, 64);
        offs.push_back(ws_bytes);
        ws_bytes += align256((size_t)(Kp / 2) * sizeof(PointRec));
        ws_bytes += 2 * align256((size_t)pr.Nx * Kp * 2);
        ws_bytes += 2 * align256((size_t)pr.Ny * Kp * 2);
        SepPrep sp{};
        sp.points = pr.points;
        sp.A = pr.A;
        sp.z = pr.z;
        sp.K = fresnel_scale(pr.lambda, pr.p);
        sp.N = pr.N;
        sp.Npad = Kp / 2;
        sp.Nx = pr.Nx;
        sp.Ny = pr.Ny;
        sp.Kp = Kp;
        prep.push_back(sp);
    }
    cgh_status st = ensure(bws, ws_bytes > 0 ? ws_bytes : 256, s, "batch workspace");
    if (st) return st;
    const bool pairs = pairs_override >= 0 ? pairs_override != 0
                                           : batch_sep_pairs(probs, count, nullptr);
    const int TM = pairs ? group_pair_tile_m() : 128;
    const int BN = pairs ? group_pair_tile_n() : group_tile_n();
    const int b_box = pairs ? group_pair_box_b() : group_tile_n();
    cudaError_t e = pairs ? prepare_umma_grouped_pair() : prepare_umma_grouped();
    if (e != cudaSuccess) return cuda_fail(e, "grouped GEMM set-up");
    std::vector<GroupProb> gps(prep.size());
    std::vector<GemmOperands> ops(prep.size());
    std::vector<int> pidx;
    for (int i = 0, k = 0; i < count; ++i)
        if (probs[i].N) pidx.push_back(i), ++k;
    for (size_t k = 0; k < prep.size(); ++k) {
        SepPrep &sp = prep[k];
        char *base = (char *)bws.ptr + offs[k];
        const size_t rec_b = align256((size_t)sp.Npad * sizeof(PointRec));
        const size_t l_b = align256((size_t)sp.Nx * sp.Kp * 2);
        const size_t r_b = align256((size_t)sp.Ny * sp.Kp * 2);
        sp.rec = (PointRec *)base;
        sp.Lhi = base + rec_b;
        sp.Llo = base + rec_b + l_b;
        sp.Rhi = base + rec_b + 2 * l_b;
        sp.Rlo = base + rec_b + 2 * l_b + r_b;
        GemmOperands op{};
        op.A_hi = sp.Rhi;
        op.A_lo = sp.Rlo;
        op.B_hi = sp.Lhi;
        op.B_lo = sp.Llo;
        op.M = sp.Ny;
        op.N = sp.Nx;
        op.K = sp.Kp;
        op.lda = sp.Kp;
        op.ldb = sp.Kp;
        op.bf16 = false;
        op.split = true;
        op.lo_scale = 1.0f / LO_SCALE;
        op.D = probs[pidx[k]].out;
        op.ldd = sp.Nx;
        op.tiles = gemm_tiles == CGH_GEMM_PAIRS_GEN ? CGH_GEMM_PAIRS : gemm_tiles;
        ops[k] = op;
        if (!encode_group_prob(&gps[k], op, b_box))
            return fail(CGH_ERR_CUDA, "problem %d: tensor map encoding failed", pidx[k]);
    }
    // items: (problem, m tile, n tile), largest K first
    std::vector<int> order(prep.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c) { return prep[a].Kp > prep[c].Kp; });
    // a problem whose product is longer than one K chunk runs as its own
    // chunked GEMM launches after the grouped kernel (same graph)
    std::vector<int> long_k;
    for (int k : order)
        if (prep[k].Kp > gemm_k_chunk(true)) long_k.push_back(k);
    std::vector<uint2> items;
    for (int k : order)
        if (prep[k].Kp <= gemm_k_chunk(true))
        for (int mt = 0; mt < (prep[k].Ny + TM - 1) / TM; ++mt)
            for (int nt = 0; nt < (prep[k].Nx + BN - 1) / BN; ++nt)
                items.push_back(make_uint2((unsigned)k, (unsigned)mt | ((unsigned)nt << 16)));
    const int nitems = (int)items.size();
    const size_t prep_b = align256(prep.size() * sizeof(SepPrep));
    const size_t gp_b = align256(gps.size() * sizeof(GroupProb));
    const size_t item_b = align256(items.size() * sizeof(uint2));
    const size_t meta_b = prep_b + gp_b + item_b + 256;
    st = ensure(meta, meta_b, s, "batch metadata");
    if (st) return st;
    st = ensure_host_stage(meta_b);
    if (st) return st;
    char *mb = (char *)meta.ptr;
    SepPrep *d_prep = (SepPrep *)mb;
    GroupProb *d_gp = (GroupProb *)(mb + prep_b);
    uint2 *d_items = (uint2 *)(mb + prep_b + gp_b);
    // the tensor maps hold the workspace addresses, so the key does too
    uint64_t key = 1469598103934665603ull;
    const int method = CGH_SEP_FP16X3;
    key = fnv1a(key, &method, sizeof(method));
    key = fnv1a(key, &count, sizeof(count));
    key = fnv1a(key, &pairs, sizeof(pairs));
    key = fnv1a(key, probs, sizeof(cgh_problem) * (size_t)count);
    int maxNpad = 1, max_blocks = 1;
    for (auto &sp : prep) {
        maxNpad = std::max(maxNpad, sp.Npad);
        // work items of the table kernel: point pairs x groups of rows
        long long n = (long long)(sp.Kp / 4) * ((sp.Nx + sp.Ny + ST_ROWS - 1) / ST_ROWS);
        max_blocks = (int)std::max<long long>(max_blocks, (n + 255) / 256);
    }
    const int np = (int)prep.size();
    auto fill = [&](char *hb) {
        memcpy(hb, prep.data(), prep.size() * sizeof(SepPrep));
        memcpy(hb + prep_b, gps.data(), gps.size() * sizeof(GroupProb));
        memcpy(hb + prep_b + gp_b, items.data(), items.size() * sizeof(uint2));
    };
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        for (int i = 0; i < count && r == cudaSuccess; ++i)
            if (probs[i].N == 0)
                r = cudaMemsetAsync(probs[i].out, 0,
                                    (size_t)probs[i].Nx * probs[i].Ny * sizeof(float), q);
        if (r != cudaSuccess || np == 0) return r;
        sep_batch_prologue_kernel<<<dim3((maxNpad + 127) / 128, np), 128, 0, q>>>(
            d_prep, d_status);
        r = cudaGetLastError();
        if (r != cudaSuccess) return r;
        sep_batch_tables_kernel<<<dim3(std::min(max_blocks, 1024), np), 256, 0, q>>>(
            d_prep);
        r = cudaGetLastError();
        if (r != cudaSuccess) return r;
        r = pairs ? launch_umma_grouped_pair(d_gp, d_items, nitems, d_status, sm_count, q)
                  : launch_umma_grouped(d_gp, d_items, nitems, d_status, sm_count, q);
        for (size_t i = 0; i < long_k.size() && r == cudaSuccess; ++i)
            r = launch_umma_gemm(ops[long_k[i]], d_status, q);
        return r;
    };
    int nkernels = np ? 3 : 0;
    for (int k : long_k) nkernels += gemm_k_chunks(prep[k].Kp, true);
    return run_batch_graph(key, meta_b, nkernels, fill, enqueue, s, CGH_K_BATCH_SEP);
}
