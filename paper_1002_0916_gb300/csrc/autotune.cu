// autotune.cu -- tile-shape choice for the direct kernel: a wave-count
// heuristic by default, and a measuring autotuner (cgh_tune) whose choices
// are kept per size bucket in the handle and, optionally, in a JSON-lines
// cache file named by CGH_TUNE_CACHE.
//
// The paper fixed its shapes at compile time (16 x 16 items per group,
// 256 points per shared-memory stage, Section 2); here the best shape
// depends on how many CTAs a frame gives relative to the 152 SMs.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "api_internal.h"
#include "common.cuh"

using namespace cgh;

std::string size_bucket(int method, int N, int Nx, int Ny) {
    int nb = 1;
    while (nb < N) nb <<= 1;
    char buf[96];
    snprintf(buf, sizeof(buf), "m%d_n%d_x%d_y%d", method, nb, (Nx + 63) / 64 * 64,
             (Ny + 63) / 64 * 64);
    return buf;
}

double direct_tile_cost(int i, int N, int Nx, int Ny, int sm_count) {
    (void)N;
    const DirectTile t = direct_tile_get(i);
    // CTAs are handed to SMs as earlier ones finish, so an SM's share is
    // about ceil(CTAs / SMs) CTAs of equal work
    long long ctas = (long long)((Nx + t.tx - 1) / t.tx) * ((Ny + t.ty - 1) / t.ty);
    const double waves = (double)((ctas + sm_count - 1) / sm_count);
    // Per-update cost model (in MUFU-cosine units), from the measured
    // rates: a quarter of the cosines on the FMA pipe saves about a
    // sixth, packed FP32x2 arithmetic a further 7-9%, shared-memory loads
    // (2 vectors + 1 broadcast per point per thread) cost in proportion
    // to 1 / (pixels per thread).
    const double share = (double)t.np / (t.vx * t.vy);
    double per_pp = 1.0 - 0.65 * std::min(share, 0.25) + 0.3 * std::max(0.0, share - 0.25);
    // packed: degree-6 0.93, degree-5 (one FMA less) 0.91, interleaved
    // 0.89; an extra polynomial pair on every fourth point (a share of
    // 9/32) 1.2% less again, on every second point (5/16) no change
    static const double pk_factor[6] = {1.0, 0.93, 0.91, 0.89, 0.89, 0.879};
    if (t.pk > 0 && t.pk < 6) per_pp *= pk_factor[t.pk];
    per_pp += 0.5 / (t.vx * t.vy) + 0.25 / (t.pt / t.g);
    if (t.pk == 6) per_pp = 0.69;  // measured: 0.88 of the packed degree-5 tile
    if (t.pk >= 7) {
        // the two-axis rotation forms run on the FMA pipe: per update
        // 2 + 3 / VX FP32 operations (8 per MUFU cosine unit), at the
        // measured 0.58 of the pipe's rate
        const double f = 2.0 + 3.0 / t.vx;
        per_pp = f / 8.0 / 0.58;
    }
    return waves * t.tx * t.ty * per_pp;
}

int default_direct_tile(int N, int Nx, int Ny, int sm_count) {
    double best = 1e300;
    int best_i = 0;
    for (int i = 0; i < direct_tile_count(); ++i) {
        const double cost = direct_tile_cost(i, N, Nx, Ny, sm_count);
        if (cost < best - 1e-9) {
            best = cost;
            best_i = i;
        }
    }
    return best_i;
}

// Fill a synthetic cloud for timing: positions spread over the frame,
// z in [0.5, 1.5] m.  Values only shape the timing, not a result.
__global__ void tune_fill_kernel(float *pts, float *A, float *z, int N, int Nx,
                                 int Ny) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    unsigned hsh = (unsigned)j * 2654435761u;
    pts[2 * j] = (float)(hsh % (unsigned)Nx);
    pts[2 * j + 1] = (float)((hsh >> 11) % (unsigned)Ny);
    A[j] = 0.5f;
    z[j] = 0.5f + (float)(hsh & 1023) / 1023.0f;
}

static const char *cache_path() {
    const char *p = getenv("CGH_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

// Time n candidates, run(i) enqueueing one call of candidate i on s: `rounds`
// rounds over all candidates, each a warm-up call and `calls` timed calls
// (CUDA events), so that slow drifts of the clock touch every candidate
// alike; a candidate's time is its fastest call.  *best: the fastest candidate --
// unless the default candidate dflt is within a factor (1 + keep) of it, in
// which case the default stays: a tuned shape must beat the built-in
// choice by a clear margin, not by noise.
cgh_status tune_pick(cgh_ctx *h, int n, int dflt, double keep, cudaStream_t s,
                     const std::function<cgh_status(int)> &run, int *best, float *best_ms,
                     int rounds, int calls) {
    std::vector<float> t(n, 1e30f);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    cgh_status st = ce == cudaSuccess ? CGH_OK : h->cuda_fail(ce, "tuning events");
    for (int round = 0; round < rounds && st == CGH_OK; ++round) {
        for (int i = 0; i < n && st == CGH_OK; ++i) {
            st = run(i);
            for (int r = 0; r < calls && st == CGH_OK; ++r) {
                cudaEventRecord(e0, s);
                st = run(i);
                cudaEventRecord(e1, s);
                if (st) break;
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                t[i] = std::min(t[i], ms);
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return h->cuda_fail(e, "tuning");
    int b = 0;
    for (int i = 1; i < n; ++i)
        if (t[i] < t[b]) b = i;
    if (dflt >= 0 && dflt < n && t[dflt] <= t[b] * (1.0 + keep)) b = dflt;
    *best = b;
    if (best_ms) *best_ms = t[b];
    return CGH_OK;
}

void cgh_ctx::load_tune_cache() {
    const char *path = cache_path();
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (fgets(line, sizeof(line), f)) {
        char dev[256] = {0}, bucket[128] = {0};
        int tx, ty, vx, vy, pt, np, g, pk;
        // {"device": "...", "bucket": "...", "tile": [tx, ty, vx, vy, pt, np, g, pk]}
        const char *d = strstr(line, "\"device\": \"");
        const char *b = strstr(line, "\"bucket\": \"");
        const char *t = strstr(line, "\"tile\": [");
        const char *gm = strstr(line, "\"gemm\": [");
        if (!d || !b || (!t && !gm)) continue;
        if (sscanf(d + 11, "%255[^\"]", dev) != 1) continue;
        if (sscanf(b + 11, "%127[^\"]", bucket) != 1) continue;
        if (gm) {
            // {"device": "...", "bucket": "...", "gemm": [tiling, width]}
            int tiling, width;
            if (sscanf(gm + 9, "%d , %d", &tiling, &width) != 2) continue;
            if (strcmp(dev, device_name) != 0) continue;
            if (tiling >= CGH_GEMM_SINGLE && tiling <= CGH_GEMM_PAIRS_GEN && width > 0 &&
                width < 1000)
                tuned_gemm[bucket] = tiling * 1000 + width;
            continue;
        }
        if (sscanf(t + 9, "%d , %d , %d , %d , %d , %d , %d , %d", &tx, &ty, &vx,
                   &vy, &pt, &np, &g, &pk) != 8)
            continue;
        if (strcmp(dev, device_name) != 0) continue;
        int i = direct_tile_index(DirectTile{tx, ty, vx, vy, pt, np, g, pk});
        if (i >= 0) tuned[bucket] = i;
    }
    fclose(f);
}

// The separable methods: time every GEMM plan compiled in -- one-CTA tiles,
// CTA pairs, CTA pairs generating their operand tiles -- at each width, on
// the whole forward (prologue, tables if any, GEMM), and keep the fastest
// for the size bucket.
static cgh_status tune_separable(cgh_ctx *h, int N, int Nx, int Ny, int method,
                                 cudaStream_t s, const float *pts, const float *A,
                                 const float *z, float *out) {
    const int kind = method == CGH_SEP_BF16 ? 0 : method == CGH_SEP_FP16 ? 1 : 2;
    static const int widths[] = {112, 128, 144, 160, 224, 256};
    std::vector<int> plans;
    for (int tiling = CGH_GEMM_SINGLE; tiling <= CGH_GEMM_PAIRS_GEN; ++tiling)
        for (int w : widths) {
            const bool ok = tiling == CGH_GEMM_SINGLE ? (w == 112 || w == 128)
                            : tiling == CGH_GEMM_PAIRS ? pair_width_ok(w)
                                                       : gen_pair_width_ok(kind, w);
            if (ok) plans.push_back(tiling * 1000 + w);
        }
    // the heuristic's plan is the default
    const GemmPlan hp = gemm_plan(Ny, Nx, CGH_GEMM_AUTO, h->sm_count, kind);
    int dflt = -1;
    for (size_t i = 0; i < plans.size(); ++i)
        if (plans[i] == hp.tiling * 1000 + hp.bn) dflt = (int)i;
    int bi = -1;
    float best_ms = 0.0f;
    cgh_status st = tune_pick(h, (int)plans.size(), dflt, TUNE_KEEP, s,
                              [&](int i) {
                                  h->forced_plan = plans[i];
                                  return h->forward_separable(pts, A, z, N, 532e-9, 8e-6,
                                                              Nx, Ny, out, method, s);
                              },
                              &bi, &best_ms);
    h->forced_plan = -1;
    const int best = (st == CGH_OK && bi >= 0) ? plans[bi] : -1;
    if (st == CGH_OK && best >= 0) {
        const std::string b = size_bucket(method, N, Nx, Ny);
        h->tuned_gemm[b] = best;
        if (const char *path = cache_path()) {
            if (FILE *f = fopen(path, "a")) {
                fprintf(f,
                        "{\"device\": \"%s\", \"bucket\": \"%s\", \"gemm\": [%d, %d], "
                        "\"ms\": %.5f}\n",
                        h->device_name, b.c_str(), best / 1000, best % 1000, best_ms);
                fclose(f);
            }
        }
    }
    return st;
}

extern "C" cgh_status cgh_tune(cgh_handle h, int N, int Nx, int Ny, int method,
                               void *stream, cgh_direct_tile *chosen) {
    NvtxRange range("cgh_tune");
    if (!h) return CGH_ERR_INVALID_ARG;
    const bool sep = method == CGH_SEP_BF16 || method == CGH_SEP_FP16 ||
                     method == CGH_SEP_FP16X3;
    if (method != CGH_DIRECT_FP32 && !sep)
        return h->fail(CGH_ERR_UNSUPPORTED,
                       "only the direct and the tensor-core methods have tunable tiles");
    if (N < 1 || N > CGH_MAX_POINTS || Nx < 1 || Ny < 1 || Nx > CGH_MAX_SIDE ||
        Ny > CGH_MAX_SIDE)
        return h->fail(CGH_ERR_INVALID_ARG, "bad tuning size");
    int prev_dev = 0;
    cudaGetDevice(&prev_dev);
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t in_b = align256((size_t)N * 4 * sizeof(float));
    const size_t out_b = align256((size_t)Nx * Ny * sizeof(float));
    cgh_status st = h->ensure(h->ws2, in_b + out_b, s, "tuning buffers");
    if (st) {
        cudaSetDevice(prev_dev);
        return st;
    }
    float *pts = (float *)h->ws2.ptr;
    float *A = pts + 2 * (size_t)N, *z = pts + 3 * (size_t)N;
    float *out = (float *)((char *)h->ws2.ptr + in_b);
    {
        TimedLaunch tl(h, CGH_K_AUX, s);
        tune_fill_kernel<<<(N + 127) / 128, 128, 0, s>>>(pts, A, z, N, Nx, Ny);
        tl.done();
    }
    if (sep) {
        st = tune_separable(h, N, Nx, Ny, method, s, pts, A, z, out);
        if (chosen) memset(chosen, 0, sizeof(*chosen));
        cudaSetDevice(prev_dev);
        return st;
    }
    float best_ms = 0.0f;
    int best_i = -1;
    st = tune_pick(h, direct_tile_count(), default_direct_tile(N, Nx, Ny, h->sm_count),
                   TUNE_KEEP, s,
                   [&](int i) {
                       return h->forward_direct(pts, A, z, N, 532e-9, 8e-6, Nx, Ny, out,
                                                i, s);
                   },
                   &best_i, &best_ms);
    if (st == CGH_OK && best_i >= 0) {
        std::string b = size_bucket(CGH_DIRECT_FP32, N, Nx, Ny);
        h->tuned[b] = best_i;
        DirectTile t = direct_tile_get(best_i);
        if (chosen) {
            chosen->tile_x = t.tx;
            chosen->tile_y = t.ty;
            chosen->vec_x = t.vx;
            chosen->vec_y = t.vy;
            chosen->points_per_stage = t.pt;
            chosen->poly_pixels = t.np;
            chosen->point_groups = t.g;
            chosen->packed = t.pk;
        }
        if (const char *path = cache_path()) {
            if (FILE *f = fopen(path, "a")) {
                fprintf(f,
                        "{\"device\": \"%s\", \"bucket\": \"%s\", \"tile\": "
                        "[%d, %d, %d, %d, %d, %d, %d, %d], \"ms\": %.5f}\n",
                        h->device_name, b.c_str(), t.tx, t.ty, t.vx, t.vy, t.pt,
                        t.np, t.g, t.pk, best_ms);
                fclose(f);
            }
        }
    }
    cudaSetDevice(prev_dev);
    return st;
}
