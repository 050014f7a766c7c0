// api.cu -- the C ABI of libcgh (include/cgh.h): handles, argument checks,
// workspace, dispatch to the kernels.  The paper's host steps (Section 2:
// initialise, allocate, send input, run the kernel, read back, release)
// map onto cgh_create / cgh_forward(_host) / cgh_destroy.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <unordered_map>

#include "api_internal.h"
#include "common.cuh"

using namespace cgh;

namespace {

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace

// --------------------------------------------------------------- errors
cgh_status cgh_ctx::fail(cgh_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, sizeof(err), fmt, ap);
    va_end(ap);
    return st;
}

cgh_status cgh_ctx::cuda_fail(cudaError_t e, const char *where) {
    cudaGetLastError();  // clear a sticky non-fatal error
    return fail(e == cudaErrorMemoryAllocation ? CGH_ERR_NOMEM : CGH_ERR_CUDA,
                "%s: %s", where, cudaGetErrorString(e));
}

// ------------------------------------------------------------ workspace
cgh_status cgh_ctx::ensure(Buffer &b, size_t bytes, cudaStream_t s,
                           const char *what) {
    if (bytes <= b.bytes) return CGH_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
        cs != cudaStreamCaptureStatusNone)
        return fail(CGH_ERR_UNSUPPORTED,
                    "%s workspace must grow to %zu bytes during stream capture;"
                    " run one uncaptured call of this shape first",
                    what, bytes);
    if (b.ptr) {
        cudaError_t e = cudaFree(b.ptr);  // implicit device synchronisation
        b.ptr = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    }
    size_t want = bytes + bytes / 8;  // some headroom for nearby shapes
    want = (want + 4095) & ~(size_t)4095;
    if (fail_alloc_after == 0)
        return fail(CGH_ERR_NOMEM, "%s: injected allocation failure (CGH_FAIL_ALLOC_AFTER)",
                    what);
    if (fail_alloc_after > 0) --fail_alloc_after;
    cudaError_t e = cudaMalloc(&b.ptr, want);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        return cuda_fail(e, what);
    }
    b.bytes = want;
    return CGH_OK;
}

// ---------------------------------------------------------- validation
static bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

cgh_status cgh_ctx::check_problem(const float *points, const float *A,
                                  const float *z, int N, double lambda,
                                  double p, int Nx, int Ny, const void *out) {
    if (N < 0 || N > CGH_MAX_POINTS)
        return fail(CGH_ERR_INVALID_ARG, "N=%d outside [0, %d]", N, CGH_MAX_POINTS);
    if (Nx < 1 || Ny < 1 || Nx > CGH_MAX_SIDE || Ny > CGH_MAX_SIDE)
        return fail(CGH_ERR_INVALID_ARG, "Nx=%d, Ny=%d outside [1, %d]", Nx, Ny,
                    CGH_MAX_SIDE);
    if (!finite_pos(lambda) || !finite_pos(p))
        return fail(CGH_ERR_INVALID_ARG, "lambda and p must be finite and > 0");
    if (!out) return fail(CGH_ERR_INVALID_ARG, "output pointer is NULL");
    if (N > 0 && (!points || !A || !z))
        return fail(CGH_ERR_INVALID_ARG, "points, A and z must not be NULL");
    if ((((uintptr_t)points) | ((uintptr_t)A) | ((uintptr_t)z) |
         ((uintptr_t)out)) & 3)
        return fail(CGH_ERR_INVALID_ARG, "float arrays must be 4-byte aligned");
    return CGH_OK;
}

// ------------------------------------------------------------ tiles
int cgh_ctx::pick_direct_tile(int N, int Nx, int Ny) {
    if (forced_tile >= 0) return forced_tile;
    auto it = tuned.find(size_bucket(CGH_DIRECT_FP32, N, Nx, Ny));
    if (it != tuned.end()) return it->second;
    return default_direct_tile(N, Nx, Ny, sm_count);
}

// ------------------------------------------------------- direct forward
cgh_status cgh_ctx::forward_direct(const float *points, const float *A,
                                   const float *z, int N, double lambda,
                                   double p, int Nx, int Ny, float *out,
                                   int tile_index, cudaStream_t s) {
    DirectTile t = direct_tile_get(tile_index);
    const int Npad = pad_to(N, t.pt);
    const size_t rec_b = align256((size_t)Npad * sizeof(PointRec));
    const size_t tab_f = direct_phase_table_floats(t, Npad, Nx, Ny);
    const size_t tab_b = align256(tab_f * sizeof(float));
    const size_t amp_b = align256((size_t)Npad * sizeof(float));
    const int nxt = (Nx + t.tx - 1) / t.tx;
    // schedule: one CTA per tile, with the tail tiles split into point
    // chunks when the tiles do not spread evenly over the SMs
    const DirectSplit d = direct_split_plan(tile_index, sm_count, Npad, Nx, Ny,
                                            direct_schedule != CGH_SCHED_GRID);
    const int nsplit = d.tiles - d.tail;
    const size_t part_b = align256((size_t)d.chunks() * t.tx * t.ty * sizeof(float));
    const size_t cnt_b = align256((size_t)nsplit * sizeof(unsigned));
    cgh_status st = ensure(ws, rec_b + tab_b + amp_b + part_b + cnt_b, s,
                           "direct workspace");
    if (st) return st;
    char *base = (char *)ws.ptr;
    PointRec *rec = (PointRec *)base;
    float *phx = (float *)(base + rec_b);
    float *phy = phx + direct_x_floats(t, nxt, Npad);
    float *amp = (float *)(base + rec_b + tab_b);
    float *part = nsplit ? (float *)(base + rec_b + tab_b + amp_b) : nullptr;
    unsigned *count =
        nsplit ? (unsigned *)(base + rec_b + tab_b + amp_b + part_b) : nullptr;

    if (!direct_fused_tables) {
        TimedLaunch tl(this, CGH_K_PROLOGUE, s);
        cudaError_t e = launch_prologue(points, A, z, N, Npad, lambda, p, rec,
                                        d_status, s, row_origin);
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        tl.done();
    }
    {
        // by default the tables kernel builds the point records itself
        TimedLaunch tl(this, CGH_K_DIRECT_TABLES, s);
        cudaError_t e =
            direct_fused_tables
                ? launch_direct_tables_fused(
                      PointSource{points, A, z, N, fresnel_scale(lambda, p), d_status, row_origin}, Npad, Nx, Ny,
                      t, phx, phy, amp, count, nsplit, s)
                : launch_direct_tables(rec, Npad, Nx, Ny, t, phx, phy, amp, count,
                                       nsplit, s);
        if (e != cudaSuccess) return cuda_fail(e, "direct tables launch");
        tl.done();
    }
    {
        TimedLaunch tl(this, CGH_K_DIRECT, s);
        cudaError_t e = launch_direct_forward(tile_index, phx, phy, amp, Npad, Nx,
                                              Ny, out, d, part, count, d_status, s);
        if (e != cudaSuccess) return cuda_fail(e, "direct kernel launch");
        tl.done();
    }
    return CGH_OK;
}

cgh_status cgh_ctx::forward_naive(const float *points, const float *A,
                                  const float *z, int N, double lambda,
                                  double p, int Nx, int Ny, float *out,
                                  cudaStream_t s) {
    const size_t rec_b = align256((size_t)N * sizeof(PointRec));
    cgh_status st = ensure(ws, rec_b, s, "naive workspace");
    if (st) return st;
    PointRec *rec = (PointRec *)ws.ptr;
    {
        TimedLaunch tl(this, CGH_K_PROLOGUE, s);
        cudaError_t e = launch_prologue(points, A, z, N, N, lambda, p, rec,
                                        d_status, s, row_origin);
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        tl.done();
    }
    {
        TimedLaunch tl(this, CGH_K_NAIVE, s);
        cudaError_t e = launch_naive_forward(rec, N, Nx, Ny, out, s);
        if (e != cudaSuccess) return cuda_fail(e, "naive kernel launch");
        tl.done();
    }
    return CGH_OK;
}

cgh_status cgh_ctx::forward_recur(const float *points, const float *A,
                                  const float *z, int N, double lambda,
                                  double p, int Nx, int Ny, float *out,
                                  cudaStream_t s) {
    const int Npad = pad_to(N, recur_points_per_stage());
    const size_t rec_b = align256((size_t)Npad * sizeof(PointRec));
    cgh_status st = ensure(ws, rec_b, s, "recurrence workspace");
    if (st) return st;
    PointRec *rec = (PointRec *)ws.ptr;
    {
        TimedLaunch tl(this, CGH_K_PROLOGUE, s);
        cudaError_t e = launch_prologue(points, A, z, N, Npad, lambda, p, rec,
                                        d_status, s, row_origin);
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        tl.done();
    }
    {
        TimedLaunch tl(this, CGH_K_RECUR, s);
        cudaError_t e = launch_recur_forward(rec, Npad, Nx, Ny, out, s);
        if (e != cudaSuccess) return cuda_fail(e, "recurrence kernel launch");
        tl.done();
    }
    return CGH_OK;
}

cgh_status cgh_ctx::forward(const float *points, const float *A,
                            const float *z, int N, double lambda, double p,
                            int Nx, int Ny, float *out, int method,
                            cudaStream_t s) {
    cgh_status st = check_problem(points, A, z, N, lambda, p, Nx, Ny, out);
    if (st) return st;
    if (N == 0) {
        cudaError_t e = cudaMemsetAsync(out, 0, (size_t)Nx * Ny * sizeof(float), s);
        return e == cudaSuccess ? CGH_OK : cuda_fail(e, "cudaMemsetAsync");
    }
    switch (method) {
    case CGH_DIRECT_FP32:
        return forward_direct(points, A, z, N, lambda, p, Nx, Ny, out,
                              pick_direct_tile(N, Nx, Ny), s);
    case CGH_NAIVE_FP32:
        return forward_naive(points, A, z, N, lambda, p, Nx, Ny, out, s);
    case CGH_RECUR_FP32:
        return forward_recur(points, A, z, N, lambda, p, Nx, Ny, out, s);
    case CGH_SEP_FP32:
        return forward_simt(points, A, z, N, lambda, p, Nx, Ny, out, s);
    case CGH_SEP_BF16:
    case CGH_SEP_FP16:
    case CGH_SEP_FP16X3:
        return forward_separable(points, A, z, N, lambda, p, Nx, Ny, out,
                                 method, s);
    default:
        return fail(CGH_ERR_INVALID_ARG, "unknown method %d", method);
    }
}

// ------------------------------------------------------------- release
void cgh_ctx::release_all() {
    for (Buffer *b : {&ws, &ws2, &io, &part, &meta, &bws, &hout[0], &hout[1]}) {
        if (b->ptr) cudaFree(b->ptr);
        b->ptr = nullptr;
        b->bytes = 0;
    }
    if (batch_exec) cudaGraphExecDestroy(batch_exec);
    batch_exec = nullptr;
    batch_key = 0;
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    if (stage_done) cudaEventDestroy(stage_done);
    stage_done = nullptr;
    if (host_stage) cudaFreeHost(host_stage);
    host_stage = nullptr;
    host_stage_bytes = 0;
    for (int k = 0; k < 2; ++k) {
        if (hout_ready[k]) cudaEventDestroy(hout_ready[k]);
        if (hout_copied[k]) cudaEventDestroy(hout_copied[k]);
        hout_ready[k] = hout_copied[k] = nullptr;
        hout_pending[k] = false;
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
    for (cudaEvent_t &e : host_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    host_calls = host_done = 0;
}

// --------------------------------------------------------- kernel timing
cudaEvent_t cgh_ctx::get_event() {
    if (!event_pool.empty()) {
        cudaEvent_t e = event_pool.back();
        event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void cgh_ctx::timer_begin(int kernel, cudaStream_t s, cudaEvent_t *ev) {
    (void)kernel;
    *ev = get_event();
    if (*ev) cudaEventRecord(*ev, s);
}

void cgh_ctx::timer_end(int kernel, cudaStream_t s, cudaEvent_t ev) {
    if (!ev) return;
    cudaEvent_t e1 = get_event();
    if (!e1) {
        event_pool.push_back(ev);
        return;
    }
    cudaEventRecord(e1, s);
    pending[kernel].push_back({ev, e1});
}

cgh_status cgh_ctx::timer_collect(int kernel) {
    for (auto &pr : pending[kernel]) {
        cudaError_t e = cudaEventSynchronize(pr.second);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess) return cuda_fail(e, "kernel timing");
        kernel_ms[kernel] += ms;
        kernel_launches[kernel] += 1;
        event_pool.push_back(pr.first);
        event_pool.push_back(pr.second);
    }
    pending[kernel].clear();
    return CGH_OK;
}

void cgh_ctx::timer_reset() {
    for (int k = 0; k < CGH_K_COUNT; ++k) {
        for (auto &pr : pending[k]) {
            cudaEventSynchronize(pr.second);
            event_pool.push_back(pr.first);
            event_pool.push_back(pr.second);
        }
        pending[k].clear();
        kernel_ms[k] = 0.0;
        kernel_launches[k] = 0;
    }
}

// ============================================================ the C ABI
const char *method_range_name(bool host, int method) {
    // one static string per (entry, method): NVTX copies nothing
    static const char *const fwd[] = {"cgh_forward direct", "cgh_forward sep_bf16",
                                      "cgh_forward sep_fp16", "cgh_forward sep_fp16x3",
                                      "cgh_forward naive", "cgh_forward recur",
                                      "cgh_forward sep_fp32"};
    static const char *const hosts[] = {
        "cgh_forward_host direct", "cgh_forward_host sep_bf16",
        "cgh_forward_host sep_fp16", "cgh_forward_host sep_fp16x3",
        "cgh_forward_host naive", "cgh_forward_host recur", "cgh_forward_host sep_fp32"};
    const bool known = method >= 0 && method < (int)(sizeof(fwd) / sizeof(fwd[0]));
    if (host) return known ? hosts[method] : "cgh_forward_host";
    return known ? fwd[method] : "cgh_forward";
}

extern "C" {

cgh_status cgh_create(cgh_handle *out, int device) {
    if (!out) return CGH_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(device);
    cgh_ctx *h = new (std::nothrow) cgh_ctx();
    if (!h) return CGH_ERR_NOMEM;
    h->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }
    h->sm_count = prop.multiProcessorCount;
    snprintf(h->device_name, sizeof(h->device_name), "%s", prop.name);
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    if (cudaMalloc(&h->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(h->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        if (h->d_status) cudaFree(h->d_status);
        delete h;
        return CGH_ERR_CUDA;
    }
    h->load_tune_cache();
    if (const char *f = getenv("CGH_FAIL_ALLOC_AFTER")) h->fail_alloc_after = atoi(f);
    if (const char *f = getenv("CGH_SIMT_STAGE")) h->simt_stage = atoi(f);
    if (const char *f = getenv("CGH_GEMM_TILES")) {
        const int v = atoi(f);
        if (v >= CGH_GEMM_AUTO && v <= CGH_GEMM_PAIRS_GEN) h->gemm_tiles = v;
    }
    if (const char *f = getenv("CGH_BWD_STAGED")) h->bwd_staged = atoi(f) != 0;
    if (const char *f = getenv("CGH_DIRECT_FUSED_TABLES"))
        h->direct_fused_tables = atoi(f) != 0;
    if (const char *f = getenv("CGH_BWD_POLY")) {
        const int v = atoi(f);
        if (v == 0 || v == 4 || v == 6) h->bwd_poly = v;
    }
    *out = h;
    return CGH_OK;
}

cgh_status cgh_destroy(cgh_handle h) {
    if (!h) return CGH_OK;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    h->release_all();
    h->timer_reset();
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    if (h->d_status) cudaFree(h->d_status);
    cudaGetLastError();
    delete h;
    return CGH_OK;
}

cgh_status cgh_forward(cgh_handle h, const float *points, const float *A,
                       const float *z, int N, double lambda, double p, int Nx,
                       int Ny, float *out, int method, void *stream) {
    NvtxRange range(method_range_name(false, method));
    if (!h) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    h->err[0] = 0;
    return h->forward(points, A, z, N, lambda, p, Nx, Ny, out, method,
                      (cudaStream_t)stream);
}

cgh_status cgh_forward_rows(cgh_handle h, const float *points, const float *A,
                            const float *z, int N, double lambda, double p, int Nx,
                            int y0, int rows, float *out, int method, void *stream) {
    NvtxRange range("cgh_forward_rows");
    if (!h) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    h->err[0] = 0;
    if (y0 < 0 || y0 > CGH_MAX_ROW_ORIGIN)
        return h->fail(CGH_ERR_INVALID_ARG, "row origin %d outside [0, %d]", y0,
                       CGH_MAX_ROW_ORIGIN);
    h->row_origin = y0;
    const cgh_status st = h->forward(points, A, z, N, lambda, p, Nx, rows, out, method,
                                     (cudaStream_t)stream);
    h->row_origin = 0;
    return st;
}

// The device address of page-locked host memory mapped into the device's
// address space (pinned memory on this platform), else nullptr (pageable
// memory, or an error, which is cleared).
static void *mapped_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

cgh_status cgh_forward_host(cgh_handle h, const float *points_host,
                            const float *A_host, const float *z_host, int N,
                            double lambda, double p, int Nx, int Ny,
                            float *out_host, int method, void *stream) {
    NvtxRange range(method_range_name(true, method));
    if (!h) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    h->err[0] = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cgh_status st = h->check_problem(points_host, A_host, z_host, N, lambda, p,
                                     Nx, Ny, out_host);
    if (st) return st;
    // Mapped (pinned) host inputs are read in place by the per-point
    // prologue.  A mapped output is written in place by the methods whose
    // kernels store the hologram tile by tile while they run (direct,
    // recurrence, naive, FP32 separable): those stores hide under the
    // compute.  The tensor-core GEMM stores the whole hologram in one burst
    // at its end, which crosses the host link faster as one copy (measured
    // at 1920x1024: 207 us in place against 120 us staged).  Other buffers
    // are staged through the handle's workspace.
    const float *m_pts = N > 0 ? (const float *)mapped_device_ptr(points_host) : nullptr;
    const float *m_A = N > 0 ? (const float *)mapped_device_ptr(A_host) : nullptr;
    const float *m_z = N > 0 ? (const float *)mapped_device_ptr(z_host) : nullptr;
    const bool progressive = method == CGH_DIRECT_FP32 || method == CGH_NAIVE_FP32 ||
                             method == CGH_RECUR_FP32 || method == CGH_SEP_FP32;
    float *m_out = progressive ? (float *)mapped_device_ptr(out_host) : nullptr;
    const size_t pts_b = m_pts ? 0 : align256((size_t)N * 2 * sizeof(float));
    const size_t a_b = m_A ? 0 : align256((size_t)N * sizeof(float));
    const size_t z_b = m_z ? 0 : align256((size_t)N * sizeof(float));
    const size_t out_b = m_out ? 0 : align256((size_t)Nx * Ny * sizeof(float));
    st = h->ensure(h->io, pts_b + a_b + z_b + out_b + 256, s, "host-call staging");
    if (st) return st;
    char *base = (char *)h->io.ptr;
    const float *d_pts = m_pts ? m_pts : (const float *)base;
    const float *d_A = m_A ? m_A : (const float *)(base + pts_b);
    const float *d_z = m_z ? m_z : (const float *)(base + pts_b + a_b);
    float *d_out = m_out ? m_out : (float *)(base + pts_b + a_b + z_b);
    cudaError_t e = cudaSuccess;
    if (N > 0) {
        if (!m_pts)
            e = cudaMemcpyAsync((void *)d_pts, points_host, (size_t)N * 2 * sizeof(float),
                                cudaMemcpyDefault, s);
        if (e == cudaSuccess && !m_A)
            e = cudaMemcpyAsync((void *)d_A, A_host, (size_t)N * sizeof(float),
                                cudaMemcpyDefault, s);
        if (e == cudaSuccess && !m_z)
            e = cudaMemcpyAsync((void *)d_z, z_host, (size_t)N * sizeof(float),
                                cudaMemcpyDefault, s);
        if (e != cudaSuccess) return h->cuda_fail(e, "host-to-device copy");
    }
    st = h->forward(d_pts, d_A, d_z, N, lambda, p, Nx, Ny, d_out, method, s);
    if (st) return st;
    if (!m_out) {
        e = cudaMemcpyAsync(out_host, d_out, (size_t)Nx * Ny * sizeof(float),
                            cudaMemcpyDefault, s);
        if (e != cudaSuccess) return h->cuda_fail(e, "device-to-host copy");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaStreamSynchronize");
    return CGH_OK;
}

cgh_status cgh_forward_host_async(cgh_handle h, const float *points_host,
                                  const float *A_host, const float *z_host,
                                  int N, double lambda, double p, int Nx,
                                  int Ny, float *out_host, int method,
                                  void *stream) {
    NvtxRange range("cgh_forward_host_async");
    if (!h) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    h->err[0] = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cgh_status st = h->check_problem(points_host, A_host, z_host, N, lambda, p,
                                     Nx, Ny, out_host);
    if (st) return st;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return h->fail(CGH_ERR_UNSUPPORTED,
                       "cgh_forward_host_async cannot run inside stream capture");
    const float *m_pts = N > 0 ? (const float *)mapped_device_ptr(points_host) : nullptr;
    const float *m_A = N > 0 ? (const float *)mapped_device_ptr(A_host) : nullptr;
    const float *m_z = N > 0 ? (const float *)mapped_device_ptr(z_host) : nullptr;
    float *m_out = (float *)mapped_device_ptr(out_host);
    if ((N > 0 && (!m_pts || !m_A || !m_z)) || !m_out)
        return h->fail(CGH_ERR_INVALID_ARG,
                       "cgh_forward_host_async needs page-locked, mapped host buffers");
    const bool progressive = method == CGH_DIRECT_FP32 || method == CGH_NAIVE_FP32 ||
                             method == CGH_RECUR_FP32 || method == CGH_SEP_FP32;
    // this call's ticket: its event slot must be free (the call that many
    // tickets back has finished)
    const uint64_t ticket = h->host_calls + 1;
    cudaEvent_t &tev = h->host_ev[ticket % CGH_HOST_TICKETS];
    if (ticket > CGH_HOST_TICKETS && h->host_done < ticket - CGH_HOST_TICKETS) {
        st = cgh_host_wait_ticket(h, ticket - CGH_HOST_TICKETS);
        if (st) return st;
    }
    cudaError_t e = cudaSuccess;
    if (!tev) e = cudaEventCreateWithFlags(&tev, cudaEventDisableTiming);
    if (e != cudaSuccess) return h->cuda_fail(e, "ticket event");
    if (progressive) {
        st = h->forward(m_pts, m_A, m_z, N, lambda, p, Nx, Ny, m_out, method, s);
        if (st) return st;
        e = cudaEventRecord(tev, s);
        if (e != cudaSuccess) return h->cuda_fail(e, "ticket event");
        h->host_calls = ticket;
        return CGH_OK;
    }

    if (!h->copy_stream) {
        e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&h->hout_ready[k], cudaEventDisableTiming);
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&h->hout_copied[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return h->cuda_fail(e, "copy stream");
    }
    const int k = h->hout_next;
    // the copy out of this buffer two calls ago must be done before the new
    // output overwrites it (a device-side wait on the caller's stream)
    if (h->hout_pending[k]) e = cudaStreamWaitEvent(s, h->hout_copied[k], 0);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaStreamWaitEvent");
    const size_t out_b = (size_t)Nx * Ny * sizeof(float);
    // (growing the buffer frees the old one: cudaFree waits for the device)
    st = h->ensure(h->hout[k], out_b, s, "asynchronous host-call output");
    if (st) return st;
    float *d_out = (float *)h->hout[k].ptr;
    st = h->forward(m_pts, m_A, m_z, N, lambda, p, Nx, Ny, d_out, method, s);
    if (st) return st;
    e = cudaEventRecord(h->hout_ready[k], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->hout_ready[k], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, d_out, out_b, cudaMemcpyDeviceToHost, h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->hout_copied[k], h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(tev, h->copy_stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "device-to-host copy");
    h->hout_pending[k] = true;
    h->hout_next = k ^ 1;
    h->host_calls = ticket;
    return CGH_OK;
}

uint64_t cgh_host_ticket(cgh_handle h) { return h ? h->host_calls : 0; }

cgh_status cgh_host_wait_ticket(cgh_handle h, uint64_t ticket) {
    if (!h) return CGH_ERR_INVALID_ARG;
    if (ticket > h->host_calls)
        return h->fail(CGH_ERR_INVALID_ARG, "ticket %llu was not issued (last %llu)",
                       (unsigned long long)ticket, (unsigned long long)h->host_calls);
    DeviceGuard g(h->device);
    // calls finish out of order across the two streams: wait for each
    // outstanding call up to the ticket (the ring holds the last
    // CGH_HOST_TICKETS of them, all of which are outstanding or done)
    uint64_t u = h->host_done + 1;
    if (ticket > CGH_HOST_TICKETS && u < ticket - CGH_HOST_TICKETS + 1)
        u = ticket - CGH_HOST_TICKETS + 1;
    for (; u <= ticket; ++u) {
        cudaError_t e = cudaEventSynchronize(h->host_ev[u % CGH_HOST_TICKETS]);
        if (e != cudaSuccess) return h->cuda_fail(e, "cgh_host_wait_ticket");
    }
    if (ticket > h->host_done) h->host_done = ticket;
    return CGH_OK;
}

cgh_status cgh_host_wait(cgh_handle h, void *stream) {
    if (!h) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess && h->copy_stream) e = cudaStreamSynchronize(h->copy_stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "cgh_host_wait");
    h->hout_pending[0] = h->hout_pending[1] = false;
    h->host_done = h->host_calls;
    return CGH_OK;
}

cgh_status cgh_last_device_status(cgh_handle h, void *stream) {
    if (!h) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaStreamSynchronize");
    unsigned v = 0;
    e = cudaMemcpy(&v, h->d_status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) return h->cuda_fail(e, "device status read");
    if (v & DEV_TIMEOUT)
        return h->fail(CGH_ERR_TIMEOUT, "a bounded device wait gave up");
    if (v & DEV_BOUNDS)
        return h->fail(CGH_ERR_CUDA, "a device bounds check failed");
    if (v & DEV_BAD_POINT)
        return h->fail(CGH_ERR_INVALID_ARG,
                       "a point had z <= 0 or a non-finite value; it was skipped");
    return CGH_OK;
}

uint64_t cgh_launch_count(cgh_handle h) { return h ? h->launches : 0; }

cgh_status cgh_kernel_timing(cgh_handle h, int enable) {
    return cgh_kernel_timing_mask(h, enable ? 0xffffffffu : 0u);
}

cgh_status cgh_kernel_timing_mask(cgh_handle h, uint32_t mask) {
    if (!h) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    h->timer_reset();
    h->timing = mask != 0;
    h->timing_mask = mask;
    return CGH_OK;
}

cgh_status cgh_kernel_time(cgh_handle h, int kernel, double *total_ms,
                           uint64_t *launches) {
    if (!h || kernel < 0 || kernel >= CGH_K_COUNT) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cgh_status st = h->timer_collect(kernel);
    if (st) return st;
    if (total_ms) *total_ms = h->kernel_ms[kernel];
    if (launches) *launches = h->kernel_launches[kernel];
    return CGH_OK;
}

const char *cgh_status_string(int status) {
    switch (status) {
    case CGH_OK: return "CGH_OK";
    case CGH_ERR_INVALID_ARG: return "CGH_ERR_INVALID_ARG: invalid argument";
    case CGH_ERR_CUDA: return "CGH_ERR_CUDA: a CUDA call failed";
    case CGH_ERR_NOMEM: return "CGH_ERR_NOMEM: out of device memory";
    case CGH_ERR_UNSUPPORTED: return "CGH_ERR_UNSUPPORTED: not supported";
    case CGH_ERR_TIMEOUT: return "CGH_ERR_TIMEOUT: a device wait timed out";
    default: return "unknown cgh_status";
    }
}

const char *cgh_last_error(cgh_handle h) { return h ? h->err : ""; }

int cgh_direct_tile_count(void) { return direct_tile_count(); }

cgh_status cgh_direct_tile_for(cgh_handle h, int N, int Nx, int Ny,
                               cgh_direct_tile *out) {
    if (!h || !out || N < 1 || N > CGH_MAX_POINTS || Nx < 1 || Ny < 1 ||
        Nx > CGH_MAX_SIDE || Ny > CGH_MAX_SIDE)
        return CGH_ERR_INVALID_ARG;
    return cgh_direct_tile_get(h->pick_direct_tile(N, Nx, Ny), out);
}

cgh_status cgh_direct_tile_get(int i, cgh_direct_tile *out) {
    if (!out || i < 0 || i >= direct_tile_count()) return CGH_ERR_INVALID_ARG;
    DirectTile t = direct_tile_get(i);
    out->tile_x = t.tx;
    out->tile_y = t.ty;
    out->vec_x = t.vx;
    out->vec_y = t.vy;
    out->points_per_stage = t.pt;
    out->poly_pixels = t.np;
    out->point_groups = t.g;
    out->packed = t.pk;
    return CGH_OK;
}

cgh_status cgh_set_direct_tile(cgh_handle h, const cgh_direct_tile *tile) {
    if (!h) return CGH_ERR_INVALID_ARG;
    if (!tile) {
        h->forced_tile = -1;
        return CGH_OK;
    }
    DirectTile t{tile->tile_x, tile->tile_y, tile->vec_x, tile->vec_y,
                 tile->points_per_stage, tile->poly_pixels, tile->point_groups,
                 tile->packed};
    int i = direct_tile_index(t);
    if (i < 0)
        return h->fail(CGH_ERR_UNSUPPORTED,
                       "tile %dx%d/%dx%d/%d/%d/%d/%d not compiled in", t.tx, t.ty,
                       t.vx, t.vy, t.pt, t.np, t.g, t.pk);
    h->forced_tile = i;
    return CGH_OK;
}

cgh_status cgh_set_direct_schedule(cgh_handle h, int schedule) {
    if (!h) return CGH_ERR_INVALID_ARG;
    if (schedule != CGH_SCHED_AUTO && schedule != CGH_SCHED_GRID &&
        schedule != CGH_SCHED_SPLIT)
        return h->fail(CGH_ERR_INVALID_ARG, "unknown direct schedule %d", schedule);
    h->direct_schedule = schedule;
    return CGH_OK;
}

cgh_status cgh_gemm_plan(cgh_handle h, int Nx, int Ny, int *tiling, int *width) {
    if (!h || !tiling || !width || Nx < 1 || Ny < 1) return CGH_ERR_INVALID_ARG;
    const GemmPlan p = gemm_plan(Ny, Nx, h->gemm_tiles, h->sm_count);
    *tiling = p.tiling;
    *width = p.bn;
    return CGH_OK;
}

cgh_status cgh_gemm_plan_for(cgh_handle h, int method, int N, int Nx, int Ny,
                             int *tiling, int *width, int *tuned) {
    if (!h || !tiling || !width || N < 1 || N > CGH_MAX_POINTS || Nx < 1 || Ny < 1 ||
        Nx > CGH_MAX_SIDE || Ny > CGH_MAX_SIDE ||
        (method != CGH_SEP_BF16 && method != CGH_SEP_FP16 && method != CGH_SEP_FP16X3))
        return CGH_ERR_INVALID_ARG;
    const cgh_ctx::GemmPlanChoice p = h->sep_plan(method, N, Nx, Ny);
    *tiling = p.tiling;
    *width = p.bn;
    if (tuned) *tuned = p.tuned ? 1 : 0;
    return CGH_OK;
}

cgh_status cgh_set_gemm_tiles(cgh_handle h, int tiles) {
    if (!h) return CGH_ERR_INVALID_ARG;
    if (tiles < CGH_GEMM_AUTO || tiles > CGH_GEMM_PAIRS_GEN)
        return h->fail(CGH_ERR_INVALID_ARG, "unknown GEMM tiling %d", tiles);
    h->gemm_tiles = tiles;
    h->gemm_bn = 0;
    return CGH_OK;
}

cgh_status cgh_set_gemm_plan(cgh_handle h, int tiling, int width) {
    if (!h) return CGH_ERR_INVALID_ARG;
    if (tiling == CGH_GEMM_AUTO) {
        h->gemm_tiles = CGH_GEMM_AUTO;
        h->gemm_bn = 0;
        return CGH_OK;
    }
    bool ok = false;
    if (tiling == CGH_GEMM_SINGLE) ok = width == 0 || width == 112 || width == 128;
    else if (tiling == CGH_GEMM_PAIRS) ok = width == 0 || pair_width_ok(width);
    else if (tiling == CGH_GEMM_PAIRS_GEN) ok = width == 0 || gen_pair_width_ok(2, width);
    if (!ok)
        return h->fail(CGH_ERR_UNSUPPORTED, "GEMM plan %d / width %d not compiled in",
                       tiling, width);
    h->gemm_tiles = tiling;
    h->gemm_bn = width;
    return CGH_OK;
}

}  // extern "C"

// ------------------------------------------------------ fault injection
// A CTA that waits on an mbarrier nothing ever arrives at.  The wait gives
// up after `limit` cycles, records DEV_TIMEOUT and the kernel returns: the
// bounded-wait path every pipelined kernel of this library uses.
__global__ void stalled_wait_kernel(long long limit, unsigned *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t0 = clock64();
        bool done = false;
        while (!(done = mbar_try_wait(&bar, 0))) {
            if (clock64() - t0 > limit) break;
        }
        if (!done) set_status(status, DEV_TIMEOUT);
    }
}

extern "C" cgh_status cgh_debug_stalled_wait(cgh_handle h, long long limit_cycles,
                                             void *stream) {
    if (!h) return CGH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (limit_cycles < 1000000LL) limit_cycles = 1000000LL;
    if (limit_cycles > 4000000000LL) limit_cycles = 4000000000LL;
    TimedLaunch tl(h, CGH_K_AUX, (cudaStream_t)stream);
    stalled_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(limit_cycles, h->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return h->cuda_fail(e, "stalled-wait launch");
    tl.done();
    return CGH_OK;
}
