// api_internal.h -- the handle behind cgh_handle (internal to libcgh).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cgh.h"

#define CGH_MAX_POINTS (1 << 24)
#define CGH_MAX_SIDE 32768
#define CGH_MAX_ROW_ORIGIN (1 << 24)

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Buffer {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct cgh_ctx {
    int device = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    char device_name[256] = {0};
    char err[512] = {0};
    unsigned *d_status = nullptr;  // device status word (DEV_* bits)
    uint64_t launches = 0;         // kernels launched by this handle

    Buffer ws;    // forward workspace: point records and tables
    Buffer ws2;   // second workspace: split planes / backward / batch
    Buffer io;    // staging for cgh_forward_host
    Buffer part;  // partial sums of the adjoint
    Buffer meta;  // small per-call metadata (tensor maps, work lists)
    Buffer bws;   // batch workspace: per-problem records and tables

    // cgh_forward_host_async: two device output buffers used in turn, the
    // copy stream, and per buffer the events after its output was computed
    // (caller's stream) and after its copy to the host (copy stream)
    Buffer hout[2];
    int hout_next = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t hout_ready[2] = {nullptr, nullptr};
    cudaEvent_t hout_copied[2] = {nullptr, nullptr};
    bool hout_pending[2] = {false, false};
    // tickets of the asynchronous host calls: the number of calls issued and
    // of calls known finished, and per call (mod CGH_HOST_TICKETS) the event
    // recorded after its last piece of work
    uint64_t host_calls = 0, host_done = 0;
    cudaEvent_t host_ev[CGH_HOST_TICKETS] = {};

    // batch: pinned staging of the work list, a private capture stream and
    // the instantiated graph of the last batch geometry
    void *host_stage = nullptr;
    size_t host_stage_bytes = 0;
    cudaEvent_t stage_done = nullptr;  // last copy out of host_stage
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t batch_exec = nullptr;
    uint64_t batch_key = 0;

    // kernel timing (cgh_kernel_timing / cgh_kernel_time)
    bool timing = false;
    uint32_t timing_mask = 0;  // kernels (bit per cgh_kernel_id) to bracket
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[CGH_K_COUNT];
    std::vector<cudaEvent_t> event_pool;
    double kernel_ms[CGH_K_COUNT] = {0};
    uint64_t kernel_launches[CGH_K_COUNT] = {0};
    cudaEvent_t get_event();
    void timer_begin(int kernel, cudaStream_t s, cudaEvent_t *ev);
    void timer_end(int kernel, cudaStream_t s, cudaEvent_t ev);
    cgh_status timer_collect(int kernel);
    void timer_reset();

    int forced_tile = -1;                         // direct tile override
    // origin of the pixel rows of the forward call in progress (nonzero only
    // inside cgh_forward_rows): every point record is built for rows
    // row_origin + v
    int row_origin = 0;
    int direct_schedule = CGH_SCHED_AUTO;         // cgh_set_direct_schedule
    int gemm_tiles = CGH_GEMM_AUTO;               // cgh_set_gemm_tiles
    int gemm_bn = 0;                              // cgh_set_gemm_plan width (0: heuristic)
    // polynomial (FMA-pipe) sin/cos columns of the direct adjoint's 16-column
    // strips: 0, 4 (default) or 6; CGH_BWD_POLY at cgh_create
    int bwd_poly = 4;
    // direct adjoint: G staged through shared memory by TMA where its layout
    // allows (1) or read row by row from global memory (0); CGH_BWD_STAGED
    int bwd_staged = 1;
    // direct forward: the tables kernel builds the point records itself (1)
    // or reads them from a prologue launch (0); CGH_DIRECT_FUSED_TABLES
    int direct_fused_tables = 1;
    // stage shape of the FP32 separable product (index into the compiled
    // shapes; 1 = 32 values of k x 2 stages, the fastest measured);
    // CGH_SIMT_STAGE at cgh_create
    int simt_stage = 1;
    // fault injection: workspace allocations left before one is made to
    // fail (-1: never); set from CGH_FAIL_ALLOC_AFTER at cgh_create
    int fail_alloc_after = -1;
    std::unordered_map<std::string, int> tuned;   // size bucket -> tile
    // size bucket (separable methods) or batch bucket -> GEMM plan, encoded
    // as tiling * 1000 + width (cgh_tune, cgh_tune_batch, the cache file)
    std::unordered_map<std::string, int> tuned_gemm;
    int forced_plan = -1;  // encoded GEMM plan while cgh_tune measures it

    cgh_status fail(cgh_status st, const char *fmt, ...);
    cgh_status cuda_fail(cudaError_t e, const char *where);
    cgh_status ensure(Buffer &b, size_t bytes, cudaStream_t s, const char *what);
    cgh_status check_problem(const float *points, const float *A, const float *z,
                             int N, double lambda, double p, int Nx, int Ny,
                             const void *out);
    int pick_direct_tile(int N, int Nx, int Ny);

    cgh_status forward(const float *points, const float *A, const float *z,
                       int N, double lambda, double p, int Nx, int Ny,
                       float *out, int method, cudaStream_t s);
    cgh_status forward_direct(const float *points, const float *A,
                              const float *z, int N, double lambda, double p,
                              int Nx, int Ny, float *out, int tile_index,
                              cudaStream_t s);
    cgh_status forward_naive(const float *points, const float *A,
                             const float *z, int N, double lambda, double p,
                             int Nx, int Ny, float *out, cudaStream_t s);
    cgh_status forward_recur(const float *points, const float *A,
                             const float *z, int N, double lambda, double p,
                             int Nx, int Ny, float *out, cudaStream_t s);
    cgh_status forward_simt(const float *points, const float *A,
                            const float *z, int N, double lambda, double p,
                            int Nx, int Ny, float *out, cudaStream_t s);
    cgh_status forward_separable(const float *points, const float *A,
                                 const float *z, int N, double lambda, double p,
                                 int Nx, int Ny, float *out, int method,
                                 cudaStream_t s);
    // The GEMM plan of a separable forward (CGH_SEP_*) of this size: the
    // plan being tuned, else the forced tiling's, else the tuned one for the
    // size bucket, else the heuristic's.  *tuned (may be null): from the tuner.
    struct GemmPlanChoice {
        int tiling, bn;
        bool tuned;
    };
    GemmPlanChoice sep_plan(int method, int N, int Nx, int Ny);
    // split-FP16 batch plan: CTA-pair items (true) or one-CTA items
    bool batch_sep_pairs(const cgh_problem *probs, int count, bool *tuned);
    int default_batch_tile(const cgh_problem *probs, int count);

    cgh_status batch(const cgh_problem *probs, int count, int method,
                     cudaStream_t s, int forced_tile_index, int forced_pairs = -1);
    cgh_status batch_direct(const cgh_problem *probs, int count, cudaStream_t s,
                            int tile_index);
    cgh_status batch_separable(const cgh_problem *probs, int count,
                               cudaStream_t s, int pairs_override = -1);
    cgh_status ensure_host_stage(size_t bytes);
    cgh_status run_batch_graph(uint64_t key, size_t meta_b, int nkernels,
                               const std::function<void(char *)> &fill_stage,
                               const std::function<cudaError_t(cudaStream_t)> &enqueue,
                               cudaStream_t s, int timer);

    void load_tune_cache();
    void release_all();
};

// autotune.cu
std::string size_bucket(int method, int N, int Nx, int Ny);
// The measuring loop of the tuners: the fastest of n candidates (run(i)
// enqueues one call of candidate i), keeping candidate dflt unless another
// beats it by more than the fraction `keep`.
cgh_status tune_pick(cgh_ctx *h, int n, int dflt, double keep, cudaStream_t s,
                     const std::function<cgh_status(int)> &run, int *best, float *best_ms,
                     int rounds = 3, int calls = 3);
constexpr double TUNE_KEEP = 0.01;
// batch.cu: tuning-cache key of a batch geometry (sizes only)
std::string batch_bucket(const cgh_problem *probs, int count);
int default_direct_tile(int N, int Nx, int Ny, int sm_count);
// autotune.cu: the heuristic's modelled cost of direct tile i for a frame
double direct_tile_cost(int i, int N, int Nx, int Ny, int sm_count);

// An NVTX range named after a public entry point (and, for the forward
// calls, the method), open for the life of the call: visible to ncu --nvtx
// and other NVTX tools, close to free when no tool is attached.
const char *method_range_name(bool host, int method);
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Brackets one kernel launch with events when the handle's timing is on,
// and counts the launch.
struct TimedLaunch {
    cgh_ctx *h;
    int kernel;
    cudaStream_t s;
    cudaEvent_t ev = nullptr;
    bool on;
    TimedLaunch(cgh_ctx *h_, int k, cudaStream_t s_)
        : h(h_), kernel(k), s(s_), on(h_->timing && ((h_->timing_mask >> k) & 1u)) {
        if (on) h->timer_begin(kernel, s, &ev);
    }
    void done() {
        ++h->launches;
        if (on) h->timer_end(kernel, s, ev);
    }
};
