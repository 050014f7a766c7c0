// noalloc.cu -- cgh_forward_noalloc: the direct FP32 hologram without any
// device-memory allocation.
//
// Who needs it: callers that must not allocate device memory while they
// run.  Two examples: a display loop feeding a spatial light modulator at a
// fixed frame rate, where cudaMalloc can take an unbounded time and cudaFree
// stalls the whole device; and a plug-in living inside a host application
// that owns all GPU memory through its own allocator and forbids plug-ins to
// call cudaMalloc.  Such callers cannot create a cgh_handle (its workspace
// and status word are allocated with cudaMalloc), so this entry point takes
// no handle at all.
//
// Where its scratch lives: the per-axis angle tables, the amplitudes, the
// split schedule's partial tiles and arrival counters, and a status word of
// the direct path (whose tables kernel builds the per-point records in
// shared memory) are carved out of one file-scope __device__ array of
// CGH_NOALLOC_SCRATCH_BYTES.  That array exists on every GPU on which this
// library's device code is loaded, for the life of the process (of the
// CUDA context that loaded it).  Its device address is looked up with
// cudaGetSymbolAddress, with the device current, the first time the entry
// point runs in a CUDA context, and remembered together with that context's
// unique id: when the context changes (cudaDeviceReset, or a primary
// context released and created again), the module is loaded again and the
// array may sit elsewhere, so the next call looks the address up again.
// Host code never hands the array's own name to a kernel, because on the
// host that name is only a stand-in, not a device address.
//
// Sharing: every call on a device uses the same array and leaves its
// contents behind.  The kernels overwrite every byte they later read, the
// tables kernel zeroes the split schedule's counters and the status word is
// cleared at the start of each call, so stale contents never leak into a
// result; but two calls whose work overlaps on the GPU (different streams,
// or different host threads) race on the array and may produce wrong
// holograms.  Serialise them.
//
// The kernels are the ones cgh_forward runs for CGH_DIRECT_FP32, with the
// tile shape its built-in heuristic picks for the frame and its default
// schedule (the last, uneven wave of tiles split into point chunks) when
// the scratch of that schedule fits, so results match cgh_forward within
// the direct path's tolerance (bit for bit when cgh_forward runs the same
// shape and schedule).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <mutex>

#include "api_internal.h"
#include "common.cuh"

using namespace cgh;

namespace {

static __device__ __align__(256) unsigned char
    g_noalloc_scratch[CGH_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchSlot {
    unsigned long long ctx_id;  // CUDA context the address belongs to
    void *addr;                 // device address of g_noalloc_scratch there
};
ScratchSlot g_slot[kMaxDevices];

// Unique id of the calling thread's current CUDA context (driver entry
// points reached through the runtime; no library to link).  False if there
// is no current context or it cannot be queried.
bool current_context_id(unsigned long long *id) {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (PFN_cuCtxGetCurrent_v4000)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)p;
        cudaGetLastError();
        looked_up = true;
    }
    if (!get_current || !get_id) return false;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_noalloc_scratch on device `dev`, which must be
// current.  Looked up once per CUDA context: again whenever the current
// context is not the one the remembered address came from.
cudaError_t scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    ScratchSlot &s = g_slot[dev];
    if (s.addr && have_id && s.ctx_id == id) {
        *out = s.addr;
        return cudaSuccess;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    // (the lookup makes the device's primary context current if no context
    // was: take the id after it)
    if (current_context_id(&id)) {
        s.ctx_id = id;
        s.addr = p;
    } else {
        s.addr = nullptr;  // cannot tell contexts apart: look up every call
    }
    *out = p;
    return cudaSuccess;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// Byte layout of one call's scratch: status word, angle tables, amplitudes,
// then (split schedule only) partial tiles and arrival counters.
struct ScratchPlan {
    size_t tab_off, amp_off, part_off, cnt_off, total;
};

ScratchPlan plan_scratch(const DirectTile &t, int Npad, int Nx, int Ny,
                         const DirectSplit &d) {
    ScratchPlan s;
    s.tab_off = 256;
    s.amp_off = s.tab_off +
                align256(direct_phase_table_floats(t, Npad, Nx, Ny) * sizeof(float));
    s.part_off = s.amp_off + align256((size_t)Npad * sizeof(float));
    const int nsplit = d.tiles - d.tail;
    s.cnt_off = s.part_off + align256((size_t)d.chunks() * t.tx * t.ty * sizeof(float));
    s.total = s.cnt_off + align256((size_t)nsplit * sizeof(unsigned));
    return s;
}

// The tile for N > 0 points: the heuristic's, or its cheapest whose scratch
// without the split tail fits the array; -1 if none fits.
int noalloc_tile(int N, int Nx, int Ny, int sms) {
    const auto fits = [&](int i) {
        const DirectTile t = direct_tile_get(i);
        const int Npad = pad_to(N, t.pt);
        const DirectSplit d = direct_split_plan(i, sms, Npad, Nx, Ny, false);
        return plan_scratch(t, Npad, Nx, Ny, d).total <= (size_t)CGH_NOALLOC_SCRATCH_BYTES;
    };
    const int first = default_direct_tile(N, Nx, Ny, sms);
    if (fits(first)) return first;
    int best = -1;
    double best_cost = 0.0;
    for (int i = 0; i < direct_tile_count(); ++i) {
        if (!fits(i)) continue;
        const double c = direct_tile_cost(i, N, Nx, Ny, sms);
        if (best < 0 || c < best_cost - 1e-9) {
            best = i;
            best_cost = c;
        }
    }
    return best;
}

}  // namespace

extern "C" cgh_status cgh_forward_noalloc(const float *points, const float *A,
                                          const float *z, int N, double lambda,
                                          double p, int Nx, int Ny, float *out,
                                          void *stream) {
    NvtxRange range("cgh_forward_noalloc");
    if (N < 0 || N > CGH_MAX_POINTS || Nx < 1 || Ny < 1 || Nx > CGH_MAX_SIDE ||
        Ny > CGH_MAX_SIDE || !finite_pos(lambda) || !finite_pos(p) || !out ||
        (N > 0 && (!points || !A || !z)))
        return CGH_ERR_INVALID_ARG;
    if ((((uintptr_t)points) | ((uintptr_t)A) | ((uintptr_t)z) |
         ((uintptr_t)out)) & 3)
        return CGH_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return CGH_ERR_UNSUPPORTED;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
        cudaSuccess) {
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }

    // the heuristic's tile if its tables fit the array, else the
    // heuristic's best among the tiles whose tables fit; with the split
    // tail, else without it, if that scratch fits too (N = 0 needs none)
    const int tile_index =
        N > 0 ? noalloc_tile(N, Nx, Ny, sms) : default_direct_tile(N, Nx, Ny, sms);
    if (tile_index < 0) return CGH_ERR_UNSUPPORTED;  // no tile's tables fit the array
    const DirectTile t = direct_tile_get(tile_index);
    const int Npad = pad_to(N > 0 ? N : 1, t.pt);
    DirectSplit d = direct_split_plan(tile_index, sms, Npad, Nx, Ny, true);
    ScratchPlan sp = plan_scratch(t, Npad, Nx, Ny, d);
    if (N > 0 && sp.total > (size_t)CGH_NOALLOC_SCRATCH_BYTES) {
        d = direct_split_plan(tile_index, sms, Npad, Nx, Ny, false);
        sp = plan_scratch(t, Npad, Nx, Ny, d);
        if (sp.total > (size_t)CGH_NOALLOC_SCRATCH_BYTES)
            return CGH_ERR_UNSUPPORTED;  // this frame needs more scratch than exists
    }

    void *base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    char *b = (char *)base;
    unsigned *status = (unsigned *)b;
    const int nxt = (Nx + t.tx - 1) / t.tx;
    float *phx = (float *)(b + sp.tab_off);
    float *phy = phx + direct_x_floats(t, nxt, Npad);
    float *amp = (float *)(b + sp.amp_off);
    const int nsplit = d.tiles - d.tail;
    float *part = nsplit ? (float *)(b + sp.part_off) : nullptr;
    unsigned *count = nsplit ? (unsigned *)(b + sp.cnt_off) : nullptr;

    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
    if (e == cudaSuccess && N == 0)
        e = cudaMemsetAsync(out, 0, (size_t)Nx * Ny * sizeof(float), s);
    if (e == cudaSuccess && N > 0) {
        // (the tables kernel also zeroes the split schedule's counters)
        e = launch_direct_tables_fused(PointSource{points, A, z, N, fresnel_scale(lambda, p), status},
                                       Npad, Nx, Ny, t, phx, phy, amp, count, nsplit, s);
        if (e == cudaSuccess)
            e = launch_direct_forward(tile_index, phx, phy, amp, Npad, Nx, Ny, out, d,
                                      part, count, status, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }
    return CGH_OK;
}
