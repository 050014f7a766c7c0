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
// Where its scratch lives: the per-axis angle tables, the amplitudes and a
// status word of the direct path (whose tables kernel builds the per-point
// records in shared memory) are carved out of one file-scope
// __device__ array of CGH_NOALLOC_SCRATCH_BYTES.  That array exists on every
// GPU on which this library's device code is loaded, for the life of the
// process.  Its device address is looked up with cudaGetSymbolAddress the
// first time the entry point runs on a device (with that device current)
// and remembered; host code never hands the array's own name to a kernel,
// because on the host that name is only a stand-in, not a device address.
//
// Sharing: every call on a device uses the same array and leaves its
// contents behind.  The kernels overwrite every byte they later read, and
// the status word is cleared at the start of each call, so stale contents
// never leak into a result; but two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array and may
// produce wrong holograms.  Serialise them.
//
// The kernels are the ones cgh_forward runs for CGH_DIRECT_FP32, with the
// tile shape fixed (the first compiled shape), so results match cgh_forward
// within the direct path's tolerance.
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
void *g_scratch_addr[kMaxDevices];

// Device address of g_noalloc_scratch on device `dev`, which must be
// current.  The lookup runs once per device.
cudaError_t scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

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

    const int tile_index = 0;
    const DirectTile t = direct_tile_get(tile_index);
    const int Npad = pad_to(N, t.pt);
    const size_t status_b = 256;
    const size_t tab_b = align256(direct_phase_table_floats(t, Npad, Nx, Ny) *
                                  sizeof(float));
    const size_t amp_b = align256((size_t)Npad * sizeof(float));
    if (status_b + tab_b + amp_b > (size_t)CGH_NOALLOC_SCRATCH_BYTES)
        return CGH_ERR_UNSUPPORTED;  // this frame needs more scratch than exists

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return CGH_ERR_UNSUPPORTED;
    void *base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    char *b = (char *)base;
    unsigned *status = (unsigned *)b;
    const int nxt = (Nx + t.tx - 1) / t.tx;
    float *phx = (float *)(b + status_b);
    float *phy = phx + (size_t)nxt * Npad * t.tx;
    float *amp = (float *)(b + status_b + tab_b);

    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
    if (e == cudaSuccess && N == 0)
        e = cudaMemsetAsync(out, 0, (size_t)Nx * Ny * sizeof(float), s);
    if (e == cudaSuccess && N > 0) {
        e = launch_direct_tables_fused(PointSource{points, A, z, N, lambda, p, status},
                                       Npad, Nx, Ny, t, phx, phy, amp, nullptr, 0, s);
        if (e == cudaSuccess)
            e = launch_direct_forward(tile_index, phx, phy, amp, Npad, Nx, Ny, out,
                                      direct_split_plan(tile_index, 0, Npad, Nx,
                                                        Ny, false),
                                      nullptr, nullptr, status, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CGH_ERR_CUDA;
    }
    return CGH_OK;
}
