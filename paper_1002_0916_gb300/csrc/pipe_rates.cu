// pipe_rates.cu -- microbenchmarks of the two SM pipes that bound the ALU
// kernels of this library (the direct forward and adjoint, the recurrence
// kernel and the FP32 separable product): hardware cosines (MUFU) and packed
// FP32 multiply-adds (fma.rn.f32x2), per SM per SM clock.  The kernel's span
// is taken from the global nanosecond timer (first CTA start to last CTA
// end, so CTAs that do not overlap are not double counted) and converted to
// SM cycles with the rate at which the SMs' own cycle counters advanced
// during the run, so the result does not depend on the clock the GPU runs
// at.  The rooflines of those kernels are derived from these two rates.
#include "api_internal.h"
#include "common.cuh"

namespace cgh {

constexpr int PR_THREADS = 1024;
constexpr int PR_CHAINS = 8;   // independent dependency chains per thread

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 of each CTA records {start ns, end ns, SM cycles elapsed}.
__device__ __forceinline__ void pr_record(long long *rec, long long g0, long long g1,
                                          long long c0, long long c1) {
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = g0;
        rec[3 * blockIdx.x + 1] = g1;
        rec[3 * blockIdx.x + 2] = c1 - c0;
    }
}

// Each thread runs PR_CHAINS independent chains of x <- cos(x) (one MUFU
// operation and one argument scale each).
__global__ void __launch_bounds__(PR_THREADS)
mufu_rate_kernel(float seed, int iters, float *sink, long long *cycles) {
    float a[PR_CHAINS];
#pragma unroll
    for (int i = 0; i < PR_CHAINS; ++i) a[i] = seed + 0.1f * i + 1e-4f * threadIdx.x;
    __syncthreads();
    const long long g0 = global_ns(), t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < PR_CHAINS; ++i) a[i] = __cosf(a[i]);
    }
    __syncthreads();
    const long long t1 = clock64(), g1 = global_ns();
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < PR_CHAINS; ++i) s += a[i];
    if (s == 1234.5f) sink[threadIdx.x] = s;  // keeps the chains alive
    pr_record(cycles, g0, g1, t0, t1);
}

// The same with chains of packed multiply-adds (two FP32 FMAs each).
__global__ void __launch_bounds__(PR_THREADS)
fma_rate_kernel(float seed, int iters, float *sink, long long *cycles) {
    float2 a[PR_CHAINS];
#pragma unroll
    for (int i = 0; i < PR_CHAINS; ++i)
        a[i] = make_float2(seed + 0.1f * i, seed - 1e-4f * threadIdx.x);
    const float2 b = make_float2(0.9999f, 0.9998f), c = make_float2(1e-4f, 2e-4f);
    __syncthreads();
    const long long g0 = global_ns(), t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < PR_CHAINS; ++i) a[i] = __ffma2_rn(a[i], b, c);
    }
    __syncthreads();
    const long long t1 = clock64(), g1 = global_ns();
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < PR_CHAINS; ++i) s += a[i].x + a[i].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;
    pr_record(cycles, g0, g1, t0, t1);
}

}  // namespace cgh

using namespace cgh;

extern "C" cgh_status cgh_debug_pipe_rates(cgh_handle h, double *mufu_per_clk,
                                           double *fma_per_clk, void *stream) {
    if (!h || !mufu_per_clk || !fma_per_clk) return CGH_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cgh_status st = CGH_OK;
    for (int pass = 0; pass < 2 && st == CGH_OK; ++pass) {
        void (*kern)(float, int, float *, long long *) =
            pass == 0 ? mufu_rate_kernel : fma_rate_kernel;
        // as many 1024-thread CTAs as the SMs hold at once
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                                      PR_THREADS, 0);
        if (e != cudaSuccess || per_sm < 1) {
            st = h->cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidConfiguration,
                              "pipe-rate occupancy");
            break;
        }
        const int ctas = per_sm * h->sm_count;
        const size_t rec_b = align256((size_t)ctas * 3 * sizeof(long long));
        const size_t sink_b = align256(PR_THREADS * sizeof(float));
        // the host-call staging buffer holds nothing between calls
        st = h->ensure(h->io, rec_b + sink_b, s, "pipe-rate scratch");
        if (st) break;
        long long *rec = (long long *)h->io.ptr;
        float *sink = (float *)((char *)h->io.ptr + rec_b);
        std::vector<long long> host((size_t)ctas * 3);
        const int iters = 4096;
        for (int rep = 0; rep < 2 && st == CGH_OK; ++rep) {  // the first run warms up
            kern<<<ctas, PR_THREADS, 0, s>>>(0.5f, iters, sink, rec);
            ++h->launches;
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(host.data(), rec, host.size() * sizeof(long long),
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = h->cuda_fail(e, "pipe-rate kernels");
        }
        if (st) break;
        long long first = host[0], last = host[1];
        double cyc = 0.0, ns = 0.0;
        for (int c = 0; c < ctas; ++c) {
            first = host[3 * c] < first ? host[3 * c] : first;
            last = host[3 * c + 1] > last ? host[3 * c + 1] : last;
            ns += (double)(host[3 * c + 1] - host[3 * c]);
            cyc += (double)host[3 * c + 2];
        }
        const double cycles_per_ns = ns > 0 ? cyc / ns : 0.0;
        const double span_cycles = (double)(last - first) * cycles_per_ns;
        // operations per SM: its CTAs x threads x iterations x chains (x 2 FMAs
        // per packed instruction)
        const double ops = (double)per_sm * PR_THREADS * iters * PR_CHAINS * (pass ? 2.0 : 1.0);
        (pass == 0 ? *mufu_per_clk : *fma_per_clk) =
            span_cycles > 0 ? ops / span_cycles : 0.0;
    }
    if (prev != h->device) cudaSetDevice(prev);
    return st;
}
