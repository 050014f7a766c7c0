/*
 * cgh.h -- C ABI of libcgh: point-source Fresnel computer-generated
 * holograms on one sm_103a GPU.
 *
 * The computation (Shimobaba et al., Section 1, Eq. 1):
 *
 *     I(x_h, y_h) = sum_{j<N} A_j cos( P_j ((x_h - x_j)^2 + (y_h - y_j)^2) ),
 *     P_j = pi p^2 / (lambda z_j),
 *
 * for every pixel x_h = 0..Nx-1, y_h = 0..Ny-1 (integer pixel indices; the
 * object coordinates x_j, y_j are in units of the pixel pitch p, as the paper
 * normalises them).  lambda (wavelength), p (pixel pitch) and z_j (depth) are
 * in metres.  The hologram is stored row-major: out[y_h * Nx + x_h].
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Pointers marked "device" must be CUDA device (or managed) memory of
 *    the handle's device; "host" pointers are ordinary process memory.
 *    The caller owns every buffer it passes; the library never frees them.
 *  * points: N x 2 floats, interleaved (x_0, y_0, x_1, y_1, ...).
 *    A, z: N floats.  4-byte alignment suffices for all float arrays.
 *  * Calls taking a `stream` (a cudaStream_t passed as void*, NULL = the
 *    legacy default stream) are asynchronous on that stream and never
 *    synchronise it, unless stated.  One handle must not be used from two
 *    streams at once: its workspace is shared between calls.
 *  * Argument errors are detected on the host and returned before any work
 *    is enqueued; outputs are untouched then.  Values that only the device
 *    sees (z_j <= 0, non-finite x_j, y_j, A_j, z_j, or z_j <= p^2/(2 lambda),
 *    i.e. P_j >= 2 pi per pixel^2 -- tens of micrometres at visible
 *    wavelengths and micrometre pitches, far inside the distance where the
 *    Fresnel form holds) make the affected point contribute nothing and
 *    raise a bit in the handle's device status word, which
 *    cgh_last_device_status() reports.
 *  * The library never aborts the process, traps the GPU, or waits without
 *    a bound: every device-side wait gives up after about one second and
 *    records CGH_ERR_TIMEOUT in the device status word.
 *  * Workspace (point records, phase/exponential tables, partial sums) is
 *    owned by the handle, grows on demand with cudaMalloc, and is freed by
 *    cgh_destroy.  Growth is refused (CGH_ERR_UNSUPPORTED) while the stream
 *    is being captured into a CUDA graph: run one uncaptured call of the same
 *    shape first.
 */
#ifndef CGH_H
#define CGH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cgh_ctx *cgh_handle;

typedef enum {
    CGH_OK = 0,
    CGH_ERR_INVALID_ARG = 1,  /* rejected argument (host) or bad point (device) */
    CGH_ERR_CUDA = 2,         /* a CUDA call failed; cgh_last_error() has text   */
    CGH_ERR_NOMEM = 3,        /* workspace allocation failed                     */
    CGH_ERR_UNSUPPORTED = 4,  /* valid request this library cannot serve         */
    CGH_ERR_TIMEOUT = 5       /* a bounded device-side wait gave up              */
} cgh_status;

typedef enum {
    /* Direct sum of Eq. 1 in FP32: exact fixed-point phase per image axis
     * (the separable form of the paper's Eq. 2 recurrence, Section 2.1),
     * point tiles staged in shared memory by bulk copies (the paper's
     * shared-memory staging, Section 2.1), hardware cosine (the paper's
     * "native cos").  max |I - I_ref| <= 1e-4 sum|A_j|. */
    CGH_DIRECT_FP32 = 0,
    /* Separable form I = Re(U diag(A) V^T), U[x,j] = exp(i P_j (x - x_j)^2),
     * V[y,j] = exp(i P_j (y - y_j)^2) (exact because the phase of Eq. 1 is
     * a sum of an x part and a y part), as a tcgen05 tensor-core GEMM with
     * FP32 accumulation.  Operands in BF16 / FP16 (single pass, relative RMS
     * error about 1e-2 / 1e-3) or split hi+lo FP16 (three products,
     * relative RMS error <= 1e-4).  Tensor memory accumulates at most
     * 16,384 values of k (8,192 points; single pass: 131,072) per launch;
     * larger N runs as consecutive launches whose partial products are
     * added in FP32. */
    CGH_SEP_BF16 = 1,
    CGH_SEP_FP16 = 2,
    CGH_SEP_FP16X3 = 3,
    /* One thread per pixel, plain loop over points, 64-bit fixed-point phase
     * and cospif (the unoptimised kernel of the paper's Fig. 2b, restated).
     * Slow; for checking. */
    CGH_NAIVE_FP32 = 4,
    /* The paper's optimised kernel design (Section 2.1) restated: groups of
     * 16 x 16 threads, eight consecutive pixels per thread along x, 256
     * points per shared-memory stage, point loop unrolled by four, the phase
     * advanced from pixel to pixel by the two recurrences of Eq. 2 (here in
     * 32-bit fixed-point turns), hardware cosine.  A comparison point for
     * CGH_DIRECT_FP32 (same accuracy bound). */
    CGH_RECUR_FP32 = 5,
    /* The separable form in FP32 on the FMA pipe: with per-axis tables of
     * A_j (cos, -sin) theta_x and (cos, sin) theta_y (exact fixed-point
     * phase, accurate sincospi), cos(theta_x + theta_y) is two FP32
     * multiply-adds per point-pixel update, no special-function operation;
     * an FP32 matrix product of depth 2N on the SIMT cores.  Same accuracy
     * bound as CGH_DIRECT_FP32. */
    CGH_SEP_FP32 = 6
} cgh_method;

/* Create a handle bound to CUDA device `device` (made current on the calling
 * thread).  *out receives the handle.  Errors: CGH_ERR_INVALID_ARG (out NULL,
 * bad device), CGH_ERR_CUDA.
 * Paper: host steps (1) and (2) of Section 2 (initialise the GPU, allocate
 * device memory).  Here the handle records the device and its SM count and
 * allocates the device status word; the workspace of step (2) is allocated
 * later, on the first call of each shape, and kept. */
cgh_status cgh_create(cgh_handle *out, int device);

/* Free the handle and its workspace.  Synchronises the device first.
 * NULL is accepted and ignored.
 * Paper: host step (6) of Section 2 (release the device memory and the GPU
 * resources). */
cgh_status cgh_destroy(cgh_handle h);

/* Eq. 1 for one hologram.  points, A, z: device, N points (N >= 0; N = 0
 * yields zeros).  out: device, Ny*Nx floats, written completely.  lambda, p:
 * finite and > 0.  1 <= Nx, Ny <= 32768, N <= 2^24.  method: a cgh_method.
 * Errors: CGH_ERR_INVALID_ARG (NULL pointer, bad size or constant, unknown
 * method), CGH_ERR_UNSUPPORTED, CGH_ERR_NOMEM, CGH_ERR_CUDA. */
cgh_status cgh_forward(cgh_handle h, const float *points, const float *A,
                       const float *z, int N, double lambda, double p,
                       int Nx, int Ny, float *out, int method, void *stream);

/* Rows y0 .. y0 + rows - 1 of the hologram of Eq. 1 (any height): the same
 * values cgh_forward computes for those rows of a frame of at least
 * y0 + rows rows, written to `out` (device, rows*Nx floats, row-major, row
 * y0 first).  For a row split of one hologram over several GPUs, one
 * process each: each computes its own slab with no exchange between them
 * (pixel rows of Eq. 1 are independent).  The row origin is folded into the
 * per-point records exactly (fixed-point turns, modulo one turn), so every
 * method computes each pixel as cgh_forward does.  0 <= y0 <= 2^24;
 * 1 <= rows <= 32768; other arguments and errors as cgh_forward. */
cgh_status cgh_forward_rows(cgh_handle h, const float *points, const float *A,
                            const float *z, int N, double lambda, double p, int Nx,
                            int y0, int rows, float *out, int method, void *stream);

/* cgh_forward from HOST buffers (Ny*Nx floats out), synchronising the
 * stream before returning.  Page-locked host buffers that are mapped into
 * the device's address space (cudaHostAlloc / cudaHostRegister memory,
 * e.g. PyTorch pinned tensors, on a unified-addressing system) are used in
 * place: the kernels read such inputs over the host link, and the methods
 * that store the hologram tile by tile as they run (CGH_DIRECT_FP32,
 * CGH_RECUR_FP32, CGH_NAIVE_FP32, CGH_SEP_FP32) write such an output there
 * directly.  The tensor-core methods, and any other buffer (pageable
 * memory, device memory), go through the handle's workspace and one copy.
 * The result is the same either way. */
cgh_status cgh_forward_host(cgh_handle h, const float *points_host,
                            const float *A_host, const float *z_host, int N,
                            double lambda, double p, int Nx, int Ny,
                            float *out_host, int method, void *stream);

/* cgh_forward_host without the synchronisation, for pipelines that compute
 * hologram after hologram into host memory (a display loop feeding a
 * spatial light modulator, a server).  All four host buffers must be
 * page-locked and mapped (as above); otherwise CGH_ERR_INVALID_ARG and
 * nothing is launched.  Inputs are read in place.  The methods that store
 * the hologram tile by tile write out_host in place on `stream`; the
 * tensor-core methods compute into one of two device buffers of the handle
 * (used in turn) and copy it to out_host on a copy stream of the handle, so
 * that the copy runs while the next call's kernels do.  A call waits on the
 * device (not the host) for the copy out of its buffer two tensor-core
 * calls earlier.  The inputs must stay unchanged, and out_host unread, until
 * cgh_host_wait (or cgh_host_wait_ticket for this call) returns.  Not
 * inside stream capture
 * (CGH_ERR_UNSUPPORTED).  Results are bit for bit those of
 * cgh_forward_host.  Other errors as cgh_forward. */
cgh_status cgh_forward_host_async(cgh_handle h, const float *points_host,
                                  const float *A_host, const float *z_host,
                                  int N, double lambda, double p, int Nx,
                                  int Ny, float *out_host, int method,
                                  void *stream);

/* Blocks until `stream` and every copy of earlier cgh_forward_host_async
 * calls of the handle have finished: their host outputs are then complete.
 * CGH_ERR_CUDA if either failed. */
cgh_status cgh_host_wait(cgh_handle h, void *stream);

/* Tickets, for pipelines that keep more than one call in flight: the
 * cgh_forward_host_async calls of a handle are numbered 1, 2, ...;
 * cgh_host_ticket returns the number of the last one (0 before any).
 * cgh_host_wait_ticket blocks until every call up to and including `ticket`
 * has finished, its output copy included (their host outputs are then
 * complete, their inputs free), leaving later calls running.  A ticket that
 * was already waited for returns at once; one beyond the last call is
 * CGH_ERR_INVALID_ARG.  The handle remembers the last CGH_HOST_TICKETS calls;
 * a new call first waits for the call that many before it.  CGH_ERR_CUDA if
 * the work failed. */
#define CGH_HOST_TICKETS 16
uint64_t cgh_host_ticket(cgh_handle h);
cgh_status cgh_host_wait_ticket(cgh_handle h, uint64_t ticket);

/* Adjoint of Eq. 1.  grad_out: device, Ny*Nx floats, dL/dI for some loss L.
 * Writes (device, N entries each; grad_points N x 2 interleaved):
 *   grad_A[j]          = sum_pix G cos(phi)
 *   grad_points[2j]    = 2 P_j A_j sum_pix G sin(phi) (x_h - x_j)
 *   grad_points[2j+1]  = 2 P_j A_j sum_pix G sin(phi) (y_h - y_j)
 *   grad_z[j]          = (P_j A_j / z_j) sum_pix G sin(phi) r^2
 * with phi = P_j r^2, r^2 = (x_h - x_j)^2 + (y_h - y_j)^2 (derivatives of
 * Eq. 1; dP_j/dz_j = -P_j/z_j).  Any of the three outputs may be NULL to
 * skip it.  method: CGH_DIRECT_FP32 (FP32, point-owned sums, deterministic),
 * CGH_SEP_FP32 (the same point-owned FP32 sums with cos(phi) and sin(phi)
 * expanded by angle addition into per-column sums of G cos, G sin of the
 * row angle and per-row sums of G cos, G sin of the column angle;
 * deterministic) or CGH_SEP_FP16X3 (two split-FP16 tensor-core GEMMs, G V and
 * G^T U, with the pixel sums fused into their epilogues).  Other methods:
 * CGH_ERR_INVALID_ARG.  Errors as cgh_forward. */
cgh_status cgh_backward(cgh_handle h, const float *points, const float *A,
                        const float *z, int N, double lambda, double p,
                        int Nx, int Ny, const float *grad_out,
                        float *grad_points, float *grad_A, float *grad_z,
                        int method, void *stream);

/* One problem of a batch; every pointer is device memory (see cgh_forward). */
typedef struct {
    const float *points;
    const float *A;
    const float *z;
    int N;
    double lambda;
    double p;
    int Nx;
    int Ny;
    float *out;
} cgh_problem;

/* Many holograms of uneven size, N and wavelength in one persistent launch
 * (after one prologue launch).  Each problem is one evaluation of Eq. 1
 * (Section 1) with its own points, constants and frame; the paper's
 * Table 1 runs the same 1,920 x 1,024 frame once per point count, and this
 * call runs many such frames (of any size) as one piece of device work.  probs: host array of `count` problems
 * (1 <= count <= 4096).  The work list of (problem, tile) items is built on
 * the host, sorted longest-first, and pulled by the persistent CTAs from an
 * atomic counter.  method: CGH_DIRECT_FP32 or CGH_SEP_FP16X3.
 * The launches are captured once per batch geometry (problem count, sizes,
 * constants and buffer addresses) into a CUDA graph that later calls of the
 * same geometry replay; the graph reads the buffers' current contents.
 * The call may itself be captured into a caller's graph once an uncaptured
 * call of the same geometry has run (else CGH_ERR_UNSUPPORTED); such a
 * captured graph stays valid until the handle runs a batch of another
 * geometry.  Errors as cgh_forward; an argument error names the problem. */
cgh_status cgh_batch(cgh_handle h, const cgh_problem *probs, int count,
                     int method, void *stream);

/* Size in bytes of the fixed device scratch array behind
 * cgh_forward_noalloc (16 MiB, present on every GPU that loads this
 * library, for the life of the process). */
#define CGH_NOALLOC_SCRATCH_BYTES (16u << 20)

/* The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate GPU memory while they run -- for example a display
 * loop driving a spatial light modulator at a fixed frame rate (cudaMalloc
 * can take unbounded time, cudaFree stalls the whole device), or a plug-in
 * inside an application that owns all device memory itself.  They cannot
 * create a cgh_handle, so this call needs none.
 *
 * Computes the same hologram as cgh_forward(..., CGH_DIRECT_FP32, ...) on
 * the calling thread's current device, using the same kernels (the tile
 * shape cgh_forward's built-in heuristic picks for the frame when its
 * tables fit the array, else the heuristic's best among the shapes whose
 * tables fit; the default schedule when that schedule's scratch fits too),
 * but takes all
 * scratch (angle tables, amplitudes, the schedule's partial tiles and
 * counters, status word) from one fixed __device__ array of
 * CGH_NOALLOC_SCRATCH_BYTES.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  points, A, z, out: device memory owned by the
 * caller, layouts as cgh_forward; stream: cudaStream_t or NULL.
 * Asynchronous on `stream`.
 *
 * The first call in a CUDA context looks up the array's device address
 * (cudaGetSymbolAddress, with the device current) and remembers it with the
 * context's id; make that first call before any stream capture.  After
 * cudaDeviceReset, or when the primary context is released and created
 * again, the next call is again a first call: it looks the address up anew.
 * Every call on a device shares the array and leaves its contents behind;
 * each call clears what it needs cleared, but calls whose work overlaps on
 * the GPU (other streams, other threads) race on the array and must be
 * serialised by the caller.  There is no status read-back in this variant:
 * points with z <= 0 or non-finite values are skipped unreported, and if a
 * bounded device-side wait ever gave up (see the conventions above), the
 * tiles of the CTAs concerned would be left unwritten, also unreported.
 *
 * Returns CGH_OK; CGH_ERR_INVALID_ARG for the argument errors cgh_forward
 * rejects; CGH_ERR_UNSUPPORTED when the frame needs more scratch than the
 * array holds (about (Nx + Ny) * N * 4 bytes of angle tables plus 4 bytes
 * per point, with Nx, Ny rounded up to 64 and N to 64) -- nothing is
 * launched then; CGH_ERR_CUDA if a CUDA call fails. */
cgh_status cgh_forward_noalloc(const float *points, const float *A,
                               const float *z, int N, double lambda, double p,
                               int Nx, int Ny, float *out, void *stream);

/* Tile shape of the direct kernel (also used by the persistent batch). */
typedef struct {
    int tile_x;            /* pixels per CTA along x           */
    int tile_y;            /* pixels per CTA along y           */
    int vec_x;             /* pixels per thread along x        */
    int vec_y;             /* pixels per thread along y        */
    int points_per_stage;  /* points per shared-memory stage   */
    int poly_pixels;       /* pixels per thread whose cosine is a
                              polynomial on the FMA pipe instead of
                              the MUFU (special-function) unit     */
    int point_groups;      /* thread groups splitting each stage's
                              points (partial sums added in order) */
    int packed;            /* 0: scalar FP32; 1: packed FP32x2
                              arithmetic on pixel pairs along x,
                              degree-6 polynomial; 2: packed,
                              degree-5 polynomial; 3: as 2 with the
                              polynomial pixel pairs spread over the
                              thread's block; 4, 5: as 3 with
                              poly_pixels + 2 polynomial pixels for
                              every second (4) or fourth (5) point;
                              6-8: the rotation forms (Eq. 1's phase
                              split into its x and y parts, cos of a
                              sum): per point, one hardware sincos
                              per thread row (6) or per thread (7
                              scalar, 8 packed), every other pixel of
                              the thread's block by angle addition
                              with the tabulated cosine and sine of
                              its exact phase offset (poly_pixels 0) */
} cgh_direct_tile;

/* How the direct kernel spreads its pixel tiles over the SMs (a scheduling
 * choice of this implementation; the paper launches one work group per
 * 16 x 16 pixel block, Section 2.1).
 *   CGH_SCHED_GRID:  one CTA per pixel tile.  When the tile count is not a
 *                    multiple of the SM count the last wave leaves SMs idle.
 *   CGH_SCHED_SPLIT: one CTA per pixel tile, except for the last
 *                    (tiles mod SMs) tiles: their points are cut into chunks
 *                    of point stages, one CTA per chunk, run at the end of
 *                    the grid; each such tile is the sum of its chunks'
 *                    partial tiles added in chunk order (deterministic; the
 *                    rounding differs from GRID's by the summation order
 *                    only).
 *   CGH_SCHED_AUTO:  SPLIT (the default).
 * The batch entry point (cgh_batch) has its own persistent schedule. */
typedef enum {
    CGH_SCHED_AUTO = 0,
    CGH_SCHED_GRID = 1,
    CGH_SCHED_SPLIT = 2
} cgh_direct_schedule;

/* Select the direct kernel's schedule for later calls on this handle.
 * CGH_ERR_INVALID_ARG for a null handle or an unknown value. */
cgh_status cgh_set_direct_schedule(cgh_handle h, int schedule);

/* How the tensor-core GEMM of the separable forward methods (CGH_SEP_BF16,
 * CGH_SEP_FP16, CGH_SEP_FP16X3) tiles its output (a scheduling choice of
 * this implementation; the paper has no tensor-core form):
 *   CGH_GEMM_SINGLE: one CTA per 128 x BN tile (BN = 112 or 128);
 *   CGH_GEMM_PAIRS:  two CTAs of a cluster per 256 x BN tile, the MMAs
 *                    issued for both SMs at once (tcgen05 cta_group::2), so
 *                    that each SM loads half as many operand bytes per
 *                    multiply-add;
 *   CGH_GEMM_PAIRS_GEN: CTA pairs whose producer warps compute each K
 *                    block's U and V tiles (the separable form's operand
 *                    tables, Eq. 1 split into its x and y phases) straight
 *                    into shared memory from the point records, instead of
 *                    a table kernel writing them to global memory and the
 *                    GEMM reading them back; same entry values bit for bit,
 *                    so the same hologram (single hologram forward only;
 *                    the adjoint and cgh_batch take CGH_GEMM_PAIRS then);
 *   CGH_GEMM_AUTO:   the handle's tuned plan for the size (cgh_tune), else
 *                    CTA pairs for single holograms and adjoints of more
 *                    than 128 rows, one-CTA tiles otherwise and for
 *                    cgh_batch (whose persistent work list balances better
 *                    with the smaller items).
 * Every mode computes the same products with FP32 accumulation; results
 * agree to rounding. */
typedef enum {
    CGH_GEMM_AUTO = 0,
    CGH_GEMM_SINGLE = 1,
    CGH_GEMM_PAIRS = 2,
    CGH_GEMM_PAIRS_GEN = 3
} cgh_gemm_tiles;

/* Select the GEMM tiling for later calls on this handle (also used by
 * cgh_debug_gemm).  CGH_ERR_INVALID_ARG for a null handle or an unknown
 * value. */
cgh_status cgh_set_gemm_tiles(cgh_handle h, int tiles);

/* Force a GEMM tiling and tile width for the separable forward methods of
 * this handle (CGH_GEMM_AUTO: back to the tuned plan or the heuristic).
 * Widths: 112 or 128 for CGH_GEMM_SINGLE; 112, 144, 160, 224 or 256 for
 * CGH_GEMM_PAIRS and CGH_GEMM_PAIRS_GEN (the single-pass generating kernel
 * has 112 and 256 only: other widths fall back to its heuristic there);
 * width 0: the heuristic's width for the tiling.
 * CGH_ERR_UNSUPPORTED for a plan not compiled in, CGH_ERR_INVALID_ARG for a
 * null handle. */
cgh_status cgh_set_gemm_plan(cgh_handle h, int tiling, int width);

/* The tiling a separable forward GEMM of an Ny-row, Nx-column hologram
 * takes on this handle under its current setting: *tiling receives
 * CGH_GEMM_SINGLE or CGH_GEMM_PAIRS and *width the tile width (hologram
 * columns per tile).  CGH_ERR_INVALID_ARG for a null pointer or a size
 * below 1. */
cgh_status cgh_gemm_plan(cgh_handle h, int Nx, int Ny, int *tiling, int *width);

/* The GEMM plan a separable forward of `method` (CGH_SEP_BF16, CGH_SEP_FP16,
 * CGH_SEP_FP16X3) with N points on an Nx x Ny frame takes on this handle:
 * the forced tiling's, else the plan cgh_tune measured fastest for the size
 * bucket, else the heuristic's.  *tiling receives CGH_GEMM_SINGLE,
 * CGH_GEMM_PAIRS or CGH_GEMM_PAIRS_GEN, *width the tile width, *tuned (may
 * be NULL) 1 if the plan came from the tuner.  CGH_ERR_INVALID_ARG for a
 * null pointer, bad sizes or another method. */
cgh_status cgh_gemm_plan_for(cgh_handle h, int method, int N, int Nx, int Ny,
                             int *tiling, int *width, int *tuned);

/* Number of direct-kernel tile shapes compiled into this library, and the
 * i-th of them (0 <= i < count). */
int cgh_direct_tile_count(void);
cgh_status cgh_direct_tile_get(int i, cgh_direct_tile *out);

/* The tile shape this handle's CGH_DIRECT_FP32 calls use for N points on
 * an Nx x Ny frame (the forced shape, else the tuned one for that size
 * bucket, else the built-in heuristic's).  Errors: CGH_ERR_INVALID_ARG for
 * a null pointer or sizes cgh_forward would reject (N = 0 included). */
cgh_status cgh_direct_tile_for(cgh_handle h, int N, int Nx, int Ny,
                               cgh_direct_tile *out);

/* Force a tile shape for CGH_DIRECT_FP32 (NULL: back to automatic choice).
 * Errors: CGH_ERR_UNSUPPORTED if the shape is not compiled in. */
cgh_status cgh_set_direct_tile(cgh_handle h, const cgh_direct_tile *tile);

/* Autotuner (the paper fixed its shapes -- 16 x 16 items per group, 256
 * points per stage -- Section 2.1; here they are measured per size).
 * method CGH_DIRECT_FP32: time every compiled direct tile shape (CUDA events
 * on `stream`, synchronising it) for a problem of this size, remember the
 * fastest for the size bucket, and write it to *chosen (may be NULL).
 * method CGH_SEP_BF16 / CGH_SEP_FP16 / CGH_SEP_FP16X3: time the whole
 * separable forward under every GEMM plan compiled in (one-CTA tiles 112
 * and 128 wide, CTA pairs 112-256 wide, CTA pairs generating their operand
 * tiles) and remember the fastest for the size bucket; later calls of that
 * method and size on this handle use it while the GEMM tiling is
 * CGH_GEMM_AUTO (read it back with cgh_gemm_plan_for); *chosen, if not NULL,
 * is zeroed.  Every candidate is timed in three rounds over all of them
 * (a warm-up call and three timed calls each, its fastest call counting);
 * the built-in heuristic's choice is kept unless another candidate is more
 * than 1% faster.  Choices are kept in the handle and, if the environment
 * variable CGH_TUNE_CACHE names a file, appended there as one JSON object
 * per line (device name, size bucket, tile or GEMM plan) and read back by
 * later handles.  Other methods: CGH_ERR_UNSUPPORTED. */
cgh_status cgh_tune(cgh_handle h, int N, int Nx, int Ny, int method,
                    void *stream, cgh_direct_tile *chosen);

/* Kernels whose launches the handle can time (cgh_kernel_time). */
typedef enum {
    CGH_K_PROLOGUE = 0,       /* per-point records                      */
    CGH_K_DIRECT_TABLES = 1,  /* per-axis angle tables (direct path)    */
    CGH_K_DIRECT = 2,         /* direct point loop                      */
    CGH_K_NAIVE = 3,          /* naive one-thread-per-pixel loop        */
    CGH_K_SEP_TABLES = 4,     /* U / V exponential tables               */
    CGH_K_GEMM = 5,           /* tcgen05 GEMM (forward)                 */
    CGH_K_BWD_DIRECT = 6,     /* direct adjoint point-owned sums        */
    CGH_K_BWD_GEMM = 7,       /* separable adjoint GEMMs + fused sums   */
    CGH_K_BWD_REDUCE = 8,     /* adjoint partial-sum reduction          */
    CGH_K_BATCH = 9,          /* direct batch (its whole graph)         */
    CGH_K_AUX = 10,           /* small helpers (conversions, fills)     */
    CGH_K_BATCH_SEP = 11,     /* separable batch (its whole graph)      */
    CGH_K_RECUR = 12,         /* Eq. 2 recurrence kernel                */
    CGH_K_SIMT = 13,          /* FP32 separable product (FMA pipe)      */
    CGH_K_BWD_SIMT = 14,      /* FP32 separable adjoint (FMA pipe)      */
    CGH_K_COUNT = 16
} cgh_kernel_id;

/* enable != 0: from now on bracket every kernel launch of this handle with
 * CUDA events recorded on the launch's own stream; enable == 0: stop.  Both
 * reset the accumulated times. */
cgh_status cgh_kernel_timing(cgh_handle h, int enable);

/* As cgh_kernel_timing, but only the kernels whose bit (1 << cgh_kernel_id)
 * is set in `mask` are bracketed (0: stop).  Events between two kernels
 * order them fully, so leaving a kernel unbracketed keeps its launch
 * overlapped with the kernel before it. */
cgh_status cgh_kernel_timing_mask(cgh_handle h, uint32_t mask);

/* Total device time (ms, from the events) and number of launches of kernel
 * `kernel` (a cgh_kernel_id) since timing was enabled.  Synchronises on the
 * recorded events. */
cgh_status cgh_kernel_time(cgh_handle h, int kernel, double *total_ms,
                           uint64_t *launches);

/* Autotuner for cgh_batch.  CGH_DIRECT_FP32: time every compiled tile
 * shape on this batch (its geometry and data; synchronises `stream`), keep
 * the fastest for batches of the same sizes, write it to *chosen (may be
 * NULL).  CGH_SEP_FP16X3: time the persistent grouped GEMM's two item
 * shapes (one-CTA 128 x 128 items and CTA-pair 256 x 128 items) and keep
 * the faster for batches of the same sizes (*chosen, if not NULL, is
 * zeroed).  The built-in choice (the heuristic's tile; one-CTA items) is
 * kept unless another is more than 1% faster.  Later cgh_batch calls of
 * that method and these sizes use the choice (with the GEMM tiling
 * CGH_GEMM_AUTO for the separable batch);
 * cgh_batch_plan reports it.  Errors as cgh_batch. */
cgh_status cgh_tune_batch(cgh_handle h, const cgh_problem *probs, int count,
                          int method, void *stream, cgh_direct_tile *chosen);

/* What cgh_batch would run for this batch: CGH_DIRECT_FP32 writes the
 * direct tile shape to *tile (forced, tuned or the heuristic's) and 0 to
 * *gemm_tiling; CGH_SEP_FP16X3 writes CGH_GEMM_SINGLE (one-CTA items) or
 * CGH_GEMM_PAIRS (CTA-pair items) to *gemm_tiling and zeroes *tile.  *tuned
 * = 1 when the choice came from cgh_tune_batch (or its cache file), else 0.
 * Any output pointer may be NULL.  CGH_ERR_INVALID_ARG for a null handle or
 * problem array, a count outside [1, 4096] or another method. */
cgh_status cgh_batch_plan(cgh_handle h, const cgh_problem *probs, int count,
                          int method, cgh_direct_tile *tile, int *gemm_tiling,
                          int *tuned);

/* Synchronise `stream`, then read and clear the handle's device status
 * word: CGH_OK, CGH_ERR_INVALID_ARG (a point had z <= 0 or a non-finite
 * value), CGH_ERR_TIMEOUT (a bounded wait gave up), CGH_ERR_CUDA.
 * Paper: host step (5) of Section 2 (receive the result from the device)
 * says nothing of errors; this call is the read-back of what only the
 * device sees.  Eq. 1 needs z_j > 0 (P_j = pi p^2 / (lambda z_j)), so a
 * point that breaks it is skipped and reported here. */
cgh_status cgh_last_device_status(cgh_handle h, void *stream);

/* Number of kernels this handle has launched since creation. */
uint64_t cgh_launch_count(cgh_handle h);

/* Static text for a status code (never NULL).  The paper's host steps
 * (Section 2, steps (1)-(6)) define no error codes; these are the outcomes
 * of this library's argument checks and of the CUDA calls behind those
 * steps. */
const char *cgh_status_string(int status);

/* Text of the handle's most recent error (never NULL; "" if none). */
const char *cgh_last_error(cgh_handle h);

/* Diagnostic: D[m*N + n] = sum_k A[m*K + k] * B[n*K + k] on the tcgen05
 * GEMM used by the separable methods.  A: device, M x K, B: device, N x K,
 * both 16-bit (is_bf16 = 0: FP16, 1: BF16), K-major; D: device FP32 M x N.
 * K must be a positive multiple of 64; M, N >= 1. */
cgh_status cgh_debug_gemm(cgh_handle h, const void *A, const void *B,
                          float *D, int M, int N, int K, int is_bf16,
                          void *stream);

/* Diagnostic for failure handling: launch one CTA that waits on an mbarrier
 * nothing ever arrives at.  The wait gives up after limit_cycles SM clock
 * cycles (clamped to [1e6, 4e9]), records CGH_ERR_TIMEOUT in the device
 * status word (read it with cgh_last_device_status) and the kernel exits;
 * the context stays usable.  This is the same bounded-wait path as every
 * pipelined kernel of the library.
 *
 * Host-side fault injection: if the environment variable
 * CGH_FAIL_ALLOC_AFTER=n is set when a handle is created, that handle's
 * (n+1)-th workspace allocation fails with CGH_ERR_NOMEM. */
cgh_status cgh_debug_stalled_wait(cgh_handle h, long long limit_cycles,
                                  void *stream);

/* Diagnostic: the two SM pipe rates that bound this library's ALU kernels,
 * measured on the handle's device by two short microbenchmarks (two CTAs of
 * 1024 threads per SM, eight independent dependency chains per thread):
 * *mufu_per_clk = hardware cosines (__cosf: one MUFU operation each) per SM
 * clock, *fma_per_clk = FP32 multiply-adds per SM clock issued as packed
 * fma.rn.f32x2.  Counted with the SMs' own cycle counters, so independent
 * of the clock the GPU runs at.  Synchronises `stream`; uses the handle's
 * host-call staging workspace.  Errors: CGH_ERR_INVALID_ARG (null
 * pointer), CGH_ERR_NOMEM, CGH_ERR_CUDA. */
cgh_status cgh_debug_pipe_rates(cgh_handle h, double *mufu_per_clk,
                                double *fma_per_clk, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CGH_H */
