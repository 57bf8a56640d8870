/*
 * stencil.h -- C ABI of the GB300 star-stencil sweep library (libstencil.so).
 *
 * The operation (Zohouri, Podobas, Matsuoka, "High-Performance High-Order
 * Stencil Computation on FPGAs Using OpenCL", Section IV.A, Eq. 1): `iters`
 * Jacobi steps of a 2D or 3D star stencil of radius r = 1..6,
 *
 *   g(p) = c[0] f(p) + sum_{i=1..r} sum_{d} c[1 + (i-1)*2*dim + d] f(clamp(p + i*e_d)),
 *
 * d = 0:W(-x) 1:E(+x) 2:S(-y) 3:N(+y) [4:B(-z) 5:A(+z)], one coefficient per
 * (distance, direction) as in the paper's no-sharing worst case, out-of-grid
 * neighbours clamped to the border cell at every step (Sections III.B, IV.B).
 * Each cell is evaluated as one FP32 multiply followed by 2*dim*r FP32 fused
 * multiply-adds in exactly that order (Section V.A's multiply-then-FMA
 * chain), so every schedule -- any temporal degree, tile or launch shape --
 * returns bit-identical FP32 results.  Sums run i = 1..r (Eq. 1 prints i = 0;
 * Table I's 12r+1 / 8r+1 FLOP count fixes 1..r).
 *
 * Grids: contiguous, x fastest, element (x, y, z) at x + nx*(y + ny*z);
 * 2D grids pass nz = 1.  Storage is FP32, BF16 or FP16; arithmetic is always
 * FP32 in registers and 16-bit storage is rounded (to nearest even) only
 * when a pass writes the grid back, i.e. once per `t` steps.
 *
 * Conventions for every call:
 *  - Return value: STENCIL_OK (0) or a negative STENCIL_ERR_* code.  No
 *    exception or abort crosses the ABI.  After STENCIL_ERR_CUDA,
 *    stencil_last_cuda_error() gives the cudaError_t value.
 *  - Device pointers are plain CUDA device addresses on the current device;
 *    `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *    work is enqueued asynchronously on `stream` unless stated otherwise.
 *  - The caller owns `in` and `out`; `in` is never written; overlapping `in`
 *    and `out` is rejected (STENCIL_ERR_ALIAS).
 *  - The handle owns a scratch grid (the second buffer of the ping-pong
 *    between passes), allocated with cudaMalloc when a run first needs it
 *    and freed by stencil_destroy.  A handle must not be used from two host
 *    threads at once; runs on different streams with the same handle share
 *    the scratch grid and must not overlap on the GPU.
 */
#ifndef STENCIL_H
#define STENCIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STENCIL_OK                 0
#define STENCIL_ERR_INVALID_ARG  (-1) /* bad dim/radius/sizes/pointer/dtype/schedule field */
#define STENCIL_ERR_ALIAS        (-2) /* in and out overlap */
#define STENCIL_ERR_UNSUPPORTED  (-3) /* schedule not available for this problem */
#define STENCIL_ERR_OOM          (-4) /* device allocation failed */
#define STENCIL_ERR_CUDA         (-5) /* a CUDA runtime call failed */
#define STENCIL_ERR_TIMEOUT      (-6) /* a kernel's bounded wait expired (device status) */
#define STENCIL_ERR_NO_DEVICE    (-7) /* no usable GPU */
#define STENCIL_ERR_BOUNDS       (-8) /* a bounds-checked kernel skipped an out-of-range access (device status) */

typedef struct stencil_plan *stencil_handle;

typedef enum { STENCIL_F32 = 0, STENCIL_BF16 = 1, STENCIL_F16 = 2 } stencil_dtype;

typedef enum {
    STENCIL_KERNEL_AUTO = 0,   /* streaming kernel when the grid allows it, else naive */
    STENCIL_KERNEL_STREAM = 1, /* blocked streaming kernel (error if not applicable) */
    STENCIL_KERNEL_NAIVE = 2   /* one thread per cell, one step per launch (t = 1) */
} stencil_kernel;

/*
 * Explicit schedule of the streaming kernel (Sections III.A and V.A: spatial
 * block size, temporal degree par_time).  Every field 0 = chosen by the
 * library.  Blocks have a compiled shape: 2D 128 threads, each owning 4
 * consecutive x cells (a 512-cell row strip streamed along y); 3D 16 x 8
 * threads, each owning 4 x cells times rows_per_thread y rows (a 64-cell
 * wide tile streamed along z).  The strip/tile includes a halo of r*(t-1)
 * cells per side (x halo rounded up to 16 bytes) recomputed by neighbouring
 * blocks (overlapped blocking, Eq. 2).  Block order: the stream axis is cut
 * into slabs of `seg` rows/planes, one block per (slab, strip/tile), the
 * strips/tiles of a slab in consecutive blocks; except for 2D kernels with a
 * long unrolled body ((2r+1)*t*4*(4r+1) > 400 FMA, e.g. r >= 2 at t >= 2) or
 * t >= 5, where the strips' y axes are laid end to end and block b streams
 * rows [b*seg, (b+1)*seg) of that sequence (one piece per strip it touches);
 * there the default `seg` gives every resident block slot of the device the
 * same number of rows (once for long bodies, else in ~200-row blocks).  Every
 * piece also streams r*t halo planes.
 */
typedef struct {
    int kernel;          /* stencil_kernel */
    int t;               /* temporal degree: time steps per pass over the grid, >= 1 */
    int threads_x;       /* 0, or the compiled block width (2D 128, 3D 16) */
    int threads_y;       /* 0, or the compiled block height (3D 8) */
    int rows_per_thread; /* 3D: 2 or 4 */
    int seg;             /* stream-axis rows/planes per block, >= 1 */
    int prefetch;        /* 0, or the compiled number of planes loaded ahead by the kernel
                            of degree t (a remainder pass of another degree runs with
                            its own kernel's depth) */
    int planes_per_step; /* 2D: rows every time level advances per step of the block's loop,
                            1, 2 (t = 1..5) or 4 (t = 1): the rows of a step share one
                            barrier, one copy wait and the loop's bookkeeping; 3D: 1.  A
                            degree compiled with fewer rows per step runs with the next
                            smaller count that is compiled (4 -> 2 -> 1). */
} stencil_schedule;

/* Number of features describing one (problem, schedule) pair for the cost model. */
#define STENCIL_NFEAT 18

/* One measured or predicted schedule of a problem (stencil_tune output). */
typedef struct {
    stencil_schedule sched;          /* fully resolved (no 0 fields) */
    float features[STENCIL_NFEAT];   /* stencil_schedule_features of it */
    float ns_per_cell;               /* measured ns per cell update (exhaustive), else -1 */
    float analytic_ns_per_cell;      /* the analytic model's estimate */
    float model_ns_per_cell;         /* the cost model's estimate, else -1 */
} stencil_timing;

typedef struct stencil_model *stencil_model_handle;

typedef enum {
    STENCIL_TUNE_ANALYTIC = 0,   /* pick the minimum of the analytic bandwidth/compute model */
    STENCIL_TUNE_EXHAUSTIVE = 1, /* time every candidate on the GPU, pick the fastest */
    STENCIL_TUNE_MODEL = 2       /* pick the minimum predicted by a trained cost model */
} stencil_tune_mode;

/* Create a stencil of dimension `dim` (2 or 3) and radius 1..6 with
 * K = 2*dim*radius + 1 FP32 coefficients read from host memory `coeffs`
 * (layout above; copied, the caller keeps ownership).  Allocates no device
 * memory.  Errors: INVALID_ARG. */
int stencil_create(stencil_handle *out, int dim, int radius, const float *coeffs);

/* Create a stencil with one coefficient per distance: K = radius + 1 FP32
 * coefficients, c[0] for the centre and c[i] for every neighbour at distance
 * i, the form of the stencils the paper compares against in Section IV.C
 * (its Sections IV.A and V.A note that sharing removes multiplications but
 * no additions).  Reordering is allowed there; this library fixes one order:
 *
 *   g(p) = c[0] f(p) + sum_{i=1..r} c[i] * s_i(p),
 *   s_i = (((W + E) + S) + N) [+ B) + A],
 *
 * the 2*dim neighbours at distance i (clamped as above) summed left to right
 * in FP32, then one FMA per distance (FP32 path: one rounded multiply, then per
 * distance 2*dim-1 rounded adds and one FMA).  Streaming kernels exist for FP32
 * storage, radius 1..4; other cases run the one-step-per-launch kernel.
 * Errors: INVALID_ARG. */
int stencil_create_shared(stencil_handle *out, int dim, int radius, const float *coeffs);

/* Free the handle and its scratch grid.  Synchronises the device first so
 * that no enqueued run still uses the scratch grid.  NULL is accepted. */
int stencil_destroy(stencil_handle h);

/* `iters` steps from `in` to `out` (device pointers, nx*ny*nz elements of
 * `dtype`), with the schedule stencil_default_schedule reports (a pick that
 * stencil_tune stored on the handle, else one in the tuning-cache file, else
 * the library's rule).
 * iters == 0 copies in to out.  Errors: INVALID_ARG (sizes <= 0, dim 2 with
 * nz != 1, NULL pointers, iters < 0, bad dtype), ALIAS, OOM, CUDA. */
int stencil_run(stencil_handle h, const void *in, void *out, int64_t nx, int64_t ny,
                int64_t nz, int iters, int dtype, void *stream);

/* As stencil_run with an explicit schedule (`sched` may be NULL = auto).
 * Errors as stencil_run plus UNSUPPORTED (temporal degree or tile shape not
 * compiled in, shared memory exceeded, grid not 16-byte aligned for the
 * streaming kernel) and INVALID_ARG for out-of-range fields. */
int stencil_run_ex(stencil_handle h, const void *in, void *out, int64_t nx, int64_t ny,
                   int64_t nz, int iters, int dtype, void *stream, const stencil_schedule *sched);

/* End-to-end form on HOST buffers: copies `in_host` to the device, runs
 * `iters` steps and copies the result to `out_host`, all on `stream`, and
 * returns after the stream has finished.  Device buffers are held by the
 * handle and reused across calls (grown on demand).  Pinned host memory gives
 * full copy bandwidth; pageable memory works.  Errors as stencil_run_ex. */
int stencil_run_host(stencil_handle h, const void *in_host, void *out_host, int64_t nx,
                     int64_t ny, int64_t nz, int iters, int dtype, void *stream,
                     const stencil_schedule *sched);

/* The schedule stencil_run would use for this problem when given none: a pick
 * stored on the handle (stencil_tune with store != 0), else one stored in the
 * tuning-cache file (see stencil_tune), else the proposal of the cost model set
 * with stencil_use_cost_model, else the library's rule (2D: radius 1 at t = 4
 * with one row per step, radius 2..4 at t = 3, 2, 2 with two rows per step --
 * 16-bit storage radius 3 at t = 3 --, radius 5, 6 at t = 2; 3D: t = 2 for
 * radius 1, else t = 1; 2 rows per thread, 4 for FP32 radius 3 and 4). */
int stencil_default_schedule(stencil_handle h, int64_t nx, int64_t ny, int64_t nz, int dtype,
                             stencil_schedule *out);

/* Schedule tuner (the model-guided parameter choice of Sections V.A and VI.A,
 * re-done for the GPU).  Candidates: every compiled temporal degree, one or two
 * rows per step (2D), several stream-segment lengths and, in 3D, 2 or 4 rows
 * per thread.
 *  - ANALYTIC: time per cell update = max(HBM bytes / bandwidth, issue time)
 *    per pass, divided by the cell updates of the pass; the issue time counts
 *    per step and level every thread's FP32 chains (halo cells included) and
 *    its bookkeeping instructions, at a share of the SM issue rate that falls
 *    with the resident warps per SM; no device work.
 *  - EXHAUSTIVE: allocates an input and output grid of the problem's size
 *    (cudaMalloc), runs each candidate after a warm-up for >= 16 steps and
 *    >= 2^30 cell updates (at most 1000 steps: small grids get longer runs, so
 *    launch latency does not decide the timing), takes the best of two
 *    CUDA-event timings, frees the grids; synchronous.
 *  - MODEL: needs `model` (stencil_model_train), trained to predict
 *    log(measured / analytic time) from the features; the prediction of a
 *    candidate is its analytic time times exp(model output).  The candidate
 *    with the lowest prediction is picked if it is predicted at least 5 % faster
 *    than the analytic model's pick, else the analytic pick (a trust region:
 *    smaller predicted gains are within the model's fit error).  No device
 *    work besides the model's forward pass.
 * `chosen` receives the pick; `rows` (capacity `cap`, may be NULL) receives one
 * stencil_timing per candidate and *nrows their number.  With `store` != 0 the
 * pick is kept in the handle and used by later stencil_run calls on the same
 * (nx, ny, nz, dtype); if the environment variable STENCIL_TUNE_CACHE names a
 * file, the pick is also appended to it as one text line keyed by the GPU's
 * name, dim, radius, coefficient form, dtype and (nx, ny, nz), and every handle
 * in any process with the same setting uses it (the handle's own pick first).
 * Errors: INVALID_ARG, UNSUPPORTED (no streaming kernel for this shape), OOM,
 * CUDA. */
int stencil_tune(stencil_handle h, int64_t nx, int64_t ny, int64_t nz, int dtype, int mode,
                 stencil_model_handle model, int store, stencil_schedule *chosen,
                 stencil_timing *rows, int cap, int *nrows);

/* The fully resolved streaming schedule of one pass of degree t (sched->t, else the
 * default's) that stencil_run_ex would launch for this problem with `sched` (NULL or
 * partial: 0 fields = library choice): compiled block shape, segment length, prefetch
 * depth and the rows per step actually compiled for that degree.  No device work.
 * Errors: INVALID_ARG, UNSUPPORTED (no streaming kernel for this schedule or rows not
 * 16-byte aligned). */
int stencil_resolve_schedule(stencil_handle h, int64_t nx, int64_t ny, int64_t nz, int dtype,
                             const stencil_schedule *sched, stencil_schedule *out);

/* Features of (problem, schedule) for the cost model: dim, radius, log2 nx,
 * log2 ny, log2 nz, bytes per element, t, resident warps per SM, tile height
 * (rows, 1 in 2D), log2 of the unrolled loop body's FMA count (queue period x
 * t x 4 x rows x (2*dim*r+1)), log2 segment length, log2 analytic ns per cell
 * update, block order (1: 2D strips laid end to end, 0: slabs), log2 of the
 * launch's blocks per resident block slot (waves), rows per step, log2 halo
 * redundancy (thread region over compute tile), registers per thread / 64,
 * log2 dynamic shared memory in KiB.  `sched` may be partial (0 = library
 * choice). */
int stencil_schedule_features(stencil_handle h, int64_t nx, int64_t ny, int64_t nz, int dtype,
                              const stencil_schedule *sched, float *features);

/* Cost model: `n_features` -> hidden -> hidden -> 1 multilayer perceptron with
 * ReLU, trained by full-batch Adam on the mean-squared error of its
 * (standardised) target, with hand-written CUDA forward, backward and update
 * kernels on the current device.  Host arrays: X is row-major n x n_features,
 * y has n entries.  Training standardises features and targets on its first
 * call unless stencil_model_normalization set them.  Errors: INVALID_ARG,
 * OOM, CUDA. */
int stencil_model_create(stencil_model_handle *out, int n_features, int hidden, int seed);
int stencil_model_destroy(stencil_model_handle m);
int stencil_model_train(stencil_model_handle m, const float *X, const float *y, int n, int epochs,
                        float lr, float *final_loss);
int stencil_model_predict(stencil_model_handle m, const float *X, float *y, int n);
/* Fixed standardisation (x - fmean) / fstd, (y - ymean) / ystd. */
int stencil_model_normalization(stencil_model_handle m, const float *fmean, const float *fstd,
                                float ymean, float ystd);
/* Copy the flat parameters (W1, b1, W2, b2, w3, b3; row-major, input index
 * first) to (set = 0) or from (set != 0) host memory; returns the parameter
 * count instead when `count` does not match it. */
int stencil_model_params(stencil_model_handle m, float *host, int count, int set);
/* Loss (mean squared error in standardised units) and its gradient with
 * respect to the flat parameters, for testing the backward kernels. */
int stencil_model_grad(stencil_model_handle m, const float *X, const float *y, int n, float *loss,
                       float *grad);

/* Make `m` (trained as stencil_tune's MODEL mode expects) the process-wide cost
 * model that proposes schedules: stencil_run, stencil_run_batched and
 * stencil_default_schedule then use, for a problem with no pick stored on the
 * handle or in the tuning-cache file, the candidate with the lowest predicted
 * time (computed once per handle and problem; one small forward pass of the
 * model on the current device).  NULL restores the library's built-in rule.
 * The model must stay alive while it is in use.  Never fails (STENCIL_OK). */
int stencil_use_cost_model(stencil_model_handle m);

/* Largest temporal degree compiled in for (dim, radius, dtype) and, in 3D,
 * rows_per_thread; 0 if none.  */
int stencil_max_t(int dim, int radius, int dtype, int rows_per_thread);

/* One grid of a batch: `in` -> `out` (device pointers, nx*ny*nz elements of
 * dtype), `iters` steps of the stencil of handle `h`. */
typedef struct {
    stencil_handle h;
    const void *in;
    void *out;
    int64_t nx, ny, nz;
    int iters;
    int dtype;
} stencil_batch_item;

/* Sweep many independent grids of mixed dimension, radius and storage type
 * together (not in the paper; a serving-style batch of the paper's sweep).
 * Each grid runs exactly the passes stencil_run would: iters / t passes of its
 * handle's tuned or default degree t, then one remainder pass of degree
 * iters mod t, so results equal stencil_run's bit for bit.  Passes are grouped
 * by kernel class (dim, radius, dtype, temporal degree, rows per thread or per
 * step); each class runs as ONE persistent launch whose blocks take tiles from
 * a device-side queue ordered pass by pass over all grids of the class,
 * largest grids first; a tile of pass p of a grid starts only when all tiles
 * of its pass p-1 are done (bounded wait: on expiry the device status is set,
 * see stencil_get_device_status).  All class launches of the full passes are
 * captured as parallel branches of one CUDA graph, so the classes run side by
 * side and one class's last wave overlaps the others' work; the remainder
 * passes follow as a second set of parallel branches once every full pass is
 * done.  The graph is cached for this exact item list (same pointers, sizes,
 * handles, schedules) and replayed on `stream` by later calls.  The batch owns
 * one scratch grid per item (allocated on the first call for an item list,
 * before capture) and keeps up to four cached lists.
 * Every grid must allow the streaming kernel (rows 16-byte aligned: nx % 4
 * FP32, nx % 8 16-bit; 16-byte aligned pointers), else STENCIL_ERR_UNSUPPORTED.
 * Items may share a handle; `in` of one item must not overlap any `out`.
 * Errors as stencil_run plus UNSUPPORTED. */
int stencil_run_batched(const stencil_batch_item *items, int n, void *stream);

/* Synchronise `stream`, then read and return the sticky device status of the
 * current device: STENCIL_OK, STENCIL_ERR_TIMEOUT when a kernel gave up a
 * bounded wait (it then stopped early and its output is not valid), or
 * STENCIL_ERR_BOUNDS when a bounds-checked kernel skipped an access.  The
 * status covers every entry point, stencil_run_noalloc included.
 * `clear` != 0 resets the status to OK afterwards. */
int stencil_get_device_status(void *stream, int clear);

/* Test hook for failure detection: while `plane` >= 0, streaming kernels on
 * this handle never issue the copy of that input plane (with two rows per
 * step: of the step holding it), so the wait for it expires after `timeout_ms`
 * milliseconds (1..10000), the kernel records STENCIL_ERR_TIMEOUT in the
 * device status and returns without hanging.  plane < 0 restores normal
 * operation (and the default 2000 ms limit).  In stencil_run_batched the same
 * setting makes full pass number `plane` of the grids swept with this handle
 * never report completion, so the bounded waits of their next full pass
 * expire. */
int stencil_set_fault_injection(stencil_handle h, int plane, int timeout_ms);

/* Memory-checker substitute: with on = 1, streaming sweeps on this handle use
 * the bounds-checked kernel instantiations, which test every shared-memory
 * access, global store and TMA copy against its buffer and, instead of
 * performing an out-of-range one, record STENCIL_ERR_BOUNDS in the device
 * status (read with stencil_get_device_status).  Only a few configurations
 * are compiled checked (2D FP32 r=1 t=1,5, r=4 t=2, r=6 t=2; 2D BF16 r=2
 * t=3; 3D FP32 r=1 t=2 2 rows, r=3 t=1 4 rows, r=5 t=1 2 rows; 3D FP16 r=2
 * t=1 2 rows); other schedules return UNSUPPORTED.  on = 0 restores the
 * normal kernels.  Errors: INVALID_ARG. */
int stencil_set_checked(stencil_handle h, int on);

/* stencil_run without any device memory allocation, for callers that cannot
 * allocate: code inside an allocator's out-of-memory path (where a cudaMalloc
 * would recurse or fail), or processes whose device memory is handed out by an
 * external budget that the library must not draw on.  The paper has no
 * counterpart; this is a library-level variant.
 *  - The second grid of the ping-pong between passes is a 16 MiB array
 *    compiled into the library (every GPU that loads the library holds it until
 *    the process exits), so nx*ny*nz*sizeof(dtype) must be at most 16 MiB (4M
 *    FP32 cells, 8M BF16/FP16 cells); larger grids are rejected with
 *    STENCIL_ERR_INVALID_ARG before any device work.
 *  - The first call on a device looks up the array's device address and the
 *    device attributes; make that first call before any stream capture.
 *  - All calls on a device share the array, which keeps the last call's
 *    contents: calls whose work overlaps on the GPU (different streams, or
 *    different handles at the same time) race and give wrong results.
 *  - The schedule is the library's default rule (stencil_default_schedule
 *    without picks stored by stencil_tune or read from the tuning-cache file);
 *    every FP32 schedule gives the same bits, so results equal stencil_run's.
 *  - A kernel whose bounded wait expires records it in a status word of this
 *    entry point (sticky, like the library's main status word);
 *    stencil_get_device_status reports it as STENCIL_ERR_TIMEOUT and clears
 *    it with clear != 0.
 * Arguments and other errors as stencil_run. */
int stencil_run_noalloc(stencil_handle h, const void *in, void *out, int64_t nx, int64_t ny,
                        int64_t nz, int iters, int dtype, void *stream);

/* Measured peaks of the current device, the denominators of the roofline
 * R(t) = min(P_fp32 / F, BW * t / (2 s)) (Table IV/V's roofline ratio, re-done
 * for the GPU): fp32_flops is the FP32 fused multiply-add throughput of the
 * CUDA cores (independent FMA chains in every thread, 2 FLOP per FMA, CUDA-event
 * timed), copy_bytes_per_s the bytes read plus written per second by a 16-byte
 * copy kernel over 1 GiB buffers (above the L2 size).  sms and sm_clock_khz are
 * the device attributes.  Allocates two 1 GiB buffers for the call (cudaMalloc)
 * and synchronises `stream`.  Errors: INVALID_ARG, OOM, CUDA. */
typedef struct {
    double fp32_flops;
    double copy_bytes_per_s;
    int sms;
    int sm_clock_khz;
} stencil_peaks;
int stencil_measure_peaks(void *stream, stencil_peaks *out);

/* cudaError_t of the last failed CUDA call on this host thread (0 if none). */
int stencil_last_cuda_error(void);

/* Static description of a status code. */
const char *stencil_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_H */
