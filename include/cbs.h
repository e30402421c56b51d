/*
 * cbs.h -- C-ABI of the GB300 cyclic compact banded solver.
 *
 * The library solves many independent cyclic (periodic) compact banded linear
 * systems A x = b, tridiagonal (bandwidth w = 3), pentadiagonal (w = 5) or
 * heptadiagonal (w = 7, the generalised bands of Sec. 2, Eq. 3-6), or
 * block-tridiagonal with 2 x 2 block entries (Sec. 1; CBS_LHS_BLOCK), one
 * per grid line of a 3-D field, with the two-level partition method of Song et
 * al., "Scalable Parallel Linear Solver for Compact Banded Systems on
 * Heterogeneous Architectures" (arXiv 2101.02286):
 *
 *   - each line is split into p partitions (Sec. 3, Fig. 3); the first r =
 *     (w-1)/2 rows of a partition are its interface unknowns, the rest its
 *     bulk block D_i;
 *   - y_i = D_i^{-1} b_i inside each partition (Eq. 17);
 *   - the reduced cyclic block-tridiagonal interface system A-hat x~ = b-hat
 *     (Eq. 11, 18-21) is solved by block PCR with detach/reattach
 *     (Algorithms 1-4), in the precision of the solve: FP64 for CBS_FP64 and
 *     CBS_FP32_REFINE_I64, FP32 for CBS_FP32 and CBS_FP32_REFINE (see the
 *     precision enum);
 *   - back-substitution x_i = y_i - S_i x~_i - R_i x~_{i+1} (Eq. 22).
 *
 * Everything RHS-independent (S_i, R_i, the reduced blocks and the PCR
 * coefficients of every stage) is pre-factorised once per plan (Sec. 4, last
 * paragraph).  Optionally the right-hand side is produced in the same launch
 * from a field f by the periodic central stencil of Eq. 1.
 *
 * Conventions for every entry point:
 *   - Array arguments named "device" are device pointers owned by the caller;
 *     the library never frees or keeps them beyond the call (except
 *     cbs_desc.bands, see below).  Host arrays are plain host pointers.
 *   - A field has dims (nx, ny, nz) with x contiguous: element (i, j, k) is at
 *     offset i + nx * (j + ny * k).  Lines run along `direction`.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Launches are asynchronous; device-side errors (a singular
 *     variable-band system, values outside the range of the FP32 modes, an
 *     expired wait) are reported through cbs_status_poll.
 *   - Every call returns a cbs_status; no C++ exception crosses the ABI.
 *     cbs_last_error_string() describes the last failure of the calling thread.
 *   - A plan may be used from several host threads, but concurrent launches on
 *     one plan must be ordered by the caller's streams (the plan's device
 *     status word is shared).
 */
#ifndef CBS_H
#define CBS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cbs_status;
enum {
    CBS_OK = 0,
    CBS_ERR_INVALID_ARG = 1, /* a descriptor field or pointer is invalid      */
    CBS_ERR_UNSUPPORTED = 2, /* valid request outside what is implemented     */
    CBS_ERR_SINGULAR = 3,    /* zero / non-finite pivot or interface block    */
    CBS_ERR_TIMEOUT = 4,     /* a bounded device wait expired                 */
    CBS_ERR_CUDA = 5,        /* a CUDA runtime call failed                    */
    CBS_ERR_NO_MEMORY = 6,   /* host or device allocation failed              */
    CBS_ERR_RANGE = 7        /* device: an input or result outside the range
                                of the FP32 modes (magnitude >= 2^126, inf or
                                nan); the affected lines' output is not valid */
};

/* Arithmetic of the solve. */
enum {
    CBS_FP64 = 0,        /* everything in FP64                                    */
    CBS_FP32 = 1,        /* FP32 (interface system included), no refinement
                            (error ~ cond * 2^-24)                                */
    CBS_FP32_REFINE = 2, /* FP32 solves + `refine_sweeps` iterative-refinement
                            sweeps whose residual b - A x is evaluated to FP64
                            accuracy; output FP64.  The interface system of each
                            FP32 solve is FP32 too: the refinement, not the
                            correction solve, carries the accuracy             */
    CBS_FP32_REFINE_I64 = 3 /* as CBS_FP32_REFINE, with the interface system of
                            every FP32 solve in FP64 (slower, same accuracy;
                            on-chip and long-line plans, not batches or
                            variable bands)                                      */
};

/* Element type of the caller's arrays. */
enum { CBS_DTYPE_F64 = 0, CBS_DTYPE_F32 = 1 };

/* Left-hand side. */
enum {
    CBS_LHS_TOEPLITZ = 0,    /* constant bands: (beta,) alpha, 1, alpha (, beta)      */
    CBS_LHS_VARIABLE = 1,    /* tridiagonal, row-wise alpha_i read from cbs_desc.bands:
                                A[i,i-1] = A[i,i+1] = alpha_i, A[i,i] = 1            */
    CBS_LHS_BLOCK = 2        /* block-tridiagonal with 2 x 2 block entries (Sec. 1),
                                see cbs_desc.block_size / blocks                     */
};

/* Right-hand side.  The staggered kinds (App. A.2; Eq. 2) map a field on one
 * grid to the grid shifted by half a spacing, selected by cbs_desc.rhs_shift
 * = s: with s = 0 input element j holds f at x_{j+1/2} and output element i
 * is at x_i; with s = 1 input element j holds f at x_j and output element i
 * is at x_{i+1/2}.  Term k couples input elements i+k-1+s and i-k+s. */
enum {
    CBS_RHS_NONE = 0,        /* the input array already holds b                       */
    CBS_RHS_CENTRAL = 1,     /* b_i = sum_k c_k (f_{i+k} - f_{i-k}) / (2 k h), Eq. 1 */
    CBS_RHS_STAGGERED = 2,   /* b_i = sum_k c_k (f_{i+k-1+s} - f_{i-k+s}) / ((2k-1) h):
                                the staggered first derivative (App. A.2: alpha =
                                9/62, c = 63/62, 17/62)                              */
    CBS_RHS_MIDPOINT = 3     /* b_i = sum_k c_k (f_{i+k-1+s} + f_{i-k+s}) / 2: the
                                compact interpolation of Eq. 2 (App. A.2: alpha =
                                3/10, c = 3/2, 1/10); h is not used                */
};

typedef struct cbs_desc {
    /* geometry */
    int64_t dims[3];        /* nx, ny, nz (>= 1); x contiguous                     */
    int32_t direction;      /* 0 = x, 1 = y, 2 = z: the solve axis; n = dims[dir]  */
    /* matrix */
    int32_t bandwidth;      /* 3, 5 or 7 (7: Toeplitz, on-chip lines of <= 32
                               partitions, no batches)                             */
    int32_t cyclic;         /* 1 = periodic; 0 = acyclic (corner blocks zero)      */
    int32_t lhs_kind;       /* CBS_LHS_*                                            */
    double  alpha, beta, gamma; /* Toeplitz bands a_{+-1}, a_{+-2}, a_{+-3} (diagonal
                               1; beta ignored below bandwidth 5, gamma below 7) */
    const void* bands;      /* CBS_LHS_VARIABLE: device array of alpha_i, same dims
                               and dtype as the input; read at every solve (the
                               caller keeps it alive and may change its values)    */
    /* right-hand side */
    int32_t rhs_kind;       /* CBS_RHS_*                                            */
    int32_t rhs_terms;      /* K = 1..3 stencil terms (CBS_RHS_CENTRAL); 1..2 for
                               the staggered kinds                                 */
    double  rhs_coef[3];    /* c_1..c_K (Lele's a, b, c)                           */
    double  h;              /* grid spacing (> 0)                                  */
    /* solver */
    int32_t segments;       /* p partitions per line; 0 = choose automatically     */
    int32_t precision;      /* CBS_FP64 / CBS_FP32 / CBS_FP32_REFINE(_I64)         */
    int32_t refine_sweeps;  /* refinement modes: 1 or 2                             */
    int32_t in_dtype;       /* CBS_DTYPE_* of the input (f or b)                   */
    int32_t out_dtype;      /* CBS_DTYPE_* of the output x (F64 for FP32_REFINE)   */
    int32_t rhs_shift;      /* staggered kinds: s = 0 (half points -> nodes) or 1
                               (nodes -> half points); ignored otherwise.  The
                               staggered kinds need cyclic = 1, a Toeplitz LHS and
                               on-chip lines (no batches)                          */
    /* One-sided boundary closures of an acyclic derivative (cyclic = 0 with
     * CBS_RHS_CENTRAL; 0 rows = none).  The first closure_rows rows of every
     * line carry their own equations, read from the host array `closure` by
     * cbs_plan_create (not kept): row k < closure_rows is
     *     sum_j L[k][j] x_j = sum_j R[k][j] f_j / h,   j < closure_width,
     * stored as closure[k*2W + j] = L[k][j], closure[k*2W + W + j] = R[k][j]
     * (W = closure_width).  The last closure_rows rows are the mirror image:
     * row n-1-k has L[k][j] on x_{n-1-j} and -R[k][j] / h on f_{n-1-j} (a
     * first derivative changes sign under reflection).  Rows in between use
     * the Toeplitz bands and the central stencil, which must stay inside the
     * line: closure_rows >= max(r, rhs_terms).  On-chip lines only.        */
    int32_t closure_rows;   /* 0..4                                                */
    int32_t closure_width;  /* 1..16                                               */
    const double* closure;  /* host array, 2 * closure_width doubles per row      */
    /* CBS_LHS_BLOCK: a line of n = dims[direction] unknowns is n / b points of
     * b = block_size unknowns each, point-major (unknown c of point m is
     * element m b + c along the line), and point m couples to points m - 1, m
     * and m + 1 through the b x b blocks L, D, U (the same for every point):
     *     L x_{m-1} + D x_m + U x_{m+1} = d_m   (cyclic: point indices mod n/b).
     * `blocks` is a host array of 3 b^2 doubles, L, D, U row-major, read by
     * cbs_plan_create (not kept).  b = 2 (the flattened system has half
     * bandwidth 2b - 1 = 3: set bandwidth = 7); n even; right-hand side given
     * (CBS_RHS_NONE); CBS_FP64 or CBS_FP32; on-chip lines (partitions of at
     * most 32 rows, made of whole points); cyclic or acyclic; no batches,
     * closures or transposes.  Partitions are counted in whole points (the
     * `segments` partitions split the n / b points as evenly as possible). */
    int32_t block_size;     /* b: 2 for CBS_LHS_BLOCK; ignored otherwise          */
    const double* blocks;   /* CBS_LHS_BLOCK: host array L | D | U (3 b^2 doubles) */
} cbs_desc;

typedef struct cbs_plan cbs_plan;
typedef struct cbs_batch cbs_batch;

/* Plan introspection: what the plan chose, and the interface schedule. */
typedef struct cbs_plan_info {
    int32_t n, bandwidth, segments;
    int32_t rows_big, rows_small, count_big; /* partition sizes (first count_big get rows_big) */
    int32_t pcr_steps;        /* block-PCR steps on the interface system            */
    int32_t detach_steps;     /* detach rounds (= reattach rounds)                  */
    int32_t detached_rows;    /* rows detached over the whole solve                 */
    int32_t stage_count;      /* stages the device executes on x~ per solve         */
    int32_t kernel;           /* implementation id (0 = on-chip lines, 1 = long lines) */
    int32_t threads_per_line;
    int64_t lines;            /* independent systems in one solve                   */
    /* Stages of the interface solve that exchange values between partitions:
     * a stage whose coupling blocks are below 2^-60 (FP64) or 2^-30 (FP32) of
     * its diagonal blocks reduces to a local product (the blocks shrink
     * geometrically with the partition size and square at every PCR step).
     * inner_*: the segment-level system of a long-line plan (kernel 1). */
    int32_t message_stages, message_stages_f32;
    int32_t inner_message_stages, inner_message_stages_f32;
    /* Kernel variant setting (cbs_plan_set_variant), whether the plan
     * qualifies for the TMA-fed refinement kernel (1: it runs when the arrays
     * start on 16-byte boundaries and the variant is 0), and the lines per
     * tile of that kernel for y/z lines (0: the default). */
    int32_t variant, tma, tile_lines;
    /* Long-line plans (kernel 1) of x-lines whose segments hold 32 (or 31)
     * inner partitions of 16 rows and whose outer interface system is
     * decoupled to FP64 rounding: 1 when a solve runs one warp per segment
     * (one launch per segment size, variant 0), 0 for the end-row /
     * interface / segment launches. */
    int32_t segment_warp;
} cbs_plan_info;

/* Create a plan: validates the descriptor, chooses p when segments == 0,
 * pre-factorises everything RHS-independent in FP64 on the host (Sec. 4) and
 * uploads the tables to the current device.  Allocates device memory.
 * Lines of up to 32 partitions of at most 32 rows (16 for FP32 + refinement)
 * run one partition per thread of a warp (kernel 0); longer lines run one
 * segment per CTA (kernel 1: x-lines, cyclic Toeplitz bands, right-hand side
 * given, segments of at most 8192 rows).  Kernel 1 segments: when n - p r
 * is a multiple of 16 they have 16 K + r or 16 (K - 1) + r rows (whole
 * 16-row inner partitions); otherwise the first n mod p get ceil(n / p) rows
 * and the rest floor(n / p) (larger ones first, as cbs_plan_info reports in
 * rows_big / rows_small / count_big).  Two segment sizes need the truncated
 * rows of D^-1 to agree (UNSUPPORTED for segments too short for the band's
 * decay).
 * Errors: INVALID_ARG (n < 2 r p, bad enum, ...), UNSUPPORTED, SINGULAR (a
 * zero or non-finite pivot in D_i or an interface block), CUDA, NO_MEMORY. */
cbs_status cbs_plan_create(cbs_plan** out, const cbs_desc* desc);

/* Rebind the alpha field of a CBS_LHS_VARIABLE plan (device pointer, same
 * dims and dtype as the plan's input; the caller keeps it alive).  Takes
 * effect for launches issued after the call.  INVALID_ARG for Toeplitz
 * plans or NULL. */
cbs_status cbs_plan_set_bands(cbs_plan* plan, const void* bands);

/* Autotuner: times every admissible partition count for `desc` (p = 1..32
 * lanes for lines that fit one warp, divisors giving 64..8192-row segments
 * for long lines), and for on-chip plans both kernel variants
 * (cbs_plan_set_variant), on scratch buffers it allocates and frees on the
 * current device (inputs filled with a fixed pattern), with `reps` timed
 * solves each after two warm-ups, and records the fastest in a per-process
 * cache keyed by (dims, direction, bandwidth, precision, dtypes, stencil,
 * bands kind).  Later cbs_plan_create calls with segments == 0 use the
 * cached choice (partition count and variant).
 * Writes the choice to *best_segments and its time per solve to *best_ms
 * (either may be NULL).  Synchronises the device.  Errors: as
 * cbs_plan_create, CUDA, NO_MEMORY. */
cbs_status cbs_autotune(const cbs_desc* desc, int32_t reps, int32_t* best_segments, double* best_ms);

/* Kernel variant and tile walk of an on-chip plan (cbs_plan_info kernel ==
 * 0), used by cbs_solve and cbs_solve_transpose.  variant:
 *   0 = automatic (default): the TMA-fed refinement kernel when the plan
 *       qualifies -- FP32_REFINE(_I64) with one sweep, cyclic tridiagonal
 *       Toeplitz bands, 32 partitions of 8 or 16 rows (n = 256 or 512), the
 *       central stencil of at most two terms or none, FP64 in and out, both
 *       arrays on 16-byte boundaries, even nx for y/z lines -- otherwise the
 *       pipelined / staged line kernels;
 *   1 = always the pipelined / staged line kernels.
 * For long-line plans (kernel 1): 0 runs a warp per segment where the plan
 * qualifies (cbs_plan_info.segment_warp), 1 always the end-row / interface /
 * segment launches.
 * Both give results within the refinement's tolerance of the FP64 solution
 * (they round differently).  tile_lines: the tile shape of the TMA kernel,
 * adjacent lines per tile (for y/z lines also the contiguous bytes per row of
 * a tile load: 8 bytes per line): x-lines 4 or 8 (a warp per line, two tile
 * buffers per CTA); y/z lines 4, 8 (as x), 16 (one buffer, 8 warps of two
 * lines each) or 32 (16 lines, 16 warps, two buffers); 0 = the default of
 * the direction.  Only the arrangement of the work changes, not the
 * results.  cbs_autotune times the variants and tile shapes with the
 * partition counts and records the fastest.  Errors: INVALID_ARG (variant
 * not 0 or 1, tile_lines not 0, 4, 8, 16 or 32, NULL plan). */
cbs_status cbs_plan_set_variant(cbs_plan* plan, int32_t variant, int32_t tile_lines);

/* Fault injection for tests of the device timeout path (no GPU fault is
 * involved).  kind 1: in solves that run the TMA-fed refinement kernel
 * (cbs_plan_info tma == 1, variant 0), CTA 0 does not issue its first tile
 * load and the limit of the tile waits drops from 1 s to 1 ms, so that wait
 * expires: the kernel sets CBS_ERR_TIMEOUT in the status word, lets its
 * other load in flight land (bounded wait), and the CTA returns; the
 * context stays usable and the output of the affected CTA's tiles is not
 * written.  kind 0: no fault (default).  Errors: INVALID_ARG. */
cbs_status cbs_plan_inject_fault(cbs_plan* plan, int32_t kind);

/* Destroy a plan and free its device memory (synchronises the device). */
cbs_status cbs_plan_destroy(cbs_plan* plan);

/* x = A^{-1} b along every line, with b = S f when the plan has a stencil.
 * in: device, in_dtype, the field f (or b); out: device, out_dtype, same dims.
 * `out` must not alias `in`.  Asynchronous on `stream`.  Arrays need only
 * element alignment: x-line plans with whole-size partitions move rows in
 * 16-byte units when both arrays start on a 16-byte boundary and otherwise
 * run a staged kernel (same results, slower). */
cbs_status cbs_solve(cbs_plan* plan, const void* in, void* out, void* stream);

/* Adjoint of cbs_solve (Sec. 3 operators transposed):
 *   lambda = A^{-T} g, and, when the plan has a stencil, grad_in = S^T lambda.
 * Any of lambda / grad_in may be NULL (not written).  For CBS_LHS_VARIABLE,
 * when x and grad_bands are both non-NULL, also writes the band gradient
 * grad_bands_i = -lambda_i (x_{i-1} + x_{i+1}) (same as cbs_band_grad).
 * g, x, lambda, grad_in, grad_bands: device, the plan's dims; g and x of
 * out_dtype, lambda / grad_in / grad_bands of in_dtype.  UNSUPPORTED for
 * long-line and CBS_LHS_BLOCK plans. */
cbs_status cbs_solve_transpose(cbs_plan* plan, const void* g, const void* x,
                               void* lambda, void* grad_in, void* grad_bands,
                               void* stream);

/* grad_bands_i = -lambda_i (x_{i-1} + x_{i+1}) along the plan's lines
 * (periodic), the gradient of <g, x> with respect to row-wise alpha_i when
 * lambda = A^{-T} g.  Device arrays of the plan's dims, in_dtype.
 * UNSUPPORTED for CBS_LHS_BLOCK plans. */
cbs_status cbs_band_grad(cbs_plan* plan, const void* lambda, const void* x,
                         void* grad_bands, void* stream);

/* Read (and clear) the plan's device status word from kernels that already
 * ran: CBS_OK; CBS_ERR_SINGULAR (a variable-band solve met a zero or
 * non-finite pivot or interface block); CBS_ERR_RANGE (an FP32 mode met an
 * input or result outside its range); CBS_ERR_TIMEOUT (a bounded wait of the
 * TMA-fed kernel for its tile expired -- the only device wait in the
 * library).  Synchronises the device. */
cbs_status cbs_status_poll(cbs_plan* plan, int32_t* device_status);

/* Fill *info with the plan's choices and interface schedule counts. */
cbs_status cbs_plan_info_get(const cbs_plan* plan, cbs_plan_info* info);

/* Interface schedule of Algorithm 1 for p partitions (host only, no device):
 * writes up to `cap` stages as triples (type, s, n_a) into `stages`
 * (type 0 = detach, 1 = PCR step, 2 = final block solve, 3 = reattach) and
 * their count into *count.  cyclic selects the cyclic (floor(log2 p) PCR
 * steps) or acyclic (ceil(log2 p)) variant (Sec. 4). */
cbs_status cbs_schedule(int32_t p, int32_t cyclic, int32_t* stages, int32_t cap,
                        int32_t* count);

/* Host-only model of a plan's interface system (no device work, no GPU
 * needed): builds the tables cbs_plan_create would build for `desc` with
 * p partitions (desc->segments is ignored) and
 *   - writes the reduced blocks D-hat_i, L-hat_i, U-hat_i of Eq. 18-20
 *     (r x r row-major, partition-major, p*r*r doubles each) when non-NULL;
 *   - when bhat and xt are non-NULL, applies the pre-factorised stage
 *     coefficients (Algorithms 2-4) to b-hat (p*r doubles) and writes
 *     x~ = A-hat^{-1} b-hat to xt, exactly as the device kernels do.
 * Toeplitz or block-entry LHS (CBS_LHS_BLOCK: partitions of whole points,
 * as cbs_plan_create makes them).  Errors: INVALID_ARG, UNSUPPORTED,
 * SINGULAR. */
cbs_status cbs_interface_model(const cbs_desc* desc, int32_t p, double* dhat, double* lhat,
                               double* uhat, const double* bhat, double* xt);

/* Ragged batch: up to `count` (<= 256) independent problems (each its own
 * cbs_desc, in and out arrays) solved together: by one persistent launch
 * over a work table, or by each problem's own launches (cbs_batch_set_mode).
 * Any problem cbs_plan_create takes can be batched (the batch pre-builds
 * every problem's plan).  The persistent launch takes: Toeplitz bands of
 * bandwidth 3 or 5; CBS_FP64 or CBS_FP32_REFINE with FP64 in and out, or
 * CBS_FP32 with FP32 in and out; the central stencil or the right-hand side
 * given; lines that fit one warp (on-chip plans), and long x-lines whose
 * plan runs a warp per segment (cbs_plan_info.segment_warp = 1: right-hand
 * side given, segments of 32 x 16 + r rows), which enter the work table as
 * (chunk of 4 segments, line) items.  A batch holding any other problem
 * runs per problem.  Allocates device memory, a stream and two events at
 * creation, none per solve.  Errors: those of cbs_plan_create for a
 * problem (the message names it). */
cbs_status cbs_batch_create(cbs_batch** out, const cbs_desc* descs, int32_t count);
cbs_status cbs_batch_destroy(cbs_batch* batch);
/* How cbs_batch_solve runs a batch (the results are the same: every problem
 * goes through its own plan's arithmetic):
 *   CBS_BATCH_PERSISTENT: one persistent launch over the work table of line
 *     tiles (the cheapest for many small problems: one launch in all);
 *   CBS_BATCH_PER_PROBLEM: each problem's own kernels, those cbs_solve runs
 *     for its plan (TMA tiles, pipelined lines, ...), the FP64 problems on a
 *     stream of the batch forked from `stream` and joined back into it
 *     within the call, so that they share the GPU with the others; one launch
 *     or more per problem;
 *   CBS_BATCH_AUTO (the default): per-problem launches when the problems
 *     hold 2^20 unknowns or more on average or the persistent launch does
 *     not take one of them, else the persistent launch.
 * Errors: INVALID_ARG (NULL, mode not 0..2), UNSUPPORTED (persistent
 * launch asked for a batch holding a problem it does not take; the message
 * names the first one). */
enum { CBS_BATCH_AUTO = 0, CBS_BATCH_PERSISTENT = 1, CBS_BATCH_PER_PROBLEM = 2 };
cbs_status cbs_batch_set_mode(cbs_batch* batch, int32_t mode);
/* ins[k] / outs[k]: device arrays of problem k (host array of `count`
 * pointers).  No allocation and no host synchronisation: capturable in a CUDA
 * graph when the pointers are fixed.  Per-problem launches need the device
 * current that the batch was created on (INVALID_ARG otherwise). */
cbs_status cbs_batch_solve(cbs_batch* batch, const void* const* ins,
                           void* const* outs, void* stream);
/* Read (and clear) the device status words of every problem of the batch,
 * as cbs_status_poll does for a plan; *device_status is the first non-OK
 * value found (problem order), else CBS_OK.  Synchronises the device. */
cbs_status cbs_batch_status_poll(cbs_batch* batch, int32_t* device_status);

/* Allocation-free variant of cbs_solve for long-line plans (cbs_plan_info
 * kernel == 1).  The paper has no counterpart: this serves callers that must
 * not call cudaMalloc when they solve -- applications that hand all device
 * memory to their own allocator at start-up, and loops with a fixed memory
 * footprint.  The solve's scratch (5 r doubles per segment of every line) is
 * one fixed 4 MiB array inside the library's device image instead of the
 * plan's buffer; lines x segments x 5 r above 524288 is rejected with
 * CBS_ERR_INVALID_ARG.  No cudaMalloc / cudaFree or other allocating call;
 * each call looks up the array's address in the current context.  All calls
 * share the array: calls whose launches may overlap on the GPU race with
 * each other, so order them (one stream, or events).  Plans that run a warp
 * per segment (cbs_plan_info.segment_warp = 1) use no scratch: the call then
 * runs that path for any plan size.  in / out / stream as for cbs_solve. */
cbs_status cbs_solve_noalloc(cbs_plan* plan, const void* in, void* out, void* stream);

/* Solves from host memory.  A pipe holds plans that read the same field
 * (same dims and input type: say the x, y and z derivatives of one field)
 * and, on the device, two input buffers and two output buffers per plan,
 * allocated by cbs_pipe_create (count 1..64; NO_MEMORY / CUDA on failure);
 * cbs_pipe_solve allocates nothing.  Each call copies host_in (the field,
 * host memory; page-locked for the copies to run asynchronously) to the
 * device on an internal upload stream, runs every plan's solve on `stream`,
 * and copies result k to host_outs[k] (host arrays of each plan's output
 * size and type) on an internal download stream as soon as solve k is done;
 * `stream` then waits for the downloads, so work issued on it after the call
 * -- or a synchronize of it -- sees the results in host memory.  Successive
 * calls alternate the device buffers: the upload of one call overlaps the
 * downloads of the previous one.  Call with the device current that the
 * pipe was created on.  Host buffers must stay valid until `stream` passes
 * the call.  The paper has no counterpart (its data live on the device). */
typedef struct cbs_pipe cbs_pipe;
cbs_status cbs_pipe_create(cbs_pipe** out, cbs_plan* const* plans, int32_t count);
cbs_status cbs_pipe_solve(cbs_pipe* pipe, const void* host_in, void* const* host_outs, void* stream);
/* Synchronises the device, then frees the pipe's buffers (not its plans). */
cbs_status cbs_pipe_destroy(cbs_pipe* pipe);

/* Measurement support for rooflines (not part of the method): the current
 * device's FP64 fused multiply-add throughput, timed with CUDA events on a
 * register-resident kernel of independent fma chains (4 CTAs of 256
 * threads per SM, 2^14 steps of 8 chains per thread, after a warm-up
 * launch).  Writes TFLOP/s (2 flops per fma) to *tflops.  Allocates and
 * frees a small device buffer; synchronises the device.  Errors:
 * INVALID_ARG, CUDA. */
cbs_status cbs_probe_fp64_peak(double* tflops);

/* Number of kernel launches the last cbs_solve / cbs_batch_solve of this
 * thread issued (for launch accounting). */
int32_t cbs_last_launch_count(void);

/* Description of the last error on the calling thread ("" if none). */
const char* cbs_last_error_string(void);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int32_t cbs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CBS_H */
