/*
 * oo.h -- C ABI of the GB300 offload-pattern library (liboo.so).
 *
 * The library executes "offload patterns" in the sense of Yamato, "Study of
 * Automatic GPU Offloading Method from Various Language Applications"
 * (arXiv:2011.03602):
 *   - loop offload (Sec. 3.2.1, Sec. 4.2.2): a gene holds one bit per
 *     parallelisable loop nest (1 = run on the GPU, 0 = on the CPU); the
 *     CPU<->GPU copies the placement implies are derived from which side sets
 *     and which side references each variable, and are hoisted to the
 *     outermost level the variable allows; a GA searches genes by measured
 *     time, a result outside tolerance counting as infinitely slow;
 *   - function-block offload (Sec. 3.2.2, Sec. 4.2.1): a callee found by name
 *     in a code-pattern table (a matrix product, a Fourier transform) is
 *     replaced by a GPU implementation behind a CPU-side interface;
 *   - the language-independent common part (Sec. 4.3): loop/variable tables,
 *     gene handling and name matching live here, behind one C ABI that C,
 *     Python (ctypes) and Java (JNI) front-ends call.
 *
 * Conventions for every entry point:
 *   - Every call returns an oo_status; OO_OK (0) on success, a negative code
 *     otherwise.  No C++ exception crosses this boundary.  On error the
 *     context's oo_last_error() holds a one-line description.
 *   - Host pointers are caller-owned and only read/written during the call.
 *     "_dev" variants take device pointers the caller owns (for example
 *     torch tensors' data_ptr()); work is queued on the context's stream and
 *     the call returns without synchronising unless stated otherwise.
 *   - The library owns the device memory and pinned host memory it allocates
 *     for its own workspaces and frees them in oo_destroy().
 *   - A context is used by one host thread at a time.
 *   - There is no CPU fallback: if the CUDA path fails, the call returns
 *     OO_ECUDA.  CPU execution of gene bits set to 0 is the method itself.
 */
#ifndef OO_H
#define OO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */
typedef int oo_status;
enum {
    OO_OK = 0,
    OO_EINVAL = -1,      /* bad argument (size, pointer, gene, mode)          */
    OO_ENOMEM = -2,      /* device or pinned host allocation failed           */
    OO_ECUDA = -3,       /* a CUDA call or kernel failed                      */
    OO_ETIMEOUT = -4,    /* a bounded device or host wait ran out             */
    OO_ETOLERANCE = -5,  /* result outside the correctness tolerance          */
    OO_EBUSY = -6,       /* no slot / memory free right now (back-pressure)   */
    OO_ENOTFOUND = -7,   /* name not in the code-pattern table                */
    OO_ESTATE = -8,      /* call not valid in the context's current state     */
    OO_EUSER = -9        /* a caller-supplied nest function reported failure  */
};

typedef struct oo_ctx oo_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to queue work on, or NULL for a stream the context creates
 * and owns.  *out receives the context.  OO_ECUDA if the device cannot be
 * used (no GPU, driver missing), OO_EINVAL for a NULL `out`.
 * device == -1 makes a host-only context: loop tables, transfer plans and
 * lookups work, any call that needs the GPU returns OO_ESTATE.             */
oo_status oo_create(int device, void *cuda_stream, oo_ctx **out);
/* Free every resource of the context (NULL is ignored). */
void oo_destroy(oo_ctx *ctx);
/* Static text for a status code. */
const char *oo_status_str(oo_status s);
/* Detail of the last error on this context; valid until the next call. */
const char *oo_last_error(const oo_ctx *ctx);
/* Block until all work queued on the context's stream is done. */
oo_status oo_sync(oo_ctx *ctx);

/* ----------------------------------------------- loop / variable table */
/* Sec. 4.3: loops and the variables each one reads and sets are kept in a
 * language-independent table.  A nest's variable sets are bit masks over
 * the variable list (at most 64 variables, 64 nests).
 *   level          0 = runs once before the loop, 1 = runs every iteration
 *   parallelisable 1 if the nest can run on the GPU at all (Sec. 4.2.2:
 *                  loops that fail to compile with a GPU directive get no
 *                  gene bit); the gene length is the count of these
 *   reads          variables the nest references
 *   writes         variables the nest sets
 *   partial        subset of writes that the nest only partly overwrites
 *                  (the rest of the variable must be current on the side
 *                  that runs the nest)                                      */
typedef struct {
    const char *name;
    uint64_t bytes;
} oo_var;

typedef struct {
    const char *name;
    int32_t level;
    int32_t parallelisable;
    uint64_t reads;
    uint64_t writes;
    uint64_t partial;
} oo_nest;

/* Replace the context's table.  `outputs` = variables the program's caller
 * reads on the host at the end.  *gene_len_out (may be NULL) receives the
 * gene length.  Copies the table; the caller keeps ownership of its arrays. */
oo_status oo_load_nests(oo_ctx *ctx, const oo_nest *nests, int n_nests,
                        const oo_var *vars, int n_vars, uint64_t outputs,
                        int *gene_len_out);

/* Load the table of the built-in Jacobi program (six nests: coef, pinit,
 * stencil, copyback, bc_ij, bc_k; fifteen variables a0..a3, b0..b2,
 * c0..c2, bnd, wrk1, p, wrk2, res) for an I x J x K grid and `iters`
 * iterations. */
oo_status oo_load_jacobi_nests(oo_ctx *ctx, int I, int J, int K, int iters,
                               int *gene_len_out);

/* One planned copy: before program point `point` (the point-th nest
 * invocation: setup nests once, then the loop nests `iters` times; point ==
 * number of invocations is the program end), copy variable `var` in
 * direction `dir` (+1 host->device, -1 device->host), `bytes` bytes.      */
typedef struct {
    int32_t point;
    int32_t var;
    int32_t dir;
    int32_t pad;
    uint64_t bytes;
} oo_xfer;

/* Sec. 4.2.2 transfer rules with Sec. 3.2.1 hoisting.  hoist = 1: a copy is
 * made only when the side about to run a nest lacks a current copy of a
 * variable the nest reads or partly writes (so loop-invariant data moves
 * once, outside the loop); hoist = 0: each GPU nest invocation copies its
 * reads and partial writes in and all its writes out.  Writes up to `cap`
 * records to `out` (may be NULL with cap 0 to count); *n_out receives the
 * full count, *h2d / *d2h (may be NULL) the byte totals.                  */
oo_status oo_transfer_plan(oo_ctx *ctx, uint64_t gene, int hoist, int iters,
                           oo_xfer *out, int cap, int *n_out, uint64_t *h2d,
                           uint64_t *d2h);

/* ------------------------------------------------ Jacobi offload patterns */
/* The loop program: a 19-point 3D Jacobi pressure solver on an I x J x K
 * float grid (k fastest).  Setup: a0=a1=a2=1, a3=1/6, b*=0, c*=1, bnd=1,
 * wrk1=0, p = wrk2 = (k/(K-1))^2.  Each iteration: stencil on the interior
 *   s0 = a0 p[i+1,j,k] + a1 p[i,j+1,k] + a2 p[i,j,k+1]
 *      + b0 Xij + b1 Xjk + b2 Xik + c0 p[i-1,j,k] + c1 p[i,j-1,k]
 *      + c2 p[i,j,k-1] + wrk1,
 *   Xuv = p(+u,+v) - p(+u,-v) - p(-u,+v) + p(-u,-v),
 *   ss = (s0 a3 - p) bnd,  res[it] += ss^2 (FP64),  wrk2 = p + omega ss;
 * copy-back p = wrk2 on the interior; faces reset to (k/(K-1))^2.
 * Per-point arithmetic is carried in float-float (about 44 significant
 * bits) and rounded once at each float store.                             */
typedef struct {
    int32_t I, J, K, iters;
    float omega;
    int32_t timing;       /* 1: record per-nest device times (adds events) */
} oo_jacobi;

typedef struct {
    double wall_ms;       /* whole pattern, host wall clock, synchronised   */
    double nest_ms[6];    /* per nest: summed event time (GPU) or host time */
    double xfer_ms;       /* host wall time spent waiting on copies          */
    uint64_t h2d_bytes;
    uint64_t d2h_bytes;
    int32_t n_xfers;
    int32_t n_launches;   /* kernels launched by the pattern                */
} oo_run_stats;

/* Run the Jacobi program with nest placement `gene` (bit b = nest b on the
 * GPU) and the transfer plan for `hoist`, synchronously.  p_out (host,
 * I*J*K floats) and res_out (host, iters doubles) receive the final
 * pressure and the per-iteration residuals; either may be NULL.  stats may
 * be NULL.  Grids need I, J, K >= 3; K <= 4096; iters >= 0.               */
oo_status oo_run_pattern(oo_ctx *ctx, uint64_t gene, int hoist,
                         const oo_jacobi *prob, float *p_out, double *res_out,
                         oo_run_stats *stats);

/* Same, but the results go to caller-owned DEVICE buffers (p_dev: I*J*K
 * floats, unpadded, k fastest; res_dev: iters doubles), so no final copy to
 * the host is made for GPU-resident results.  Synchronous.                */
oo_status oo_run_pattern_dev(oo_ctx *ctx, uint64_t gene, int hoist,
                             const oo_jacobi *prob, float *p_dev,
                             double *res_dev, oo_run_stats *stats);

/* ------------------------------------------------- generic loop programs */
/* Sec. 4.3: the method on any program described by the loaded table
 * (oo_load_nests).  The caller supplies the nests' bodies as one function:
 *   fn(user, nest, on_gpu, iter, vars, stream) runs nest `nest` (index in
 *   the table) for iteration `iter` (-1 for setup nests); on_gpu = 1: vars
 *   are the DEVICE buffers and the work must be enqueued on `stream` (the
 *   context's CUDA stream, a cudaStream_t), asynchronously; on_gpu = 0:
 *   vars are the HOST buffers and the work is done before returning.
 *   Returns 0, or nonzero to abort the run (OO_EUSER).                     */
typedef int (*oo_nest_fn)(void *user, int nest, int on_gpu, int64_t iter, void *const *vars,
                          void *stream);
/* Result check of a finished run on the host buffers: 0 = acceptable.    */
typedef int (*oo_check_fn)(void *user, void *const *host_vars);

/* Run the loaded program once: setup nests (level 0) once, then level-1
 * nests `iters` times, each on the side its gene bit chooses
 * (non-parallelisable nests on the CPU), with the copies of
 * oo_transfer_plan(gene, hoist, iters) made before each program point
 * between host_vars[v] and dev_vars[v] (caller-owned, vars[v].bytes each;
 * pinned host memory makes the copies asynchronous).  At the start the
 * host buffers hold the current values; at the end every table output is
 * current on the host.  A buffer may be NULL only for a variable no copy
 * and no nest on that side uses.  Synchronous; stats (may be NULL) gets the
 * wall time, copy bytes and count, and the number of GPU nest calls.       */
oo_status oo_run_program(oo_ctx *ctx, uint64_t gene, int hoist, int iters, oo_nest_fn fn, void *user,
                         void *const *host_vars, void *const *dev_vars, oo_run_stats *stats);

/* Sec. 4.2.2 GA over the loaded program's genes (gene length 1..20):
 * fitness from the measured wall time of oo_run_program, a gene whose
 * result fails `check` (may be NULL) counting as infinitely slow.  The host
 * buffers are re-initialised by the program's setup nests on every run, so
 * the program must compute all of its state from its setup nests.
 * history (gens x pop genes) and gene_ms (2^L, infinity = not measured or
 * failed) may be NULL.                                                    */
oo_status oo_ga_program(oo_ctx *ctx, int hoist, int iters, oo_nest_fn fn, oo_check_fn check, void *user,
                        void *const *host_vars, void *const *dev_vars, int pop, int gens, double pc,
                        double pm, uint64_t seed, uint64_t *best_gene, double *best_ms, uint64_t *history,
                        double *gene_ms);

/* One stencil sweep (nest N2) on caller-owned device arrays.  Every array is
 * I x J x pitch floats (pitch >= K, pitch % 4 == 0, k fastest, base 16-byte
 * aligned); coef points to 12 device pointers in the order a0 a1 a2 a3 b0
 * b1 b2 c0 c1 c2 bnd wrk1.  Writes wrk2 on the interior only and stores the
 * FP64 sum of ss^2 into *res_dev (device).  Asynchronous on the context's
 * stream; the tile variant is the context's (OO_OPT_STENCIL_VARIANT, else
 * the oo_tune_stencil choice for the grid, else the default rule).        */
oo_status oo_stencil_dev(oo_ctx *ctx, int I, int J, int K, int pitch,
                         const float *const *coef, const float *p, float omega,
                         float *wrk2, double *res_dev);
/* After oo_stencil_dev sweeps: synchronise the context's stream and report
 * OO_ETIMEOUT if a bounded pipeline wait of the last plan's sweeps ran out
 * (their wrk2 / residual are then incomplete); the error word is cleared. */
oo_status oo_stencil_check(oo_ctx *ctx);

/* The same stencil sweep as oo_stencil_dev, for callers that cannot
 * allocate device memory at the time they call: for example serving loops
 * that draw on a fixed, pre-reserved memory pool, or language runtimes that
 * own every device allocation.  The paper has no
 * counterpart; this is a deployment variant of the same nest.
 * It calls no cudaMalloc, cudaFree or allocating library routine: its
 * scratch (per-warp partial residuals, a completion counter, an error word)
 * lives in one static device array of 512 KB + 256 B that every device
 * loading the library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.
 * The first call looks the address up under a lock, so threads may make it
 * together; a device reset between calls invalidates the cached address.
 * Every call shares the array and clears its counter and error word first,
 * so calls that overlap on the GPU (other streams, other contexts on the
 * same device) race and must not be issued.  The tile variant and work
 * split are oo_stencil_dev's (same wrk2 bits; the same residual bits while
 * that split fits the array, else the residual is summed over fewer
 * i-segments and agrees to about 1e-12 relative).  Grids whose tiles
 * alone need more than 65536 partial slots (ceil((K-1)/TK) *
 * ceil((J-2)/TJ) * consumer warps; TK x TJ = 128 x 8 with 16 warps by
 * default for K > 65) are rejected with OO_EINVAL.  Arguments and layout as
 * for oo_stencil_dev; asynchronous on the context's stream.  A bounded
 * pipeline wait that runs out is reported by oo_stencil_noalloc_check, not
 * by this call.                                                          */
oo_status oo_stencil_noalloc_dev(oo_ctx *ctx, int I, int J, int K, int pitch,
                                 const float *const *coef, const float *p, float omega,
                                 float *wrk2, double *res_dev);
/* Synchronise the context's stream and report OO_ETIMEOUT if a bounded
 * pipeline wait of an oo_stencil_noalloc_dev sweep on this device ran out
 * since the last check (that sweep's wrk2 / residual are incomplete); the
 * word is cleared.  Allocates nothing.                                   */
oo_status oo_stencil_noalloc_check(oo_ctx *ctx);

/* Tile-shape autotuner for the stencil nest: times each of the
 * OO_STENCIL_VARIANTS tile variants (tile shape, consumer warps, points per
 * thread, CTAs per SM) for an I x J x K grid on the context's workspace (one
 * warm-up and three timed sweeps each, CUDA events on the context's
 * stream), and keeps the fastest for that grid: every later pattern run of
 * the context on that grid uses it, and so do the context's served Jacobi
 * requests (tune before oo_serve_start, not while serving).  All variants
 * compute bit-identical
 * results, so tuning changes speed only.  Outputs the chosen variant and,
 * if ms_per_variant is not NULL, the mean sweep time of each variant
 * (OO_STENCIL_VARIANTS entries).  Without tuning a grid uses the default
 * rule (variant 1 when K - 1 > 64, else 4), which is the tuner's choice at
 * the benchmarked sizes.  Synchronous.                                     */
enum { OO_STENCIL_VARIANTS = 5 };
oo_status oo_tune_stencil(oo_ctx *ctx, int I, int J, int K, int *variant, double *ms_per_variant);

/* Fault injection for tests of the bounded device waits; nothing faults,
 * traps or hangs.  Arms a one-shot failure on the context:
 *   OO_INJECT_STENCIL_LOAD  the next stencil sweep launched by
 *                           oo_run_pattern / oo_run_pattern_dev /
 *                           oo_stencil_dev / oo_stencil_noalloc_dev never
 *                           issues its first p-tile copy, so the consumer
 *                           warps' bounded wait (about one second) runs out;
 *   OO_INJECT_FUSED_BARRIER the next fused-iteration launch (small grids,
 *                           all iteration nests on the GPU) waits at its first
 *                           grid barrier for one block more than it launched.
 *   OO_INJECT_SERVE_STALL   the device-resident serving loop started next
 *                           (oo_serve_start_resident) gives the first request
 *                           it admits a work entry whose dependency never
 *                           completes, so the workers' bounded waits run out:
 *                           every request in flight fails with OO_ETIMEOUT.
 * Either kernel then sets its error word, waits (bounded) for its own copies
 * in flight and returns; the pattern call (or oo_stencil_check /
 * oo_stencil_noalloc_check after a single sweep) returns OO_ETIMEOUT and the
 * context stays usable.  OO_INJECT_NONE disarms; OO_EINVAL for other values. */
enum { OO_INJECT_NONE = 0, OO_INJECT_STENCIL_LOAD = 1, OO_INJECT_FUSED_BARRIER = 2, OO_INJECT_SERVE_STALL = 3 };
oo_status oo_inject_wait_timeout(oo_ctx *ctx, int what);

/* Context options (per context, never read from the process environment):
 *   OO_OPT_JACOBI_FUSED     -1 (default) fuse all iterations of the all-GPU
 *                           iteration nests into one cooperative launch for
 *                           grids of at most 2^20 points; 0 never; 1
 *                           whenever the placement and copies allow it.
 *   OO_OPT_STENCIL_VARIANT  -1 (default) the oo_tune_stencil choice for the
 *                           grid, else the default rule; 0 ..
 *                           OO_STENCIL_VARIANTS - 1 that tile variant for
 *                           every stencil sweep of the context (pattern
 *                           runs, oo_stencil_dev, oo_stencil_noalloc_dev,
 *                           served Jacobi requests started afterwards).
 *   OO_OPT_GEMM_PAIR        1 (default) the split-BF16 products of
 *                           oo_gemm_f64 / oo_gemm_f64_dev run on CTA pairs
 *                           (256-row tiles, each SM of a pair loading half
 *                           of the tile's B columns), the tile width (160,
 *                           192, 224 or 256 columns) chosen per problem;
 *                           160, 192, 224 or 256: CTA pairs with that tile
 *                           width; 0: single CTAs (128 x 128 tiles).  All
 *                           form the same products in the same order, so
 *                           the results are the same bits.
 * OO_EINVAL for an unknown option or value.                               */
enum { OO_OPT_JACOBI_FUSED = 1, OO_OPT_STENCIL_VARIANT = 2, OO_OPT_GEMM_PAIR = 3 };
oo_status oo_set_option(oo_ctx *ctx, int option, int value);
oo_status oo_get_option(oo_ctx *ctx, int option, int *value);

/* Device row pitch (floats) the library uses for a row of K floats. */
int oo_jacobi_pitch(int K);

/* ------------------------------------------------------------------- GA */
/* Sec. 4.2.2 GA over genes, with fitness from measured time.  Readings the
 * paper leaves open: fitness t^-1/2 (0 when the result failed the
 * tolerance check against the all-CPU run or the run exceeded
 * eval_timeout_ms); elitism 1; roulette selection; one-point crossover
 * (probability pc); per-bit mutation (probability pm); random numbers from
 * xoshiro256** seeded by splitmix64(seed).  Each distinct gene is measured
 * once.  history (gens*pop genes) and gene_ms (2^L entries, INFINITY for
 * genes never measured or failed) may be NULL.                            */
oo_status oo_ga_search(oo_ctx *ctx, const oo_jacobi *prob, int hoist, int pop,
                       int gens, double pc, double pm, uint64_t seed,
                       double eval_timeout_ms, uint64_t *best_gene,
                       double *best_ms, uint64_t *history, double *gene_ms);

/* oo_ga_search resumed from a saved table (checkpoint / resume): known_ms
 * has 2^6 entries, the gene_ms output of an earlier search (or any
 * measured times): a finite time or INFINITY is taken as that gene's
 * measured time and the gene is not run again; NaN marks a gene still to
 * be measured.  With the same seed and the same times the GA makes the same
 * choices, so a search interrupted after some evaluations continues where
 * it stopped.  A table that leaves no gene to measure needs no GPU (a
 * host-only context, device -1, will do).  OO_EINVAL for a NULL table or a
 * time <= 0.  Other arguments and outputs as for oo_ga_search.            */
oo_status oo_ga_search_resume(oo_ctx *ctx, const oo_jacobi *prob, int hoist, int pop,
                              int gens, double pc, double pm, uint64_t seed,
                              double eval_timeout_ms, const double *known_ms,
                              uint64_t *best_gene, double *best_ms,
                              uint64_t *history, double *gene_ms);

/* The same GA driven by a given time table time_of_gene[2^L] instead of
 * measurements (L <= 20).  No context needed.                             */
oo_status oo_ga_table(int L, int pop, int gens, double pc, double pm,
                      uint64_t seed, const double *time_of_gene,
                      uint64_t *history, uint64_t *best_gene,
                      double *best_time);

/* ------------------------------------------------------- function blocks */
enum { OO_BLOCK_GEMM = 1, OO_BLOCK_FFT = 2 };
enum { OO_LANG_C = 0, OO_LANG_PYTHON = 1, OO_LANG_JAVA = 2 };

/* Sec. 3.2.2 / Sec. 4.2.1 name match: look a callee name up in the
 * code-pattern table for language `lang`.  Spelling variants of a table
 * entry are accepted: Python import aliases (np., sp., la.) and module
 * re-exports, C BLAS names in any case, Java Class.method without its
 * package when that suffix names one block.  OO_ENOTFOUND if absent.     */
oo_status oo_lookup_block(const char *callee, int lang, int *block_id);

/* Sec. 3.2.2 matrix-product block: C = A B for FP64 row-major A (m x k,
 * leading dimension lda >= k), B (k x n, ldb >= n), C (m x n, ldc >= n).
 * An entry of C whose row of A or column of B holds a NaN or an infinity
 * is NaN (as a compensated FP64 dot product gives it); the other entries
 * are unaffected.  prec selects the precision pattern:
 *   OO_PREC_SPLIT3_BF16  A and B are scaled per row / column by powers of
 *                        two (a column of B whose largest entry lies in
 *                        [2^-20, 2^40) by 1) and split into BF16 hi + lo; C = A1 B1 +
 *                        (A1 B2 + A2 B1) on the tensor cores (FP32
 *                        accumulators in tensor memory), the two partial
 *                        products summed in FP64.  Error about 5e-5 of
 *                        sum_l |a_il b_lj| per element; callers needing
 *                        FP64 accuracy must not use this mode.
 *   OO_PREC_FP64EQ       FP64-equivalent (Ozaki-type splitting): every row
 *                        of A / column of B is cut into s signed BF16 digit
 *                        slices of beta bits relative to its power-of-two
 *                        scale; the products of slices with level p + q <= L
 *                        are formed on the tensor cores in K-blocks small
 *                        enough that FP32 accumulation is exact, and summed
 *                        in float-float before widening to FP64.  How the
 *                        products share FP32 accumulators is fixed by k
 *                        (oo_gemm_scheme), so a product gives the same bits
 *                        alone and inside a batch.  Error at
 *                        most ~2.3e-13 of sum_l |a_il b_lj| when the entries
 *                        of each row of A and column of B are of comparable
 *                        magnitude (bound ~4 (L+2) 2^(-beta (L-1)) of
 *                        k max_l|a_il| max_l|b_lj| in general).  oo_gemm_plan
 *                        reports beta, L and the number of BF16 products.
 *   OO_PREC_SPLIT3_TF32  the split-BF16 pattern with TF32 hi + lo operands
 *                        (FP32 with 10 fraction bits, rounded to nearest,
 *                        ties away; kind::tf32 tensor-core products, half the
 *                        BF16 rate): ~22 significant bits of every entry;
 *                        the error is about 1e-6 of sum_l |a_il b_lj| or
 *                        less (measured 3.1e-7 at k = 256, four times below
 *                        the BF16 pattern's; 8.6e-7 at k = 4096, where the
 *                        tensor cores' FP32 accumulation dominates both
 *                        split patterns).  Single calls only (batches and
 *                        the serving loops take the other two patterns).
 * oo_gemm_f64: host buffers, synchronous.                                 */
enum { OO_PREC_SPLIT3_BF16 = 0, OO_PREC_SPLIT3_TF32 = 1, OO_PREC_FP64EQ = 2 };
oo_status oo_gemm_f64(oo_ctx *ctx, int prec, int m, int n, int k, const double *A, int lda,
                      const double *B, int ldb, double *C, int ldc);
/* Device buffers (caller-owned), asynchronous on the context's stream; the
 * library's scratch for the split operands is reused across calls.        */
oo_status oo_gemm_f64_dev(oo_ctx *ctx, int prec, int m, int n, int k, const double *dA, int lda,
                          const double *dB, int ldb, double *dC, int ldc);
/* After oo_gemm_f64_dev calls of shape (m, n, k) in the precision pattern
 * last used on this context: synchronise and report OO_ETIMEOUT if a
 * bounded pipeline wait inside the kernel ran out.                        */
oo_status oo_gemm_check(oo_ctx *ctx, int m, int n, int k);
/* The tensor-core work of a product with inner dimension k in pattern prec:
 * number of BF16 products (each 2 m n k flops; 3 for SPLIT3), digit width
 * beta (bits, 0 for SPLIT3), level bound L (0 for SPLIT3) and the K-block
 * over which FP32 accumulation is exact (0 for SPLIT3).  No context needed;
 * any output pointer may be NULL.                                         */
oo_status oo_gemm_plan(int prec, int k, int *products, int *beta, int *levels, int *k_block);
/* How an FP64-equivalent product with inner dimension k accumulates its
 * digit products: OO_EQ_PAIRS (one FP32 accumulator per product, products
 * sharing an A slice paired into one MMA; k > 512) or OO_EQ_LEVELS (every
 * product of one level p + q summed in the same accumulator, which stays
 * exact because per_accumulator * k_block * (2^beta - 1)^2 < 2^24: 7-bit
 * digits and 128-deep K-blocks for k <= 128, 6-bit digits and 512-deep
 * K-blocks for k <= 512).  *per_accumulator (may be NULL) receives the
 * most products one accumulator sums (1 for pairs, L - 1 for levels).
 * The level schemes read fewer accumulators back, which is what bounds
 * products with short inner dimensions.  No context needed.              */
enum { OO_EQ_PAIRS = 0, OO_EQ_LEVELS = 1 };
oo_status oo_gemm_scheme(int k, int *scheme, int *per_accumulator);

/* Tile widths of the FP64-equivalent product in batches and in the single
 * products of a level scheme: output tiles are 128 rows by 32, 64 or 128
 * columns.  The width of a problem's full tiles is looked up by its n and k
 * in a table of OO_TILE_NBUCKETS x OO_TILE_KBUCKETS entries, entry
 * [nb * OO_TILE_KBUCKETS + kb] with nb for n <= 32, 64, 128, 256, 512 or
 * more and kb for k <= 64, 128, 256, 512 or more; a problem's last column
 * tile takes the narrowest width that covers it.  Widths change speed only,
 * never a result bit.  A context starts with the library's built-in table
 * (the autotuner's choices measured on GB300).
 * oo_tune_gemm_tiles: the autotuner.  For every bucket it times each width
 * on a synthetic group of products drawn in the bucket (one warm-up and
 * three timed launches, CUDA events on the context's stream), keeps the
 * fastest in the context's table and writes it to widths (may be NULL);
 * ms (may be NULL) receives OO_TILE_NBUCKETS x OO_TILE_KBUCKETS x 3 mean
 * launch times (widths 32, 64, 128).  Batches created afterwards use the
 * table.  Synchronous; allocates device memory for the trial.
 * oo_get_gemm_tiles / oo_set_gemm_tiles read / replace the context's table
 * (entries 32, 64 or 128, else OO_EINVAL).                                */
enum { OO_TILE_NBUCKETS = 6, OO_TILE_KBUCKETS = 5 };
oo_status oo_tune_gemm_tiles(oo_ctx *ctx, int *widths, double *ms);
oo_status oo_get_gemm_tiles(oo_ctx *ctx, int *widths);
oo_status oo_set_gemm_tiles(oo_ctx *ctx, const int *widths);

/* Sec. 3.2.2 Fourier-transform block: complex128 FFT of length n = 2^k,
 * 0 <= k <= 24, interleaved (re, im) doubles.  dir -1: forward,
 * X_k = sum_j x_j exp(-2 pi i jk/n); dir +1: inverse with exp(+...) and 1/n.
 * Butterflies run in float-float arithmetic (relative L2 error ~1e-14 for
 * normal inputs); inputs are scaled internally by powers of two (one per
 * transform, or per column of a long transform's first pass), so any finite
 * input is accepted (components more than ~2^126 below the transform's
 * largest one are flushed).  A transform of length n >= 2 with
 * a NaN or an infinity among its inputs gives NaN in every output component
 * (as the FP64 definition does); n = 1 returns its input unchanged.
 * oo_fft_c128: host buffers, synchronous; in may equal out.               */
oo_status oo_fft_c128(oo_ctx *ctx, int64_t n, int dir, const double *in, double *out);
/* batch contiguous transforms on caller device buffers (16-byte aligned,
 * batch * n complex values each; din may equal dout), asynchronous on the
 * context's stream.  batch <= 65535.                                      */
oo_status oo_fft_c128_dev(oo_ctx *ctx, int64_t n, int batch, int dir, const double *din,
                          double *dout);

/* ------------------------------------ function-block trial (Sec. 4.2.1) */
/* One call site of a library function in the source, as the code analysis
 * finds it: the callee's name (matched against the code-pattern table for
 * `lang`, oo_lookup_block), how often one program run calls it, and the
 * shape of its arguments.                                                  */
typedef struct {
    const char *callee;
    int32_t lang;        /* OO_LANG_*                                        */
    int32_t calls;       /* calls per program run, 1..1000                   */
    int64_t m, n, k;     /* GEMM: C (m x n) = A (m x k) B (k x n), each
                            1..8192; FFT: forward length n = 2^e <= 2^22     */
} oo_fb_site;

/* Sec. 4.2.1: every site whose callee the table knows is a candidate; each
 * combination of candidates offloaded (bit i of a mask = site i runs the
 * GPU block in precision pattern `prec`, host buffers, synchronous; the
 * other sites run the original CPU code, an OpenMP DGEMM / radix-2 FFT in
 * FP64) is run on seeded inputs of the sites' shapes (seed) and timed (wall
 * ms of all calls of the known sites).  An offloaded result that differs
 * from the all-CPU result by more than tol (GEMM: max |C-C*|/(|A||B|);
 * FFT: relative L2) makes that combination infinitely slow.
 * n_sites 1..12.  Outputs: block_ids[n_sites] (0 = not in the table; may
 * be NULL), mask_ms[2^n_sites] (infinity for masks that offload an unknown
 * site or fail tol; may be NULL), the fastest mask (ties: the lower mask)
 * and its time.                                                            */
oo_status oo_fb_search(oo_ctx *ctx, const oo_fb_site *sites, int n_sites, int prec, double tol,
                       uint64_t seed, int32_t *block_ids, double *mask_ms, uint32_t *best_mask,
                       double *best_ms);
/* The decision of oo_fb_search on a given table mask_ms[2^n_sites]
 * (infinity = not allowed), without measuring.  No context needed.         */
oo_status oo_fb_best(int n_sites, const double *mask_ms, uint32_t *best_mask, double *best_ms);
/* Sec. 4.2 trial order: function blocks first (oo_fb_search on the sites;
 * n_sites may be 0), then the loop GA (oo_ga_search) on the Jacobi
 * program's loop nests, which lie outside every library call site.
 * Outputs the fastest site mask with its time and the fastest loop gene
 * with its time.                                                           */
oo_status oo_offload_search(oo_ctx *ctx, const oo_fb_site *sites, int n_sites, int prec, double tol,
                            uint64_t seed, const oo_jacobi *prob, int hoist, int pop, int gens, double pc,
                            double pm, uint64_t ga_seed, double eval_timeout_ms, uint32_t *best_mask,
                            uint64_t *best_gene, double *fb_ms, double *loop_ms);

/* ----------------------------------------------------------------- serving */
/* Mixed requests from any number of client threads (C, Python ctypes, Java
 * JNI front-ends alike), admitted continuously onto the GPU: whenever one of
 * `slots` CUDA streams is free, the oldest waiting requests whose device
 * footprint fits the free part of a `hbm_budget_bytes` device arena start
 * (a request that has waited 50 ms at the head of the queue is not
 * overtaken); their copies and kernels overlap on the device.  Inputs are
 * copied into a pinned staging pool (as large as the budget) by oo_submit;
 * results are copied into the caller's buffer by oo_wait.
 *   kind OO_BLOCK_GEMM   : C (m x n) = A (m x k) B (k x n), host row-major
 *                          contiguous; in0 = A, in1 = B, out = C; prec
 *                          OO_PREC_SPLIT3_BF16 or OO_PREC_FP64EQ.
 *   kind OO_BLOCK_FFT    : length n, dir; in0 = x, out = X (complex128).
 *   kind OO_BLOCK_JACOBI : the Jacobi program on an m x n x k grid (I, J, K)
 *                          for `iters` iterations with `omega`, every nest
 *                          on the GPU; out = final p (I*J*K floats), res =
 *                          residuals (iters doubles, may be NULL).
 * Host buffers must stay valid until oo_wait returns for the ticket, and
 * every ticket must be waited for (that releases its staging).           */
enum { OO_BLOCK_JACOBI = 3 };
typedef struct {
    int32_t kind;
    int32_t prec;
    int64_t m, n, k;
    int32_t dir;
    int32_t iters;
    float omega;
    int32_t client;  /* front-end tag for the caller's statistics */
    const void *in0;
    const void *in1;
    void *out;
    double *res;
} oo_serve_req;
typedef struct {
    uint64_t submitted, completed, rejected_busy, failed, queued, running;
    uint64_t device_free_bytes, device_budget_bytes;
    /* mean time (ms) of completed requests in each stage: [0] queued (to
     * admission), [1] input copies, [2] staging until the work is published
     * (device-resident loop), [3] on the device (host-scheduled loop: from
     * its start on a slot, copies included), [4] output copies; 0 where a
     * loop has no such stage */
    double stage_ms[5];
} oo_serve_stats_t;
/* Start the scheduler thread; allocates the device arena and pinned pool. */
oo_status oo_serve_start(oo_ctx *ctx, int slots, uint64_t hbm_budget_bytes, int queue_cap);
/* Thread-safe.  OO_EBUSY: queue or staging pool full (back-pressure, retry
 * later); OO_EINVAL: malformed, or larger than the device budget.        */
oo_status oo_submit(oo_ctx *ctx, const oo_serve_req *req, uint64_t *ticket);
/* Thread-safe.  Waits up to timeout_ms; *latency_ms (may be NULL) is the
 * time from submission to completion.  OO_ETIMEOUT if not done in time (the
 * ticket stays valid); other errors are the request's own status.  Only one
 * thread may wait for a given ticket, and oo_serve_stop must not be called
 * while waits are in progress.                                           */
oo_status oo_wait(oo_ctx *ctx, uint64_t ticket, int timeout_ms, double *latency_ms);
oo_status oo_serve_stats(oo_ctx *ctx, oo_serve_stats_t *out);
/* Finish admitted and queued work, stop the scheduler, free the arena.
 * Tickets not yet waited for are discarded.  Stops either kind of service. */
oo_status oo_serve_stop(oo_ctx *ctx);

/* The same service (oo_submit, oo_wait, oo_serve_stats, oo_serve_stop) with
 * the request loop resident on the device: two persistent worker kernels are
 * launched here, once, and take their work from rings in device memory --
 * one of `tensor_ctas` CTAs (0: an eighth of the SMs) runs the tensor-core tiles of
 * FP64-equivalent GEMMs, the other (the remaining SMs, 512 threads each) the
 * digit splits, FFT passes and Jacobi sweeps.  A scheduler thread admits the
 * oldest waiting requests whose device footprint fits the free part of the
 * `hbm_budget_bytes` budget (a quarter of it holds GEMM digit slices),
 * copies their inputs, descriptors and work entries to the device and
 * publishes the entries through a control block in mapped host memory; it
 * launches no kernel per request.  Requests' entries interleave in the rings,
 * so requests that arrive while others run share the SMs (continuous
 * batching).  The workers write each finished request's flag to mapped
 * memory.  Inputs are copied from the caller's buffers to the device when a
 * request is admitted and outputs into them as soon as it completes, by the
 * library's I/O threads (no staging copy on the host), so the buffers must
 * stay valid until oo_wait returns.  Host threads: one scheduler, which
 * polls without sleeping while requests are in flight (it holds a host core
 * then; idle, it sleeps and wakes at least every millisecond), and four I/O
 * threads.  Served here: GEMMs in
 * OO_PREC_FP64EQ with k <= 2048 (the same bits as oo_gemm_f64), FFTs up to
 * 2^22 points (the same bits as oo_fft_c128), Jacobi programs (the tiled
 * kernels' p bits; residuals summed in chunk order, within ~1e-12 relative of
 * the tiled kernels'); other requests give OO_EINVAL.  Every device wait is
 * bounded (about a second); an idle server publishes keep-alive entries.
 * If a wait runs out, every request in flight fails with OO_ETIMEOUT and
 * later submissions with OO_ESTATE until oo_serve_stop.  While serving, the
 * workers hold every SM of the device: the context's other GPU calls return
 * OO_ESTATE until oo_serve_stop (a kernel loaded lazily at its first launch
 * could wait for the workers).  OO_ESTATE if the context already serves.  */
oo_status oo_serve_start_resident(oo_ctx *ctx, uint64_t hbm_budget_bytes, int queue_cap, int tensor_ctas);

/* ------------------------------------------------------- serving replicas */
/* Requests routed over several serving contexts (one per GPU; each already
 * serving with oo_serve_start or oo_serve_start_resident) by free device
 * memory (Sec. 3: the same method on whichever destination is free):
 * requests are independent, so replicas share nothing.  A replica's free
 * bytes are its arena's free bytes, but at most its budget less the
 * footprints (oo_serve_footprint) of the requests this router sent there and
 * that are not yet waited for (queued requests do not occupy the arena yet).
 * A request goes to the replica with the most free bytes among those with
 * room for its footprint (ties: fewer requests queued or running there, then the
 * lower index); when none has room, to the replica with the fewest requests
 * in flight, where it queues.  On OO_EBUSY or OO_ESTATE from that replica the
 * next best is tried.  The contexts stay owned by the caller and must
 * outlive the router.  Thread-safe.                                        */
typedef struct oo_router oo_router;
oo_status oo_router_create(oo_ctx *const *ctxs, int n, oo_router **out);
/* *replica: the index (into ctxs) that took the request, for oo_router_wait */
oo_status oo_router_submit(oo_router *r, const oo_serve_req *req, int *replica, uint64_t *ticket);
oo_status oo_router_wait(oo_router *r, int replica, uint64_t ticket, int timeout_ms, double *latency_ms);
void oo_router_destroy(oo_router *r);
/* The routing decision alone, host-only: free_bytes[n] and queued[n] (queued
 * or running) per replica, `need` the request's footprint -> *replica.       */
oo_status oo_route_pick(const uint64_t *free_bytes, const uint64_t *queued, int n, uint64_t need, int *replica);
/* m requests routed in order, each decision charging its replica with the
 * request's bytes and one more request in flight: with one process per GPU,
 * every process computes the same owners from the same all-gathered figures
 * and serves the requests it owns.  Host-only.                             */
oo_status oo_route_batch(const uint64_t *free_bytes, const uint64_t *queued, int n, const uint64_t *needs, int m,
                         int *replicas);
/* The routing estimate of a request's device footprint (bytes).  Host-only. */
oo_status oo_serve_footprint(const oo_serve_req *req, uint64_t *bytes);

/* --------------------------------------------------- batched function blocks */
/* Many GEMM and FFT requests of uneven sizes, on caller-owned device buffers.
 *   GEMM (kind OO_BLOCK_GEMM): C (m x n) = A (m x k) B (k x n), row-major,
 *        contiguous (leading dimensions k, n, n); in0 = A, in1 = B, out = C;
 *        prec OO_PREC_SPLIT3_BF16 (all such requests share the grouped
 *        split-BF16 tensor-core kernel) or OO_PREC_FP64EQ (m, n, k <=
 *        65536; all such requests share one split launch and one grouped
 *        FP64-equivalent tensor-core launch, with tile widths from the
 *        context's table, oo_tune_gemm_tiles).
 *   FFT  (kind OO_BLOCK_FFT): length n = 2^e (e <= 24), in0 = x, out = X
 *        (interleaved complex128, 16-byte aligned), dir -1 / +1; m, k unused.
 * oo_batch_create builds the grouped plan once (tensor maps, split-operand
 * arena, tile and item lists; it allocates device memory).                */
typedef struct {
    int32_t kind;
    int32_t prec;
    int64_t m, n, k;
    const void *in0;
    const void *in1;
    void *out;
    int32_t dir;
    int32_t pad;
} oo_req;
typedef struct oo_batch oo_batch;
oo_status oo_batch_create(oo_ctx *ctx, const oo_req *reqs, int n_req, oo_batch **out);
/* mode 0: grouped persistent kernels (GEMM split passes + one tensor-core
 *         kernel over every split-BF16 tile, one split launch + one
 *         tensor-core kernel over every FP64-equivalent tile; FFT maxima
 *         pass + three item launches), the GEMM and FFT groups on forked
 *         streams;
 * mode 1: the same, captured into a CUDA graph on first use and replayed;
 * mode 2: one library call per request (oo_gemm_f64_dev / oo_fft_c128_dev).
 * Asynchronous on the context's stream.                                  */
oo_status oo_batch_run(oo_batch *b, int mode);
/* Synchronise; OO_ETIMEOUT if a bounded wait in a grouped kernel ran out. */
oo_status oo_batch_check(oo_batch *b);
/* Totals of the batch: 2 m n k summed over GEMMs (both patterns), points
 * summed over FFTs. */
oo_status oo_batch_info(const oo_batch *b, double *gemm_flops, double *fft_points, int *n_gemm,
                        int *n_fft);
void oo_batch_destroy(oo_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* OO_H */
