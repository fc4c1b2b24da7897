/*
 * oracle.h -- plain, slow, obviously-correct FP64 C oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA/C++ library under paper_2011_03602_gb300/.
 *
 * What it computes (paper: Yamato, "Study of Automatic GPU Offloading Method
 * from Various Language Applications"):
 *   - the loop program whose parallelisable nests a gene places on CPU or GPU
 *     (Sec. 3.2.1, Sec. 4.2.2): a 19-point 3D Jacobi pressure solver
 *     (coefficient setup, stencil update with residual, copy-back, boundary);
 *   - the CPU<->GPU transfer list a gene implies, with and without hoisting
 *     transfers to the outermost level the variable allows (Sec. 3.2.1,
 *     Sec. 4.2.2);
 *   - the GA over genes (Sec. 4.2.2): random initial genes, fitness from
 *     time, selection, crossover, mutation, copy-as-is, generations;
 *   - the function blocks a code-pattern lookup replaces (Sec. 3.2.2):
 *     dense matrix product and complex FFT, in FP64.
 *
 * Parity status of each function is stated beside it and in the design notes.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- Jacobi */
/* Coefficient array order, 12 arrays of I*J*K floats, k fastest:
 *   0..3 a0..a3, 4..6 b0..b2, 7..9 c0..c2, 10 bnd, 11 wrk1.                */
enum { ORC_NCOEF = 12 };

/* Fill the coefficient arrays and p as the setup nests define them:
 * a0=a1=a2=1, a3=fl32(1/6), b*=0, c*=1, bnd=1, wrk1=0;
 * p[i,j,k] = fl32(k^2 / (K-1)^2).                                          */
void oracle_jacobi_setup(int I, int J, int K, float *coef12, float *p);

/* One stencil sweep (nest N2) over the interior, in FP64 arithmetic on the
 * float inputs.  wrk2_out (I*J*K doubles) receives p + omega*ss on the
 * interior and p elsewhere (exact FP64 values, not rounded).  *res_out is
 * the FP64 sum of ss^2 in i-j-k order.  p is given in double so the same
 * routine serves the FP64-storage mode.                                      */
void oracle_stencil(int I, int J, int K, const float *coef12, const double *p,
                    double omega, double *wrk2_out, double *res_out);

/* The whole Jacobi program: setup, then iters x (stencil, copy-back,
 * boundary faces).  mode 0: p and wrk2 kept in FP64 ("oracle-64");
 * mode 1: every store of p and wrk2 rounded to float ("oracle-s32").
 * coef12 / p0 may be NULL for the setup values.  res_out[iters];
 * p_out[I*J*K] may be NULL.  Returns 0 on success, -1 on bad sizes.         */
int oracle_jacobi_run(int I, int J, int K, int iters, float omega, int mode,
                      const float *coef12, const float *p0,
                      double *res_out, double *p_out);

/* --------------------------------------------------------- transfer plan */
typedef struct {
    int32_t point;   /* program point the copy runs before (see below)   */
    int32_t var;     /* variable index                                    */
    int32_t dir;     /* +1 host->device, -1 device->host                  */
    int32_t pad;
    uint64_t bytes;
} oracle_xfer;

/* Program order: setup nests (level 0) once in table order, then `iters`
 * passes over the loop nests (level 1) in table order.  Program point q is
 * the q-th nest invocation; point == n_invocations is the program end.
 * gene bit g belongs to the g-th parallelisable nest (1 = GPU).
 * Per nest: reads, writes (full overwrite), partial (writes that keep the
 * rest of the variable; a subset of writes) as variable bit masks.
 * outputs: variables that must be valid on the host at the end.
 * hoist 1: a copy happens only when the executing side lacks a valid copy
 *          (transfers rise to the outermost point the data flow allows);
 * hoist 0: every GPU nest invocation copies its reads and partial writes in
 *          and all of its writes out.
 * Returns the number of transfers (written up to cap), -1 on bad input.   */
int oracle_plan(int n_nests, const int *level, const int *parallelisable,
                const uint64_t *reads, const uint64_t *writes,
                const uint64_t *partial, int n_vars, const uint64_t *var_bytes,
                uint64_t outputs, uint64_t gene, int hoist, int iters,
                oracle_xfer *out, int cap, uint64_t *h2d_total,
                uint64_t *d2h_total);

/* --------------------------------------------------------------------- GA */
uint64_t oracle_splitmix64(uint64_t *state);
/* xoshiro256** seeded from four successive splitmix64(seed) outputs. */
typedef struct { uint64_t s[4]; } oracle_rng;
void oracle_rng_seed(oracle_rng *r, uint64_t seed);
uint64_t oracle_rng_next(oracle_rng *r);

/* GA over genes of length L (<= 20) with a fitness table time_of_gene[2^L]
 * (INFINITY = failed the correctness gate).  history[g*pop + i] receives the
 * gene of individual i evaluated in generation g.  Returns 0 on success.    */
int oracle_ga(int L, int pop, int gens, double pc, double pm, uint64_t seed,
              const double *time_of_gene, uint64_t *history,
              uint64_t *best_gene, double *best_time);

/* ----------------------------------------------------------- FB: GEMM */
/* C = A*B, row-major, A m x k (lda), B k x n (ldb), C m x n (ldc).
 * Each dot product is a compensated (Dot2) FP64 sum.  rows [r0, r1) only. */
void oracle_gemm(int m, int n, int k, const double *A, int lda,
                 const double *B, int ldb, double *C, int ldc, int r0, int r1);

/* ------------------------------------------------------------ FB: FFT */
/* Interleaved complex (re, im).  dir -1: X_k = sum_n x_n e^{-2 pi i nk/N};
 * dir +1: x_n = (1/N) sum_k X_k e^{+2 pi i nk/N}.                         */
void oracle_dft(int64_t n, int dir, const double *in, double *out);
/* Recursive radix-2 FFT, n a power of two, same conventions.  0 / -1.    */
int oracle_fft(int64_t n, int dir, const double *in, double *out);

/* --------------------------------------------- function-block decision */
/* Sec. 4.2.1: given times[2^n_sites] of every combination of offloaded
 * blocks (bit i = block i on the GPU; INFINITY = result failed the check or
 * not replaceable), the fastest combination, the lowest mask on ties.
 * Returns -1 on bad arguments or a NaN entry.  Parity: pinned by hand-made
 * tables (tests/test_fb.py).                                             */
int oracle_fb_best(int n_sites, const double *times, uint32_t *best_mask, double *best_time);

#ifdef __cplusplus
}
#endif
#endif
