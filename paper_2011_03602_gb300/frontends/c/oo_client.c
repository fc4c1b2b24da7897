/*
 * oo_client.c -- the C front-end of the offload library (Sec. 3.3.1, Sec.
 * 4.3.1: a C program's loops and function blocks offloaded through the
 * common, language-independent part).  It links liboo.so and:
 *   1. looks its callees up in the code-pattern table (Sec. 4.2.1),
 *   2. runs one offload pattern of the Jacobi program (all nests on the GPU,
 *      hoisted transfers) and prints the residuals,
 *   3. calls the GEMM and FFT function blocks on host buffers,
 *   4. submits a mixed batch to the serving loop from NTHREADS threads.
 * Output is one line per step, "key value ...", for the test that runs it.
 * Usage: oo_client [device]
 */
#define _POSIX_C_SOURCE 200809L
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oo.h"

#define CHECK(x)                                                                      \
    do {                                                                              \
        oo_status s_ = (x);                                                           \
        if (s_ != OO_OK) {                                                            \
            fprintf(stderr, "%s failed: %s (%s)\n", #x, oo_status_str(s_),            \
                    oo_last_error(ctx));                                              \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

#define NTHREADS 3
#define PER_THREAD 8

static uint64_t sm_state = 12345;
static double uniform(void) {  /* splitmix64 -> [0, 1) */
    uint64_t z = (sm_state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

typedef struct {
    oo_ctx *ctx;
    int tag;
    int ok;
    double worst_latency_ms;
} client_arg;

static void *client(void *p) {
    client_arg *a = (client_arg *)p;
    enum { N = 96 };
    double *A = malloc(sizeof(double) * N * N), *B = malloc(sizeof(double) * N * N);
    double *C = malloc(sizeof(double) * N * N * PER_THREAD);
    uint64_t tickets[PER_THREAD];
    for (int i = 0; i < N * N; ++i) {
        A[i] = (double)((i * 7 + a->tag) % 17) - 8.0; /* small integers: exact products */
        B[i] = (double)((i * 5 + 3 * a->tag) % 13) - 6.0;
    }
    a->ok = 1;
    for (int r = 0; r < PER_THREAD; ++r) {
        oo_serve_req q;
        memset(&q, 0, sizeof(q));
        q.kind = OO_BLOCK_GEMM;
        q.prec = OO_PREC_SPLIT3_BF16;
        q.m = q.n = q.k = N;
        q.client = OO_LANG_C;
        q.in0 = A;
        q.in1 = B;
        q.out = C + (size_t)r * N * N;
        while (oo_submit(a->ctx, &q, &tickets[r]) == OO_EBUSY) {
        }
    }
    for (int r = 0; r < PER_THREAD; ++r) {
        double lat = 0;
        if (oo_wait(a->ctx, tickets[r], 60000, &lat) != OO_OK) a->ok = 0;
        if (lat > a->worst_latency_ms) a->worst_latency_ms = lat;
        /* check one entry exactly: small-integer products are exact */
        const int i = (r * 31) % N, j = (r * 17) % N;
        double ref = 0;
        for (int l = 0; l < N; ++l) ref += A[i * N + l] * B[l * N + j];
        if (C[(size_t)r * N * N + i * N + j] != ref) a->ok = 0;
    }
    free(A);
    free(B);
    free(C);
    return NULL;
}

int main(int argc, char **argv) {
    const int device = argc > 1 ? atoi(argv[1]) : 0;
    oo_ctx *ctx = NULL;
    if (oo_create(device, NULL, &ctx) != OO_OK) {
        fprintf(stderr, "oo_create failed: %s\n", oo_last_error(NULL));
        return 1;
    }
    /* 1. code-pattern lookup of this program's callees */
    int gemm_block = 0, fft_block = 0;
    CHECK(oo_lookup_block("cblas_dgemm", OO_LANG_C, &gemm_block));
    CHECK(oo_lookup_block("fftw_execute", OO_LANG_C, &fft_block));
    printf("lookup %d %d\n", gemm_block, fft_block);

    /* 2. an offload pattern of the Jacobi program */
    const int I = 33, J = 33, K = 65, iters = 10;
    oo_jacobi prob = {I, J, K, iters, 0.8f, 0};
    float *p = malloc(sizeof(float) * I * J * K);
    double res[10];
    oo_run_stats st;
    CHECK(oo_run_pattern(ctx, 0x3f, 1, &prob, p, res, &st));
    printf("pattern %.17g %.17g %llu\n", res[0], res[iters - 1], (unsigned long long)st.d2h_bytes);

    /* 3. function blocks on host buffers */
    enum { M = 64 };
    double *A = malloc(sizeof(double) * M * M), *Cm = malloc(sizeof(double) * M * M);
    for (int i = 0; i < M * M; ++i) A[i] = 2.0 * uniform() - 1.0;
    double *I64 = calloc(M * M, sizeof(double));
    for (int i = 0; i < M; ++i) I64[i * M + i] = 1.0;
    CHECK(oo_gemm_f64(ctx, OO_PREC_SPLIT3_BF16, M, M, M, A, M, I64, M, Cm, M));
    double maxerr = 0;
    for (int i = 0; i < M * M; ++i) maxerr = fmax(maxerr, fabs(Cm[i] - A[i]));
    printf("gemm_identity_maxerr %.3e\n", maxerr);
    enum { NF = 4096 };
    double *x = malloc(sizeof(double) * 2 * NF), *X = malloc(sizeof(double) * 2 * NF);
    for (int t = 0; t < NF; ++t) {
        x[2 * t] = cos(2.0 * 3.14159265358979323846 * 37.0 * t / NF);
        x[2 * t + 1] = sin(2.0 * 3.14159265358979323846 * 37.0 * t / NF);
    }
    CHECK(oo_fft_c128(ctx, NF, -1, x, X));
    printf("fft_tone %.12f %.3e\n", X[2 * 37], fabs(X[2 * 38]) + fabs(X[2 * 38 + 1]));

    /* 4. serving from NTHREADS client threads */
    CHECK(oo_serve_start(ctx, 4, (uint64_t)256 << 20, 64));
    pthread_t th[NTHREADS];
    client_arg args[NTHREADS];
    for (int t = 0; t < NTHREADS; ++t) {
        args[t].ctx = ctx;
        args[t].tag = t;
        args[t].ok = 0;
        args[t].worst_latency_ms = 0;
        pthread_create(&th[t], NULL, client, &args[t]);
    }
    int all_ok = 1;
    double worst = 0;
    for (int t = 0; t < NTHREADS; ++t) {
        pthread_join(th[t], NULL);
        all_ok &= args[t].ok;
        if (args[t].worst_latency_ms > worst) worst = args[t].worst_latency_ms;
    }
    oo_serve_stats_t ss;
    CHECK(oo_serve_stats(ctx, &ss));
    printf("serve %d %llu %.3f\n", all_ok, (unsigned long long)ss.completed, worst);
    CHECK(oo_serve_stop(ctx));

    free(p);
    free(A);
    free(Cm);
    free(I64);
    free(x);
    free(X);
    oo_destroy(ctx);
    printf("done\n");
    return 0;
}
