/*
 * oo_loadgen.c -- a C client of the serving loop (Sec. 3.3.1, Sec. 4.3.1:
 * C programs reach the common back end through its C ABI), built as a
 * shared object so that a load generator in another language can run it in
 * the same process, against the same serving context, beside its own
 * clients.  The client submits its share of a request stream at the given
 * arrival times with oo_submit, allocates every output buffer itself (as a
 * C program would), waits with oo_wait, and records per request the latency,
 * the status and a digest of the output words (XOR and sum of the 64-bit
 * words of each output array), so that its results can be compared bit for
 * bit with those of the other front ends.
 */
#define _POSIX_C_SOURCE 200809L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "oo.h"

/* input pools, by size index */
typedef struct {
    const double *gemm_a[16], *gemm_b[16];
    int32_t gemm_n[16];
    const double *fft_x[32];
    int32_t fft_log2[32];
    int32_t jac_i[8], jac_j[8], jac_k[8];
    int32_t jac_iters;
    int32_t prec;         /* GEMM pattern */
    int32_t client;       /* front-end tag written into every request */
    int32_t max_in_flight;
} oo_load_pools;

/* one request of the stream: kind (OO_BLOCK_*), size index into the pools,
 * arrival time (seconds on CLOCK_MONOTONIC) */
typedef struct {
    int32_t kind, size;
    double arrival;
} oo_load_item;

typedef struct {
    double latency_ms;
    int32_t status;
    int32_t pad;
    uint64_t digest_xor, digest_sum;
} oo_load_result;

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static void sleep_until(double t) {
    for (;;) {
        const double d = t - now_s();
        if (d <= 0.0) return;
        struct timespec ts;
        ts.tv_sec = (time_t)d;
        ts.tv_nsec = (long)((d - (double)ts.tv_sec) * 1e9);
        nanosleep(&ts, NULL);
    }
}

typedef struct {
    uint64_t ticket;
    int index;
    void *out;
    double *res;
    size_t out_words, res_words;
} pending;

static void digest(const void *p, size_t words, uint64_t *x, uint64_t *s) {
    const uint64_t *w = (const uint64_t *)p;
    for (size_t i = 0; i < words; ++i) {
        *x ^= w[i];
        *s += w[i];
    }
}

static void finish(oo_ctx *ctx, pending *q, oo_load_result *results) {
    oo_load_result *r = &results[q->index];
    double lat = 0.0;
    r->status = oo_wait(ctx, q->ticket, 600000, &lat);
    r->latency_ms = lat;
    r->digest_xor = 0;
    r->digest_sum = 0;
    if (r->status == OO_OK) {
        digest(q->out, q->out_words, &r->digest_xor, &r->digest_sum);
        if (q->res) digest(q->res, q->res_words, &r->digest_xor, &r->digest_sum);
    }
    free(q->out);
    free(q->res);
}

/* Submit items[0 .. n) in order at their arrival times, at most
 * max_in_flight unfinished (the oldest is waited for first); returns the
 * number of requests refused with OO_EBUSY (their status says so too). */
int oo_load_run(oo_ctx *ctx, const oo_load_pools *P, const oo_load_item *items, int n, oo_load_result *results) {
    const int cap = P->max_in_flight > 0 ? P->max_in_flight : 256;
    pending *ring = calloc((size_t)cap, sizeof(pending));
    int head = 0, count = 0, busy = 0;
    if (!ring) return -1;
    for (int i = 0; i < n; ++i) {
        const oo_load_item *it = &items[i];
        oo_serve_req r;
        memset(&r, 0, sizeof(r));
        r.client = P->client;
        r.kind = it->kind;
        pending q;
        memset(&q, 0, sizeof(q));
        q.index = i;
        if (it->kind == OO_BLOCK_GEMM) {
            const int64_t m = P->gemm_n[it->size];
            r.prec = P->prec;
            r.m = r.n = r.k = m;
            r.in0 = P->gemm_a[it->size];
            r.in1 = P->gemm_b[it->size];
            q.out_words = (size_t)(m * m);
            q.out = malloc(q.out_words * 8);
            r.out = q.out;
        } else if (it->kind == OO_BLOCK_FFT) {
            r.n = (int64_t)1 << P->fft_log2[it->size];
            r.dir = -1;
            r.in0 = P->fft_x[it->size];
            q.out_words = (size_t)r.n * 2;
            q.out = malloc(q.out_words * 8);
            r.out = q.out;
        } else {
            r.m = P->jac_i[it->size];
            r.n = P->jac_j[it->size];
            r.k = P->jac_k[it->size];
            r.iters = P->jac_iters;
            r.omega = 0.8f;
            const size_t pts = (size_t)(r.m * r.n * r.k);
            q.out_words = pts / 2; /* p is float: whole 64-bit words of it */
            q.out = malloc(pts * 4 + 8);
            r.out = q.out;
            q.res_words = (size_t)P->jac_iters;
            q.res = malloc(q.res_words * 8 + 8);
            r.res = q.res;
        }
        if (!q.out || (it->kind == OO_BLOCK_JACOBI && !q.res)) {
            free(q.out);
            free(q.res);
            results[i].status = OO_ENOMEM;
            continue;
        }
        sleep_until(it->arrival);
        const oo_status st = oo_submit(ctx, &r, &q.ticket);
        if (st != OO_OK) {
            results[i].status = st;
            results[i].latency_ms = 0.0;
            busy += st == OO_EBUSY;
            free(q.out);
            free(q.res);
            continue;
        }
        if (count == cap) {
            finish(ctx, &ring[head], results);
            head = (head + 1) % cap;
            --count;
        }
        ring[(head + count) % cap] = q;
        ++count;
    }
    while (count > 0) {
        finish(ctx, &ring[head], results);
        head = (head + 1) % cap;
        --count;
    }
    free(ring);
    return busy;
}
