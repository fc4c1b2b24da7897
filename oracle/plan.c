/*
 * plan.c -- oracle for the CPU<->GPU transfer list a gene implies.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Sec. 4.2.2: data set on the CPU side and referenced on the GPU side must be
 * copied host->device; data set on the GPU side and referenced, set or
 * defined on the CPU side must be copied device->host.  Sec. 3.2.1: copies
 * are not repeated at inner nest levels when a variable allows moving them
 * to an upper level, so they happen once, in bulk.
 *
 * hoist = 1 is the lazy walk: each variable carries a valid flag per side;
 * a copy is made only right before a nest that needs the variable on a side
 * where it is stale.  hoist = 0 copies every GPU nest's reads (and the
 * variables it only partly overwrites) in before it and all it writes out
 * after it, as a per-region copy clause would.
 *
 * Parity: pinned by hand-derived plans for chosen genes and by the
 * executed-program invariant (tests/test_oracle_plan.py).
 */
#include "oracle.h"

static int emit(oracle_xfer *out, int cap, int n, int point, int var, int dir,
                uint64_t bytes)
{
    if (n < cap) {
        out[n].point = point;
        out[n].var = var;
        out[n].dir = dir;
        out[n].pad = 0;
        out[n].bytes = bytes;
    }
    return n + 1;
}

int oracle_plan(int n_nests, const int *level, const int *parallelisable,
                const uint64_t *reads, const uint64_t *writes,
                const uint64_t *partial, int n_vars, const uint64_t *var_bytes,
                uint64_t outputs, uint64_t gene, int hoist, int iters,
                oracle_xfer *out, int cap, uint64_t *h2d_total,
                uint64_t *d2h_total)
{
    if (n_nests < 1 || n_nests > 64 || n_vars < 1 || n_vars > 64 || iters < 0) return -1;
    int on_gpu[64];
    int g = 0;
    for (int n = 0; n < n_nests; ++n) {
        on_gpu[n] = 0;
        if (parallelisable[n]) {
            on_gpu[n] = (int)((gene >> g) & 1u);
            ++g;
        }
    }
    /* the invocation sequence: setup nests once, then the loop nests iters times */
    int seq_len = 0;
    for (int n = 0; n < n_nests; ++n) if (level[n] == 0) ++seq_len;
    int n_loop = 0;
    for (int n = 0; n < n_nests; ++n) if (level[n] == 1) ++n_loop;
    seq_len += n_loop * iters;

    int host_valid[64], dev_valid[64];
    for (int v = 0; v < n_vars; ++v) { host_valid[v] = 1; dev_valid[v] = 0; }
    uint64_t h2d = 0, d2h = 0;
    int nx = 0;
    int q = 0;
    for (int pass = -1; pass < iters; ++pass) {
        for (int n = 0; n < n_nests; ++n) {
            if (pass < 0 && level[n] != 0) continue;
            if (pass >= 0 && level[n] != 1) continue;
            uint64_t need = reads[n] | partial[n];
            if (hoist) {
                if (on_gpu[n]) {
                    for (int v = 0; v < n_vars; ++v)
                        if (((need >> v) & 1u) && !dev_valid[v]) {
                            nx = emit(out, cap, nx, q, v, +1, var_bytes[v]);
                            h2d += var_bytes[v];
                            dev_valid[v] = 1;
                        }
                    for (int v = 0; v < n_vars; ++v)
                        if ((writes[n] >> v) & 1u) { dev_valid[v] = 1; host_valid[v] = 0; }
                } else {
                    for (int v = 0; v < n_vars; ++v)
                        if (((need >> v) & 1u) && !host_valid[v]) {
                            nx = emit(out, cap, nx, q, v, -1, var_bytes[v]);
                            d2h += var_bytes[v];
                            host_valid[v] = 1;
                        }
                    for (int v = 0; v < n_vars; ++v)
                        if ((writes[n] >> v) & 1u) { host_valid[v] = 1; dev_valid[v] = 0; }
                }
            } else if (on_gpu[n]) {
                for (int v = 0; v < n_vars; ++v)
                    if ((need >> v) & 1u) {
                        nx = emit(out, cap, nx, q, v, +1, var_bytes[v]);
                        h2d += var_bytes[v];
                    }
                for (int v = 0; v < n_vars; ++v)
                    if ((writes[n] >> v) & 1u) {
                        nx = emit(out, cap, nx, q + 1, v, -1, var_bytes[v]);
                        d2h += var_bytes[v];
                    }
            }
            ++q;
        }
    }
    if (hoist) {
        for (int v = 0; v < n_vars; ++v)
            if (((outputs >> v) & 1u) && !host_valid[v]) {
                nx = emit(out, cap, nx, seq_len, v, -1, var_bytes[v]);
                d2h += var_bytes[v];
                host_valid[v] = 1;
            }
    }
    if (h2d_total) *h2d_total = h2d;
    if (d2h_total) *d2h_total = d2h;
    return nx;
}
