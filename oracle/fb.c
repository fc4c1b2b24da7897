/*
 * fb.c -- the function-block offload decision (Sec. 4.2.1) and the trial
 * order (Sec. 4.2).  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Sec. 4.2.1: each replaceable block is measured offloaded and not, and
 * with several blocks every combination is measured; the fastest one is
 * kept.  A combination whose result fails the check counts as infinitely
 * slow (the rule of Sec. 4.2.2).  Here the measurements are given as a table
 * times[mask] over the 2^n combinations (bit i = block i offloaded); the
 * decision is the minimum, the first (lowest) mask on ties.
 */
#include <math.h>

#include "oracle.h"

int oracle_fb_best(int n_sites, const double *times, uint32_t *best_mask, double *best_time) {
    if (n_sites < 1 || n_sites > 20 || !times || !best_mask) return -1;
    uint32_t best = 0;
    const uint32_t count = 1u << n_sites;
    for (uint32_t m = 0; m < count; ++m) {
        if (isnan(times[m])) return -1;
        if (times[m] < times[best]) best = m;
    }
    *best_mask = best;
    if (best_time) *best_time = times[best];
    return 0;
}
