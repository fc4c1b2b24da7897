/*
 * ga.c -- oracle for the genetic search over offload genes.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Sec. 4.2.2: genes hold one bit per parallelisable loop (1 = GPU); the
 * initial population is random 0/1; each individual is measured (a result
 * outside tolerance counts as infinite time); fitness follows from time;
 * individuals are selected by fitness and the next generation is made by
 * crossover, mutation and copying as-is; after the given number of
 * generations the fastest gene is the answer.
 *
 * The paper leaves the operators' details open.  The readings used here
 * (and, written separately, by the library):
 *   fitness f = t^(-1/2), f = 0 for t = inf;
 *   the fittest individual (lowest index on ties) is copied unchanged;
 *   parents by roulette over f (uniform when all f are 0);
 *   one-point crossover with probability pc, cut c uniform in [1, L-1]:
 *     child1 = low c bits of parent a + high bits of parent b, child2 the
 *     converse; then each bit of each child flips with probability pm;
 *   random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded with four
 *     successive splitmix64 outputs (Steele, Lea & Flood, 2014);
 *     uniform u = (x >> 11) * 2^-53; randint(n) = floor(u * n);
 *     an initial gene bit is the top bit of one 64-bit output.
 *   The best gene is the lowest time seen; ties keep the earliest.
 *
 * Parity: pinned by the published splitmix64 output for seed 0 and by
 * special cases (pc = pm = 0, pm = 1, single-finite tables, elitism, roulette
 * frequencies) in tests/test_oracle_ga.py.
 */
#include "oracle.h"
#include <math.h>

uint64_t oracle_splitmix64(uint64_t *state)
{
    uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

void oracle_rng_seed(oracle_rng *r, uint64_t seed)
{
    uint64_t s = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = oracle_splitmix64(&s);
}

uint64_t oracle_rng_next(oracle_rng *r)
{
    uint64_t *s = r->s;
    const uint64_t result = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

static double uniform01(oracle_rng *r) { return (double)(oracle_rng_next(r) >> 11) * 0x1.0p-53; }
static int randint(oracle_rng *r, int n) { return (int)(uniform01(r) * (double)n); }

static int roulette(oracle_rng *r, const double *f, int pop)
{
    double total = 0.0;
    for (int i = 0; i < pop; ++i) total += f[i];
    if (total <= 0.0) return randint(r, pop);
    double x = uniform01(r) * total;
    double c = 0.0;
    int last = 0;
    for (int i = 0; i < pop; ++i) {
        if (f[i] > 0.0) last = i;
        c += f[i];
        if (x < c) return i;
    }
    return last;
}

int oracle_ga(int L, int pop, int gens, double pc, double pm, uint64_t seed,
              const double *time_of_gene, uint64_t *history,
              uint64_t *best_gene, double *best_time)
{
    if (L < 1 || L > 20 || pop < 1 || pop > 4096 || gens < 1) return -1;
    oracle_rng rng;
    oracle_rng_seed(&rng, seed);
    uint64_t cur[4096], nxt[4096];
    double f[4096];
    for (int i = 0; i < pop; ++i) {
        uint64_t gene = 0;
        for (int b = 0; b < L; ++b) gene |= (oracle_rng_next(&rng) >> 63) << b;
        cur[i] = gene;
    }
    uint64_t bg = cur[0];
    double bt = INFINITY;
    int have_best = 0;
    const uint64_t full = (L == 64) ? ~0ULL : ((1ULL << L) - 1ULL);
    for (int g = 0; g < gens; ++g) {
        for (int i = 0; i < pop; ++i) {
            const double t = time_of_gene[cur[i]];
            history[(size_t)g * pop + i] = cur[i];
            f[i] = (isfinite(t) && t > 0.0) ? 1.0 / sqrt(t) : 0.0;
            if (!have_best || t < bt) { bt = t; bg = cur[i]; have_best = 1; }
        }
        if (g == gens - 1) break;
        int elite = 0;
        for (int i = 1; i < pop; ++i) if (f[i] > f[elite]) elite = i;
        int m = 0;
        nxt[m++] = cur[elite];
        while (m < pop) {
            const uint64_t pa = cur[roulette(&rng, f, pop)];
            const uint64_t pb = cur[roulette(&rng, f, pop)];
            uint64_t c1 = pa, c2 = pb;
            if (uniform01(&rng) < pc && L > 1) {
                const int cut = 1 + randint(&rng, L - 1);
                const uint64_t low = (1ULL << cut) - 1ULL;
                c1 = (pa & low) | (pb & ~low & full);
                c2 = (pb & low) | (pa & ~low & full);
            }
            for (int b = 0; b < L; ++b) if (uniform01(&rng) < pm) c1 ^= 1ULL << b;
            for (int b = 0; b < L; ++b) if (uniform01(&rng) < pm) c2 ^= 1ULL << b;
            nxt[m++] = c1;
            if (m < pop) nxt[m++] = c2;
        }
        for (int i = 0; i < pop; ++i) cur[i] = nxt[i];
    }
    *best_gene = bg;
    *best_time = bt;
    return 0;
}
