// Genetic search over offload genes (Sec. 4.2.2).
//
// The paper fixes the outline: random 0/1 initial genes; measure each
// individual (out-of-tolerance results count as infinite time); fitness from
// time; select by fitness; make the next generation by crossover, mutation
// and copying as-is; repeat for the given number of generations; the fastest
// gene is the answer.  The details it leaves open are fixed as follows:
//   fitness t^(-1/2), 0 for infinite time; the fittest individual (first on
//   ties) is copied unchanged; parents are drawn by roulette over fitness
//   (uniformly when every fitness is 0); with probability pc a one-point
//   crossover at a cut drawn uniformly from [1, L-1] swaps the high parts of
//   the two parents; then each bit of each child flips with probability pm.
// Random numbers: xoshiro256** (Blackman & Vigna 2018), state from four
// splitmix64 draws (Steele, Lea & Flood 2014); a uniform is the top 53 bits
// scaled by 2^-53; randint(n) = floor(uniform * n); an initial gene bit is
// the top bit of one draw.
#include <cmath>

#include "oo_internal.h"

namespace oo {

uint64_t splitmix64(uint64_t &state) {
    state += 0x9e3779b97f4a7c15ull;
    uint64_t z = state;
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ull;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t v, int r) { return (v << r) | (v >> (64 - r)); }

void Rng::seed(uint64_t sd) {
    uint64_t st = sd;
    for (auto &w : s) w = splitmix64(st);
}

uint64_t Rng::next() {
    const uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
    const uint64_t sh = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= sh;
    s[3] = rotl64(s[3], 45);
    return out;
}

double Rng::uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }

int Rng::randint(int n) { return (int)(uniform() * (double)n); }

namespace {

int spin_roulette(Rng &rng, const std::vector<double> &fit) {
    double total = 0.0;
    for (double f : fit) total += f;
    const int pop = (int)fit.size();
    if (!(total > 0.0)) return rng.randint(pop);
    const double x = rng.uniform() * total;
    double acc = 0.0;
    int last_positive = 0;
    for (int i = 0; i < pop; ++i) {
        if (fit[i] > 0.0) last_positive = i;
        acc += fit[i];
        if (x < acc) return i;
    }
    return last_positive;
}

}  // namespace

GaResult ga_run(int L, int pop, int gens, double pc, double pm, uint64_t seed,
                const std::function<double(uint64_t)> &time_of) {
    OO_REQUIRE(L >= 1 && L <= 63, OO_EINVAL, "gene length must be 1..63");
    OO_REQUIRE(pop >= 1 && pop <= 4096 && gens >= 1, OO_EINVAL, "bad population / generations");
    OO_REQUIRE(pc >= 0 && pc <= 1 && pm >= 0 && pm <= 1, OO_EINVAL, "pc, pm must be in [0, 1]");
    Rng rng;
    rng.seed(seed);
    const uint64_t mask = (1ull << L) - 1ull;
    std::vector<uint64_t> cur(pop), nxt;
    for (auto &g : cur) {
        g = 0;
        for (int b = 0; b < L; ++b) g |= (rng.next() >> 63) << b;
    }
    GaResult r;
    r.history.reserve((size_t)gens * pop);
    bool seen = false;
    std::vector<double> fit(pop);
    for (int gen = 0; gen < gens; ++gen) {
        for (int i = 0; i < pop; ++i) {
            const double t = time_of(cur[i]);
            r.history.push_back(cur[i]);
            fit[i] = (std::isfinite(t) && t > 0.0) ? 1.0 / std::sqrt(t) : 0.0;
            if (!seen || t < r.best_time) {
                r.best_time = t;
                r.best_gene = cur[i];
                seen = true;
            }
        }
        if (gen + 1 == gens) break;
        int elite = 0;
        for (int i = 1; i < pop; ++i)
            if (fit[i] > fit[elite]) elite = i;
        nxt.clear();
        nxt.push_back(cur[elite]);
        while ((int)nxt.size() < pop) {
            const uint64_t a = cur[spin_roulette(rng, fit)];
            const uint64_t b = cur[spin_roulette(rng, fit)];
            uint64_t x = a, y = b;
            if (rng.uniform() < pc && L > 1) {
                const int cut = 1 + rng.randint(L - 1);
                const uint64_t lo = (1ull << cut) - 1ull;
                x = (a & lo) | (b & ~lo & mask);
                y = (b & lo) | (a & ~lo & mask);
            }
            for (int bit = 0; bit < L; ++bit)
                if (rng.uniform() < pm) x ^= 1ull << bit;
            for (int bit = 0; bit < L; ++bit)
                if (rng.uniform() < pm) y ^= 1ull << bit;
            nxt.push_back(x);
            if ((int)nxt.size() < pop) nxt.push_back(y);
        }
        cur.swap(nxt);
    }
    return r;
}

}  // namespace oo
