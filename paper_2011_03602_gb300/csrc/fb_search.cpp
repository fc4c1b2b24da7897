// Function-block offload trial and the whole trial order (Sec. 4.2,
// Sec. 4.2.1).
//
// The method tries function-block offload before loop offload, since a
// block replaced by a GPU implementation written for its algorithm beats
// offloading its loops one by one (Sec. 4.2).  Every call site whose callee
// the code-pattern table knows is a candidate; each candidate is measured
// offloaded and not offloaded and, when there are several, every
// combination of them is measured too (Sec. 4.2.1).  A combination whose
// results differ from the all-CPU run beyond the tolerance counts as
// infinitely slow, like a failing loop pattern (Sec. 4.2.2).  The loop GA
// then runs on the code outside the offloaded blocks, and the fastest
// pattern is the answer (Sec. 4.2).
//
// Not-offloaded sites run the program's original CPU code: here a plain
// OpenMP DGEMM and an iterative radix-2 FFT in FP64 (stand-ins for the CPU
// library the source calls).  Inputs are seeded synthetic data of the
// sites' shapes.  Sites the table does not know keep their CPU code in
// every combination, so they add the same time to each and are not run.
#include <omp.h>

#include <chrono>
#include <cmath>
#include <complex>
#include <limits>
#include <vector>

#include "oo_internal.h"

namespace oo {

namespace {

void cpu_dgemm(int m, int n, int k, const double *A, const double *B, double *C) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        double *c = C + (size_t)i * n;
        for (int j = 0; j < n; ++j) c[j] = 0.0;
        for (int l = 0; l < k; ++l) {
            const double a = A[(size_t)i * k + l];
            const double *b = B + (size_t)l * n;
            for (int j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

// in place, iterative radix-2 decimation in time, e^{-2 pi i jk/n}
void cpu_fft(long long n, std::complex<double> *x) {
    for (long long i = 1, j = 0; i < n; ++i) {
        long long bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(x[i], x[j]);
    }
    std::vector<std::complex<double>> w;
    for (long long len = 2; len <= n; len <<= 1) {
        const long long half = len >> 1;
        w.resize(half);
        for (long long t = 0; t < half; ++t) {
            const double ang = -6.283185307179586 * (double)t / (double)len;
            w[t] = std::complex<double>(std::cos(ang), std::sin(ang));
        }
#pragma omp parallel for schedule(static) if (n >= (1 << 14))
        for (long long s = 0; s < n; s += len)
            for (long long t = 0; t < half; ++t) {
                const std::complex<double> u = x[s + t], v = x[s + t + half] * w[t];
                x[s + t] = u + v;
                x[s + t + half] = u - v;
            }
    }
}

struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    double sym() { return 2.0 * (double)(next() >> 11) * 0x1.0p-53 - 1.0; }  // [-1, 1)
};

struct Site {
    int block = 0;
    std::vector<double> a, b, ref, out, absab;
};

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

void fb_trial(const oo_fb_site *sites, int n_sites, int prec, double tol, uint64_t seed,
              std::vector<double> &mask_ms, std::vector<int> &block_ids, const FbGpu &gpu) {
    OO_REQUIRE(n_sites >= 1 && n_sites <= 12, OO_EINVAL, "1..12 function-block sites");
    OO_REQUIRE(sites != nullptr, OO_EINVAL, "null site list");
    OO_REQUIRE(tol > 0.0, OO_EINVAL, "tolerance must be positive");
    std::vector<Site> D(n_sites);
    block_ids.assign(n_sites, 0);
    SplitMix rng{seed};
    uint32_t cand = 0;
    for (int i = 0; i < n_sites; ++i) {
        const oo_fb_site &s = sites[i];
        const std::string at = "site " + std::to_string(i) + ": ";
        OO_REQUIRE(s.callee != nullptr, OO_EINVAL, at + "null callee");
        OO_REQUIRE(s.lang >= OO_LANG_C && s.lang <= OO_LANG_JAVA, OO_EINVAL, at + "unknown language");
        OO_REQUIRE(s.calls >= 1 && s.calls <= 1000, OO_EINVAL, at + "calls must be 1..1000");
        Site &d = D[i];
        d.block = lookup_block(s.callee, s.lang);
        block_ids[i] = d.block;
        if (d.block == OO_BLOCK_GEMM) {
            OO_REQUIRE(s.m >= 1 && s.n >= 1 && s.k >= 1 && s.m <= 8192 && s.n <= 8192 && s.k <= 8192, OO_EINVAL,
                       at + "GEMM dimensions must be 1..8192");
            const size_t m = s.m, n = s.n, k = s.k;
            d.a.resize(m * k);
            d.b.resize(k * n);
            for (auto &v : d.a) v = rng.sym();
            for (auto &v : d.b) v = rng.sym();
            d.ref.resize(m * n);
            d.out.resize(m * n);
            cpu_dgemm((int)m, (int)n, (int)k, d.a.data(), d.b.data(), d.ref.data());
            std::vector<double> aa(d.a.size()), bb(d.b.size());
            for (size_t x = 0; x < aa.size(); ++x) aa[x] = std::fabs(d.a[x]);
            for (size_t x = 0; x < bb.size(); ++x) bb[x] = std::fabs(d.b[x]);
            d.absab.resize(m * n);
            cpu_dgemm((int)m, (int)n, (int)k, aa.data(), bb.data(), d.absab.data());
            cand |= 1u << i;
        } else if (d.block == OO_BLOCK_FFT) {
            OO_REQUIRE(s.n >= 1 && s.n <= (1 << 22) && (s.n & (s.n - 1)) == 0, OO_EINVAL,
                       at + "FFT length must be a power of two <= 2^22");
            d.a.resize(2 * (size_t)s.n);
            for (auto &v : d.a) v = rng.sym();
            d.ref = d.a;
            cpu_fft(s.n, reinterpret_cast<std::complex<double> *>(d.ref.data()));
            d.out.resize(d.ref.size());
            cand |= 1u << i;
        }
    }
    mask_ms.assign((size_t)1 << n_sites, std::numeric_limits<double>::infinity());
    for (uint32_t mask = 0; mask < (1u << n_sites); ++mask) {
        if (mask & ~cand) continue;  // only known sites can be offloaded
        bool ok = true;
        const double t0 = now_ms();
        for (int i = 0; i < n_sites; ++i) {
            const oo_fb_site &s = sites[i];
            Site &d = D[i];
            if (d.block == 0) continue;
            const bool on_gpu = (mask >> i) & 1u;
            for (int call = 0; call < s.calls; ++call) {
                if (on_gpu) {
                    gpu(prec, d.block, s, d.a.data(), d.b.data(), d.out.data());
                } else if (d.block == OO_BLOCK_GEMM) {
                    cpu_dgemm((int)s.m, (int)s.n, (int)s.k, d.a.data(), d.b.data(), d.out.data());
                } else {
                    d.out = d.a;
                    cpu_fft(s.n, reinterpret_cast<std::complex<double> *>(d.out.data()));
                }
            }
        }
        const double t1 = now_ms();
        // results of the offloaded sites against the all-CPU run
        for (int i = 0; i < n_sites && ok; ++i) {
            const Site &d = D[i];
            if (!((mask >> i) & 1u)) continue;
            if (d.block == OO_BLOCK_GEMM) {
                double e = 0.0;
                for (size_t x = 0; x < d.out.size(); ++x)
                    e = std::max(e, std::fabs(d.out[x] - d.ref[x]) / std::max(d.absab[x], 1e-300));
                ok = e <= tol;
            } else {
                double num = 0.0, den = 0.0;
                for (size_t x = 0; x < d.out.size(); ++x) {
                    num += (d.out[x] - d.ref[x]) * (d.out[x] - d.ref[x]);
                    den += d.ref[x] * d.ref[x];
                }
                ok = std::sqrt(num) <= tol * std::sqrt(den);
            }
        }
        if (ok) mask_ms[mask] = t1 - t0;
    }
}

uint32_t fb_best(const double *mask_ms, int n_sites, double *best_ms) {
    uint32_t best = 0;
    for (uint32_t m = 1; m < (1u << n_sites); ++m)
        if (mask_ms[m] < mask_ms[best]) best = m;  // ties keep the lower mask
    if (best_ms) *best_ms = mask_ms[best];
    return best;
}

}  // namespace oo
