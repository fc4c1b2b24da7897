// CPU execution of the Jacobi program's nests, used for gene bits set to 0.
//
// Sec. 3.2.1: a gene bit of 0 leaves its loop on the CPU.  These are the
// program's own loops, run on the host cores with OpenMP over i: per-point
// arithmetic in FP64 on the float inputs, stores rounded to float, the
// residual summed in FP64 per i-plane and then over planes in i order (so the
// sum does not depend on the thread count).
#include <omp.h>

#include <vector>

#include "oo_internal.h"

namespace oo {

namespace {
inline size_t at(const JacobiDims &d, int i, int j, int k) {
    return ((size_t)i * d.J + j) * d.K + k;
}
inline float dirichlet(int k, int K) {
    // (k/(K-1))^2 as one correctly rounded float division of exact integers
    return (float)(k * k) / (float)((K - 1) * (K - 1));
}
}  // namespace

void host_coef(const JacobiDims &d, float *const coef[NCOEF]) {
    static const float val[NCOEF] = {1.0f, 1.0f, 1.0f, (float)(1.0 / 6.0), 0.0f, 0.0f,
                                     0.0f, 1.0f, 1.0f, 1.0f,               1.0f, 0.0f};
    const long long n = (long long)d.n_host();
#pragma omp parallel for schedule(static)
    for (long long x = 0; x < n; ++x)
        for (int a = 0; a < NCOEF; ++a) coef[a][x] = val[a];
}

void host_pinit(const JacobiDims &d, float *p, float *wrk2) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < d.I; ++i)
        for (int j = 0; j < d.J; ++j)
            for (int k = 0; k < d.K; ++k) {
                const float g = dirichlet(k, d.K);
                p[at(d, i, j, k)] = g;
                wrk2[at(d, i, j, k)] = g;
            }
}

double host_stencil(const JacobiDims &d, const float *const coef[NCOEF], const float *p,
                    float omega, float *wrk2) {
    std::vector<double> plane(d.I, 0.0);
    const float *a0 = coef[0], *a1 = coef[1], *a2 = coef[2], *a3 = coef[3];
    const float *b0 = coef[4], *b1 = coef[5], *b2 = coef[6];
    const float *c0 = coef[7], *c1 = coef[8], *c2 = coef[9];
    const float *bnd = coef[10], *wrk1 = coef[11];
    const size_t sj = d.K, si = (size_t)d.J * d.K;
    const double om = omega;
#pragma omp parallel for schedule(static)
    for (int i = 1; i < d.I - 1; ++i) {
        double acc = 0.0;
        for (int j = 1; j < d.J - 1; ++j)
            for (int k = 1; k < d.K - 1; ++k) {
                const size_t c = at(d, i, j, k);
                const double xij = ((double)p[c + si + sj] - (double)p[c + si - sj]) -
                                   (double)p[c - si + sj] + (double)p[c - si - sj];
                const double xjk = ((double)p[c + sj + 1] - (double)p[c - sj + 1]) -
                                   (double)p[c + sj - 1] + (double)p[c - sj - 1];
                const double xik = ((double)p[c + si + 1] - (double)p[c - si + 1]) -
                                   (double)p[c + si - 1] + (double)p[c - si - 1];
                const double s0 = (double)a0[c] * p[c + si] + (double)a1[c] * p[c + sj] +
                                  (double)a2[c] * p[c + 1] + (double)b0[c] * xij +
                                  (double)b1[c] * xjk + (double)b2[c] * xik +
                                  (double)c0[c] * p[c - si] + (double)c1[c] * p[c - sj] +
                                  (double)c2[c] * p[c - 1] + (double)wrk1[c];
                const double ss = (s0 * (double)a3[c] - (double)p[c]) * (double)bnd[c];
                acc += ss * ss;
                wrk2[c] = (float)((double)p[c] + om * ss);
            }
        plane[i] = acc;
    }
    double res = 0.0;
    for (int i = 1; i < d.I - 1; ++i) res += plane[i];
    return res;
}

void host_copyback(const JacobiDims &d, float *p, const float *wrk2) {
#pragma omp parallel for schedule(static)
    for (int i = 1; i < d.I - 1; ++i)
        for (int j = 1; j < d.J - 1; ++j)
            for (int k = 1; k < d.K - 1; ++k) p[at(d, i, j, k)] = wrk2[at(d, i, j, k)];
}

void host_bc_ij(const JacobiDims &d, float *p) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < d.I; ++i)
        for (int j = 0; j < d.J; ++j) {
            if (i != 0 && i != d.I - 1 && j != 0 && j != d.J - 1) continue;
            for (int k = 0; k < d.K; ++k) p[at(d, i, j, k)] = dirichlet(k, d.K);
        }
}

void host_bc_k(const JacobiDims &d, float *p) {
    const float g0 = dirichlet(0, d.K), g1 = dirichlet(d.K - 1, d.K);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < d.I; ++i)
        for (int j = 0; j < d.J; ++j) {
            p[at(d, i, j, 0)] = g0;
            p[at(d, i, j, d.K - 1)] = g1;
        }
}

}  // namespace oo
