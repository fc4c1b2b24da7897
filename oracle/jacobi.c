/*
 * jacobi.c -- oracle for the loop program whose nests a gene offloads.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper (Sec. 3.2.1, Sec. 4.2.2) offloads the parallelisable loop nests
 * of an ordinary CPU program.  The program used here is a 19-point 3D Jacobi
 * pressure solver with six nests: coefficient setup, pressure init, stencil
 * update with residual, copy-back, and two boundary-face nests.  Arithmetic
 * is FP64 on the float-valued inputs, in the plain loop order below (i, then
 * j, then k), with no blocking, fusion or reordering.
 *
 * Parity: pinned by a hand-computed 4x4x4 step, per-term closed forms on
 * polynomial fields, the closed-form first residual of the setup field, and
 * the constant-field fixed point (tests/test_oracle_jacobi.py).
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, k) (((size_t)(i) * (size_t)J + (size_t)(j)) * (size_t)K + (size_t)(k))

void oracle_jacobi_setup(int I, int J, int K, float *coef12, float *p)
{
    const size_t N = (size_t)I * J * K;
    const float one_sixth = (float)(1.0 / 6.0);
    for (size_t n = 0; n < N; ++n) {
        coef12[0 * N + n] = 1.0f;        /* a0 */
        coef12[1 * N + n] = 1.0f;        /* a1 */
        coef12[2 * N + n] = 1.0f;        /* a2 */
        coef12[3 * N + n] = one_sixth;   /* a3 */
        coef12[4 * N + n] = 0.0f;        /* b0 */
        coef12[5 * N + n] = 0.0f;        /* b1 */
        coef12[6 * N + n] = 0.0f;        /* b2 */
        coef12[7 * N + n] = 1.0f;        /* c0 */
        coef12[8 * N + n] = 1.0f;        /* c1 */
        coef12[9 * N + n] = 1.0f;        /* c2 */
        coef12[10 * N + n] = 1.0f;       /* bnd */
        coef12[11 * N + n] = 0.0f;       /* wrk1 */
    }
    if (p) {
        const double den = (double)(K - 1) * (double)(K - 1);
        for (int i = 0; i < I; ++i)
            for (int j = 0; j < J; ++j)
                for (int k = 0; k < K; ++k)
                    p[IDX(i, j, k)] = (float)(((double)k * (double)k) / den);
    }
}

void oracle_stencil(int I, int J, int K, const float *coef12, const double *p,
                    double omega, double *wrk2_out, double *res_out)
{
    const size_t N = (size_t)I * J * K;
    const float *a0 = coef12 + 0 * N, *a1 = coef12 + 1 * N, *a2 = coef12 + 2 * N;
    const float *a3 = coef12 + 3 * N;
    const float *b0 = coef12 + 4 * N, *b1 = coef12 + 5 * N, *b2 = coef12 + 6 * N;
    const float *c0 = coef12 + 7 * N, *c1 = coef12 + 8 * N, *c2 = coef12 + 9 * N;
    const float *bnd = coef12 + 10 * N, *wrk1 = coef12 + 11 * N;
    double res = 0.0;
    for (size_t n = 0; n < N; ++n) wrk2_out[n] = p[n];
    for (int i = 1; i < I - 1; ++i)
        for (int j = 1; j < J - 1; ++j)
            for (int k = 1; k < K - 1; ++k) {
                const size_t c = IDX(i, j, k);
                /* cross differences in the (i,j), (j,k) and (i,k) planes */
                double xij = p[IDX(i + 1, j + 1, k)] - p[IDX(i + 1, j - 1, k)]
                           - p[IDX(i - 1, j + 1, k)] + p[IDX(i - 1, j - 1, k)];
                double xjk = p[IDX(i, j + 1, k + 1)] - p[IDX(i, j - 1, k + 1)]
                           - p[IDX(i, j + 1, k - 1)] + p[IDX(i, j - 1, k - 1)];
                double xik = p[IDX(i + 1, j, k + 1)] - p[IDX(i - 1, j, k + 1)]
                           - p[IDX(i + 1, j, k - 1)] + p[IDX(i - 1, j, k - 1)];
                double s0 = (double)a0[c] * p[IDX(i + 1, j, k)]
                          + (double)a1[c] * p[IDX(i, j + 1, k)]
                          + (double)a2[c] * p[IDX(i, j, k + 1)]
                          + (double)b0[c] * xij
                          + (double)b1[c] * xjk
                          + (double)b2[c] * xik
                          + (double)c0[c] * p[IDX(i - 1, j, k)]
                          + (double)c1[c] * p[IDX(i, j - 1, k)]
                          + (double)c2[c] * p[IDX(i, j, k - 1)]
                          + (double)wrk1[c];
                double ss = (s0 * (double)a3[c] - p[c]) * (double)bnd[c];
                res += ss * ss;
                wrk2_out[c] = p[c] + omega * ss;
            }
    *res_out = res;
}

int oracle_jacobi_run(int I, int J, int K, int iters, float omega, int mode,
                      const float *coef12, const float *p0,
                      double *res_out, double *p_out)
{
    if (I < 3 || J < 3 || K < 3 || iters < 0) return -1;
    const size_t N = (size_t)I * J * K;
    float *coef = (float *)malloc(sizeof(float) * N * ORC_NCOEF);
    float *g = (float *)malloc(sizeof(float) * N);       /* setup p = boundary values */
    double *p = (double *)malloc(sizeof(double) * N);
    double *wrk2 = (double *)malloc(sizeof(double) * N);
    float *gk = (float *)malloc(sizeof(float) * (size_t)K);
    if (!coef || !g || !p || !wrk2 || !gk) {
        free(coef); free(g); free(p); free(wrk2); free(gk);
        return -1;
    }
    for (int k = 0; k < K; ++k)
        gk[k] = (float)(((double)k * (double)k) / ((double)(K - 1) * (double)(K - 1)));

    /* nest N0 (coefficients) and N1 (pressure init) */
    oracle_jacobi_setup(I, J, K, coef, g);
    if (coef12) memcpy(coef, coef12, sizeof(float) * N * ORC_NCOEF);
    if (p0) memcpy(g, p0, sizeof(float) * N);
    for (size_t n = 0; n < N; ++n) p[n] = (double)g[n];

    for (int it = 0; it < iters; ++it) {
        /* N2: stencil + residual into wrk2 */
        oracle_stencil(I, J, K, coef, p, (double)omega, wrk2, &res_out[it]);
        if (mode == 1)
            for (size_t n = 0; n < N; ++n) wrk2[n] = (double)(float)wrk2[n];
        /* N3: copy-back on the interior */
        for (int i = 1; i < I - 1; ++i)
            for (int j = 1; j < J - 1; ++j)
                for (int k = 1; k < K - 1; ++k) p[IDX(i, j, k)] = wrk2[IDX(i, j, k)];
        /* N4: faces i in {0, I-1} and j in {0, J-1} re-set to the
         * Dirichlet value fl32(k^2 / (K-1)^2) */
        for (int i = 0; i < I; ++i)
            for (int j = 0; j < J; ++j) {
                if (i != 0 && i != I - 1 && j != 0 && j != J - 1) continue;
                for (int k = 0; k < K; ++k) p[IDX(i, j, k)] = (double)gk[k];
            }
        /* N5: faces k in {0, K-1} */
        for (int i = 0; i < I; ++i)
            for (int j = 0; j < J; ++j) {
                p[IDX(i, j, 0)] = (double)gk[0];
                p[IDX(i, j, K - 1)] = (double)gk[K - 1];
            }
    }
    if (p_out) memcpy(p_out, p, sizeof(double) * N);
    free(coef); free(g); free(p); free(wrk2); free(gk);
    return 0;
}
