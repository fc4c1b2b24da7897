/*
 * gemm.c -- oracle for the dense matrix-product function block.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Sec. 3.2.2 / Sec. 4.2.1: a library call found by name (a matrix product)
 * is replaced by a GPU implementation behind the same CPU interface.  The
 * operation itself is the textbook product C[i][j] = sum_l A[i][l] B[l][j].
 * Each dot product is summed with the compensated Dot2 scheme of Ogita,
 * Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput.,
 * 2005): every product is split exactly with an FMA and every addition
 * exactly with Knuth's two-sum, and the error terms are added up separately,
 * so the result is as accurate as if computed in twice the working precision.
 *
 * Parity: pinned by exact identity / permutation products, by exact small-
 * integer products and by a long-double triple loop on small sizes
 * (tests/test_oracle_gemm.py).
 */
#include "oracle.h"
#include <math.h>

void oracle_gemm(int m, int n, int k, const double *A, int lda,
                 const double *B, int ldb, double *C, int ldc, int r0, int r1)
{
    if (r0 < 0) r0 = 0;
    if (r1 > m) r1 = m;
    for (int i = r0; i < r1; ++i)
        for (int j = 0; j < n; ++j) {
            double sum = 0.0, err = 0.0;
            for (int l = 0; l < k; ++l) {
                const double x = A[(size_t)i * lda + l];
                const double y = B[(size_t)l * ldb + j];
                const double h = x * y;                 /* product, rounded  */
                const double r = fma(x, y, -h);         /* its exact error   */
                const double s = sum + h;               /* two-sum of sum+h  */
                const double bb = s - sum;
                const double q = (sum - (s - bb)) + (h - bb);
                sum = s;
                err += q + r;
            }
            C[(size_t)i * ldc + j] = sum + err;
        }
}
