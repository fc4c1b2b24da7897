/*
 * fft.c -- oracle for the complex FFT function block.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Sec. 3.2.2 names the Fourier transform as a function block that a GPU
 * library replaces.  Definition used (unnormalised forward, 1/N inverse):
 *   forward  X_k = sum_{n<N} x_n exp(-2 pi i n k / N)
 *   inverse  x_n = (1/N) sum_{k<N} X_k exp(+2 pi i n k / N)
 * oracle_dft is that definition summed term by term, the angle reduced
 * exactly as (n k mod N) / N in integers before the FP64 cos / sin.
 * oracle_fft is the plain recursive radix-2 decimation-in-time split
 * X_k = E_k + w^k O_k, X_{k+N/2} = E_k - w^k O_k with every twiddle w^k taken
 * directly from cos / sin (no recurrences).
 *
 * Parity: pinned against closed forms (delta, constant, single tones),
 * Parseval, linearity, shift-phase, inverse round trip and, for the FFT,
 * against the DFT on N <= 4096 (tests/test_oracle_fft.py).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>

static const double TWO_PI = 6.283185307179586476925286766559;

void oracle_dft(int64_t n, int dir, const double *in, double *out)
{
    const double sgn = dir < 0 ? -1.0 : 1.0;
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t t = 0; t < n; ++t) {
            const int64_t m = (int64_t)(((unsigned __int128)t * (unsigned __int128)k) % (unsigned __int128)n);
            const double ang = TWO_PI * (double)m / (double)n;
            const double c = cos(ang), s = sgn * sin(ang);
            const double xr = in[2 * t], xi = in[2 * t + 1];
            sr += xr * c - xi * s;
            si += xr * s + xi * c;
        }
        if (dir > 0) { sr /= (double)n; si /= (double)n; }
        out[2 * k] = sr;
        out[2 * k + 1] = si;
    }
}

/* out[k] for the length-n transform of x[0], x[stride], ... (unscaled) */
static void fft_rec(int64_t n, int64_t stride, double sgn, const double *x, double *out)
{
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        return;
    }
    const int64_t h = n / 2;
    double *e = (double *)malloc(sizeof(double) * 2 * (size_t)h);
    double *o = (double *)malloc(sizeof(double) * 2 * (size_t)h);
    fft_rec(h, stride * 2, sgn, x, e);
    fft_rec(h, stride * 2, sgn, x + 2 * stride, o);
    for (int64_t k = 0; k < h; ++k) {
        const double ang = TWO_PI * (double)k / (double)n;
        const double wr = cos(ang), wi = sgn * sin(ang);
        const double tr = wr * o[2 * k] - wi * o[2 * k + 1];
        const double ti = wr * o[2 * k + 1] + wi * o[2 * k];
        out[2 * k] = e[2 * k] + tr;
        out[2 * k + 1] = e[2 * k + 1] + ti;
        out[2 * (k + h)] = e[2 * k] - tr;
        out[2 * (k + h) + 1] = e[2 * k + 1] - ti;
    }
    free(e);
    free(o);
}

int oracle_fft(int64_t n, int dir, const double *in, double *out)
{
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    fft_rec(n, 1, dir < 0 ? -1.0 : 1.0, in, out);
    if (dir > 0)
        for (int64_t t = 0; t < 2 * n; ++t) out[t] /= (double)n;
    return 0;
}
