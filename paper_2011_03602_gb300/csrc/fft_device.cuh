// Device code of the Fourier-transform block shared by its kernels
// (fft.cu) and the device-resident serving loop (serve_resident.cu):
// float-float complex values in shared memory, Stockham stages (a first
// stage of radix 2, 4 or 8, then radix 8) with per-stage twiddle tables, the
// exact power-of-two input scaling, and one work item of a group of
// transforms.  The design is described in fft.cu.
#pragma once

#include <cuda_runtime.h>

#include "ff.cuh"

namespace oo {
namespace ff {

// Lazy forms for chains of operations (the FFT's butterflies): the same
// error-free hi-part transforms, without the final renormalisation.  A lazy
// result (h, l) is an unevaluated sum whose l may exceed ulp(h) after
// cancellation; every operation below takes such inputs (two-sum on the hi
// parts, the lo parts added), and the chain ends with norm().  The error of
// each step stays a few units of 2^-48 relative to the magnitudes of its
// operands, which is what a normwise bound for the transform needs.
__device__ __forceinline__ void add_lazy(float ah, float al, float bh, float bl, float &h, float &l) {
    float e;
    two_sum(ah, bh, h, e);
    l = __fadd_rn(e, __fadd_rn(al, bl));
}
__device__ __forceinline__ cplx cadd_lazy(const cplx &a, const cplx &b) {
    cplx r;
    add_lazy(a.rh, a.rl, b.rh, b.rl, r.rh, r.rl);
    add_lazy(a.ih, a.il, b.ih, b.il, r.ih, r.il);
    return r;
}
__device__ __forceinline__ cplx csub_lazy(const cplx &a, const cplx &b) {
    cplx r;
    add_lazy(a.rh, a.rl, -b.rh, -b.rl, r.rh, r.rl);
    add_lazy(a.ih, a.il, -b.ih, -b.il, r.ih, r.il);
    return r;
}
// a * w as cmul, without its final renormalisation
__device__ __forceinline__ cplx cmul_lazy(const cplx &a, const cplx &w) {
    cplx r;
    {
        float p1, e1, p2, e2, e3;
        two_prod(a.rh, w.rh, p1, e1);
        two_prod(a.ih, w.ih, p2, e2);
        two_sum(p1, -p2, r.rh, e3);
        float e = __fadd_rn(__fsub_rn(e1, e2), e3);
        e = __fmaf_rn(a.rh, w.rl, e);
        e = __fmaf_rn(a.rl, w.rh, e);
        e = __fmaf_rn(-a.ih, w.il, e);
        r.rl = __fmaf_rn(-a.il, w.ih, e);
    }
    {
        float p1, e1, p2, e2, e3;
        two_prod(a.rh, w.ih, p1, e1);
        two_prod(a.ih, w.rh, p2, e2);
        two_sum(p1, p2, r.ih, e3);
        float e = __fadd_rn(__fadd_rn(e1, e2), e3);
        e = __fmaf_rn(a.rh, w.il, e);
        e = __fmaf_rn(a.rl, w.ih, e);
        e = __fmaf_rn(a.ih, w.rl, e);
        r.il = __fmaf_rn(a.il, w.rh, e);
    }
    return r;
}
// renormalise both components (|l| <= ulp(h) / 2 afterwards when |h| >= |l|)
__device__ __forceinline__ cplx norm(const cplx &a) {
    cplx r;
    fast_two_sum(a.rh, a.rl, r.rh, r.rl);
    fast_two_sum(a.ih, a.il, r.ih, r.il);
    return r;
}

}  // namespace ff

namespace {

constexpr int kFftThreads = 512;
constexpr int kFftBpt = 2;                               // (8 values per thread: 8 / R radix-R butterflies)
constexpr int kFftElems = 4 * kFftThreads * kFftBpt;     // 4096 values per CTA
// The values sit in shared memory with one float4 of padding after every
// eight (value i at sp(i, 3)), so the strided stores of the Stockham stages
// (R or R Ls float4 apart) and the loads across short columns fall in eight
// different 16-byte bank groups of a quarter warp instead of one.  Passes of
// 2048 points keep the unpadded layout (sp(i, 30) = i): with their 32 KB
// twiddle table the padding would take two CTAs past 196 KB of shared
// memory per SM, and the smaller L1 that leaves costs more (measured: 2^22
// 0.205 -> 0.227 ms) than the conflicts.
constexpr int kFftElemsPad = kFftElems + kFftElems / 8;
__host__ __device__ __forceinline__ bool fft_padded(int log2L) { return log2L != 11; }
__host__ __device__ __forceinline__ int fft_pad_shift(int log2L) { return fft_padded(log2L) ? 3 : 30; }
__host__ __device__ __forceinline__ int fft_data_slots(int log2L) { return fft_padded(log2L) ? kFftElemsPad : kFftElems; }
__host__ __device__ __forceinline__ int sp(int i, int ps) { return ps >= 30 ? i : i + (i >> ps); }
constexpr int kTwSplit = 11;                             // four-step twiddle split: 2^11

using ff::cplx;

__device__ __forceinline__ cplx ld_cplx(const float4 *p) {
    const float4 v = *p;
    return cplx{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ void st_cplx(float4 *p, const cplx &c) { *p = make_float4(c.rh, c.rl, c.ih, c.il); }

// x * 2^-S split into a float pair (hi: top 24 mantissa bits; lo: the rest
// rounded to 24 bits), integer-only; values below 2^-126 after scaling flush.
__device__ __forceinline__ void split_scaled(double x, int S, float &h, float &l) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
    const unsigned sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7ffu);
    const int fe = e - 1023 - S + 127;  // biased float exponent of the scaled value
    if (e == 0 || e == 0x7ff || fe <= 0) {
        h = 0.0f;
        l = 0.0f;
        return;
    }
    const unsigned mtop = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
    h = __uint_as_float(sign | ((unsigned)fe << 23) | mtop);
    const unsigned r = lo32 & 0x1fffffffu;
    const int le = fe - 52;  // biased exponent of 2^(unbiased(fe) - 52)
    float lf = 0.0f;
    if (le > 0 && r != 0) lf = __fmul_rn(__uint2float_rn(r), __uint_as_float((unsigned)le << 23));
    l = sign ? -lf : lf;
}

// (h + l) * 2^S as a double, integer-only conversion
__device__ __forceinline__ double widen_scaled(float h, float l, int S) {
    return ff::scale_pow2(ff::to_double(h, l), S);
}

// A transform holding a NaN or an infinity: its maximum exponent reads 0x7ff.
// Every butterfly then sees zeros (split_scaled flushes non-finite values and
// the scale flushes the rest) and every output component is written as NaN,
// which is what the FP64 definition gives for any length above one.
constexpr int kNonFiniteExpo = 0x7ff;
__device__ __forceinline__ double2 nan2() {
    const double q = __longlong_as_double(0x7ff8000000000000ll);
    return make_double2(q, q);
}

__device__ __forceinline__ cplx twiddle(const float4 *stw, int idx, bool inv) {
    cplx w = ld_cplx(stw + idx);
    return inv ? ff::conj(w) : w;
}

// ---- stages.  A length-L transform runs a first stage of radix 2^b0,
// b0 = ((log2 L - 1) mod 3) + 1 (the whole transform when L <= 8), then
// radix-8 stages with sub-lengths Ls = 2^b0, 8 * 2^b0, ...  A Stockham stage
// of radix R and sub-length Ls takes inputs j + q L/R (q < R) of butterfly
// j, multiplies input q by W_{R Ls}^{k q} (k = j mod Ls; none in the first
// stage, Ls = 1) from its slice of the per-stage table, stw[(q - 1) Ls + k]
// (lanes with consecutive k read consecutive entries), and writes output p
// to (j - k) R + k + p Ls.  Fewer, wider stages than radix 4 mean fewer
// shared-memory round trips and barriers per point.

__host__ __device__ __forceinline__ int first_radix_log2(int log2L) {
    return log2L <= 3 ? log2L : ((log2L - 1) % 3) + 1;
}
// entries of the per-stage twiddle table of a length-2^log2L transform: 7 Ls
// per radix-8 stage after the first
__host__ __device__ __forceinline__ int stage_table_count(int log2L) {
    return log2L <= 3 ? 0 : (1 << log2L) - (1 << first_radix_log2(log2L));
}

// Where a pass reads its per-stage table.  Up to L = 2048 (2040 entries,
// 32 KB) it is staged in shared memory beside the 64 KB of data; the
// 4096-point table (4088 entries, 64 KB) is read in place from global memory,
// cached in L1: staged, it would double the CTA's shared memory to 128 KB and
// leave one CTA per SM, while in place two CTAs fit and one's global loads and
// stores overlap the other's butterflies.  Same entries, same arithmetic: the
// results do not depend on where the table is read from.
__host__ __device__ __forceinline__ bool twiddles_staged(int log2L) { return log2L < 12; }
// Shared memory of a CTA running a pass of length 2^log2L: the data, the
// staged table (if any), then one int per column of the CTA (its largest
// input exponent), 16-byte aligned.
__host__ __device__ __forceinline__ size_t fft_colmax_bytes(int log2L) {
    return ((size_t)(kFftElems >> log2L) * 4 + 15) / 16 * 16;
}
__host__ __device__ __forceinline__ size_t fft_smem_bytes(int log2L) {
    return (size_t)(fft_data_slots(log2L) + (twiddles_staged(log2L) ? (1 << log2L) : 0)) * 16 +
           fft_colmax_bytes(log2L);
}
// the largest of those (L = 2048, unpadded: 96 KB + 16 bytes)
constexpr size_t kFftSmemMax = (size_t)(kFftElems + 2048) * 16 + 16;

// 1 / sqrt(2) as a float pair (hi, lo)
constexpr double kInvSqrt2 = 0.70710678118654752440084436210485;
constexpr float kS2h = (float)kInvSqrt2;
constexpr float kS2l = (float)(kInvSqrt2 - (double)kS2h);

// (h + l) / sqrt(2), lazy
__device__ __forceinline__ void mul_inv_sqrt2(float h, float l, float &rh, float &rl) {
    float e;
    ff::two_prod(h, kS2h, rh, e);
    e = __fmaf_rn(h, kS2l, e);
    rl = __fmaf_rn(l, kS2h, e);
}

// 4-point DFT of lazy inputs, lazy outputs (no renormalisation)
__device__ __forceinline__ void dft4_lazy(const cplx &x0, const cplx &x1, const cplx &x2, const cplx &x3, cplx *y,
                                          bool inv) {
    const cplx a0 = ff::cadd_lazy(x0, x2), a1 = ff::csub_lazy(x0, x2);
    const cplx b0 = ff::cadd_lazy(x1, x3), b1 = ff::csub_lazy(x1, x3);
    const cplx rb1 = inv ? ff::mul_pos_i(b1) : ff::mul_neg_i(b1);
    y[0] = ff::cadd_lazy(a0, b0);
    y[2] = ff::csub_lazy(a0, b0);
    y[1] = ff::cadd_lazy(a1, rb1);
    y[3] = ff::csub_lazy(a1, rb1);
}

// R-point DFT (R = 2, 4, 8) of lazy inputs in place, x[p] <- Y_p = sum_q
// x_q W_R^{+-p q}, each output renormalised once.  R = 8: two 4-point DFTs
// (even and odd inputs) and Y_p = E_p + W_8^p O_p, Y_{p+4} = E_p - W_8^p O_p,
// where W_8^{+-1}, W_8^{+-3} are a sum and a difference of O's parts times
// 1 / sqrt(2) and W_8^{+-2} = -+i is exact.
template <int R>
__device__ __forceinline__ void dft_small(cplx *x, bool inv) {
    if constexpr (R == 2) {
        const cplx y0 = ff::cadd_lazy(x[0], x[1]), y1 = ff::csub_lazy(x[0], x[1]);
        x[0] = ff::norm(y0);
        x[1] = ff::norm(y1);
    } else if constexpr (R == 4) {
        cplx y[4];
        dft4_lazy(x[0], x[1], x[2], x[3], y, inv);
#pragma unroll
        for (int p = 0; p < 4; ++p) x[p] = ff::norm(y[p]);
    } else {
        cplx E[4], O[4];
        dft4_lazy(x[0], x[2], x[4], x[6], E, inv);
        dft4_lazy(x[1], x[3], x[5], x[7], O, inv);
        cplx t[4];
        t[0] = O[0];
        t[2] = inv ? ff::mul_pos_i(O[2]) : ff::mul_neg_i(O[2]);
        {
            float sh, sl, dh, dl;  // s = re + im, d = im - re
            ff::add_lazy(O[1].rh, O[1].rl, O[1].ih, O[1].il, sh, sl);
            ff::add_lazy(O[1].ih, O[1].il, -O[1].rh, -O[1].rl, dh, dl);
            if (inv) {  // (1 + i) / sqrt 2: (-d + i s) / sqrt 2
                mul_inv_sqrt2(-dh, -dl, t[1].rh, t[1].rl);
                mul_inv_sqrt2(sh, sl, t[1].ih, t[1].il);
            } else {    // (1 - i) / sqrt 2: (s + i d) / sqrt 2
                mul_inv_sqrt2(sh, sl, t[1].rh, t[1].rl);
                mul_inv_sqrt2(dh, dl, t[1].ih, t[1].il);
            }
        }
        {
            float sh, sl, dh, dl;
            ff::add_lazy(O[3].rh, O[3].rl, O[3].ih, O[3].il, sh, sl);
            ff::add_lazy(O[3].ih, O[3].il, -O[3].rh, -O[3].rl, dh, dl);
            if (inv) {  // (-1 + i) / sqrt 2: (-s - i d) / sqrt 2
                mul_inv_sqrt2(-sh, -sl, t[3].rh, t[3].rl);
                mul_inv_sqrt2(-dh, -dl, t[3].ih, t[3].il);
            } else {    // (-1 - i) / sqrt 2: (d - i s) / sqrt 2
                mul_inv_sqrt2(dh, dl, t[3].rh, t[3].rl);
                mul_inv_sqrt2(-sh, -sl, t[3].ih, t[3].il);
            }
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            x[p] = ff::norm(ff::cadd_lazy(E[p], t[p]));
            x[p + 4] = ff::norm(ff::csub_lazy(E[p], t[p]));
        }
    }
}

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

// One Stockham stage of radix R over the CTA's kFftElems values (C columns of
// length L): 8 / R butterflies per thread; value i at sd[sp(i, ps)].
template <int R>
__device__ __forceinline__ void stage_radix(float4 *sd, const float4 *stw, int log2L, int Ls, bool inv, int ps) {
    constexpr int B = kFftElems / (R * kFftThreads);
    const int log2lr = log2L - ilog2c(R), lr = 1 << log2lr;
    cplx Y[B][R];
    int base_c[B], jj[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int bidx = threadIdx.x + b * kFftThreads;
        const int c = bidx >> log2lr, j = bidx & (lr - 1);
        base_c[b] = c << log2L;
        jj[b] = j;
#pragma unroll
        for (int q = 0; q < R; ++q) Y[b][q] = ld_cplx(sd + sp(base_c[b] + j + q * lr, ps));
        if (Ls > 1) {
            const int k = j & (Ls - 1);
#pragma unroll
            for (int q = 1; q < R; ++q) Y[b][q] = ff::cmul_lazy(Y[b][q], twiddle(stw, (q - 1) * Ls + k, inv));
        }
        dft_small<R>(Y[b], inv);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = jj[b], k = j & (Ls - 1);
        const int o = base_c[b] + (j - k) * R + k;
#pragma unroll
        for (int p = 0; p < R; ++p) st_cplx(sd + sp(o + p * Ls, ps), Y[b][p]);
    }
    __syncthreads();
}

// the radix-8 stages after the first stage (which the caller has done);
// inlined, so a caller's constant layout shift ps stays a constant
__device__ __forceinline__ void fft_in_smem_after_first(float4 *sd, const float4 *stw, int log2L, bool inv, int ps) {
    for (int Ls = 1 << first_radix_log2(log2L); Ls < (1 << log2L); Ls *= 8) {
        stage_radix<8>(sd, stw, log2L, Ls, inv, ps);
        stw += 7 * Ls;
    }
}

// the whole transform of every column in shared memory
__device__ __forceinline__ void fft_in_smem(float4 *sd, const float4 *stw, int log2L, bool inv, int ps) {
    if (log2L == 0) return;
    const int b0 = first_radix_log2(log2L);
    if (b0 == 1)
        stage_radix<2>(sd, stw, log2L, 1, inv, ps);
    else if (b0 == 2)
        stage_radix<4>(sd, stw, log2L, 1, inv, ps);
    else
        stage_radix<8>(sd, stw, log2L, 1, inv, ps);
    fft_in_smem_after_first(sd, stw, log2L, inv, ps);
}

// largest biased exponent among the 64-bit words [x0, x1) of p (stride
// `step` between a thread's 16-byte loads, four loads in flight per thread);
// kNonFiniteExpo (0x7ff, above every finite exponent) if any word is a NaN or
// an infinity
__device__ __forceinline__ int max_exponent(const ulonglong2 *p, long long x0, long long x1, long long step) {
    int m = 0;
    auto ex = [](unsigned long long w) { return (int)((w >> 52) & 0x7ffu); };
    long long x = x0;
    for (; x + 3 * step < x1; x += 4 * step) {
        ulonglong2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = p[x + u * step];
#pragma unroll
        for (int u = 0; u < 4; ++u) m = max(m, max(ex(v[u].x), ex(v[u].y)));
    }
    for (; x < x1; x += step) {
        const ulonglong2 v = p[x];
        m = max(m, max(ex(v.x), ex(v.y)));
    }
    return m;
}

// Per-column scales.  Every column of a CTA -- a whole transform, or one
// column of a four-step transform's first pass -- is scaled by the power of
// two that brings its own largest component into [1/2, 1); the exponents are
// found in shared memory from the values the CTA has loaded anyway, so no
// pass over the input precedes the transform.  A first pass records each
// column's largest exponent and raises the transform's (atomicMax); the
// second pass brings every column's float-float values to the transform's
// scale, an exact multiplication by a power of two (values more than 2^126
// below the transform's largest component become zero).  Where nothing
// over- or underflows, the per-column scale changes no rounding: the bits
// are those of one scale for the whole transform.

// largest biased exponent of a complex value's parts (0x7ff: NaN or infinity)
__device__ __forceinline__ int expo_of(double2 v) {
    const int a = (int)(((unsigned long long)__double_as_longlong(v.x) >> 52) & 0x7ffu);
    const int b = (int)(((unsigned long long)__double_as_longlong(v.y) >> 52) & 0x7ffu);
    return max(a, b);
}
// Combine a warp's exponents m over lanes that hold the same column (lanes
// equal modulo `period`, a power of two <= 32, when `low` is false; lanes in
// the same aligned group of `period` when `low` is true) and raise smax[col]
// once per column from the lowest such lane.
__device__ __forceinline__ void colmax_warp(int m, int period, bool low, int *smax, int col) {
    const int lane = threadIdx.x & 31;
    if (low) {
        if (period == 32)
            m = __reduce_max_sync(0xffffffffu, m);
        else
            for (int o = period >> 1; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((lane & (period - 1)) == 0 && m > 0) atomicMax(smax + col, m);
    } else {
        for (int o = 16; o >= period; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane < period && m > 0) atomicMax(smax + col, m);
    }
}
// (h, l) pairs of a lazy float-float complex times 2^d, d <= 0
__device__ __forceinline__ float4 scale_down(float4 v, int d) {
    if (d == 0) return v;
    const float f = d >= -126 ? __uint_as_float((unsigned)(127 + d) << 23) : 0.0f;
    return make_float4(__fmul_rn(v.x, f), __fmul_rn(v.y, f), __fmul_rn(v.z, f), __fmul_rn(v.w, f));
}
// the shift from a first-pass column's scale to its transform's: column
// largest exponent cm, transform's em (0: all zero)
__device__ __forceinline__ int col_shift(int cm, int em) { return cm == 0 ? 0 : cm - em; }

// ------------------------------------------------- grouped transforms
// A CTA's worth of work in a batch of transforms of different lengths:
// mode 0: `count` whole transforms of length 2^log2L (request ids at
// tlist[first ..]); mode 1 / 2: the four-step column / row pass of request
// `first` starting at column / row c0.
struct FftItem {
    int mode, log2L, first, count, c0, pad0, pad1, pad2;
};
struct FftGroupReq {
    const double *in;
    double *out;
    float4 *mid;
    const float4 *tw, *tw_n1, *tw_n2, *tw_hi, *tw_lo;
    int *colmax;  // four-step transforms: N2 first-pass column exponents
    int log2n, log2n1, log2n2, inverse;
};

__device__ __forceinline__ int scale_from(int e) { return e == 0 ? 0 : e - 1023 + 1; }

// One work item of a group of transforms (grouped launches and the device-
// resident serving loop alike): mode 0, `count` whole transforms of length
// 2^log2L (request ids at tlist[first ..]); mode 1 / 2, the four-step column /
// row pass of request `first` starting at column / row c0.  512 threads; sd
// is the dynamic shared memory: the item's kFftElems values in its layout
// (fft_data_slots float4), then room for the pass's per-stage twiddle table,
// then the columns' exponents: every table is staged there when stage_all is
// set (callers whose global loads bypass L1), else the 4096-point one is
// read in place.  Mode 1 raises expo[first] (zero before
// the request's first pass) and writes the request's column exponents;
// mode 2 reads both.
__device__ __forceinline__ void fft_group_item(const FftItem &item, const FftGroupReq *reqs, const int *tlist,
                                               int *expo, float4 *sd, bool stage_all) {
    const int log2L = item.log2L, L = 1 << log2L;
    const int C = kFftElems >> log2L;
    const int ps = fft_pad_shift(log2L);
    float4 *stw = sd + fft_data_slots(log2L);  // the table after this item's data layout
    const FftGroupReq &R0 = reqs[item.mode == 0 ? tlist[item.first] : item.first];
    const float4 *tw = item.mode == 0 ? R0.tw : (item.mode == 1 ? R0.tw_n1 : R0.tw_n2);
    const bool inv = R0.inverse != 0;
    __syncthreads();  // previous item's shared-memory reads are done
    const bool staged = stage_all || twiddles_staged(log2L);
    if (staged)
        for (int t = threadIdx.x; t < stage_table_count(log2L); t += kFftThreads) stw[t] = tw[t];
    int *smax = reinterpret_cast<int *>(stw + (staged ? L : 0));
    for (int t = threadIdx.x; t < C; t += kFftThreads) smax[t] = 0;
    const float4 *tws = staged ? stw : tw;
    const int N1 = 1 << R0.log2n1, N2 = 1 << R0.log2n2;
    constexpr int kPer = kFftElems / kFftThreads;
    // value r of this thread: column c, position t
    auto coords = [&](int r, int &c, int &t) {
        const int q = threadIdx.x + r * kFftThreads;
        if (item.mode == 1) {
            c = q & (C - 1);
            t = q >> (31 - __clz(C));
        } else {
            c = q >> log2L;
            t = q & (L - 1);
        }
    };
    __syncthreads();  // smax cleared
    // ---- load.  Mode 2: the first pass's float-float values, brought from
    // their column's scale to the transform's.  Modes 0, 1: every load
    // issued first, the columns' largest exponents gathered, then each value
    // split at its column's scale straight into shared memory.
    if (item.mode == 2) {
        const int em = expo[item.first];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            int c, t;
            coords(r, c, t);
            const float4 v = R0.mid[(long long)(item.c0 + c) * N2 + t];
            sd[sp((c << log2L) + t, ps)] = scale_down(v, col_shift(R0.colmax[t], em));
        }
    } else {
        double2 raw[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            int c, t;
            coords(r, c, t);
            raw[r] = make_double2(0.0, 0.0);
            if (item.mode == 0) {
                if (c < item.count) raw[r] = reinterpret_cast<const double2 *>(reqs[tlist[item.first + c]].in)[t];
            } else {
                raw[r] = reinterpret_cast<const double2 *>(R0.in)[(long long)t * N2 + item.c0 + c];
            }
        }
        if (item.mode == 1) {  // a thread's values are all of column tid mod C
            int m = 0;
#pragma unroll
            for (int r = 0; r < kPer; ++r) m = max(m, expo_of(raw[r]));
            colmax_warp(m, min(C, 32), false, smax, (int)threadIdx.x & (C - 1));
        } else {
#pragma unroll
            for (int r = 0; r < kPer; ++r)
                colmax_warp(expo_of(raw[r]), min(L, 32), true, smax, ((int)threadIdx.x + r * kFftThreads) >> log2L);
        }
        __syncthreads();
        if (item.mode == 1 && (int)threadIdx.x < C) {
            const int e = smax[threadIdx.x];
            R0.colmax[item.c0 + threadIdx.x] = e;
            if (e > 0) atomicMax(expo + item.first, e);
        }
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            int c, t;
            coords(r, c, t);
            const int S = scale_from(smax[c]);
            float4 v;
            split_scaled(raw[r].x, S, v.x, v.y);
            split_scaled(raw[r].y, S, v.z, v.w);
            sd[sp((c << log2L) + t, ps)] = v;
        }
    }
    __syncthreads();
    fft_in_smem(sd, tws, log2L, inv, ps);
    // ---- store
    for (int q = threadIdx.x; q < kFftElems; q += kFftThreads) {
        int c, t;
        if (item.mode == 0) {
            c = q >> log2L;
            t = q & (L - 1);
        } else {
            c = q & (C - 1);
            t = q >> (31 - __clz(C));
        }
        cplx v = ld_cplx(sd + sp((c << log2L) + t, ps));
        if (item.mode == 1) {
            const long long m = (long long)t * (item.c0 + c);
            const int mh = (int)(m >> kTwSplit), ml = (int)(m & ((1 << kTwSplit) - 1));
            cplx w = ff::cmul_lazy(ld_cplx(R0.tw_hi + mh), ld_cplx(R0.tw_lo + ml));
            if (inv) w = ff::conj(w);
            st_cplx(R0.mid + (long long)t * N2 + item.c0 + c, ff::cmul_lazy(v, w));  // pass 2 takes lazy pairs
        } else if (item.mode == 0) {
            if (c >= item.count) continue;
            const int r = tlist[item.first + c];
            const int S = scale_from(smax[c]) - (inv ? log2L : 0);
            double2 y = make_double2(widen_scaled(v.rh, v.rl, S), widen_scaled(v.ih, v.il, S));
            if (log2L == 0)  // length 1: the transform is the identity, exactly
                y = reinterpret_cast<const double2 *>(reqs[r].in)[0];
            else if (smax[c] == kNonFiniteExpo)
                y = nan2();
            reinterpret_cast<double2 *>(reqs[r].out)[t] = y;
        } else {
            const int em = expo[item.first];
            const int S = scale_from(em) - (inv ? R0.log2n : 0);
            reinterpret_cast<double2 *>(R0.out)[(item.c0 + c) + (long long)N1 * t] =
                em == kNonFiniteExpo ? nan2()
                                     : make_double2(widen_scaled(v.rh, v.rl, S), widen_scaled(v.ih, v.il, S));
        }
    }
}

}  // namespace
}  // namespace oo
