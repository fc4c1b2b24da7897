// Float-float ("double-float") arithmetic: a value is an unevaluated sum
// hi + lo of two floats.  Error-free transforms: Knuth's two-sum and the
// FMA two-product (Dekker / Ogita-Rump-Oishi).  These carry about 44-48
// significant bits on the FP32 pipes, which on GB300 run ~59x faster than
// the FP64 pipe (69 vs 1.18 TFLOP/s measured).  Translation units using them
// must be compiled without FMA contraction (-fmad=false); intended FMAs are
// written explicitly.
#pragma once

namespace oo {
namespace ff {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// (H, L) += (th, tl), lo parts accumulated without renormalisation
__device__ __forceinline__ void acc(float &H, float &L, float th, float tl) {
    float e;
    two_sum(H, th, H, e);
    L = __fadd_rn(L, __fadd_rn(e, tl));
}
// (ah, al) + (bh, bl), renormalised
__device__ __forceinline__ void add(float ah, float al, float bh, float bl, float &h, float &l) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, h, l);
}

// complex float-float: (re.hi, re.lo, im.hi, im.lo)
struct cplx {
    float rh, rl, ih, il;
};

__device__ __forceinline__ cplx cadd(const cplx &a, const cplx &b) {
    cplx r;
    add(a.rh, a.rl, b.rh, b.rl, r.rh, r.rl);
    add(a.ih, a.il, b.ih, b.il, r.ih, r.il);
    return r;
}
__device__ __forceinline__ cplx csub(const cplx &a, const cplx &b) {
    cplx r;
    add(a.rh, a.rl, -b.rh, -b.rl, r.rh, r.rl);
    add(a.ih, a.il, -b.ih, -b.il, r.ih, r.il);
    return r;
}
// a * (-i) = (a.im, -a.re) and a * (+i) = (-a.im, a.re): exact
__device__ __forceinline__ cplx mul_neg_i(const cplx &a) { return cplx{a.ih, a.il, -a.rh, -a.rl}; }
__device__ __forceinline__ cplx mul_pos_i(const cplx &a) { return cplx{-a.ih, -a.il, a.rh, a.rl}; }
__device__ __forceinline__ cplx conj(const cplx &a) { return cplx{a.rh, a.rl, -a.ih, -a.il}; }

// a * w: each component is an exact two-term product difference plus the
// first-order cross terms, renormalised once
__device__ __forceinline__ cplx cmul(const cplx &a, const cplx &w) {
    cplx r;
    {
        float p1, e1, p2, e2, s, e3;
        two_prod(a.rh, w.rh, p1, e1);
        two_prod(a.ih, w.ih, p2, e2);
        two_sum(p1, -p2, s, e3);
        float e = __fadd_rn(__fsub_rn(e1, e2), e3);
        e = __fmaf_rn(a.rh, w.rl, e);
        e = __fmaf_rn(a.rl, w.rh, e);
        e = __fmaf_rn(-a.ih, w.il, e);
        e = __fmaf_rn(-a.il, w.ih, e);
        fast_two_sum(s, e, r.rh, r.rl);
    }
    {
        float p1, e1, p2, e2, s, e3;
        two_prod(a.rh, w.ih, p1, e1);
        two_prod(a.ih, w.rh, p2, e2);
        two_sum(p1, p2, s, e3);
        float e = __fadd_rn(__fadd_rn(e1, e2), e3);
        e = __fmaf_rn(a.rh, w.il, e);
        e = __fmaf_rn(a.rl, w.ih, e);
        e = __fmaf_rn(a.ih, w.rl, e);
        e = __fmaf_rn(a.il, w.rh, e);
        fast_two_sum(s, e, r.ih, r.il);
    }
    return r;
}

// h + l as a double (faithfully rounded) using integer operations only: on
// GB300 the FP64 pipe converts ~2.6x slower than this path.  Zero, subnormal
// and non-finite h take the plain widening.
__device__ __forceinline__ double to_double(float h, float l) {
    float s, e;
    two_sum(h, l, s, e);  // renormalise: |e| <= ulp(s) / 2
    const unsigned hb = __float_as_uint(s), lb = __float_as_uint(e);
    const unsigned eh = (hb >> 23) & 0xffu;
    if (eh == 0 || eh == 0xffu) return (double)s;
    unsigned long long M = (1ull << 52) | ((unsigned long long)(hb & 0x7fffffu) << 29);
    int E = (int)eh - 127 + 1023;
    const unsigned el = (lb >> 23) & 0xffu;
    if (el != 0) {
        const unsigned long long ml = (1ull << 23) | (lb & 0x7fffffu);
        const int sh = (int)el - (int)eh + 29;  // ml * 2^(el-150) in units of 2^(eh-127-52)
        const unsigned long long L = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> (-sh)) : 0ull);
        if ((lb ^ hb) & 0x80000000u)
            M -= L;
        else
            M += L;
        if (M >> 53) {
            M >>= 1;
            E += 1;
        } else if (!(M >> 52)) {
            M <<= 1;
            E -= 1;
        }
    }
    const unsigned long long bits = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                    ((unsigned long long)E << 52) | (M & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// d * 2^S by exponent arithmetic when the result stays normal
__device__ __forceinline__ double scale_pow2(double d, int S) {
    const long long b = __double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return d == 0.0 ? d : ldexp(d, S);
    const int ne = e + S;
    if (e == 0x7ff || ne <= 0 || ne >= 0x7ff) return ldexp(d, S);
    return __longlong_as_double(b + ((long long)S << 52));
}

}  // namespace ff
}  // namespace oo
