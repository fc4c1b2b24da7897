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

}  // namespace ff
}  // namespace oo
