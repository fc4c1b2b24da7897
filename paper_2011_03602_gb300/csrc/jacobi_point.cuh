// The Jacobi stencil nest's per-point arithmetic without tiling: the
// cooperative all-iterations kernel (jacobi.cu) and the device-resident
// serving loop (serve_resident.cu) share it.  The same float-float terms in
// the same order as the tiled kernel, so wrk2 is bit-identical to it.
#pragma once

#include <cuda_runtime.h>

#include "ff.cuh"
#include "oo_internal.h"

namespace oo {
namespace {

// The 19 values of p one interior point's update reads: planes i-1, i, i+1
// (W, C, E), each as a 3 x 3 window over (j - 1 .. j + 1) x (k - 1 .. k + 1),
// [dj][dk].  Of planes i +- 1 only the centre cross is read.
struct PWin {
    float w[3][3];
};

// The update of one interior point from its windows: wrk2 = p + omega ss,
// rounded once (returned); ss^2 is added to the float-float residual
// (RH, RL).  The float-float terms in the same order as the tiled kernel,
// so the value is bit-identical to it.
__device__ __forceinline__ float stencil_point_core(const float cf[NCOEF], const PWin &W, const PWin &C,
                                                    const PWin &E, float omega, float &RH, float &RL) {
    using ff::two_prod;
    using ff::two_sum;
    auto ff_acc = [](float &H, float &L, float th, float tl) { ff::acc(H, L, th, tl); };
    const float pc = C.w[1][1], pE = E.w[1][1], pW = W.w[1][1], pN = C.w[2][1], pS = C.w[0][1];
    const float pKp = C.w[1][2], pKm = C.w[1][0];
    float H, L, th, tl, t1, xh, xl, e;
    two_prod(cf[0], pE, H, L);                                   // a0 p[i+1]
    two_prod(cf[1], pN, th, tl); ff_acc(H, L, th, tl);           // a1 p[j+1]
    two_prod(cf[2], pKp, th, tl); ff_acc(H, L, th, tl);          // a2 p[k+1]
    {   // b0 Xij: D(i+1) - D(i-1), D = p(j+1) - p(j-1) exact pairs
        float dnh, dnl, gh, gl;
        two_sum(E.w[2][1], -E.w[0][1], dnh, dnl);
        two_sum(W.w[2][1], -W.w[0][1], gh, gl);
        two_sum(dnh, -gh, xh, e);
        xl = __fadd_rn(e, __fsub_rn(dnl, gl));
        two_prod(cf[4], xh, th, t1);
        tl = __fmaf_rn(cf[4], xl, t1);
        ff_acc(H, L, th, tl);
    }
    {   // b1 Xjk: D(k+1) - D(k-1) on plane i
        float dph, dpl, dmh, dml;
        two_sum(C.w[2][2], -C.w[0][2], dph, dpl);
        two_sum(C.w[2][0], -C.w[0][0], dmh, dml);
        two_sum(dph, -dmh, xh, e);
        xl = __fadd_rn(e, __fsub_rn(dpl, dml));
        two_prod(cf[5], xh, th, t1);
        tl = __fmaf_rn(cf[5], xl, t1);
        ff_acc(H, L, th, tl);
    }
    {   // b2 Xik: F(k+1) - F(k-1), F = p(i+1) - p(i-1) on row j
        float fph, fpl, fmh, fml;
        two_sum(E.w[1][2], -W.w[1][2], fph, fpl);
        two_sum(E.w[1][0], -W.w[1][0], fmh, fml);
        two_sum(fph, -fmh, xh, e);
        xl = __fadd_rn(e, __fsub_rn(fpl, fml));
        two_prod(cf[6], xh, th, t1);
        tl = __fmaf_rn(cf[6], xl, t1);
        ff_acc(H, L, th, tl);
    }
    two_prod(cf[7], pW, th, tl); ff_acc(H, L, th, tl);           // c0 p[i-1]
    two_prod(cf[8], pS, th, tl); ff_acc(H, L, th, tl);           // c1 p[j-1]
    two_prod(cf[9], pKm, th, tl); ff_acc(H, L, th, tl);          // c2 p[k-1]
    ff_acc(H, L, cf[11], 0.0f);                                  // wrk1
    // ss = (s0 a3 - p) bnd; wrk2 = p + omega ss, rounded once
    float dh, dl, e1, sh, s1;
    two_prod(H, cf[3], th, t1);
    tl = __fmaf_rn(L, cf[3], t1);
    two_sum(th, -pc, dh, e1);
    dl = __fadd_rn(e1, tl);
    two_prod(dh, cf[10], sh, s1);
    const float sl = __fmaf_rn(dl, cf[10], s1);
    float wh, w1, yh, e2;
    two_prod(omega, sh, wh, w1);
    const float wl = __fmaf_rn(omega, sl, w1);
    two_sum(pc, wh, yh, e2);
    const float out = __fadd_rn(yh, __fadd_rn(e2, wl));
    float nh, nl, qh, q1;
    two_sum(sh, sl, nh, nl);
    two_prod(nh, nh, qh, q1);
    const float ql = __fmaf_rn(__fadd_rn(nh, nh), nl, q1);
    ff_acc(RH, RL, qh, ql);
    return out;
}

// Plane window around element c, read through L2 (p is rewritten by other
// SMs between iterations, so never a stale L1 line); `full` false reads the
// centre cross only (planes i +- 1).
__device__ __forceinline__ void load_pwin(const float *p, size_t c, size_t sj, bool full, PWin &P) {
    P.w[1][1] = __ldcg(p + c);
    P.w[2][1] = __ldcg(p + c + sj);
    P.w[0][1] = __ldcg(p + c - sj);
    P.w[1][2] = __ldcg(p + c + 1);
    P.w[1][0] = __ldcg(p + c - 1);
    if (full) {
        P.w[2][2] = __ldcg(p + c + sj + 1);
        P.w[0][2] = __ldcg(p + c - sj + 1);
        P.w[2][0] = __ldcg(p + c + sj - 1);
        P.w[0][0] = __ldcg(p + c - sj - 1);
    } else {
        P.w[2][2] = P.w[0][2] = P.w[2][0] = P.w[0][0] = 0.0f;
    }
}

// One interior point c (element offset; si, sj the i and j strides in
// elements), without tiling: wrk2[c] from p; ss^2 added to (RH, RL).
__device__ __forceinline__ void stencil_point_ff(const float *const *coef, const float *p, size_t c, size_t si,
                                                 size_t sj, float omega, float *wrk2, float &RH, float &RL) {
    float cf[NCOEF];
#pragma unroll
    for (int q = 0; q < NCOEF; ++q) cf[q] = coef[q][c];
    PWin W, C, E;
    load_pwin(p, c - si, sj, false, W);
    load_pwin(p, c, sj, true, C);
    load_pwin(p, c + si, sj, false, E);
    wrk2[c] = stencil_point_core(cf, W, C, E, omega, RH, RL);
}

// face value of the Dirichlet boundary: (k / (K - 1))^2 as one correctly
// rounded float division of exact integers
__device__ __forceinline__ float jacobi_face_value(int k, int K) {
    return __fdiv_rn((float)(k * k), (float)((K - 1) * (K - 1)));
}

}  // namespace
}  // namespace oo
