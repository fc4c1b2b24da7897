// FP64-equivalent matrix product: the shared parts of its single-problem
// kernel (gemm_fp64eq.cu) and its grouped, tile-width-tuned kernel
// (gemm_eq_group.cu) -- the digit split of an FP64 entry and the
// accumulation schemes.
//
// Ozaki-type error-free splitting (Ozaki, Ogita, Oishi, Rump 2012): an entry
// of row i of A is a_il = 2^ea_i sum_p d_p 2^(-beta p) + r, with signed
// beta-bit integer digits d_p read straight from its fixed-point mantissa
// relative to the row scale 2^ea_i (columns of B alike); every digit is
// exact in BF16, every digit product exact in FP32, and a sum of such
// products stays exact in an FP32 accumulator while it holds fewer than 2^24
// units.  C_ij = 2^(ea_i + eb_j) sum_{p + q <= L} 2^(-beta (p + q)) D_pq(i, j),
// D_pq = sum_l d^A_p d^B_q over K-blocks of kb terms.  Dropping the levels
// p + q > L and the split remainders costs at most about
// (L + 2) 2^(-beta (L - 1)) of k max|a_i.| max|b_.j|; L is the smallest level
// with 4 (L + 2) 2^(-beta (L - 1)) <= 2^-42.
//
// Three ways to accumulate the products (a "scheme", a fixed function of k
// so that a problem gives the same bits alone and inside a batch):
//   kSchemePairs  one accumulator per product D_pq, products sharing A_p
//                 paired into one N = 2 BN MMA (kb <= 1024: beta 8 when
//                 kb <= 256, else 7); the epilogue reads every product.
//   kSchemeLevel7 one accumulator per level s = p + q: every D_pq of the
//                 level summed in the same FP32 accumulator, which stays
//                 exact with beta = 7 and kb = 128 ((L - 1) kb 127^2 < 2^24);
//                 the epilogue reads L - 1 levels per K-block, not every
//                 product.
//   kSchemeLevel6 the same with beta = 6 and kb = 512 (8 * 512 * 63^2 <
//                 2^24): more products (L = 9), fewer K-blocks.
#pragma once

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "tc.cuh"

namespace oo {
namespace eq {

constexpr int kBK = 64;  // K elements per pipeline stage (one 128-byte swizzled row)
enum { kSchemePairs = 0, kSchemeLevel7 = 1, kSchemeLevel6 = 2, kSchemes = 3 };

struct Shape {
    int scheme, beta, levels, slices, kb, nkb, nprod;
};

// smallest L with 4 (L + 2) 2^(-beta (L - 1)) <= 2^-42
inline int level_bound(int beta) {
    int L = 2;
    while (std::log2(4.0 * (L + 2)) - beta * (L - 1) > -42.0) ++L;
    return L;
}

inline Shape shape(int scheme, int k) {
    Shape e{};
    e.scheme = scheme;
    const int kp = (k + kBK - 1) / kBK * kBK;
    if (scheme == kSchemeLevel7) {
        e.kb = std::min(kp, 128);
        e.beta = 7;
    } else if (scheme == kSchemeLevel6) {
        e.kb = std::min(kp, 512);
        e.beta = 6;
    } else {
        e.kb = std::min(kp, 1024);
        e.beta = e.kb <= 256 ? 8 : 7;
    }
    e.levels = level_bound(e.beta);
    e.slices = e.levels - 1;
    e.nkb = (kp + e.kb - 1) / e.kb;
    e.nprod = e.levels * (e.levels - 1) / 2;
    return e;
}

// Exponent field used for the scale: subnormals count as exponent 1, zero
// as 0 (no contribution), NaN and infinities as tc::kNonFiniteExp.
__device__ __forceinline__ int eff_exp(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e != 0) return e == 0x7ff ? tc::kNonFiniteExp : e;
    return (b & 0x000fffffffffffffull) ? 1 : 0;
}

// |x| * 2^(64 - E) as a 64-bit fixed-point fraction (truncated), where
// 2^E = 2^(mx - 1022) bounds the row / column; the sign separately.
__device__ __forceinline__ unsigned long long fixed_frac(double x, int mx, unsigned &neg) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    neg = (unsigned)(b >> 63);
    int e = (int)((b >> 52) & 0x7ff);
    unsigned long long m = b & 0x000fffffffffffffull;
    if (e == 0) {
        if (m == 0) return 0ull;
        e = 1;
    } else {
        m |= 1ull << 52;
    }
    // x = m 2^(e - 1075), X = x 2^(64 - (mx - 1022)) = m 2^(e - mx + 11)
    const int sh = e - mx + 11;
    if (sh >= 0) return m << sh;  // sh <= 11: m < 2^53 keeps X < 2^64
    if (sh <= -64) return 0ull;
    return m >> (-sh);
}

// digit p (0-based) of X as a signed BF16 integer
__device__ __forceinline__ __nv_bfloat16 digit(unsigned long long X, unsigned neg, int beta, int p) {
    const unsigned d = (unsigned)(X >> (64 - beta * (p + 1))) & ((1u << beta) - 1u);
    const float f = __uint2float_rn(d);
    return __float2bfloat16_rn(neg ? -f : f);
}

// The same digits of two entries packed as a BF16 pair (first entry in the
// low half), by exponent arithmetic: d < 2^8 is exact as 2^23 + d - 2^23 in
// FP32 and in that float's top 16 bits, which are its BF16 bits; the sign is
// OR-ed in (a zero digit of a negative entry is -0, as the conversion above
// gives).  Bit for bit what digit() gives, without the integer-to-float and
// float-to-BF16 conversion instructions.
__device__ __forceinline__ unsigned digit_bits(unsigned long long X, unsigned neg, int beta, int p) {
    const unsigned d = (unsigned)(X >> (64 - beta * (p + 1))) & ((1u << beta) - 1u);
    const float f = __fsub_rn(__uint_as_float(0x4b000000u | d), 8388608.0f);
    return (__float_as_uint(f) >> 16) | (neg << 15);
}
__device__ __forceinline__ unsigned digit_pair(unsigned long long X0, unsigned n0, unsigned long long X1, unsigned n1,
                                               int beta, int p) {
    return digit_bits(X0, n0, beta, p) | (digit_bits(X1, n1, beta, p) << 16);
}

}  // namespace eq
}  // namespace oo
