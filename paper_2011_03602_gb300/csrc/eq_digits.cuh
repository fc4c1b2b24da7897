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

// One product's split job arguments (grouped products and the serving loop)
struct GSplit {
    const double *A, *B;
    long long lda, ldb, pitch;  // pitch: row pitch (elements) of the stacked operands
    int m, n, k, kp, beta, slices;
    __nv_bfloat16 *As, *Bs;     // row 0 of slice 0 of this problem: slice p of row r at As[(p m + r) pitch]
    int *ea, *eb;
};

// Rows [r0, r0 + warps) of A, one warp per row: the row's scale exponent ea
// and its digit slices (zero digits fill [k, kp)).
__device__ __forceinline__ void split_rows_job(const GSplit &G, int r0) {
    const int lane = threadIdx.x & 31;
    const int row = r0 + (threadIdx.x >> 5);
    if (row >= G.m) return;
    const double *src = G.A + (long long)row * G.lda;
    int mx = 0;
#pragma unroll 4
    for (int l = lane; l < G.k; l += 32) mx = max(mx, eff_exp(src[l]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) G.ea[row] = mx == 0 ? 0 : mx - 1022;
    const size_t plane2 = (size_t)G.m * G.pitch / 2;
    unsigned *dst = reinterpret_cast<unsigned *>(G.As + (size_t)row * G.pitch);
    for (int l2 = lane; l2 < G.kp / 2; l2 += 32) {
        const int l = 2 * l2;
        unsigned n0 = 0, n1 = 0;
        const unsigned long long X0 = (mx != 0 && l < G.k) ? fixed_frac(src[l], mx, n0) : 0ull;
        const unsigned long long X1 = (mx != 0 && l + 1 < G.k) ? fixed_frac(src[l + 1], mx, n1) : 0ull;
        for (int p = 0; p < G.slices; ++p) dst[p * plane2 + l2] = digit_pair(X0, n0, X1, n1, G.beta, p);
    }
}

// Columns [c0, c0 + 64) of B: each column's scale exponent eb (largest over
// all k) and its transposed digit slices through 64 x 64 shared-memory
// tiles.  Every thread of the block calls it (it synchronises the block);
// blockDim.x a multiple of 64, t and red shared arrays of 64 x 65 doubles and
// (blockDim.x / 64) x 64 ints.
__device__ __forceinline__ void split_cols_job(const GSplit &G, int c0, double (*t)[65], int (*red)[64]) {
    const int lane = threadIdx.x & 31;
    const int ny = blockDim.x >> 6, nw = blockDim.x >> 5;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 columns x ny row groups
    const int col = c0 + tx;
    int mx = 0;
    if (col < G.n)
#pragma unroll 4
        for (int l = ty; l < G.k; l += ny) mx = max(mx, eff_exp(G.B[(long long)l * G.ldb + col]));
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0) {
        for (int y = 1; y < ny; ++y) mx = max(mx, red[y][tx]);
        red[0][tx] = mx;
        if (col < G.n) G.eb[col] = mx == 0 ? 0 : mx - 1022;
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, cpw = 64 / nw;  // columns written per warp
    const size_t plane2 = (size_t)G.n * G.pitch / 2;
    for (int l0 = 0; l0 < G.kp; l0 += 64) {
#pragma unroll 4
        for (int yy = ty; yy < 64; yy += ny) {
            const int l = l0 + yy;
            t[yy][tx] = (l < G.k && col < G.n) ? G.B[(long long)l * G.ldb + col] : 0.0;
        }
        __syncthreads();
        for (int cc = w * cpw; cc < w * cpw + cpw; ++cc) {
            const int c = c0 + cc;
            if (c >= G.n) break;
            const int cm = red[0][cc];
            unsigned n0 = 0, n1 = 0;
            const unsigned long long X0 = cm != 0 ? fixed_frac(t[2 * lane][cc], cm, n0) : 0ull;
            const unsigned long long X1 = cm != 0 ? fixed_frac(t[2 * lane + 1][cc], cm, n1) : 0ull;
            unsigned *dst = reinterpret_cast<unsigned *>(G.Bs + (size_t)c * G.pitch + l0) + lane;
            for (int p = 0; p < G.slices; ++p) dst[p * plane2] = digit_pair(X0, n0, X1, n1, G.beta, p);
        }
        __syncthreads();
    }
}

}  // namespace eq
}  // namespace oo
