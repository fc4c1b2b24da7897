// FP64-equivalent matrix product (precision pattern OO_PREC_FP64EQ) for the
// matrix-product function block (Sec. 3.2.2): C = A B for FP64 row-major
// A (m x k) and B (k x n), computed on the BF16 tensor cores by an
// Ozaki-type error-free splitting (Ozaki, Ogita, Oishi, Rump 2012):
//
//   a_il = 2^ea_i * sum_{p=1..s} d^A_p(i,l) 2^(-beta p) + r   (|r| < 2^(ea_i - beta s))
//   b_lj = 2^eb_j * sum_{q=1..s} d^B_q(l,j) 2^(-beta q) + r'
//
// Each digit d is a signed integer with |d| <= 2^beta - 1, read directly
// as a beta-bit group of the entry's fixed-point mantissa relative to its
// row (A) or column (B) scale 2^e (no floating-point arithmetic in the
// split).  Digits are exact in BF16 (beta <= 8), their products exact in
// FP32, and with K-blocks of kb terms, kb (2^beta - 1)^2 < 2^24, every
// product's K-block sum D_pq = sum_l d^A_p d^B_q accumulates exactly in the
// FP32 accumulators of tensor memory, whatever order the hardware adds in.
//
//   C_ij = 2^(ea_i + eb_j) sum_{p + q <= L} 2^(-beta (p + q)) D_pq(i, j)
//
// The terms are summed in float-float (about 48 bits) in tensor memory,
// smallest level first, then widened to FP64 and scaled.  Dropping the
// levels p + q > L and the split remainders costs at most about
// (L + 2) 2^(-beta (L - 1)) 2^(ea_i + eb_j) k per element; L is the
// smallest level for which 4 (L + 2) 2^(-beta (L - 1)) <= 2^-42, i.e. at
// most ~2.3e-13 of sum_l |a_il| |b_lj| when the entries of a row (column)
// are of comparable size.
//
//   K-block kb = min(roundup64(k), 1024);  beta = 8 (kb <= 256) or 7;
//   beta 8: L = 7 (21 products); beta 7: L = 8 (28 products).
//
// Kernel: persistent, one CTA per SM over 128 x 128 output tiles.  The
// products are grouped in units that share the A slice: (p, q1) and
// (p, q2) become one M = 128, N = 256 MMA whose B operand is the two B
// slices' tiles stacked (a product without a partner runs alone at
// N = 128).  A unit of work is one such group over one K-block (K-blocks
// outermost, so one K-block's slices serve all groups while in L2): warp 0
// streams its A_p and B_q tiles (TMA, 128-byte swizzle) through a 4-stage
// ring, warp 1 issues tcgen05.mma (K = 16) into one of two 256-column FP32
// accumulators in tensor memory (double-buffered), and eight epilogue warps
// (two per tensor-memory lane quarter, one per 64-column half) add each
// finished accumulator, scaled by 2^(-beta (p + q)), into a float-float
// running sum held in registers; after the tile's last unit they write
// FP64 C.  Sharing A_p raises the MMA work per staged byte by a third,
// which is what bounds this kernel (operand latency, not tensor rate).
// Every mbarrier wait is bounded.
// A row of A or column of B holding a NaN or an infinity gives NaN in every
// entry of C it meets (tc.cuh, kNonFiniteExp); other entries are unaffected.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ff.cuh"
#include "oo_internal.h"
#include "eq_digits.cuh"
#include "tc.cuh"

namespace oo {

namespace {

using namespace tc;
using eq::eff_exp;
using eq::fixed_frac;

constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 4;
constexpr int kThreads = 320;              // producer, MMA issuer, 8 epilogue warps
constexpr int kEpiWarps = 8;
constexpr uint32_t kTile = kBM * kBK * 2;  // 16 KB, A and B tiles alike
constexpr uint32_t kStageBytes = 3 * kTile;  // A_p, B_q1, B_q2
constexpr int kGroupM = 8;
constexpr int kMaxUnits = 24;
constexpr uint32_t kIdescPair = idesc_bf16(kBM, 2 * kBN);
constexpr uint32_t kIdescOne = idesc_bf16(kBM, kBN);
constexpr unsigned char kNone = 0xff;

using EqShape = eq::Shape;
// the pair scheme this file's kernel runs
EqShape eq_shape(int k) { return eq::shape(eq::kSchemePairs, k); }
// the scheme the library uses for inner dimension k
EqShape eq_used_shape(int k) { return eq::shape(eq_scheme_for(k), k); }

// A unit: slice p of A against slices q1 and q2 (q2 = kNone: alone) of B
struct EqUnit {
    int p, q1, q2;
};
// Products (p, q), 1-based, p + q <= L, grouped by p in pairs of
// consecutive q; ordered from the smallest contributions up.
std::vector<EqUnit> eq_units(const EqShape &e) {
    std::vector<EqUnit> u;
    for (int p = 1; p <= e.slices; ++p)
        for (int q = 1; q <= e.levels - p; q += 2)
            u.push_back({p - 1, q - 1, q + 1 <= e.levels - p ? q : (int)kNone});
    std::stable_sort(u.begin(), u.end(), [](const EqUnit &a, const EqUnit &b) { return a.p + a.q1 > b.p + b.q1; });
    return u;
}

struct EqMaps {
    CUtensorMap a, b;  // all slices stacked: slice p at rows [p m, (p + 1) m)
};

struct EqArgs {
    int m, n, ksteps, kb_steps, nkb, nunits;
    int m_tiles, n_tiles;
    double *C;
    long long ldc;
    const int *ea, *eb;
    unsigned *err;
    unsigned char up[kMaxUnits], uq1[kMaxUnits], uq2[kMaxUnits];  // 0-based slices; uq2 kNone: alone
    float us1[kMaxUnits], us2[kMaxUnits];                           // 2^(-beta (p + q)), 1-based p, q
};

__device__ __forceinline__ void eq_tile(const EqArgs &a, int t, int &m0, int &n0) {
    const int per_group = kGroupM * a.n_tiles;
    const int g = t / per_group, r = t % per_group;
    const int rows = min(kGroupM, a.m_tiles - g * kGroupM);
    m0 = (g * kGroupM + r % rows) * kBM;
    n0 = (r / rows) * kBN;
}

#define OO_TMEM_LD16(taddr, r)                                                                              \
    asm volatile(                                                                                           \
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "  \
        "[%16];"                                                                                            \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),   \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),          \
          "=r"(r[15])                                                                                       \
        : "r"(taddr))

__global__ void __launch_bounds__(kThreads, 1) gemm_fp64eq_kernel(const __grid_constant__ EqMaps maps,
                                                                 const __grid_constant__ EqArgs a) {
    extern __shared__ __align__(1024) unsigned char esm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(esm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kStages * kStageBytes);
    uint64_t *full = bars, *empty = bars + kStages;
    uint64_t *tfull = bars + 2 * kStages, *tempty = bars + 2 * kStages + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = a.m_tiles * a.n_tiles;
    const int units = a.nunits * a.nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(su32(&full[s]), 1);
            bar_init(su32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(su32(&tfull[b]), 1);
            bar_init(su32(&tempty[b]), kEpiWarps);  // one arrival per epilogue warp
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(su32(tmem_slot), 512);
        fence_before();
    }
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    int loaded = 0;      // producer: stages issued
    int units_mma = 0;   // MMA issuer: units whose accumulation was issued
    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------- TMA producer
        int it = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
            int m0, n0;
            eq_tile(a, t, m0, n0);
            for (int u = 0; ok && u < units; ++u) {
                const int kbi = u / a.nunits, pr = u % a.nunits;  // K-block outer: its slices stay in L2
                const bool pair = a.uq2[pr] != kNone;
                const int rowA = a.up[pr] * a.m + m0, rowB1 = a.uq1[pr] * a.n + n0;
                const int rowB2 = pair ? a.uq2[pr] * a.n + n0 : 0;
                const int ks1 = min(a.ksteps, (kbi + 1) * a.kb_steps);
                for (int ks = kbi * a.kb_steps; ks < ks1; ++ks, ++it) {
                    const int s = it % kStages;
                    const uint32_t use = it / kStages;
                    if (use > 0 && !bar_wait(su32(&empty[s]), (use - 1) & 1, abort_flag, a.err, 1u)) {
                        ok = false;
                        break;
                    }
                    unsigned char *st = sm + (size_t)s * kStageBytes;
                    const uint32_t fb = su32(&full[s]);
                    bar_expect_tx(fb, pair ? 3 * kTile : 2 * kTile);
                    tma_2d(su32(st), &maps.a, ks * kBK, rowA, fb);
                    tma_2d(su32(st + kTile), &maps.b, ks * kBK, rowB1, fb);
                    if (pair) tma_2d(su32(st + 2 * kTile), &maps.b, ks * kBK, rowB2, fb);
                    ++loaded;
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------- MMA issuer
        int it = 0, gu = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
            for (int u = 0; ok && u < units; ++u, ++gu) {
                const int b = gu & 1;
                const uint32_t buse = gu >> 1;
                if (buse > 0 && !bar_wait(su32(&tempty[b]), (buse - 1) & 1, abort_flag, a.err, 2u)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(b * 2 * kBN);
                const int kbi = u / a.nunits, pr = u % a.nunits;  // K-block outer: its slices stay in L2
                const bool pair = a.uq2[pr] != kNone;
                const int ks0 = kbi * a.kb_steps, ks1 = min(a.ksteps, (kbi + 1) * a.kb_steps);
                for (int ks = ks0; ks < ks1; ++ks, ++it) {
                    const int s = it % kStages;
                    if (!bar_wait(su32(&full[s]), (it / kStages) & 1, abort_flag, a.err, 2u)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t sa = su32(sm + (size_t)s * kStageBytes), sb = sa + kTile;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint32_t off = kk * 32;  // 16 BF16 along K inside the 128-byte row
                        const uint32_t acc = (ks == ks0 && kk == 0) ? 0u : 1u;
                        if (pair)  // B_q1 and B_q2 tiles stacked: one N = 256 operand
                            mma_bf16<kIdescPair>(d, sdesc_sw128(sa + off), sdesc_sw128(sb + off), acc);
                        else
                            mma_bf16<kIdescOne>(d, sdesc_sw128(sa + off), sdesc_sw128(sb + off), acc);
                    }
                    mma_commit(su32(&empty[s]));
                }
                if (!ok) break;
                mma_commit(su32(&tfull[b]));  // this unit's accumulator is complete
                ++units_mma;
            }
        }
    } else if (warp >= 2) {
        // ---------------------------------------------------- epilogue
        const int q = warp & 3;              // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;       // 64-column half of the tile
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        float Sh[64], Sl[64];                // running float-float sum of this row's 64 columns
        int gu = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
            int m0, n0;
            eq_tile(a, t, m0, n0);
            for (int u = 0; u < units; ++u, ++gu) {
                const int b = gu & 1;
                if (!bar_wait(su32(&tfull[b]), (gu >> 1) & 1, abort_flag, a.err, 4u)) {
                    ok = false;
                    break;
                }
                fence_after();
                const int pr = u % a.nunits;
                const bool pair = a.uq2[pr] != kNone, first = u == 0;
                const float f1 = a.us1[pr], f2 = a.us2[pr];
                const uint32_t acc = tmem + (uint32_t)(b * 2 * kBN) + lane_off + (uint32_t)(h * 64);
#pragma unroll
                for (int c = 0; c < 64; c += 16) {
                    uint32_t v[16];
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        if (half == 1 && !pair) break;
                        OO_TMEM_LD16(acc + half * kBN + c, v);
                        tmem_wait_ld();
                        const float f = half ? f2 : f1;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float w = __fmul_rn(__uint_as_float(v[j]), f);  // exact: power-of-two scale
                            if (first && half == 0) {
                                Sh[c + j] = w;
                                Sl[c + j] = 0.0f;
                            } else {
                                ff::add(Sh[c + j], Sl[c + j], w, 0.0f, Sh[c + j], Sl[c + j]);
                            }
                        }
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(su32(&tempty[b]));
                if (u == units - 1) {
                    // column scales: lane l holds columns l and l + 32 of this
                    // half (coalesced) and hands them out by shuffle
                    const int row = m0 + q * 32 + lane;
                    const int c0 = n0 + h * 64;
                    const int e0 = c0 + lane < a.n ? a.eb[c0 + lane] : 0;
                    const int e1 = c0 + 32 + lane < a.n ? a.eb[c0 + 32 + lane] : 0;
                    const bool row_ok = row < a.m;
                    const int sa = row_ok ? a.ea[row] : 0;
                    double *crow = a.C + (long long)row * a.ldc + c0;
#pragma unroll
                    for (int j = 0; j < 64; ++j) {
                        const int sb = __shfl_sync(0xffffffffu, j < 32 ? e0 : e1, j & 31);
                        if (row_ok && c0 + j < a.n)
                            crow[j] = nan_or_scaled(ff::to_double(Sh[j], Sl[j]), sa + sb);
                    }
                }
            }
        }
    }
    // drain on abort: wait (bounded) for issued MMAs and copies before TMEM
    // is released and the CTA exits
    if (*abort_flag) {
        if (warp == 1 && lane == 0 && units_mma > 0)
            bar_drain(su32(&tfull[(units_mma - 1) & 1]), ((units_mma - 1) >> 1) & 1);
        if (warp == 0 && lane == 0)
            for (int it = (loaded > kStages ? loaded - kStages : 0); it < loaded; ++it)
                bar_drain(su32(&full[it % kStages]), (it / kStages) & 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------ CTA pairs
// The same products on CTA pairs (cta_group::2, M = 256): a tile is 256 rows
// x 128 columns, CTA r of the pair holding rows m0 + 128 r .. +127 of the
// tile and its own accumulators and running sums.  A two-product unit
// (p, q1) + (p, q2) is one M = 256, N = 256 MMA whose B operand is B_q1's
// tile in rank 0's shared memory and B_q2's in rank 1's, so an SM stages
// 32 KB (A_p and one B slice tile) per K step where a single CTA stages
// 48 KB for the same MMA work; a one-product unit is an N = 128 MMA, each
// CTA holding 64 of the tile's columns of B_q.  Rank 0 issues the MMAs;
// the commits arrive on both CTAs' barriers; both epilogues report to rank
// 0 that their accumulator buffer is free.  The D_pq of a K-block are exact
// whatever the instruction shape, and the epilogue adds the units in the
// same order, so the result is the single-CTA kernel's bit for bit.
constexpr int kStagesPair = 6;
constexpr uint32_t kStageBytesPair = 2 * kTile;  // A_p and this CTA's B tile
constexpr uint32_t kIdescPair2 = idesc_bf16(2 * kBM, 2 * kBN);
constexpr uint32_t kIdescOne2 = idesc_bf16(2 * kBM, kBN);

struct EqPairMaps {
    CUtensorMap a, b, bh;  // bh: B slices in 64-row boxes (one-product units)
};

__device__ __forceinline__ void eq_tile_pair(const EqArgs &a, int t, int &m0, int &n0) {
    const int per_group = (kGroupM / 2) * a.n_tiles;
    const int g = t / per_group, r = t % per_group;
    const int rows = min(kGroupM / 2, a.m_tiles - g * (kGroupM / 2));
    m0 = (g * (kGroupM / 2) + r % rows) * 2 * kBM;
    n0 = (r / rows) * kBN;
}

// a.m_tiles counts 256-row slabs here
__global__ void __launch_bounds__(kThreads, 1) gemm_fp64eq_pair_kernel(const __grid_constant__ EqPairMaps maps,
                                                                      const __grid_constant__ EqArgs a) {
    extern __shared__ __align__(1024) unsigned char esm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(esm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kStagesPair * kStageBytesPair);
    uint64_t *full = bars, *empty = bars + kStagesPair;
    uint64_t *tfull = bars + 2 * kStagesPair, *tempty = tfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
    const int tiles = a.m_tiles * a.n_tiles;
    const int units = a.nunits * a.nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesPair; ++s) {
            bar_init(su32(&full[s]), 1);   // rank 0's: its expect-tx arrival + both CTAs' bytes
            bar_init(su32(&empty[s]), 1);  // the MMA commit
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(su32(&tfull[b]), 1);
            bar_init(su32(&tempty[b]), 2 * kEpiWarps);  // rank 0's: every epilogue warp of both CTAs
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc_pair(su32(tmem_slot), 512);
        fence_before();
    }
    __syncthreads();
    cluster_sync_all();  // both CTAs' barriers and TMEM exist before either uses the other's
    fence_after();
    const uint32_t tmem = *tmem_slot;

    int loaded = 0, units_mma = 0;
    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------- TMA producer (both CTAs)
        int it = 0;
        bool ok = true;
        for (int t = cid; ok && t < tiles; t += ncl) {
            int m0, n0;
            eq_tile_pair(a, t, m0, n0);
            for (int u = 0; ok && u < units; ++u) {
                const int kbi = u / a.nunits, pr = u % a.nunits;  // K-block outer: its slices stay in L2
                const bool pair = a.uq2[pr] != kNone;
                const int rowA = a.up[pr] * a.m + m0 + (int)rank * kBM;
                const int rowB = pair ? (rank ? a.uq2[pr] : a.uq1[pr]) * a.n + n0
                                      : a.uq1[pr] * a.n + n0 + (int)rank * (kBN / 2);
                const uint32_t tx = pair ? 2 * 2 * kTile : 2 * (kTile + kTile / 2);
                const int ks1 = min(a.ksteps, (kbi + 1) * a.kb_steps);
                for (int ks = kbi * a.kb_steps; ks < ks1; ++ks, ++it) {
                    const int s = it % kStagesPair;
                    const uint32_t use = it / kStagesPair;
                    if (use > 0 && !bar_wait_cluster(su32(&empty[s]), (use - 1) & 1, abort_flag, a.err, 1u)) {
                        ok = false;
                        break;
                    }
                    unsigned char *st = sm + (size_t)s * kStageBytesPair;
                    if (leader) bar_expect_tx(su32(&full[s]), tx);
                    const uint32_t fb = map_to_rank(su32(&full[s]), 0);
                    tma_2d_pair(su32(st), &maps.a, ks * kBK, rowA, fb);
                    tma_2d_pair(su32(st + kTile), pair ? &maps.b : &maps.bh, ks * kBK, rowB, fb);
                    ++loaded;
                }
            }
        }
    } else if (warp == 1 && lane == 0 && leader) {
        // ---------------------------------------------------- MMA issuer (rank 0)
        int it = 0, gu = 0;
        bool ok = true;
        for (int t = cid; ok && t < tiles; t += ncl) {
            for (int u = 0; ok && u < units; ++u, ++gu) {
                const int b = gu & 1;
                const uint32_t buse = gu >> 1;
                if (buse > 0 && !bar_wait_cluster(su32(&tempty[b]), (buse - 1) & 1, abort_flag, a.err, 2u)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(b * 2 * kBN);
                const int kbi = u / a.nunits, pr = u % a.nunits;
                const uint32_t idesc = a.uq2[pr] != kNone ? kIdescPair2 : kIdescOne2;
                const int ks0 = kbi * a.kb_steps, ks1 = min(a.ksteps, (kbi + 1) * a.kb_steps);
                for (int ks = ks0; ks < ks1; ++ks, ++it) {
                    const int s = it % kStagesPair;
                    if (!bar_wait_cluster(su32(&full[s]), (it / kStagesPair) & 1, abort_flag, a.err, 2u)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t sa = su32(sm + (size_t)s * kStageBytesPair), sb = sa + kTile;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint32_t acc = (ks == ks0 && kk == 0) ? 0u : 1u;
                        mma_bf16_pair(d, sdesc_sw128(sa + off), sdesc_sw128(sb + off), idesc, acc);
                    }
                    mma_commit_pair(su32(&empty[s]), 3);  // stage s free in both CTAs
                }
                if (!ok) break;
                mma_commit_pair(su32(&tfull[b]), 3);  // this unit's accumulators complete in both CTAs
                ++units_mma;
            }
        }
    } else if (warp >= 2) {
        // ---------------------------------------------------- epilogue (both CTAs)
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        float Sh[64], Sl[64];
        int gu = 0;
        bool ok = true;
        for (int t = cid; ok && t < tiles; t += ncl) {
            int m0, n0;
            eq_tile_pair(a, t, m0, n0);
            m0 += (int)rank * kBM;
            for (int u = 0; u < units; ++u, ++gu) {
                const int b = gu & 1;
                if (!bar_wait_cluster(su32(&tfull[b]), (gu >> 1) & 1, abort_flag, a.err, 4u)) {
                    ok = false;
                    break;
                }
                fence_after();
                const int pr = u % a.nunits;
                const bool pair = a.uq2[pr] != kNone, first = u == 0;
                const float f1 = a.us1[pr], f2 = a.us2[pr];
                const uint32_t acc = tmem + (uint32_t)(b * 2 * kBN) + lane_off + (uint32_t)(h * 64);
#pragma unroll
                for (int c = 0; c < 64; c += 16) {
                    uint32_t v[16];
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        if (half == 1 && !pair) break;
                        OO_TMEM_LD16(acc + half * kBN + c, v);
                        tmem_wait_ld();
                        const float f = half ? f2 : f1;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float w = __fmul_rn(__uint_as_float(v[j]), f);  // exact: power-of-two scale
                            if (first && half == 0) {
                                Sh[c + j] = w;
                                Sl[c + j] = 0.0f;
                            } else {
                                ff::add(Sh[c + j], Sl[c + j], w, 0.0f, Sh[c + j], Sl[c + j]);
                            }
                        }
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (leader)
                        bar_arrive(su32(&tempty[b]));
                    else
                        bar_arrive_remote(map_to_rank(su32(&tempty[b]), 0));
                }
                if (u == units - 1) {
                    const int row = m0 + q * 32 + lane;
                    const int c0 = n0 + h * 64;
                    const int e0 = c0 + lane < a.n ? a.eb[c0 + lane] : 0;
                    const int e1 = c0 + 32 + lane < a.n ? a.eb[c0 + 32 + lane] : 0;
                    const bool row_ok = row < a.m;
                    const int sa = row_ok ? a.ea[row] : 0;
                    double *crow = a.C + (long long)row * a.ldc + c0;
#pragma unroll
                    for (int j = 0; j < 64; ++j) {
                        const int sb = __shfl_sync(0xffffffffu, j < 32 ? e0 : e1, j & 31);
                        if (row_ok && c0 + j < a.n)
                            crow[j] = nan_or_scaled(ff::to_double(Sh[j], Sl[j]), sa + sb);
                    }
                }
            }
        }
    }
    // drain on abort (bounded): rank 0 waits for its issued MMAs and for the
    // copies counted on its barriers; rank 1 for the commits that free its
    // stages (its copies complete on rank 0's barriers)
    if (*abort_flag) {
        if (warp == 1 && lane == 0 && leader && units_mma > 0)
            bar_drain(su32(&tfull[(units_mma - 1) & 1]), ((units_mma - 1) >> 1) & 1);
        if (warp == 0 && lane == 0)
            for (int it = (loaded > kStagesPair ? loaded - kStagesPair : 0); it < loaded; ++it)
                bar_drain(su32(leader ? &full[it % kStagesPair] : &empty[it % kStagesPair]),
                          (it / kStagesPair) & 1);
    }
    fence_before();
    __syncthreads();
    cluster_sync_all();  // neither CTA leaves while the other may still signal it or read its TMEM
    if (warp == 1) {
        fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
}

// ------------------------------------------------------------ splitting
// A (m x k, lda) -> ea and slices As[p] (m x kp each, p < s); one warp per row
__global__ void eq_split_rows_kernel(const double *A, long long lda, int m, int k, int kp, int beta, int s,
                                     int *ea, __nv_bfloat16 *As) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= m) return;
    const int lane = threadIdx.x & 31;
    const double *src = A + (long long)row * lda;
    int mx = 0;
#pragma unroll 4
    for (int l = lane; l < k; l += 32) mx = max(mx, eff_exp(src[l]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) ea[row] = mx == 0 ? 0 : mx - 1022;
    const size_t plane = (size_t)m * kp;
    __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(As + (size_t)row * kp);
    for (int l2 = lane; l2 < kp / 2; l2 += 32) {
        const int l = 2 * l2;
        unsigned n0 = 0, n1 = 0;
        const unsigned long long X0 = (mx != 0 && l < k) ? fixed_frac(src[l], mx, n0) : 0ull;
        const unsigned long long X1 = (mx != 0 && l + 1 < k) ? fixed_frac(src[l + 1], mx, n1) : 0ull;
        for (int p = 0; p < s; ++p)
            reinterpret_cast<unsigned *>(dst)[p * (plane / 2) + l2] = eq::digit_pair(X0, n0, X1, n1, beta, p);
    }
}

// Same split, one 256-thread CTA per row and 16-byte loads (lda even, A
// 16-byte aligned): the row's second read hits L1, and each thread keeps
// eight loads in flight in the exponent pass.
__global__ void __launch_bounds__(256) eq_split_rows_v2_kernel(const double *A, long long lda, int m, int k, int kp,
                                                             int beta, int s, int *ea, __nv_bfloat16 *As) {
    const int row = blockIdx.x;
    const double2 *src = reinterpret_cast<const double2 *>(A + (long long)row * lda);
    const int k2 = k >> 1;
    int mx = 0;
#pragma unroll 8
    for (int l2 = threadIdx.x; l2 < k2; l2 += 256) {
        const double2 v = src[l2];
        mx = max(mx, max(eff_exp(v.x), eff_exp(v.y)));
    }
    if ((k & 1) && threadIdx.x == 0) mx = max(mx, eff_exp(A[(long long)row * lda + k - 1]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ int red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = max(mx, red[w]);
    if (threadIdx.x == 0) ea[row] = mx == 0 ? 0 : mx - 1022;
    const size_t plane2 = (size_t)m * kp / 2;
    __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(As + (size_t)row * kp);
#pragma unroll 2
    for (int l2 = threadIdx.x; l2 < kp / 2; l2 += 256) {
        const int l = 2 * l2;
        double2 v = make_double2(0.0, 0.0);
        if (l + 1 < k) {
            v = src[l2];
        } else if (l < k) {
            v.x = A[(long long)row * lda + l];
        }
        unsigned n0 = 0, n1 = 0;
        const unsigned long long X0 = mx != 0 ? fixed_frac(v.x, mx, n0) : 0ull;
        const unsigned long long X1 = mx != 0 ? fixed_frac(v.y, mx, n1) : 0ull;
        for (int p = 0; p < s; ++p)
            reinterpret_cast<unsigned *>(dst)[p * plane2 + l2] = eq::digit_pair(X0, n0, X1, n1, beta, p);
    }
}

// largest effective exponent of each column of B (k x n); grid.x column
// blocks of 32, grid.y row chunks
__global__ void eq_col_maxexp_kernel(const double *B, long long ldb, int k, int n, int rows_per, int *mxo) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * rows_per, r1 = min(k, r0 + rows_per);
    if (col >= n) return;
    int mx = 0;
#pragma unroll 8
    for (int l = r0 + threadIdx.y; l < r1; l += blockDim.y) mx = max(mx, eff_exp(B[(long long)l * ldb + col]));
    if (mx > 0) atomicMax(mxo + col, mx);
}

// B tile of 64 (k) x 64 (columns) -> transposed slices Bs[q] (n x kp each);
// mxo holds the column maxima (exponent fields); 256 threads
__global__ void eq_split_cols_t_kernel(const double *B, long long ldb, int k, int n, int kp, int beta, int s,
                                       const int *mxo, __nv_bfloat16 *Bs) {
    __shared__ double t[64][65];
    const int c0 = blockIdx.x * 64, l0 = blockIdx.y * 64;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
#pragma unroll
    for (int yy = ty; yy < 64; yy += 4) {
        const int l = l0 + yy, c = c0 + tx;
        t[yy][tx] = (l < k && c < n) ? B[(long long)l * ldb + c] : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t plane = (size_t)n * kp;
    for (int cc = w * 8; cc < w * 8 + 8; ++cc) {
        const int c = c0 + cc;
        if (c >= n) break;
        const int mx = mxo[c];
        unsigned n0 = 0, n1 = 0;
        const unsigned long long X0 = mx != 0 ? fixed_frac(t[2 * lane][cc], mx, n0) : 0ull;
        const unsigned long long X1 = mx != 0 ? fixed_frac(t[2 * lane + 1][cc], mx, n1) : 0ull;
        __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(Bs + (size_t)c * kp + l0) + lane;
        for (int p = 0; p < s; ++p)
            reinterpret_cast<unsigned *>(dst)[p * (plane / 2)] = eq::digit_pair(X0, n0, X1, n1, beta, p);
    }
}

__global__ void eq_col_scale_kernel(const int *mxo, int *eb, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) eb[i] = mxo[i] == 0 ? 0 : mxo[i] - 1022;
}

size_t smem_eq() { return 1024 + (size_t)kStages * kStageBytes + 256; }
constexpr size_t kSmemEqPair = 1024 + (size_t)kStagesPair * kStageBytesPair + 256;
static_assert(kSmemEqPair <= 232448, "pair kernel exceeds the shared memory of a CTA");

// 2-CTA clusters of the pair kernel that fit on the device at once (cached)
int eq_pair_clusters() {
    int dev = 0;
    OO_CUDA_TRY(cudaGetDevice(&dev));
    static std::atomic<int> max_clusters[64];
    int ncl = dev < 64 ? max_clusters[dev].load() : 0;
    if (ncl > 0) return ncl;
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)gemm_fp64eq_pair_kernel, kSmemEqPair, attr);
    int sms = 148;
    OO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(sms / 2 * 2));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemEqPair;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    OO_CUDA_TRY(cudaOccupancyMaxActiveClusters(&ncl, (const void *)gemm_fp64eq_pair_kernel, &cfg));
    OO_REQUIRE(ncl >= 1, OO_ECUDA, "no 2-CTA cluster of the FP64-equivalent kernel fits on this device");
    if (dev < 64) max_clusters[dev].store(ncl);
    return ncl;
}

struct EqLayout {
    size_t err, ea, eb, mxo, as, bs, total;
};
EqLayout eq_layout(int m, int n, int k) {
    const EqShape e = eq_used_shape(k);
    const size_t kp = (size_t)(k + kBK - 1) / kBK * kBK;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    EqLayout L{};
    L.err = 0;
    L.ea = 256;
    L.eb = L.ea + up((size_t)m * 4);
    L.mxo = L.eb + up((size_t)n * 4);
    L.as = L.mxo + up((size_t)n * 4);
    L.bs = L.as + up((size_t)e.slices * m * kp * 2);
    L.total = L.bs + up((size_t)e.slices * n * kp * 2);
    return L;
}

}  // namespace

// The grouped products' digit split (their tensor-core kernel is in
// gemm_eq_group.cu, which reads only through L2 for the device-resident
// loop's sake; the split's second pass over a row wants L1): jobs (0,
// problem, first row), eight rows of A each, in one kernel that uses no
// shared memory -- so more of its blocks fit on an SM and L1 keeps the rows
// for their second pass -- then jobs (1, problem, first column), 64 columns
// of B each, through shared-memory tiles (eq_digits.cuh).
namespace {
__global__ void __launch_bounds__(256) eq_group_split_rows_kernel(const eq::GSplit *gs, const int4 *jobs) {
    const int4 jb = jobs[blockIdx.x];
    eq::split_rows_job(gs[jb.y], jb.z);
}
__global__ void __launch_bounds__(256) eq_group_split_cols_kernel(const eq::GSplit *gs, const int4 *jobs) {
    __shared__ double t[64][65];
    __shared__ int red[4][64];
    const int4 jb = jobs[blockIdx.x];
    eq::split_cols_job(gs[jb.y], jb.z, t, red);
}
}  // namespace

void launch_eq_group_split(const eq::GSplit *gs, const int4 *jobs, int nrow_jobs, int ncol_jobs, cudaStream_t s) {
    if (nrow_jobs > 0) {
        eq_group_split_rows_kernel<<<nrow_jobs, 256, 0, s>>>(gs, jobs);
        OO_CUDA_TRY(cudaGetLastError());
    }
    if (ncol_jobs > 0) {
        eq_group_split_cols_kernel<<<ncol_jobs, 256, 0, s>>>(gs, jobs + nrow_jobs);
        OO_CUDA_TRY(cudaGetLastError());
    }
}

size_t gemm_fp64eq_scratch_bytes(int m, int n, int k) { return eq_layout(m, n, k).total; }

int gemm_fp64eq_products(int k) { return eq_used_shape(k).nprod; }

void gemm_fp64eq_shape(int k, int *beta, int *levels, int *k_block) {
    const EqShape e = eq_used_shape(k);
    if (beta) *beta = e.beta;
    if (levels) *levels = e.levels;
    if (k_block) *k_block = e.kb;
}

void launch_gemm_fp64eq(int m, int n, int k, const double *A, long long lda, const double *B, long long ldb,
                        double *C, long long ldc, void *scratch, cudaStream_t s, int width, bool pair) {
    OO_REQUIRE(m >= 1 && n >= 1 && k >= 1, OO_EINVAL, "m, n, k must be >= 1");
    OO_REQUIRE(lda >= k && ldb >= n && ldc >= n, OO_EINVAL, "leading dimensions too small");
    const EqShape e = eq_used_shape(k);
    OO_REQUIRE((long long)e.slices * m < (1ll << 31) && (long long)e.slices * n < (1ll << 31), OO_EINVAL,
               "matrix too large for the FP64-equivalent mode");
    const int kp = (k + kBK - 1) / kBK * kBK;
    const EqLayout L = eq_layout(m, n, k);
    char *p = static_cast<char *>(scratch);
    unsigned *err = reinterpret_cast<unsigned *>(p + L.err);
    int *ea = reinterpret_cast<int *>(p + L.ea), *eb = reinterpret_cast<int *>(p + L.eb);
    int *mxo = reinterpret_cast<int *>(p + L.mxo);
    auto *As = reinterpret_cast<__nv_bfloat16 *>(p + L.as);
    auto *Bs = reinterpret_cast<__nv_bfloat16 *>(p + L.bs);
    OO_CUDA_TRY(cudaMemsetAsync(err, 0, 4, s));
    OO_CUDA_TRY(cudaMemsetAsync(mxo, 0, (size_t)n * 4, s));
    {
        const int rows_per = 256;
        dim3 grid((n + 31) / 32, (k + rows_per - 1) / rows_per), block(32, 8);
        OO_REQUIRE(grid.y <= 65535, OO_EINVAL, "k too large");
        eq_col_maxexp_kernel<<<grid, block, 0, s>>>(B, ldb, k, n, rows_per, mxo);
        OO_CUDA_TRY(cudaGetLastError());
        eq_col_scale_kernel<<<(n + 255) / 256, 256, 0, s>>>(mxo, eb, n);
        OO_CUDA_TRY(cudaGetLastError());
    }
    if (lda % 2 == 0 && ((uintptr_t)A & 15u) == 0)
        eq_split_rows_v2_kernel<<<m, 256, 0, s>>>(A, lda, m, k, kp, e.beta, e.slices, ea, As);
    else
        eq_split_rows_kernel<<<(m + 7) / 8, 256, 0, s>>>(A, lda, m, k, kp, e.beta, e.slices, ea, As);
    OO_CUDA_TRY(cudaGetLastError());
    {
        dim3 grid((n + 63) / 64, kp / 64);
        OO_REQUIRE(grid.y <= 65535, OO_EINVAL, "k too large");
        eq_split_cols_t_kernel<<<grid, 256, 0, s>>>(B, ldb, k, n, kp, e.beta, e.slices, mxo, Bs);
        OO_CUDA_TRY(cudaGetLastError());
    }
    int dev = 0, sms = 148;
    OO_CUDA_TRY(cudaGetDevice(&dev));
    OO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (e.scheme != eq::kSchemePairs) {
        // level schemes: the tiled kernel (gemm_eq_group.cu), as in batches
        launch_gemm_eq_tiles(m, n, k, As, Bs, ea, eb, C, ldc, width, err, sms, s);
        return;
    }
    EqMaps maps;
    map_bf16(&maps.a, As, (long long)e.slices * m, kp, kBM);
    map_bf16(&maps.b, Bs, (long long)e.slices * n, kp, kBN);
    EqArgs ga{};
    ga.m = m;
    ga.n = n;
    ga.ksteps = kp / kBK;
    ga.kb_steps = e.kb / kBK;
    ga.nkb = e.nkb;
    ga.m_tiles = (m + kBM - 1) / kBM;
    ga.n_tiles = (n + kBN - 1) / kBN;
    ga.C = C;
    ga.ldc = ldc;
    ga.ea = ea;
    ga.eb = eb;
    ga.err = err;
    const std::vector<EqUnit> U = eq_units(e);
    OO_REQUIRE((int)U.size() <= kMaxUnits, OO_EINVAL, "too many product groups");
    ga.nunits = (int)U.size();
    for (size_t i = 0; i < U.size(); ++i) {
        ga.up[i] = (unsigned char)U[i].p;
        ga.uq1[i] = (unsigned char)U[i].q1;
        ga.uq2[i] = (unsigned char)U[i].q2;
        ga.us1[i] = std::ldexp(1.0f, -e.beta * (U[i].p + U[i].q1 + 2));
        ga.us2[i] = U[i].q2 == kNone ? 0.0f : std::ldexp(1.0f, -e.beta * (U[i].p + U[i].q2 + 2));
    }
    if (pair) {
        EqPairMaps pm;
        map_bf16(&pm.a, As, (long long)e.slices * m, kp, kBM);
        map_bf16(&pm.b, Bs, (long long)e.slices * n, kp, kBN);
        map_bf16(&pm.bh, Bs, (long long)e.slices * n, kp, kBN / 2);
        ga.m_tiles = (m + 2 * kBM - 1) / (2 * kBM);  // 256-row slabs
        const long long ptiles = (long long)ga.m_tiles * ga.n_tiles;
        OO_REQUIRE(ptiles < (1ll << 31), OO_EINVAL, "too many tiles");
        const int ncl = eq_pair_clusters();
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(2 * std::min<long long>(ptiles, ncl)));
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = kSmemEqPair;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        OO_CUDA_TRY(cudaLaunchKernelEx(&cfg, gemm_fp64eq_pair_kernel, (const EqPairMaps)pm, (const EqArgs)ga));
        return;
    }
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)gemm_fp64eq_kernel, smem_eq(), attr);
    const long long tiles = (long long)ga.m_tiles * ga.n_tiles;
    OO_REQUIRE(tiles < (1ll << 31), OO_EINVAL, "too many tiles");
    const int grid = (int)std::min<long long>(tiles, sms);
    OO_REQUIRE(grid >= 1, OO_EINVAL, "empty product");
    gemm_fp64eq_kernel<<<grid, kThreads, smem_eq(), s>>>(maps, ga);
    OO_CUDA_TRY(cudaGetLastError());
}

unsigned *gemm_fp64eq_error_word(void *scratch) { return static_cast<unsigned *>(scratch); }

unsigned gemm_fp64eq_check_error(void *scratch, cudaStream_t s) {
    unsigned *err = static_cast<unsigned *>(scratch);
    unsigned e = 0;
    OO_CUDA_TRY(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s));
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    if (e) OO_CUDA_TRY(cudaMemsetAsync(err, 0, 4, s));
    return e;
}

}  // namespace oo
