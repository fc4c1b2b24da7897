// Matrix-product function block (Sec. 3.2.2, Sec. 4.2.1): C = A B for FP64
// A (m x k), B (k x n), row-major, computed on the 5th-generation tensor
// cores with the split-precision ("precision pattern") scheme:
//
//   A = 2^sA (A1 + A2 + dA),  B = (B1 + B2 + dB) 2^sB,  A1, A2, B1, B2 in BF16
//   C ~= 2^(sA + sB) ( A1 B1 + [A1 B2 + A2 B1] )
//
// sA is a per-row power of two that brings the row's largest entry into
// [1/2, 1); sB is per column, 1 when the column's largest entry already lies
// in [2^-20, 2^40) and otherwise chosen like sA (bf16_col_scale), so the
// split keeps 16 significant bits of every entry regardless of the input's
// range, and B is split in one pass.  The three products are
// summed, K step by K step in the order A1 B1, A1 B2, A2 B1, into one FP32
// accumulator in tensor memory (TMEM); the epilogue widens it to FP64 and
// applies the power-of-two scales.  Error: about 3 * 2^-16 of sum|a||b| per
// element plus FP32 accumulation rounding (the A1 B1 sum alone carries that
// rounding; adding the two cross products to the same accumulator, 2^-8
// smaller, leaves it about the same); the result is reported against an
// FP64 oracle, not claimed to be FP64.
//
// Kernels: persistent, warp-specialised.  gemm_split3_pair_kernel (the
// default) runs 256 x 256 output tiles on CTA pairs (cta_group::2, M = 256,
// N = 256 MMAs, each SM holding half of the tile's B columns);
// gemm_split3_kernel and the grouped kernel run 128 x 128 tiles on single
// CTAs (M = 128, N = 128).  Warp 0 issues TMA loads of the four BF16 operand
// tiles (128B-swizzled, K-major) into a 3-stage ring, warp 1 allocates 512
// TMEM columns (two accumulator buffers) and one of its threads issues
// tcgen05.mma (K = 16, kind::f16, BF16 x BF16 -> FP32) and tcgen05.commit
// to release stages; eight epilogue warps (4-11, two per TMEM lane quarter)
// read finished accumulators with tcgen05.ld and write FP64 C while the
// next tile accumulates.  Every mbarrier wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "ff.cuh"
#include "oo_internal.h"
#include "tc.cuh"

namespace oo {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 3;
constexpr int kGemmThreads = 384;  // producer, MMA issuer, 2 idle, 8 epilogue warps
constexpr int kEpiWarps = 8;
constexpr uint32_t kStageOut = kEpiWarps * 32 * 16 * 8;  // per epilogue warp: 32 rows x 16 FP64 staging
constexpr uint32_t kTileA = kBM * kBK * 2;   // 16 KB
constexpr uint32_t kTileB = kBN * kBK * 2;   // 16 KB
constexpr uint32_t kStageBytes = 2 * kTileA + 2 * kTileB;  // 64 KB
constexpr int kGroupM = 8;                   // tile raster: groups of 8 m-tiles share B panels in L2

using namespace tc;
constexpr uint32_t kIdesc = idesc_bf16(kBM, kBN);
constexpr uint32_t kIdescTF32 = idesc_tf32(kBM, kBN);
constexpr int kBKTF32 = 32;  // TF32 values per 128-byte row: K per pipeline stage of the TF32 pattern

struct GemmMaps {
    CUtensorMap a1, a2, b1, b2;
};

struct GemmArgs {
    int m, n, k, kp;        // kp: padded K of the split operands (a multiple of kstage)
    int kstage;             // K values per pipeline stage: 64 (BF16) or 32 (TF32)
    int m_tiles, n_tiles;
    int nw;                 // pair kernel: tile width (columns; a multiple of 32, 160 .. 256)
    double *C;
    long long ldc;
    const int *ea;          // per-row scale exponents of A (power of two)
    const int *eb;          // per-column scale exponents of B
    unsigned *err;
};

// Persistent, warp-specialised: CTA c processes tiles c, c + G, c + 2G, ...
// (grouped raster order).  TMEM holds two accumulator buffers of 256
// columns, so the epilogue of one tile overlaps the main loop of the next:
// the split-BF16 pattern sums its three products into one FP32 accumulator
// (128 columns), the split-TF32 pattern keeps D_hh and D_x (128 each).
__device__ __forceinline__ void tile_coords(const GemmArgs &a, int t, int &m0, int &n0) {
    const int per_group = kGroupM * a.n_tiles;
    const int g = t / per_group, r = t % per_group;
    const int rows = min(kGroupM, a.m_tiles - g * kGroupM);
    m0 = (g * kGroupM + r % rows) * kBM;
    n0 = (r / rows) * kBN;
}

// One output tile: where its operands and outputs are.
struct TileJob {
    const CUtensorMap *a1, *a2, *b1, *b2;
    double *C;
    long long ldc;
    const int *ea, *eb;
    int m, n, m0, n0, ksteps;
    int ra, rb;  // first row of this problem's A / B operands in the tensor maps
};

// Single problem: tensor maps are kernel parameters, tiles in grouped raster order.
struct SingleSrc {
    const GemmMaps *maps;
    const GemmArgs *a;
    __device__ __forceinline__ int count() const { return a->m_tiles * a->n_tiles; }
    __device__ __forceinline__ int ksteps(int) const { return a->kp / a->kstage; }
    __device__ __forceinline__ TileJob job(int t) const {
        int m0, n0;
        tile_coords(*a, t, m0, n0);
        return TileJob{&maps->a1, &maps->a2, &maps->b1, &maps->b2, a->C, a->ldc, a->ea, a->eb,
                       a->m, a->n, m0, n0, a->kp / a->kstage, 0, 0};
    }
};

// Many problems: every problem's split operands are stacked in four shared
// arrays (row pitch = the group's largest padded K), so four tensor maps,
// passed as kernel parameters like the single-problem ones, cover them
// all and a problem is a row offset.  (Per-problem tensor maps read from
// global memory starved the TMA unit: ~0.76 TB/s of operand traffic.)  The
// tile list (problem, m0, n0, k steps) is sorted by work so the
// round-robin assignment to persistent CTAs stays balanced.
struct GroupProblem {
    double *C;
    long long ldc;
    const int *ea, *eb;
    int m, n, k, kp;
    int ra, rb;
};
struct GroupSrc {
    const GemmMaps *maps;
    const GroupProblem *probs;
    const int4 *tiles;
    int ntiles;
    __device__ __forceinline__ int count() const { return ntiles; }
    __device__ __forceinline__ int ksteps(int t) const { return tiles[t].w; }
    __device__ __forceinline__ TileJob job(int t) const {
        const int4 td = tiles[t];
        const GroupProblem &P = probs[td.x];
        return TileJob{&maps->a1, &maps->a2, &maps->b1, &maps->b2, P.C, P.ldc, P.ea, P.eb,
                       P.m, P.n, td.y, td.z, td.w, P.ra, P.rb};
    }
};

// f * 2^S as a double by integer operations (exact; the FP64 pipe only for
// zeros, subnormals and results outside the normal range); NaN where the
// row's and column's scales flag a non-finite input (see nan_or_scaled)
__device__ __forceinline__ double nan_or_widened(float f, int S) {
    if (S > 4096) return __longlong_as_double(0x7ff8000000000000ll);
    const unsigned b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xffu);
    const int ne = e - 127 + 1023 + S;
    if (e == 0 || e == 0xff || ne <= 0 || ne >= 0x7ff) return ldexp((double)f, S);
    return __longlong_as_double((long long)(((unsigned long long)(b & 0x80000000u) << 32) |
                                            ((unsigned long long)ne << 52) |
                                            ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// Epilogue of one tile for one warp: TMEM lane quarter q holds rows
// m0 + 32 q .. +31 of the tile; the warp takes tile columns hcol .. cend - 1
// (cend - hcol a multiple of 16 or cut by the problem's last column), in at
// most NCH 32-column chunks.  MERGED: one FP32 accumulator at d (the
// split-BF16 products); else D_hh at d and D_x at d + 128, summed exactly
// (the split-TF32 pair).  Each thread widens its row's values; 16-column
// blocks go through a per-warp shared-memory transpose (XOR-swizzled: no
// bank conflicts) so every global store writes two whole 128-byte row
// segments.  sa: the row's scale exponent; e[c]: that of column
// hcol + 32 c + lane.
template <int NCH, bool MERGED>
__device__ __forceinline__ void store_tile_quarter(const TileJob &jb, uint32_t d, int q, int hcol, int cend, int lane,
                                                   double *stg, int sa, const int (&e)[NCH]) {
    const int n0 = jb.n0, row0 = jb.m0 + q * 32;
    const int ncols = cend;  // columns of the tile this warp stores end here
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
#pragma unroll 1
    for (int cc = 0; cc < NCH; ++cc) {
        const int c = hcol + cc * 32;
        if (c >= ncols) break;
        uint32_t h[32], x[32];
        OO_TMEM_LD32(d + lane_off + c, h);
        if constexpr (!MERGED) OO_TMEM_LD32(d + 128 + lane_off + c, x);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        int ecur = e[0];
#pragma unroll
        for (int i = 1; i < NCH; ++i)
            if (cc == i) ecur = e[i];
#pragma unroll
        for (int sub = 0; sub < 2; ++sub) {
            if (c + sub * 16 >= ncols) break;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int t2 = sub * 16 + j;
                const int sb = __shfl_sync(0xffffffffu, ecur, t2);
                double v;
                if constexpr (MERGED) {
                    v = nan_or_widened(__uint_as_float(h[t2]), sa + sb);
                } else {
                    // exact two-sum of the partial products, widened and
                    // scaled without the (slow) FP64 pipe
                    v = nan_or_scaled(ff::to_double(__uint_as_float(h[t2]), __uint_as_float(x[t2])), sa + sb);
                }
                stg[lane * 16 + (j ^ (lane & 15))] = v;
            }
            __syncwarp();
            const int cl = lane & 15, col = c + sub * 16 + cl;
#pragma unroll 4
            for (int r = lane >> 4; r < 32; r += 2) {
                const double v = stg[r * 16 + (cl ^ (r & 15))];
                if (row0 + r < jb.m && col < ncols) jb.C[(long long)(row0 + r) * jb.ldc + n0 + col] = v;
            }
            __syncwarp();
        }
    }
}

// TF32: the operands are TF32-rounded FP32 (kind::tf32 MMAs, 32 K values
// per 128-byte row); the stage layout, accumulators and epilogue are the
// BF16 pattern's byte for byte.
template <class Src, bool TF32 = false>
__device__ __forceinline__ void gemm_body(const Src &src, unsigned *err) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    unsigned char *gsm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    double *stg_all = reinterpret_cast<double *>(gsm + kStages * kStageBytes);  // epilogue store staging
    uint64_t *bars = reinterpret_cast<uint64_t *>(gsm + kStages * kStageBytes + kStageOut);
    uint64_t *full = bars, *empty = bars + kStages;
    uint64_t *tfull = bars + 2 * kStages, *tempty = bars + 2 * kStages + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = src.count();

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
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        fence_before();
    }
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    int loaded = 0;          // producer: stages issued
    int tiles_mma = 0;       // MMA issuer: tiles whose accumulation was issued
    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------- TMA producer
        int it = 0;
        bool ok = true;
        // the next tile's descriptor is fetched one tile ahead so that its
        // (dependent) global loads stay off the critical path
        TileJob nx = blockIdx.x < (unsigned)tiles ? src.job(blockIdx.x) : TileJob{};
        for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
            const TileJob jb = nx;
            if (t + (int)gridDim.x < tiles) nx = src.job(t + gridDim.x);
            for (int ks = 0; ks < jb.ksteps; ++ks, ++it) {
                const int s = it % kStages;
                const uint32_t use = it / kStages;
                if (use > 0 && !bar_wait(su32(&empty[s]), (use - 1) & 1, abort_flag, err, 1u)) {
                    ok = false;
                    break;
                }
                unsigned char *st = gsm + (size_t)s * kStageBytes;
                const uint32_t fb = su32(&full[s]);
                bar_expect_tx(fb, kStageBytes);
                const int k0 = ks * (TF32 ? kBKTF32 : kBK);
                tma_2d(su32(st), jb.a1, k0, jb.ra + jb.m0, fb);
                tma_2d(su32(st + kTileA), jb.a2, k0, jb.ra + jb.m0, fb);
                tma_2d(su32(st + 2 * kTileA), jb.b1, k0, jb.rb + jb.n0, fb);
                tma_2d(su32(st + 2 * kTileA + kTileB), jb.b2, k0, jb.rb + jb.n0, fb);
                ++loaded;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------- MMA issuer
        int it = 0, lt = 0;
        bool ok = true;
        int ks_next = blockIdx.x < (unsigned)tiles ? src.ksteps(blockIdx.x) : 0;
        for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x, ++lt) {
            const int ksteps = ks_next;
            if (t + (int)gridDim.x < tiles) ks_next = src.ksteps(t + gridDim.x);
            const int b = lt & 1;
            const uint32_t buse = lt >> 1;
            if (buse > 0 && !bar_wait(su32(&tempty[b]), (buse - 1) & 1, abort_flag, err, 2u)) break;
            fence_after();
            const uint32_t d_hh = tmem + (uint32_t)(b * 256), d_x = d_hh + 128;
            for (int ks = 0; ks < ksteps; ++ks, ++it) {
                const int s = it % kStages;
                const uint32_t use = it / kStages;
                if (!bar_wait(su32(&full[s]), use & 1, abort_flag, err, 2u)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t base = su32(gsm + (size_t)s * kStageBytes);
                const uint32_t a1 = base, a2 = base + kTileA, b1 = base + 2 * kTileA, b2 = b1 + kTileB;
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
                    const uint32_t off = kk * 32;  // 16 BF16 (8 TF32) along K inside the 128-byte row
                    const uint32_t acc = (ks == 0 && kk == 0) ? 0u : 1u;
                    if constexpr (TF32) {
                        mma_tf32<kIdescTF32>(d_hh, sdesc_sw128(a1 + off), sdesc_sw128(b1 + off), acc);
                        mma_tf32<kIdescTF32>(d_x, sdesc_sw128(a1 + off), sdesc_sw128(b2 + off), acc);
                        mma_tf32<kIdescTF32>(d_x, sdesc_sw128(a2 + off), sdesc_sw128(b1 + off), 1u);
                    } else {  // one accumulator: A1 B1, A1 B2, A2 B1 in this order
                        mma_bf16<kIdesc>(d_hh, sdesc_sw128(a1 + off), sdesc_sw128(b1 + off), acc);
                        mma_bf16<kIdesc>(d_hh, sdesc_sw128(a1 + off), sdesc_sw128(b2 + off), 1u);
                        mma_bf16<kIdesc>(d_hh, sdesc_sw128(a2 + off), sdesc_sw128(b1 + off), 1u);
                    }
                }
                mma_commit(su32(&empty[s]));
            }
            mma_commit(su32(&tfull[b]));  // accumulators of this tile complete
            ++tiles_mma;
        }
    } else if (warp >= 4) {
        // ---------------------------------------------------- epilogue
        // Eight warps: warp w reads TMEM lane quarter (w & 3), i.e. rows
        // 32 (w & 3) .. +31 of the tile, and column half (w - 4) >> 2;
        // quarters with no valid row are skipped.
        const int q = warp & 3, hcol = ((warp - 4) >> 2) * 64;
        double *stg = stg_all + (size_t)(warp - 4) * 32 * 16;
        int lt = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++lt) {
            const int b = lt & 1;
            // descriptor and scales before the accumulator wait (overlaps the
            // MMAs); lane l holds the scales of columns hcol + l and hcol + 32 + l
            const TileJob jb = src.job(t);
            const int n0 = jb.n0, row0 = jb.m0 + q * 32;
            const int ncols = jb.n - n0;  // valid columns of the tile (may exceed 128)
            const int sa = row0 + lane < jb.m ? jb.ea[row0 + lane] : 0;
            const int e[2] = {hcol + lane < ncols ? jb.eb[n0 + hcol + lane] : 0,
                              hcol + 32 + lane < ncols ? jb.eb[n0 + hcol + 32 + lane] : 0};
            if (!bar_wait(su32(&tfull[b]), (lt >> 1) & 1, abort_flag, err, 4u)) break;
            fence_after();
            if (row0 < jb.m)
                store_tile_quarter<2, !TF32>(jb, tmem + (uint32_t)(b * 256), q, hcol, min(ncols, hcol + 64), lane, stg,
                                             sa, e);
            fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(su32(&tempty[b]));
        }
    }
    // drain on abort: wait (bounded) for issued MMAs and copies before TMEM
    // is released and the CTA exits
    if (*abort_flag) {
        if (warp == 1 && lane == 0 && tiles_mma > 0) {
            const int lb = (tiles_mma - 1) & 1;
            const long long t0 = clock64();
            while (!bar_try(su32(&tfull[lb]), ((tiles_mma - 1) >> 1) & 1) && clock64() - t0 < kWaitLimit) {
            }
        }
        if (warp == 0 && lane == 0) {
            for (int it = (loaded > kStages ? loaded - kStages : 0); it < loaded; ++it) {
                const long long t0 = clock64();
                while (!bar_try(su32(&full[it % kStages]), (it / kStages) & 1) && clock64() - t0 < kWaitLimit) {
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

__global__ void __launch_bounds__(kGemmThreads, 1) gemm_split3_kernel(const __grid_constant__ GemmMaps maps,
                                                                     const __grid_constant__ GemmArgs a) {
    const SingleSrc src{&maps, &a};
    gemm_body(src, a.err);
}

__global__ void __launch_bounds__(kGemmThreads, 1) gemm_split3_tf32_kernel(const __grid_constant__ GemmMaps maps,
                                                                          const __grid_constant__ GemmArgs a) {
    const SingleSrc src{&maps, &a};
    gemm_body<SingleSrc, true>(src, a.err);
}

__global__ void __launch_bounds__(kGemmThreads, 1) gemm_group_kernel(const __grid_constant__ GemmMaps maps,
                                                                    const GroupProblem *probs, const int4 *tiles,
                                                                    int ntiles, unsigned *err) {
    const GroupSrc src{&maps, probs, tiles, ntiles};
    gemm_body(src, err);
}

// ------------------------------------------------- CTA-pair split3 kernel
// The split-BF16 product on CTA pairs (cta_group::2).  A unit is a 256 x W
// tile of C (W = a.nw, 160 .. 256 columns, chosen per problem so that the
// units fill the resident clusters' waves: n = 4096 takes W = 224, 304
// units = 4 waves of 76 pairs, where W = 256 leaves the fourth wave a
// third full); CTA r of the pair loads rows m0 + 128 r .. +127 of A1 and
// A2 and rows n0 + r W/2 .. +W/2-1 of B1 and B2 (its half of the tile's
// columns).  Rank 0 issues M = 256, N = W MMAs into both CTAs' TMEM (each
// holds its 128 rows x W columns, double-buffered); the commits arrive on
// both CTAs' barriers; each CTA's epilogue stores its own rows and reports
// to rank 0 that its accumulator buffer is free.  Wide N matters: measured
// on GB300, N = 128 instructions (either tile shape) kept the tensor pipe
// ~64 % busy at most, N = 256 ones ~97 %.  Every output element sees the
// same products in the same K order as in gemm_split3_kernel, so the two
// kernels give the same bits.
constexpr int kStagesP = 3;
constexpr int kBNP = 2 * kBN;                                 // widest tile: 256 columns
constexpr uint32_t kStageBytesP = 2 * kTileA + 2 * kTileB;    // 64 KB: room for 128-row A and B tiles
constexpr int kGroupMP = 4;  // raster: groups of 4 pair rows (1024 rows of A) share B panels in L2
constexpr size_t kSmemPair = 1024 + (size_t)kStagesP * kStageBytesP + kStageOut + 256;
static_assert(kSmemPair <= 232448, "pair kernel exceeds the shared memory of a CTA");

// unit u -> first row of the pair's 256-row slab, first column of the tile
__device__ __forceinline__ void pair_coords(const GemmArgs &a, int u, int &mp, int &n0) {
    const int per_group = kGroupMP * a.n_tiles;
    const int g = u / per_group, r = u % per_group;
    const int rows = min(kGroupMP, a.m_tiles - g * kGroupMP);
    mp = (g * kGroupMP + r % rows) * 2 * kBM;
    n0 = (r / rows) * a.nw;
}

// a.m_tiles counts 256-row slabs, a.n_tiles a.nw-column panels
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_split3_pair_kernel(const __grid_constant__ GemmMaps maps,
                                                                          const __grid_constant__ GemmArgs a) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    unsigned char *gsm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    double *stg_all = reinterpret_cast<double *>(gsm + kStagesP * kStageBytesP);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gsm + kStagesP * kStageBytesP + kStageOut);
    uint64_t *full = bars, *empty = bars + kStagesP;
    uint64_t *tfull = bars + 2 * kStagesP, *tempty = tfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    unsigned *err = a.err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
    const int units = a.m_tiles * a.n_tiles;
    const int ksteps = a.kp / kBK;
    const int half = a.nw >> 1;  // B rows (tile columns) per CTA
    const uint32_t stage_tx = 2 * (2 * kTileA + 2u * (uint32_t)half * kBK * 2);  // both CTAs' bytes per stage

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesP; ++s) {
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

    int loaded = 0, tiles_mma = 0;
    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------- TMA producer (both CTAs)
        int it = 0;
        bool ok = true;
        for (int u = cid; ok && u < units; u += ncl) {
            int mp, n0;
            pair_coords(a, u, mp, n0);
            const int ma = mp + (int)rank * kBM, nb = n0 + (int)rank * half;
            for (int ks = 0; ks < ksteps; ++ks, ++it) {
                const int s = it % kStagesP;
                const uint32_t use = it / kStagesP;
                if (use > 0 && !bar_wait_cluster(su32(&empty[s]), (use - 1) & 1, abort_flag, err, 1u)) {
                    ok = false;
                    break;
                }
                unsigned char *st = gsm + (size_t)s * kStageBytesP;
                if (leader) bar_expect_tx(su32(&full[s]), stage_tx);
                const uint32_t fb = map_to_rank(su32(&full[s]), 0);
                const int k0 = ks * kBK;
                tma_2d_pair(su32(st), &maps.a1, k0, ma, fb);
                tma_2d_pair(su32(st + kTileA), &maps.a2, k0, ma, fb);
                tma_2d_pair(su32(st + 2 * kTileA), &maps.b1, k0, nb, fb);
                tma_2d_pair(su32(st + 2 * kTileA + kTileB), &maps.b2, k0, nb, fb);
                ++loaded;
            }
        }
    } else if (warp == 1 && lane == 0 && leader) {
        // ---------------------------------------------------- MMA issuer (rank 0)
        const uint32_t idesc = idesc_bf16(2 * kBM, a.nw);
        int it = 0, lt = 0;
        bool ok = true;
        for (int u = cid; ok && u < units; u += ncl, ++lt) {
            const int b = lt & 1;
            const uint32_t buse = lt >> 1;
            if (buse > 0 && !bar_wait_cluster(su32(&tempty[b]), (buse - 1) & 1, abort_flag, err, 2u)) break;
            fence_after();
            const uint32_t d = tmem + (uint32_t)(b * 256);
            for (int ks = 0; ks < ksteps; ++ks, ++it) {
                const int s = it % kStagesP;
                const uint32_t use = it / kStagesP;
                if (!bar_wait_cluster(su32(&full[s]), use & 1, abort_flag, err, 2u)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t base = su32(gsm + (size_t)s * kStageBytesP);
                const uint32_t a1 = base, a2 = base + kTileA, b1 = base + 2 * kTileA, b2 = b1 + kTileB;
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint32_t acc = (ks == 0 && kk == 0) ? 0u : 1u;
                    mma_bf16_pair(d, sdesc_sw128(a1 + off), sdesc_sw128(b1 + off), idesc, acc);
                    mma_bf16_pair(d, sdesc_sw128(a1 + off), sdesc_sw128(b2 + off), idesc, 1u);
                    mma_bf16_pair(d, sdesc_sw128(a2 + off), sdesc_sw128(b1 + off), idesc, 1u);
                }
                mma_commit_pair(su32(&empty[s]), 3);  // stage s free in both CTAs
            }
            if (!ok) break;
            mma_commit_pair(su32(&tfull[b]), 3);  // both halves of the accumulator complete
            ++tiles_mma;
        }
    } else if (warp >= 4) {
        // ---------------------------------------------------- epilogue (both CTAs)
        // warp-halves take tile columns [0, 128) and [128, W): chunk starts
        // stay multiples of 32
        const int q = warp & 3, hsel = (warp - 4) >> 2, hcol = hsel * 128;
        const int hend = hsel ? a.nw : min(128, a.nw);
        double *stg = stg_all + (size_t)(warp - 4) * 32 * 16;
        int lt = 0;
        for (int u = cid; u < units; u += ncl, ++lt) {
            const int b = lt & 1;
            int mp, n0;
            pair_coords(a, u, mp, n0);
            const TileJob jb{&maps.a1, &maps.a2, &maps.b1, &maps.b2, a.C, a.ldc, a.ea, a.eb,
                             a.m, a.n, mp + (int)rank * kBM, n0, ksteps, 0, 0};
            const int row0 = jb.m0 + q * 32, ncols = a.n - n0;
            const int sa = row0 + lane < a.m ? a.ea[row0 + lane] : 0;
            int e[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) e[c] = hcol + 32 * c + lane < ncols ? a.eb[n0 + hcol + 32 * c + lane] : 0;
            if (!bar_wait_cluster(su32(&tfull[b]), (lt >> 1) & 1, abort_flag, err, 4u)) break;
            fence_after();
            if (row0 < a.m)
                store_tile_quarter<4, true>(jb, tmem + (uint32_t)(b * 256), q, hcol, min(ncols, hend), lane, stg, sa,
                                            e);
            fence_before();
            __syncwarp();
            if (lane == 0) {
                if (leader)
                    bar_arrive(su32(&tempty[b]));
                else
                    bar_arrive_remote(map_to_rank(su32(&tempty[b]), 0));
            }
        }
    }
    // drain on abort (bounded): rank 0 waits for its issued MMAs and for the
    // copies counted on its barriers; rank 1 for the commits that free its
    // stages (its copies complete on rank 0's barriers)
    if (*abort_flag) {
        if (warp == 1 && lane == 0 && leader && tiles_mma > 0) {
            const int lb = (tiles_mma - 1) & 1;
            bar_drain(su32(&tfull[lb]), ((tiles_mma - 1) >> 1) & 1);
        }
        if (warp == 0 && lane == 0) {
            for (int it = (loaded > kStagesP ? loaded - kStagesP : 0); it < loaded; ++it)
                bar_drain(su32(leader ? &full[it % kStagesP] : &empty[it % kStagesP]), (it / kStagesP) & 1);
        }
    }
    fence_before();
    __syncthreads();
    cluster_sync_all();  // neither CTA leaves while the other may still signal it or read its TMEM
    if (warp == 1) {
        fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
}
// ---------------------------------------------------------------- splitting
// Scale exponent of a column of B in the split-BF16 pattern, from its
// largest biased exponent mx (0: every entry zero; kNonFiniteExp: a NaN or
// an infinity).  0 when the column's largest magnitude lies in
// [2^-20, 2^40): BF16 and FP32 hold such a column's splits, products and
// sums unscaled, and a power-of-two scale would change no rounding in them,
// only flush a few entries more than 2^106 below the largest; otherwise the
// power of two that brings the largest entry into [1/2, 1), and 2^20 (the
// non-finite flag) for a column holding a NaN or an infinity.  Rows of A
// always take the [1/2, 1) scale.  Unscaled columns let the split read B
// once (split_cols_strip).
__device__ __forceinline__ int bf16_col_scale(int mx) {
    if (mx == 0) return 0;
    const int u = mx - 1023;  // unbiased exponent of the largest entry
    if (u >= -20 && u < 40) return 0;
    return mx - 1023 + 1;
}
// per-column maxima of B (k x n): grid.x over column blocks of 32, grid.y over k chunks
__global__ void col_maxexp_kernel(const double *B, long long ldb, int k, int n, int rows_per, int *e) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * rows_per, r1 = min(k, r0 + rows_per);
    if (col >= n) return;
    int mx = 0;
#pragma unroll 8
    for (int l = r0 + threadIdx.y; l < r1; l += blockDim.y) {
        mx = max(mx, biased_exp_or_flag((unsigned long long)__double_as_longlong(B[(long long)l * ldb + col])));
    }
    if (mx > 0) atomicMax(e + col, mx);
}
__global__ void exp_to_scale_kernel(int *e, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) e[i] = e[i] == 0 ? 0 : e[i] - 1023 + 1;
}
// the same for the columns of B in the split-BF16 pattern (bf16_col_scale)
__global__ void exp_to_bf16_col_scale_kernel(int *e, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) e[i] = bf16_col_scale(e[i]);
}

// x * 2^-S -> (hi, lo) BF16 pair with hi + lo = x * 2^-S to ~16 bits
__device__ __forceinline__ void split_bf16(double x, int S, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
    const unsigned sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7ffu);
    const int fe = e - 1023 - S + 127;
    float h = 0.0f, l = 0.0f;
    if (e != 0 && e != 0x7ff && fe > 0) {
        h = __uint_as_float(sign | ((unsigned)fe << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29));
        const unsigned r = lo32 & 0x1fffffffu;
        const int le = fe - 52;
        if (le > 0 && r != 0) {
            const float lf = __fmul_rn(__uint2float_rn(r), __uint_as_float((unsigned)le << 23));
            l = sign ? -lf : lf;
        }
    }
    hi = __float2bfloat16_rn(h);
    const float rem = __fadd_rn(__fsub_rn(h, __bfloat162float(hi)), l);
    lo = __float2bfloat16_rn(rem);
}

// One row of A -> its scale exponent and BF16 hi / lo rows (kp entries,
// zero padding in [k, kp)); executed by one warp; the second pass re-reads
// the row from cache.
__device__ __forceinline__ void split_row_warp(const double *src, int k, int kp, int *ea_out,
                                               __nv_bfloat16 *A1row, __nv_bfloat16 *A2row) {
    const int lane = threadIdx.x & 31;
    int mx = 0;
#pragma unroll 4
    for (int l = lane; l < k; l += 32) {
        mx = max(mx, biased_exp_or_flag((unsigned long long)__double_as_longlong(src[l])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int S = mx == 0 ? 0 : mx - 1023 + 1;
    if (lane == 0) *ea_out = S;
    __nv_bfloat162 *d1 = reinterpret_cast<__nv_bfloat162 *>(A1row);
    __nv_bfloat162 *d2 = reinterpret_cast<__nv_bfloat162 *>(A2row);
#pragma unroll 2
    for (int l2 = lane; l2 < kp / 2; l2 += 32) {
        const int l = 2 * l2;
        __nv_bfloat16 h0 = __float2bfloat16_rn(0.0f), o0 = h0, h1 = h0, o1 = h0;
        if (l < k) split_bf16(src[l], S, h0, o0);
        if (l + 1 < k) split_bf16(src[l + 1], S, h1, o1);
        d1[l2] = __halves2bfloat162(h0, h1);
        d2[l2] = __halves2bfloat162(o0, o1);
    }
}

// A (m x k, lda) -> per-row scale ea and A1, A2 (m x kp); one warp per row
__global__ void split_rows_fused_kernel(const double *A, long long lda, int m, int k, int kp, int *ea,
                                        __nv_bfloat16 *A1, __nv_bfloat16 *A2) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= m) return;
    split_row_warp(A + (long long)row * lda, k, kp, ea + row, A1 + (long long)row * kp, A2 + (long long)row * kp);
}

// Same, one 256-thread CTA per row with 16-byte loads (lda even, A 16-byte
// aligned): the second read of the row hits L1 and each thread keeps eight
// loads in flight in the exponent pass.
__global__ void __launch_bounds__(256) split_rows_v2_kernel(const double *A, long long lda, int m, int k, int kp,
                                                          int *ea, __nv_bfloat16 *A1, __nv_bfloat16 *A2) {
    const int row = blockIdx.x;
    const double *base = A + (long long)row * lda;
    const double2 *src = reinterpret_cast<const double2 *>(base);
    const int k2 = k >> 1;
    int mx = 0;
    auto ex = [](double x) { return biased_exp_or_flag((unsigned long long)__double_as_longlong(x)); };
#pragma unroll 8
    for (int l2 = threadIdx.x; l2 < k2; l2 += 256) {
        const double2 v = src[l2];
        mx = max(mx, max(ex(v.x), ex(v.y)));
    }
    if ((k & 1) && threadIdx.x == 0) mx = max(mx, ex(base[k - 1]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ int red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = max(mx, red[w]);
    const int S = mx == 0 ? 0 : mx - 1023 + 1;
    if (threadIdx.x == 0) ea[row] = S;
    __nv_bfloat162 *d1 = reinterpret_cast<__nv_bfloat162 *>(A1 + (long long)row * kp);
    __nv_bfloat162 *d2 = reinterpret_cast<__nv_bfloat162 *>(A2 + (long long)row * kp);
#pragma unroll 2
    for (int l2 = threadIdx.x; l2 < kp / 2; l2 += 256) {
        const int l = 2 * l2;
        double2 v = make_double2(0.0, 0.0);
        if (l + 1 < k) {
            v = src[l2];
        } else if (l < k) {
            v.x = base[l];
        }
        __nv_bfloat16 h0, o0, h1, o1;
        split_bf16(v.x, S, h0, o0);
        split_bf16(v.y, S, h1, o1);
        d1[l2] = __halves2bfloat162(h0, h1);
        d2[l2] = __halves2bfloat162(o0, o1);
    }
}

// One 64 (k) x 64 (column) tile of B -> transposed BF16 hi / lo tiles of
// B1t, B2t (n x kp); 256 threads, through shared memory.
// (B1t, B2t rows `pitch` elements apart; columns [0, kp) written)
__device__ __forceinline__ void split_b_tile(const double *B, long long ldb, int k, int n, int kp, long long pitch,
                                             const int *eb, __nv_bfloat16 *B1t, __nv_bfloat16 *B2t, int l0, int c0) {
    __shared__ __nv_bfloat16 th[64][66], tl[64][66];
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
    const int col = c0 + tx;
    const int S = col < n ? eb[col] : 0;
#pragma unroll
    for (int yy = ty; yy < 64; yy += 4) {
        const int l = l0 + yy;
        __nv_bfloat16 h = __float2bfloat16_rn(0.0f), lo = h;
        if (l < k && col < n) split_bf16(B[(long long)l * ldb + col], S, h, lo);
        th[yy][tx] = h;
        tl[yy][tx] = lo;
    }
    __syncthreads();
    // write: each warp covers 8 columns x 64 k values (128 bytes per column)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int cc = w * 8; cc < w * 8 + 8; ++cc) {
        const int c = c0 + cc;
        const int l = l0 + 2 * lane;
        if (c < n && l < kp) {
            __nv_bfloat162 *o1 = reinterpret_cast<__nv_bfloat162 *>(B1t + (long long)c * pitch + l);
            __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(B2t + (long long)c * pitch + l);
            *o1 = __halves2bfloat162(th[2 * lane][cc], th[2 * lane + 1][cc]);
            *o2 = __halves2bfloat162(tl[2 * lane][cc], tl[2 * lane + 1][cc]);
        }
    }
}

// B (k x n, ldb) -> B1t, B2t (n x kp, transposed), zero padding in [k, kp)
__global__ void split_cols_t_kernel(const double *B, long long ldb, int k, int n, int kp, const int *eb,
                                    __nv_bfloat16 *B1t, __nv_bfloat16 *B2t) {
    split_b_tile(B, ldb, k, n, kp, kp, eb, B1t, B2t, blockIdx.y * 64, blockIdx.x * 64);
}

// B (k x n, ldb even, 16-byte aligned) -> column scales eb and B1t, B2t
// (n x kp, transposed), zero padding in [k, kp).  One CTA per strip of 16
// columns, one pass over B: every entry is split unscaled (S = 0) while the
// columns' largest exponents are gathered; a column whose scale turns out
// not to be 0 (bf16_col_scale: its largest entry outside [2^-20, 2^40), or
// a non-finite entry) is split again with its scale, re-reading the strip
// -- normally no column.  Same scales and splits as col_maxexp +
// exp_to_bf16_col_scale + split_cols_t, with B read once.
constexpr int kStripThreads = 512;
__device__ __forceinline__ void split_cols_strip(const double *B, long long ldb, int k, int n, int kp, int *eb,
                                                 __nv_bfloat16 *B1t, __nv_bfloat16 *B2t, int strip) {
    __shared__ int red[64][17];
    __shared__ int Ssh[16];
    __shared__ int redo;
    __shared__ __nv_bfloat16 th[16][258], tl[16][258];
    const int c0 = strip * 16;
    const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;  // 8 column pairs x 64 rows
    const int col = c0 + 2 * tx;
    const bool in0 = col < n, in1 = col + 1 < n;
    auto ex = [](double x) { return biased_exp_or_flag((unsigned long long)__double_as_longlong(x)); };
    auto load = [&](int l) {
        double2 v = make_double2(0.0, 0.0);
        if (l < k) {
            const double *src = B + (long long)l * ldb + col;
            if (in1)
                v = *reinterpret_cast<const double2 *>(src);
            else if (in0)
                v.x = *src;
        }
        return v;
    };
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;  // warp w writes column c0 + w
    // one pass over the strip with scales S0, S1 for this thread's columns:
    // 256 k values per step, the next step's four loads issued before this
    // step's stores; with `track`, the columns' largest exponents gathered
    auto pass = [&](int S0, int S1, bool track, int &m0, int &m1) {
        double2 nv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) nv[q] = load(64 * q + ty);
        for (int l0 = 0; l0 < kp; l0 += 256) {
            double2 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = nv[q];
            if (l0 + 256 < kp) {
#pragma unroll
                for (int q = 0; q < 4; ++q) nv[q] = load(l0 + 256 + 64 * q + ty);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (track) {
                    m0 = max(m0, ex(v[q].x));
                    m1 = max(m1, ex(v[q].y));
                }
                split_bf16(v[q].x, S0, th[2 * tx][64 * q + ty], tl[2 * tx][64 * q + ty]);
                split_bf16(v[q].y, S1, th[2 * tx + 1][64 * q + ty], tl[2 * tx + 1][64 * q + ty]);
            }
            __syncthreads();
            const int c = c0 + w;
            if (c < n) {
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int l = l0 + 64 * h + 2 * lane;
                    if (l < kp) {
                        const int q = 64 * h + 2 * lane;
                        *reinterpret_cast<__nv_bfloat162 *>(B1t + (long long)c * kp + l) =
                            __halves2bfloat162(th[w][q], th[w][q + 1]);
                        *reinterpret_cast<__nv_bfloat162 *>(B2t + (long long)c * kp + l) =
                            __halves2bfloat162(tl[w][q], tl[w][q + 1]);
                    }
                }
            }
            __syncthreads();
        }
    };
    int m0 = 0, m1 = 0;
    pass(0, 0, true, m0, m1);
    red[ty][2 * tx] = m0;
    red[ty][2 * tx + 1] = m1;
    if (threadIdx.x == 0) redo = 0;
    __syncthreads();
    if (threadIdx.x < 16) {
        int mx = 0;
        for (int y = 0; y < 64; ++y) mx = max(mx, red[y][threadIdx.x]);
        const int S = bf16_col_scale(mx);
        Ssh[threadIdx.x] = S;
        if (c0 + (int)threadIdx.x < n) {
            eb[c0 + threadIdx.x] = S;
            if (S != 0) redo = 1;
        }
    }
    __syncthreads();
    if (redo) {  // the strip again, every column with its own scale
        int u0 = 0, u1 = 0;
        pass(Ssh[2 * tx], Ssh[2 * tx + 1], false, u0, u1);
    }
}

__global__ void __launch_bounds__(kStripThreads) split_cols_strip_kernel(const double *B, long long ldb, int k, int n,
                                                                        int kp, int *eb, __nv_bfloat16 *B1t,
                                                                        __nv_bfloat16 *B2t) {
    split_cols_strip(B, ldb, k, n, kp, eb, B1t, B2t, blockIdx.x);
}

// One row of A -> its scale exponent and BF16 hi / lo rows, by 256 threads
// (half of a 512-thread CTA) synchronising on named barrier `bar`; row
// 16-byte aligned, lda even.  Same results as split_rows_v2_kernel.
__device__ __forceinline__ void split_row_half(const double *base, int k, int kp, int *ea_row, __nv_bfloat16 *a1,
                                               __nv_bfloat16 *a2, int t, int bar, int *red8) {
    const double2 *src = reinterpret_cast<const double2 *>(base);
    const int k2 = k >> 1;
    auto ex = [](double x) { return biased_exp_or_flag((unsigned long long)__double_as_longlong(x)); };
    int mx = 0;
#pragma unroll 8
    for (int l2 = t; l2 < k2; l2 += 256) {
        const double2 v = src[l2];
        mx = max(mx, max(ex(v.x), ex(v.y)));
    }
    if ((k & 1) && t == 0) mx = max(mx, ex(base[k - 1]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((t & 31) == 0) red8[t >> 5] = mx;
    asm volatile("bar.sync %0, 256;" ::"r"(bar) : "memory");
    mx = red8[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = max(mx, red8[w]);
    const int S = mx == 0 ? 0 : mx - 1023 + 1;
    if (t == 0) *ea_row = S;
    __nv_bfloat162 *d1 = reinterpret_cast<__nv_bfloat162 *>(a1);
    __nv_bfloat162 *d2 = reinterpret_cast<__nv_bfloat162 *>(a2);
#pragma unroll 2
    for (int l2 = t; l2 < kp / 2; l2 += 256) {
        const int l = 2 * l2;
        double2 v = make_double2(0.0, 0.0);
        if (l + 1 < k) {
            v = src[l2];
        } else if (l < k) {
            v.x = base[l];
        }
        __nv_bfloat16 h0, o0, h1, o1;
        split_bf16(v.x, S, h0, o0);
        split_bf16(v.y, S, h1, o1);
        d1[l2] = __halves2bfloat162(h0, h1);
        d2[l2] = __halves2bfloat162(o0, o1);
    }
}

// Both operands in one launch: CTAs [0, nstrip) split 16-column strips of
// B, the rest split two rows of A each, so the bandwidth-bound row splits
// run while the strips wait on their loads.
__global__ void __launch_bounds__(kStripThreads) split_ab_kernel(const double *A, long long lda, int m,
                                                                const double *B, long long ldb, int n, int k, int kp,
                                                                int nstrip, int *ea, int *eb, __nv_bfloat16 *A1,
                                                                __nv_bfloat16 *A2, __nv_bfloat16 *B1t,
                                                                __nv_bfloat16 *B2t) {
    if ((int)blockIdx.x < nstrip) {
        split_cols_strip(B, ldb, k, n, kp, eb, B1t, B2t, blockIdx.x);
        return;
    }
    __shared__ int red8[2][8];
    const int half = threadIdx.x >> 8;
    const int row = 2 * ((int)blockIdx.x - nstrip) + half;
    if (row >= m) return;
    split_row_half(A + (long long)row * lda, k, kp, ea + row, A1 + (long long)row * kp, A2 + (long long)row * kp,
                   threadIdx.x & 255, 1 + half, red8[half]);
}

// ----------------------------------------------------- TF32 splitting
// The TF32 pattern: A = 2^sA (A1 + A2 + dA), B likewise, A1, A2, B1, B2 TF32
// (FP32 with 10 fraction bits, rounded to nearest, ties away), so the pair
// keeps ~22 significant bits of every entry; the products and accumulators
// are the BF16 pattern's (D_hh = A1 B1, D_x = A1 B2 + A2 B1).

// effective biased exponent for the scales: subnormals count as 1, zero 0,
// NaN and infinities as the non-finite flag
__device__ __forceinline__ int eff_exp_or_flag(unsigned long long bits) {
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0x7ff) return kNonFiniteExp;
    return e != 0 ? e : ((bits & 0x000fffffffffffffull) ? 1 : 0);
}

// round an FP32 value to TF32 (10 fraction bits), to nearest with ties away
// from zero, by integer operations; zero and subnormals pass unchanged
__device__ __forceinline__ float round_tf32(float v) {
    const unsigned b = __float_as_uint(v);
    if ((b & 0x7f800000u) == 0) return v;
    return __uint_as_float((b + 0x1000u) & 0xffffe000u);
}

// x * 2^-S as a TF32 pair (hi + lo), integer operations and FP32 only: the
// scaled value's top 24 significant bits h (truncated) and the rest l
// (rounded to 24 bits), then hi = tf32(h), lo = tf32((h - hi) + l).
// Values below the FP32 range after scaling, NaN and infinities give zeros
// (the scale flags a non-finite row or column; the epilogue writes NaN).
__device__ __forceinline__ void split_tf32(double x, int S, float &hi, float &lo) {
    hi = lo = 0.0f;
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    unsigned long long M = b & 0x000fffffffffffffull;
    if (e == 0x7ff || (e == 0 && M == 0)) return;
    int E = e;
    if (e != 0) {
        M |= 1ull << 52;
    } else {  // subnormal: normalise the significand
        const int lz = __clzll((long long)M) - 11;
        M <<= lz;
        E = 1 - lz;
    }
    const int fe = E - 1023 - S + 127;  // biased FP32 exponent of x 2^-S
    if (fe <= 0 || fe >= 255) return;
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const float h = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((M >> 29) & 0x7fffffu));
    const unsigned rest = (unsigned)(M & 0x1fffffffu);
    float l = 0.0f;
    if (rest != 0 && fe > 52) l = __fmul_rn(__uint2float_rn(rest), __uint_as_float((unsigned)(fe - 52) << 23));
    if (sign) l = -l;
    hi = round_tf32(h);
    lo = round_tf32(__fadd_rn(__fsub_rn(h, hi), l));
}

// rows of A, one 256-thread block each: the row's scale exponent, then
// the TF32 pair (zeros in the padding [k, kp)); the second pass reads the
// row from L2
__global__ void __launch_bounds__(256) split_rows_tf32_kernel(const double *A, long long lda, int m, int k, int kp,
                                                             int *ea, float *A1, float *A2) {
    __shared__ int red[8];
    const int row = blockIdx.x, tid = threadIdx.x;
    const double *src = A + (long long)row * lda;
    int mx = 0;
#pragma unroll 4
    for (int l = tid; l < k; l += 256) mx = max(mx, eff_exp_or_flag((unsigned long long)__double_as_longlong(src[l])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = max(mx, red[w]);
    const int S = mx == 0 ? 0 : mx - 1023 + 1;
    if (tid == 0) ea[row] = S;
    float *d1 = A1 + (long long)row * kp, *d2 = A2 + (long long)row * kp;
#pragma unroll 4
    for (int l = tid; l < kp; l += 256) {
        float h = 0.0f, lo = 0.0f;
        if (l < k) split_tf32(src[l], S, h, lo);
        d1[l] = h;
        d2[l] = lo;
    }
}

// column maxima of B (k x n) over chunks of 256 rows: 32 columns x 8 row
// groups per block, atomicMax into eb (zeroed first); exp_to_scale_kernel
// then turns the maxima into scale exponents
__global__ void col_max_tf32_kernel(const double *B, long long ldb, int k, int n, int *eb) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    const int l0 = blockIdx.y * 256, l1 = min(k, l0 + 256);
    if (col >= n) return;
    int mx = 0;
#pragma unroll 8
    for (int l = l0 + threadIdx.y; l < l1; l += 8)
        mx = max(mx, eff_exp_or_flag((unsigned long long)__double_as_longlong(B[(long long)l * ldb + col])));
    if (mx > 0) atomicMax(eb + col, mx);
}

// B transposed and split: 32 x 32 tiles through shared memory (reads along
// n, writes along k), zeros in the padding [k, kp)
__global__ void split_cols_tf32_kernel(const double *B, long long ldb, int k, int n, int kp, const int *eb,
                                       float *B1, float *B2) {
    __shared__ float th[32][33], tl[32][33];
    const int c0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
    const int x = threadIdx.x, c = c0 + x;
    const int S = c < n ? eb[c] : 0;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int l = l0 + y;
        float h = 0.0f, lo = 0.0f;
        if (c < n && l < k) split_tf32(B[(long long)l * ldb + c], S, h, lo);
        th[y][x] = h;
        tl[y][x] = lo;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int cc = c0 + y, l = l0 + x;
        if (cc < n && l < kp) {
            B1[(long long)cc * kp + l] = th[x][y];
            B2[(long long)cc * kp + l] = tl[x][y];
        }
    }
}

// ------------------------------------------------------- grouped splitting
struct GroupSplit {
    const double *A, *B;
    long long lda, ldb;
    int m, n, k, kp;
    long long pitch;                    // row pitch of the stacked split operands
    __nv_bfloat16 *A1, *A2, *B1, *B2;   // this problem's first rows in them
    int *ea, *eb;
};

// job (problem, first row): 8 warps, one row each
__global__ void split_a_group_kernel(const GroupSplit *gs, const int2 *jobs) {
    const int2 jb = jobs[blockIdx.x];
    const GroupSplit &G = gs[jb.x];
    const int row = jb.y + (threadIdx.x >> 5);
    if (row >= G.m) return;
    split_row_warp(G.A + (long long)row * G.lda, G.k, G.kp, G.ea + row, G.A1 + (long long)row * G.pitch,
                   G.A2 + (long long)row * G.pitch);
}

// job (problem, first column): 32 x 8 threads, the whole k range of 32 columns
__global__ void colmax_b_group_kernel(const GroupSplit *gs, const int2 *jobs) {
    const int2 jb = jobs[blockIdx.x];
    const GroupSplit &G = gs[jb.x];
    const int col = jb.y + threadIdx.x;
    int mx = 0;
    if (col < G.n) {
#pragma unroll 8
        for (int l = threadIdx.y; l < G.k; l += blockDim.y) {
            mx = max(mx, biased_exp_or_flag((unsigned long long)__double_as_longlong(G.B[(long long)l * G.ldb + col])));
        }
    }
    __shared__ int red[8][33];
    red[threadIdx.y][threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.y == 0 && col < G.n) {
        for (int y = 1; y < (int)blockDim.y; ++y) mx = max(mx, red[y][threadIdx.x]);
        G.eb[col] = bf16_col_scale(mx);
    }
}

// job (problem, first column, first k): one 64 x 64 tile
__global__ void split_b_group_kernel(const GroupSplit *gs, const int3 *jobs) {
    const int3 jb = jobs[blockIdx.x];
    const GroupSplit &G = gs[jb.x];
    split_b_tile(G.B, G.ldb, G.k, G.n, G.kp, G.pitch, G.eb, G.B1, G.B2, jb.z, jb.y);
}

size_t smem_gemm() { return 1024 + (size_t)kStages * kStageBytes + kStageOut + 256; }

// 2-CTA clusters of the pair kernel that fit on the device at once (cached)
int pair_clusters() {
    int dev = 0;
    OO_CUDA_TRY(cudaGetDevice(&dev));
    static std::atomic<int> max_clusters[64];
    int ncl = dev < 64 ? max_clusters[dev].load() : 0;
    if (ncl > 0) return ncl;
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)gemm_split3_pair_kernel, kSmemPair, attr);
    int sms = 148;
    OO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(sms / 2 * 2));
    cfg.blockDim = dim3(kGemmThreads);
    cfg.dynamicSmemBytes = kSmemPair;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    OO_CUDA_TRY(cudaOccupancyMaxActiveClusters(&ncl, (const void *)gemm_split3_pair_kernel, &cfg));
    OO_REQUIRE(ncl >= 1, OO_ECUDA, "no 2-CTA cluster of the GEMM kernel fits on this device");
    if (dev < 64) max_clusters[dev].store(ncl);
    return ncl;
}

// Tile width of the pair kernel for an m x n product: the width among 256,
// 224, 192 and 160 columns with the fewest column-waves (waves of units over
// the resident clusters x width), the widest on a tie.  Narrower MMAs lose
// tensor throughput (N = 128 ran at ~64 %), so 160 is the floor.
int pair_tile_width(int m, int n, int ncl) {
    const long long slabs = (m + 2 * kBM - 1) / (2 * kBM);
    int best = kBNP;
    long long best_cost = -1;
    for (int w = kBNP; w >= 160; w -= 32) {
        const long long units = slabs * ((n + w - 1) / w);
        const long long cost = (units + ncl - 1) / ncl * w;
        if (best_cost < 0 || cost < best_cost) {
            best = w;
            best_cost = cost;
        }
    }
    return best;
}

// persistent: one 2-CTA cluster per unit, at most as many as are resident
void launch_split3_pair(const GemmMaps &maps, GemmArgs ga, int nw, int ncl, cudaStream_t s) {
    ga.nw = nw;
    ga.m_tiles = (ga.m + 2 * kBM - 1) / (2 * kBM);  // 256-row slabs
    ga.n_tiles = (ga.n + nw - 1) / nw;              // nw-column panels
    const long long units = (long long)ga.m_tiles * ga.n_tiles;
    OO_REQUIRE(units < (1ll << 31), OO_EINVAL, "too many tiles");
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(2 * std::min<long long>(units, ncl)));
    cfg.blockDim = dim3(kGemmThreads);
    cfg.dynamicSmemBytes = kSmemPair;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    OO_CUDA_TRY(cudaLaunchKernelEx(&cfg, gemm_split3_pair_kernel, maps, (const GemmArgs)ga));
}

}  // namespace

size_t gemm_scratch_bytes(int m, int n, int k) {
    const size_t kp = (size_t)(k + kBK - 1) / kBK * kBK;
    const size_t a = (size_t)m * kp * 2, b = (size_t)n * kp * 2;
    return 2 * ((a + 255) / 256 * 256) + 2 * ((b + 255) / 256 * 256) + ((size_t)m + n) * 4 + 1024;
}

void launch_gemm_split3(int m, int n, int k, const double *A, long long lda, const double *B, long long ldb,
                        double *C, long long ldc, void *scratch, cudaStream_t s, int pair) {
    OO_REQUIRE(m >= 1 && n >= 1 && k >= 1, OO_EINVAL, "m, n, k must be >= 1");
    OO_REQUIRE(lda >= k && ldb >= n && ldc >= n, OO_EINVAL, "leading dimensions too small");
    const int kp = (k + kBK - 1) / kBK * kBK;
    const size_t a_bytes = ((size_t)m * kp * 2 + 255) / 256 * 256, b_bytes = ((size_t)n * kp * 2 + 255) / 256 * 256;
    char *p = static_cast<char *>(scratch);
    auto *A1 = reinterpret_cast<__nv_bfloat16 *>(p);
    auto *A2 = reinterpret_cast<__nv_bfloat16 *>(p + a_bytes);
    auto *B1 = reinterpret_cast<__nv_bfloat16 *>(p + 2 * a_bytes);
    auto *B2 = reinterpret_cast<__nv_bfloat16 *>(p + 2 * a_bytes + b_bytes);
    int *ea = reinterpret_cast<int *>(p + 2 * a_bytes + 2 * b_bytes);
    int *eb = ea + m;
    unsigned *err = reinterpret_cast<unsigned *>(eb + n);
    OO_CUDA_TRY(cudaMemsetAsync(err, 0, 4, s));

    const bool strip_b = ldb % 2 == 0 && ((uintptr_t)B & 15u) == 0;
    const bool rows_v2 = lda % 2 == 0 && ((uintptr_t)A & 15u) == 0;
    if (strip_b && rows_v2) {
        const int nstrip = (n + 15) / 16;
        const long long grid = (long long)nstrip + (m + 1) / 2;
        OO_REQUIRE(grid < (1ll << 31), OO_EINVAL, "problem too large");
        split_ab_kernel<<<(unsigned)grid, kStripThreads, 0, s>>>(A, lda, m, B, ldb, n, k, kp, nstrip, ea, eb, A1, A2,
                                                                B1, B2);
        OO_CUDA_TRY(cudaGetLastError());
    } else if (!strip_b) {
        OO_CUDA_TRY(cudaMemsetAsync(eb, 0, (size_t)n * 4, s));
        const int rows_per = 256;
        dim3 grid((n + 31) / 32, (k + rows_per - 1) / rows_per), block(32, 8);
        OO_REQUIRE(grid.y <= 65535, OO_EINVAL, "k too large");
        col_maxexp_kernel<<<grid, block, 0, s>>>(B, ldb, k, n, rows_per, eb);
        OO_CUDA_TRY(cudaGetLastError());
        exp_to_bf16_col_scale_kernel<<<(n + 255) / 256, 256, 0, s>>>(eb, n);
        OO_CUDA_TRY(cudaGetLastError());
    }
    if (!(strip_b && rows_v2)) {
        if (rows_v2)
            split_rows_v2_kernel<<<m, 256, 0, s>>>(A, lda, m, k, kp, ea, A1, A2);
        else
            split_rows_fused_kernel<<<(m + 7) / 8, 256, 0, s>>>(A, lda, m, k, kp, ea, A1, A2);
        OO_CUDA_TRY(cudaGetLastError());
        if (strip_b) {
            split_cols_strip_kernel<<<(n + 15) / 16, kStripThreads, 0, s>>>(B, ldb, k, n, kp, eb, B1, B2);
        } else {
            dim3 grid((n + 63) / 64, kp / 64);
            OO_REQUIRE(grid.y <= 65535, OO_EINVAL, "k too large");
            split_cols_t_kernel<<<grid, 256, 0, s>>>(B, ldb, k, n, kp, eb, B1, B2);
        }
        OO_CUDA_TRY(cudaGetLastError());
    }
    GemmMaps maps;
    map_bf16(&maps.a1, A1, m, kp, kBM);
    map_bf16(&maps.a2, A2, m, kp, kBM);
    int ncl = 0, nw = kBN;
    if (pair) {
        ncl = pair_clusters();
        nw = pair == 1 ? pair_tile_width(m, n, ncl) : pair;
        OO_REQUIRE(nw >= 160 && nw <= kBNP && nw % 32 == 0, OO_EINVAL, "pair tile width must be 160, 192, 224 or 256");
    }
    // B tiles: half of a pair tile's columns per CTA, else 128 columns
    map_bf16(&maps.b1, B1, n, kp, pair ? nw / 2 : kBN);
    map_bf16(&maps.b2, B2, n, kp, pair ? nw / 2 : kBN);
    GemmArgs ga{};
    ga.m = m;
    ga.n = n;
    ga.k = k;
    ga.kp = kp;
    ga.kstage = kBK;
    ga.m_tiles = (m + kBM - 1) / kBM;
    ga.n_tiles = (n + kBN - 1) / kBN;
    ga.C = C;
    ga.ldc = ldc;
    ga.ea = ea;
    ga.eb = eb;
    ga.err = err;
    if (pair) {
        launch_split3_pair(maps, ga, nw, ncl, s);
        return;
    }
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)gemm_split3_kernel, smem_gemm(), attr);
    const long long tiles = (long long)ga.m_tiles * ga.n_tiles;
    OO_REQUIRE(tiles < (1ll << 31), OO_EINVAL, "too many tiles");
    int dev2 = 0, sms2 = 148;
    cudaGetDevice(&dev2);
    cudaDeviceGetAttribute(&sms2, cudaDevAttrMultiProcessorCount, dev2);
    const int grid = (int)std::min<long long>(tiles, sms2);
    gemm_split3_kernel<<<grid, kGemmThreads, smem_gemm(), s>>>(maps, ga);
    OO_CUDA_TRY(cudaGetLastError());
}

// ------------------------------------------------------- TF32 pattern
namespace {
struct Tf32Layout {
    int kp;
    size_t a_bytes, b_bytes, total;
};
Tf32Layout tf32_layout(int m, int n, int k) {
    Tf32Layout L{};
    L.kp = (k + kBKTF32 - 1) / kBKTF32 * kBKTF32;
    L.a_bytes = ((size_t)m * L.kp * 4 + 255) / 256 * 256;
    L.b_bytes = ((size_t)n * L.kp * 4 + 255) / 256 * 256;
    L.total = 2 * L.a_bytes + 2 * L.b_bytes + ((size_t)m + n) * 4 + 1024;
    return L;
}
}  // namespace

size_t gemm_tf32_scratch_bytes(int m, int n, int k) { return tf32_layout(m, n, k).total; }

unsigned *gemm_tf32_error_word(void *scratch, int m, int n, int k) {
    const Tf32Layout L = tf32_layout(m, n, k);
    return reinterpret_cast<unsigned *>(static_cast<char *>(scratch) + 2 * L.a_bytes + 2 * L.b_bytes +
                                        ((size_t)m + n) * 4);
}

void launch_gemm_split3_tf32(int m, int n, int k, const double *A, long long lda, const double *B, long long ldb,
                             double *C, long long ldc, void *scratch, cudaStream_t s) {
    OO_REQUIRE(m >= 1 && n >= 1 && k >= 1, OO_EINVAL, "m, n, k must be >= 1");
    OO_REQUIRE(lda >= k && ldb >= n && ldc >= n, OO_EINVAL, "leading dimensions too small");
    const Tf32Layout L = tf32_layout(m, n, k);
    const int kp = L.kp;
    char *p = static_cast<char *>(scratch);
    auto *A1 = reinterpret_cast<float *>(p);
    auto *A2 = reinterpret_cast<float *>(p + L.a_bytes);
    auto *B1 = reinterpret_cast<float *>(p + 2 * L.a_bytes);
    auto *B2 = reinterpret_cast<float *>(p + 2 * L.a_bytes + L.b_bytes);
    int *ea = reinterpret_cast<int *>(p + 2 * L.a_bytes + 2 * L.b_bytes);
    int *eb = ea + m;
    unsigned *err = reinterpret_cast<unsigned *>(eb + n);
    OO_CUDA_TRY(cudaMemsetAsync(err, 0, 4, s));
    split_rows_tf32_kernel<<<m, 256, 0, s>>>(A, lda, m, k, kp, ea, A1, A2);
    OO_CUDA_TRY(cudaGetLastError());
    OO_CUDA_TRY(cudaMemsetAsync(eb, 0, (size_t)n * 4, s));
    OO_REQUIRE((k + 255) / 256 <= 65535, OO_EINVAL, "k too large");
    col_max_tf32_kernel<<<dim3((n + 31) / 32, (k + 255) / 256), dim3(32, 8), 0, s>>>(B, ldb, k, n, eb);
    OO_CUDA_TRY(cudaGetLastError());
    exp_to_scale_kernel<<<(n + 255) / 256, 256, 0, s>>>(eb, n);
    OO_CUDA_TRY(cudaGetLastError());
    OO_REQUIRE(kp / 32 <= 65535, OO_EINVAL, "k too large");
    split_cols_tf32_kernel<<<dim3((n + 31) / 32, kp / 32), dim3(32, 8), 0, s>>>(B, ldb, k, n, kp, eb, B1, B2);
    OO_CUDA_TRY(cudaGetLastError());
    GemmMaps maps;
    map_f32(&maps.a1, A1, m, kp, kBM);
    map_f32(&maps.a2, A2, m, kp, kBM);
    map_f32(&maps.b1, B1, n, kp, kBN);
    map_f32(&maps.b2, B2, n, kp, kBN);
    GemmArgs ga{};
    ga.m = m;
    ga.n = n;
    ga.k = k;
    ga.kp = kp;
    ga.kstage = kBKTF32;
    ga.m_tiles = (m + kBM - 1) / kBM;
    ga.n_tiles = (n + kBN - 1) / kBN;
    ga.C = C;
    ga.ldc = ldc;
    ga.ea = ea;
    ga.eb = eb;
    ga.err = err;
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)gemm_split3_tf32_kernel, smem_gemm(), attr);
    const long long tiles = (long long)ga.m_tiles * ga.n_tiles;
    OO_REQUIRE(tiles < (1ll << 31), OO_EINVAL, "too many tiles");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<long long>(tiles, sms);
    gemm_split3_tf32_kernel<<<grid, kGemmThreads, smem_gemm(), s>>>(maps, ga);
    OO_CUDA_TRY(cudaGetLastError());
}

// ------------------------------------------------------------ group plans
struct GemmGroup {
    void *arena = nullptr;
    GemmMaps maps;
    GroupProblem *d_probs = nullptr;
    GroupSplit *d_split = nullptr;
    int4 *d_tiles = nullptr;
    int2 *d_ajobs = nullptr, *d_cjobs = nullptr;
    int3 *d_bjobs = nullptr;
    unsigned *d_err = nullptr;
    int ntiles = 0, na = 0, nc = 0, nb = 0, grid = 1;
    double flops = 0;
};

GemmGroup *gemm_group_create(const std::vector<GemmDesc> &v, int num_sms) {
    OO_REQUIRE(!v.empty(), OO_EINVAL, "empty GEMM group");
    auto up = [](size_t x, size_t a) { return (x + a - 1) / a * a; };
    // arena layout: A1 | A2 | B1 | B2 (every problem's rows stacked, row pitch
    // KP = the largest padded K) | scale exponents | descriptors | job lists | error word
    std::vector<int> kp(v.size()), ra(v.size()), rb(v.size());
    long long rows_a = 0, rows_b = 0;
    int KP = kBK;
    for (size_t i = 0; i < v.size(); ++i) {
        const GemmDesc &d = v[i];
        OO_REQUIRE(d.m >= 1 && d.n >= 1 && d.k >= 1 && d.lda >= d.k && d.ldb >= d.n && d.ldc >= d.n, OO_EINVAL,
                   "bad GEMM in group");
        kp[i] = (d.k + kBK - 1) / kBK * kBK;
        KP = std::max(KP, kp[i]);
        ra[i] = (int)rows_a;
        rb[i] = (int)rows_b;
        rows_a += d.m;
        rows_b += d.n;
        OO_REQUIRE(rows_a < (1ll << 30) && rows_b < (1ll << 30), OO_EINVAL, "GEMM group too large");
    }
    const size_t a_bytes = up((size_t)rows_a * KP * 2, 256), b_bytes = up((size_t)rows_b * KP * 2, 256);
    size_t at = 0;
    const size_t off_a1 = at; at += a_bytes;
    const size_t off_a2 = at; at += a_bytes;
    const size_t off_b1 = at; at += b_bytes;
    const size_t off_b2 = at; at += b_bytes;
    std::vector<size_t> off_ea(v.size()), off_eb(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        off_ea[i] = at; at += up((size_t)v[i].m * 4, 16);
        off_eb[i] = at; at += up((size_t)v[i].n * 4, 16);
    }
    at = up(at, 128);
    const size_t off_probs = at; at += up(v.size() * sizeof(GroupProblem), 16);
    const size_t off_split = at; at += up(v.size() * sizeof(GroupSplit), 16);
    std::vector<int4> tiles;
    std::vector<int2> ajobs, cjobs;
    std::vector<int3> bjobs;
    double flops = 0;
    for (size_t i = 0; i < v.size(); ++i) {
        const GemmDesc &d = v[i];
        flops += 2.0 * d.m * d.n * d.k;
        for (int m0 = 0; m0 < d.m; m0 += kBM)
            for (int n0 = 0; n0 < d.n; n0 += kBN) tiles.push_back(make_int4((int)i, m0, n0, kp[i] / kBK));
        for (int r0 = 0; r0 < d.m; r0 += 8) ajobs.push_back(make_int2((int)i, r0));
        for (int c0 = 0; c0 < d.n; c0 += 32) cjobs.push_back(make_int2((int)i, c0));
        for (int c0 = 0; c0 < d.n; c0 += 64)
            for (int l0 = 0; l0 < kp[i]; l0 += 64) bjobs.push_back(make_int3((int)i, c0, l0));
    }
    std::stable_sort(tiles.begin(), tiles.end(), [](const int4 &x, const int4 &y) { return x.w > y.w; });
    const size_t off_tiles = at; at += up(tiles.size() * sizeof(int4), 16);
    const size_t off_aj = at; at += up(ajobs.size() * sizeof(int2), 16);
    const size_t off_cj = at; at += up(cjobs.size() * sizeof(int2), 16);
    const size_t off_bj = at; at += up(bjobs.size() * sizeof(int3), 16);
    const size_t off_err = at; at += 16;
    auto *g = new GemmGroup();
    try {
        if (cudaMalloc(&g->arena, at) != cudaSuccess) {
            cudaGetLastError();
            throw Error{OO_ENOMEM, "GEMM group arena of " + std::to_string(at) + " bytes"};
        }
        char *base = static_cast<char *>(g->arena);
        auto *A1 = reinterpret_cast<__nv_bfloat16 *>(base + off_a1);
        auto *A2 = reinterpret_cast<__nv_bfloat16 *>(base + off_a2);
        auto *B1 = reinterpret_cast<__nv_bfloat16 *>(base + off_b1);
        auto *B2 = reinterpret_cast<__nv_bfloat16 *>(base + off_b2);
        map_bf16(&g->maps.a1, A1, rows_a, KP, kBM);
        map_bf16(&g->maps.a2, A2, rows_a, KP, kBM);
        map_bf16(&g->maps.b1, B1, rows_b, KP, kBN);
        map_bf16(&g->maps.b2, B2, rows_b, KP, kBN);
        std::vector<GroupProblem> probs(v.size());
        std::vector<GroupSplit> splits(v.size());
        for (size_t i = 0; i < v.size(); ++i) {
            const GemmDesc &d = v[i];
            int *ea = reinterpret_cast<int *>(base + off_ea[i]);
            int *eb = reinterpret_cast<int *>(base + off_eb[i]);
            probs[i] = GroupProblem{d.C, d.ldc, ea, eb, d.m, d.n, d.k, kp[i], ra[i], rb[i]};
            splits[i] = GroupSplit{d.A, d.B, d.lda, d.ldb, d.m, d.n, d.k, kp[i], (long long)KP,
                                   A1 + (size_t)ra[i] * KP, A2 + (size_t)ra[i] * KP,
                                   B1 + (size_t)rb[i] * KP, B2 + (size_t)rb[i] * KP, ea, eb};
        }
        OO_CUDA_TRY(cudaMemcpy(base + off_probs, probs.data(), probs.size() * sizeof(GroupProblem),
                               cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_split, splits.data(), splits.size() * sizeof(GroupSplit),
                               cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_aj, ajobs.data(), ajobs.size() * sizeof(int2), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_cj, cjobs.data(), cjobs.size() * sizeof(int2), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_bj, bjobs.data(), bjobs.size() * sizeof(int3), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemset(base + off_err, 0, 16));
        g->d_probs = reinterpret_cast<GroupProblem *>(base + off_probs);
        g->d_split = reinterpret_cast<GroupSplit *>(base + off_split);
        g->d_tiles = reinterpret_cast<int4 *>(base + off_tiles);
        g->d_ajobs = reinterpret_cast<int2 *>(base + off_aj);
        g->d_cjobs = reinterpret_cast<int2 *>(base + off_cj);
        g->d_bjobs = reinterpret_cast<int3 *>(base + off_bj);
        g->d_err = reinterpret_cast<unsigned *>(base + off_err);
        g->ntiles = (int)tiles.size();
        g->na = (int)ajobs.size();
        g->nc = (int)cjobs.size();
        g->nb = (int)bjobs.size();
        g->grid = std::max(1, std::min(g->ntiles, num_sms));
        g->flops = flops;
    } catch (...) {
        if (g->arena) cudaFree(g->arena);
        delete g;
        throw;
    }
    return g;
}

void gemm_group_launch(GemmGroup *g, cudaStream_t s) {
    split_a_group_kernel<<<g->na, 256, 0, s>>>(g->d_split, g->d_ajobs);
    OO_CUDA_TRY(cudaGetLastError());
    colmax_b_group_kernel<<<g->nc, dim3(32, 8), 0, s>>>(g->d_split, g->d_cjobs);
    OO_CUDA_TRY(cudaGetLastError());
    split_b_group_kernel<<<g->nb, 256, 0, s>>>(g->d_split, g->d_bjobs);
    OO_CUDA_TRY(cudaGetLastError());
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)gemm_group_kernel, smem_gemm(), attr);
    gemm_group_kernel<<<g->grid, kGemmThreads, smem_gemm(), s>>>(g->maps, g->d_probs, g->d_tiles, g->ntiles,
                                                                  g->d_err);
    OO_CUDA_TRY(cudaGetLastError());
}

unsigned gemm_group_check(GemmGroup *g, cudaStream_t s) {
    unsigned e = 0;
    OO_CUDA_TRY(cudaMemcpyAsync(&e, g->d_err, 4, cudaMemcpyDeviceToHost, s));
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    if (e) OO_CUDA_TRY(cudaMemsetAsync(g->d_err, 0, 4, s));
    return e;
}

double gemm_group_flops(const GemmGroup *g) { return g->flops; }

void gemm_group_destroy(GemmGroup *g) {
    if (!g) return;
    if (g->arena) cudaFree(g->arena);
    delete g;
}

unsigned *gemm_error_word(void *scratch, int m, int n, int k) {
    const int kp = (k + kBK - 1) / kBK * kBK;
    const size_t a_bytes = ((size_t)m * kp * 2 + 255) / 256 * 256, b_bytes = ((size_t)n * kp * 2 + 255) / 256 * 256;
    return reinterpret_cast<unsigned *>(static_cast<char *>(scratch) + 2 * a_bytes + 2 * b_bytes +
                                        ((size_t)m + n) * 4);
}

unsigned gemm_check_error(void *scratch, int m, int n, int k, cudaStream_t s) {
    unsigned *err = gemm_error_word(scratch, m, n, k);
    unsigned e = 0;
    OO_CUDA_TRY(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s));
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    if (e) OO_CUDA_TRY(cudaMemsetAsync(err, 0, 4, s));
    return e;
}

}  // namespace oo
