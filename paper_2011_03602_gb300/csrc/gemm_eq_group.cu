// FP64-equivalent matrix products of uneven sizes in one persistent
// tensor-core launch (the batched form of the Sec. 3.2.2 matrix-product
// block), and the single products whose accumulation scheme is a level
// scheme (eq_digits.cuh).
//
// Work list: one entry per output tile (problem, m0, n0, width).  Tiles are
// 128 rows (the M of one tcgen05.mma) by 32, 64 or 128 columns; the width of
// a problem's full tiles comes from a table indexed by the problem's n and k
// (the autotuner's choice: oo_tune_gemm_tiles), a problem's last column tile
// takes the narrowest width that covers what is left.  A tile's unit of work
// is one accumulator pair of its scheme over one K-block: a list of terms
// A_p x [B_qL | B_qR] whose products land in the pair's left half (level or
// product qL) and right half (qR), as one N = 2 w MMA when both halves are
// fed, else one N = w MMA into the half that is.  Units run K-block outer,
// so the arithmetic per element is that of the single-problem kernel for the
// pair scheme and the same for a problem alone or in a group, whatever the
// tile widths: widths change speed only.
//
// Operands: every problem's digit slices are stacked by rows in one of six
// pitch classes (padded K <= 64, 128, 256, 512, 1024, larger), so two tensor
// maps per class, passed as kernel parameters, cover every problem: A with
// 128-row boxes, B (transposed slices) with 32-row boxes, loaded w / 32 at a
// time.  Roles as in the single kernel: warp 0 streams A_p and the B tiles
// (TMA, 128-byte swizzle) through a 4-stage ring, warp 1 issues tcgen05.mma
// into two double-buffered 256-column FP32 accumulators in tensor memory,
// eight epilogue warps (two per lane quarter) add each finished unit, scaled
// by its power of two, into a float-float sum in registers and write FP64 C
// after the tile's last unit; warps whose rows or columns lie wholly outside
// the problem skip the reads.  Every mbarrier wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "eq_digits.cuh"
#include "ff.cuh"
#include "oo_internal.h"
#include "resident.h"
#include "tc.cuh"

namespace oo {

namespace {

using namespace tc;
using eq::kBK;

constexpr int kBM = 128, kStages = 4;
constexpr int kThreads = 320;  // producer, MMA issuer, 8 epilogue warps
constexpr int kEpiWarps = 8;
constexpr uint32_t kTileA = kBM * kBK * 2;               // 16 KB
constexpr int kBRows = 32;                                // B box rows
constexpr uint32_t kBox = kBRows * kBK * 2;               // 4 KB
constexpr uint32_t kStageBytes = kTileA + 2 * 128 * kBK * 2;  // A + two B tiles of up to 128 rows
constexpr int kMaxUnits = 24, kMaxTerms = 48;
constexpr unsigned char kNone = 0xff;
constexpr int kClasses = 6;
// scheme tables: 0 pairs with 8-bit digits (padded k <= 256), 1 pairs with
// 7-bit digits, 2 levels with 7-bit digits, 3 levels with 6-bit digits
constexpr int kTables = 4;

struct SchemeTab {
    int nunits, nterms;
    unsigned char ut0[kMaxUnits], unt[kMaxUnits];                 // first term, term count of each unit
    unsigned char tp[kMaxTerms], tqL[kMaxTerms], tqR[kMaxTerms];  // 0-based slices; kNone: half not fed
    float usL[kMaxUnits], usR[kMaxUnits];                         // 2^(-beta s) of each half (0: unused)
};

struct GProb {
    double *C;
    const int *ea, *eb;
    long long ldc;
    int m, n, ksteps, kb_steps;
    int nkb, ra, rb, cls;  // rows of slice 0 in its class's stacked A / B, pitch class
    int scheme, bn, m_tiles, n_tiles;  // bn, m_tiles, n_tiles: single-problem raster only
};

struct GMaps {
    CUtensorMap a[kClasses], b[kClasses];
};

struct GArgs {
    unsigned *err;
    SchemeTab sch[kTables];
};

// work list of a group: tiles[t] = (problem, m0, n0, width) in global memory
struct GroupTiles {
    const GProb *probs;
    const int4 *tiles;
    int ntiles;
    __device__ __forceinline__ int count() const { return ntiles; }
    __device__ __forceinline__ int4 tile(int t) const { return tiles[t]; }
    __device__ __forceinline__ const GProb &prob(int i) const { return probs[i]; }
};

__host__ __device__ inline int narrowest_width(int rem) { return rem <= 32 ? 32 : (rem <= 64 ? 64 : 128); }

// one problem: its descriptor is a kernel parameter, tiles in grouped raster
// order (8 m-tiles share their B panels while in L2)
struct SingleTiles {
    const GProb *P;
    __device__ __forceinline__ int count() const { return P->m_tiles * P->n_tiles; }
    __device__ __forceinline__ int4 tile(int t) const {
        constexpr int kGroupM = 8;
        const int per_group = kGroupM * P->n_tiles;
        const int g = t / per_group, r = t % per_group;
        const int rows = min(kGroupM, P->m_tiles - g * kGroupM);
        const int m0 = (g * kGroupM + r % rows) * kBM, n0 = (r / rows) * P->bn;
        const int rem = P->n - n0;
        return make_int4(0, m0, n0, rem >= P->bn ? P->bn : narrowest_width(rem));
    }
    __device__ __forceinline__ const GProb &prob(int) const { return *P; }
};

// instruction descriptor (kind::f16: D F32, A and B BF16, both K-major) of
// an M = 128 MMA with N columns
__device__ __forceinline__ uint32_t idesc_n(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_rt(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

#define OO_TMEM_LD16(taddr, r)                                                                              \
    asm volatile(                                                                                           \
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "  \
        "[%16];"                                                                                            \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),   \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),          \
          "=r"(r[15])                                                                                       \
        : "r"(taddr))

// Shared-memory pipeline of one tile CTA: a 4-stage operand ring, two
// accumulator buffers in tensor memory, an abort flag.
struct Pipe {
    unsigned char *sm;
    uint64_t *full, *empty, *tfull, *tempty;
    volatile int *abort_flag;
    uint32_t tmem;
};

// Barriers, abort flag and tensor memory of the CTA; `extra` more mbarriers
// (initialised by the caller) follow the pipeline's.
__device__ __forceinline__ Pipe pipe_setup(uint64_t **extra_bars) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    Pipe pp;
    pp.sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) &
                                              ~static_cast<uintptr_t>(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(pp.sm + kStages * kStageBytes);
    pp.full = bars;
    pp.empty = bars + kStages;
    pp.tfull = bars + 2 * kStages;
    pp.tempty = bars + 2 * kStages + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 4);
    pp.abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    // 16-byte aligned (8 mbarriers then 16-byte entries follow there)
    if (extra_bars) *extra_bars = reinterpret_cast<uint64_t *>(tmem_slot + 4);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(su32(&pp.full[s]), 1);
            bar_init(su32(&pp.empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(su32(&pp.tfull[b]), 1);
            bar_init(su32(&pp.tempty[b]), kEpiWarps);
        }
        *pp.abort_flag = 0;
    }
    if (warp == 1) {
        tmem_alloc(su32(tmem_slot), 512);
        fence_before();
    }
    return pp;
}

// TMA producer (one thread): the operand loads of one tile; false when the
// pipeline aborted
__device__ __forceinline__ bool produce_tile(const GMaps &maps, const GArgs &a, const Pipe &pp, const GProb &P,
                                             const int4 td, int &it, int &loaded) {
    const SchemeTab &S = a.sch[P.scheme];
    const CUtensorMap *ma = &maps.a[P.cls], *mb = &maps.b[P.cls];
    const int nbox = td.w / kBRows;
    const uint32_t btile = (uint32_t)td.w * kBK * 2;
    for (int kbi = 0; kbi < P.nkb; ++kbi) {
        const int ks0 = kbi * P.kb_steps, ks1 = min(P.ksteps, ks0 + P.kb_steps);
        for (int u = 0; u < S.nunits; ++u) {
            for (int tt = S.ut0[u]; tt < S.ut0[u] + S.unt[u]; ++tt) {
                const int p = S.tp[tt], qL = S.tqL[tt], qR = S.tqR[tt];
                const int rowA = P.ra + p * P.m + td.y;
                const int rowL = P.rb + (qL == kNone ? 0 : qL) * P.n + td.z;
                const int rowR = P.rb + (qR == kNone ? 0 : qR) * P.n + td.z;
                const uint32_t bytes = kTileA + (uint32_t)((qL != kNone) + (qR != kNone)) * btile;
                for (int ks = ks0; ks < ks1; ++ks, ++it) {
                    const int s = it % kStages;
                    const uint32_t use = it / kStages;
                    if (use > 0 && !bar_wait(su32(&pp.empty[s]), (use - 1) & 1, pp.abort_flag, a.err, 1u))
                        return false;
                    unsigned char *st = pp.sm + (size_t)s * kStageBytes;
                    const uint32_t fb = su32(&pp.full[s]);
                    bar_expect_tx(fb, bytes);
                    tma_2d(su32(st), ma, ks * kBK, rowA, fb);
                    if (qL != kNone)
                        for (int j = 0; j < nbox; ++j)
                            tma_2d(su32(st + kTileA + j * kBox), mb, ks * kBK, rowL + j * kBRows, fb);
                    if (qR != kNone)
                        for (int j = 0; j < nbox; ++j)
                            tma_2d(su32(st + kTileA + btile + j * kBox), mb, ks * kBK, rowR + j * kBRows, fb);
                    ++loaded;
                }
            }
        }
    }
    return true;
}

// MMA issuer (one thread): every unit of one tile into the accumulator
// buffers; false when the pipeline aborted
__device__ __forceinline__ bool mma_tile(const GArgs &a, const Pipe &pp, const GProb &P, const int4 td, int &it,
                                         int &gu, int &units_mma) {
    const SchemeTab &S = a.sch[P.scheme];
    const uint32_t btile = (uint32_t)td.w * kBK * 2;
    const uint32_t id_pair = idesc_n(2 * td.w), id_one = idesc_n(td.w);
    for (int kbi = 0; kbi < P.nkb; ++kbi) {
        const int ks0 = kbi * P.kb_steps, ks1 = min(P.ksteps, ks0 + P.kb_steps);
        for (int u = 0; u < S.nunits; ++u, ++gu) {
            const int b = gu & 1;
            const uint32_t buse = gu >> 1;
            if (buse > 0 && !bar_wait(su32(&pp.tempty[b]), (buse - 1) & 1, pp.abort_flag, a.err, 2u)) return false;
            fence_after();
            const uint32_t d = pp.tmem + (uint32_t)(b * 256);
            bool first = true;
            for (int tt = S.ut0[u]; tt < S.ut0[u] + S.unt[u]; ++tt) {
                const int qL = S.tqL[tt], qR = S.tqR[tt];
                for (int ks = ks0; ks < ks1; ++ks, ++it) {
                    const int s = it % kStages;
                    if (!bar_wait(su32(&pp.full[s]), (it / kStages) & 1, pp.abort_flag, a.err, 2u)) return false;
                    fence_after();
                    const uint32_t sa = su32(pp.sm + (size_t)s * kStageBytes);
                    const uint32_t sbL = sa + kTileA, sbR = sbL + btile;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint32_t off = kk * 32;  // 16 BF16 along K inside the 128-byte row
                        const uint32_t acc = first ? 0u : 1u;
                        if (qL != kNone && qR != kNone)  // both halves: B_qL and B_qR stacked
                            mma_rt(d, sdesc_sw128(sa + off), sdesc_sw128(sbL + off), id_pair, acc);
                        else if (qL != kNone)
                            mma_rt(d, sdesc_sw128(sa + off), sdesc_sw128(sbL + off), id_one, acc);
                        else
                            mma_rt(d + (uint32_t)td.w, sdesc_sw128(sa + off), sdesc_sw128(sbR + off), id_one, acc);
                        first = false;
                    }
                    mma_commit(su32(&pp.empty[s]));
                }
            }
            mma_commit(su32(&pp.tfull[b]));  // this unit's accumulator pair is complete
            ++units_mma;
        }
    }
    return true;
}

// One epilogue warp (of eight: lane quarter q = warp & 3, column half h):
// add every finished unit of one tile, scaled by its power of two, into a
// float-float running sum (Sh, Sl) of this row's columns, then write FP64
// C; false when the pipeline aborted
__device__ __forceinline__ bool epilogue_tile(const GArgs &a, const Pipe &pp, const GProb &P, const int4 td, int &gu,
                                              float (&Sh)[64], float (&Sl)[64]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3;         // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;  // which half of the tile's columns
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const SchemeTab &S = a.sch[P.scheme];
    const int cpw = td.w >> 1, cw0 = h * cpw;  // columns per warp, first column of this warp
    const int row0 = td.y + q * 32;
    const int ncols = min(cpw, P.n - td.z - cw0);
    const bool active = row0 < P.m && ncols > 0;  // warp-uniform
    const int units = P.nkb * S.nunits;
    for (int uu = 0; uu < units; ++uu, ++gu) {
        const int b = gu & 1;
        if (!bar_wait(su32(&pp.tfull[b]), (gu >> 1) & 1, pp.abort_flag, a.err, 4u)) return false;
        fence_after();
        const int u = uu % S.nunits;
        const float fL = S.usL[u], fR = S.usR[u];
        if (active) {
            const uint32_t acc = pp.tmem + (uint32_t)(b * 256) + lane_off + (uint32_t)cw0;
#pragma unroll
            for (int c = 0; c < 64; c += 16) {
                if (c < ncols) {
                    uint32_t v[16];
                    OO_TMEM_LD16(acc + c, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float w = __fmul_rn(__uint_as_float(v[j]), fL);  // exact: power of two
                        if (uu == 0) {
                            Sh[c + j] = w;
                            Sl[c + j] = 0.0f;
                        } else {
                            ff::add(Sh[c + j], Sl[c + j], w, 0.0f, Sh[c + j], Sl[c + j]);
                        }
                    }
                    if (fR != 0.0f) {
                        OO_TMEM_LD16(acc + (uint32_t)td.w + c, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float w = __fmul_rn(__uint_as_float(v[j]), fR);
                            ff::add(Sh[c + j], Sl[c + j], w, 0.0f, Sh[c + j], Sl[c + j]);
                        }
                    }
                }
            }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(su32(&pp.tempty[b]));
    }
    if (active) {
        // column scales: lane l holds columns l and l + 32 of this warp's
        // range and hands them out by shuffle
        const int row = row0 + lane;
        const int c0 = td.z + cw0;
        const int e0 = lane < ncols ? P.eb[c0 + lane] : 0;
        const int e1 = 32 + lane < ncols ? P.eb[c0 + 32 + lane] : 0;
        const bool row_ok = row < P.m;
        const int sa = row_ok ? P.ea[row] : 0;
        double *crow = P.C + (long long)row * P.ldc + c0;
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            if (j < ncols) {
                const int sb = __shfl_sync(0xffffffffu, j < 32 ? e0 : e1, j & 31);
                if (row_ok) crow[j] = nan_or_scaled(ff::to_double(Sh[j], Sl[j]), sa + sb);
            }
        }
    }
    return true;
}

// drain on abort: wait (bounded) for issued MMAs and copies before tensor
// memory is released and the CTA exits
__device__ __forceinline__ void pipe_teardown(const Pipe &pp, int loaded, int units_mma) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*pp.abort_flag) {
        if (warp == 1 && lane == 0 && units_mma > 0)
            bar_drain(su32(&pp.tfull[(units_mma - 1) & 1]), ((units_mma - 1) >> 1) & 1);
        if (warp == 0 && lane == 0)
            for (int it = (loaded > kStages ? loaded - kStages : 0); it < loaded; ++it)
                bar_drain(su32(&pp.full[it % kStages]), (it / kStages) & 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(pp.tmem, 512);
    }
}

template <class Src>
__device__ __forceinline__ void eq_tiles_body(const GMaps &maps, const GArgs &a, const Src &src) {
    Pipe pp = pipe_setup(nullptr);
    if (threadIdx.x == 0) {
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    fence_after();
    pp.tmem = *reinterpret_cast<uint32_t *>(pp.tempty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = src.count();
    int loaded = 0;     // producer: stages issued
    int units_mma = 0;  // MMA issuer: units whose accumulation was issued
    if (warp == 0 && lane == 0) {
        int it = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            const int4 td = src.tile(t);
            if (!produce_tile(maps, a, pp, src.prob(td.x), td, it, loaded)) break;
        }
    } else if (warp == 1 && lane == 0) {
        int it = 0, gu = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            const int4 td = src.tile(t);
            if (!mma_tile(a, pp, src.prob(td.x), td, it, gu, units_mma)) break;
        }
    } else if (warp >= 2) {
        float Sh[64], Sl[64];
        int gu = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            const int4 td = src.tile(t);
            if (!epilogue_tile(a, pp, src.prob(td.x), td, gu, Sh, Sl)) break;
        }
    }
    pipe_teardown(pp, loaded, units_mma);
}

__global__ void __launch_bounds__(kThreads, 1) gemm_eq_group_kernel(const __grid_constant__ GMaps maps,
                                                                   const __grid_constant__ GArgs a,
                                                                   const GProb *probs, const int4 *tiles,
                                                                   int ntiles) {
    const GroupTiles src{probs, tiles, ntiles};
    eq_tiles_body(maps, a, src);
}

__global__ void __launch_bounds__(kThreads, 1) gemm_eq_single_kernel(const __grid_constant__ GMaps maps,
                                                                    const __grid_constant__ GArgs a,
                                                                    const __grid_constant__ GProb P) {
    const SingleTiles src{&P};
    eq_tiles_body(maps, a, src);
}

// ------------------------------------------------ the device-resident loop
// One GEMM request of the resident serving loop (resident.h): its tile
// descriptor, the split entry its tiles wait for, and its completion count
// (eight epilogue warps per tile).
struct ResTileDesc {
    GProb P;
    uint32_t split_ctr, split_target;
    uint32_t done_ctr, done_target;
    uint32_t gen;
    int32_t slot, pad0, pad1;
};
constexpr int kTileNop = -1, kTileStop = -2;
struct ResTileArgs {
    const int4 *ring;          // res::kRingCap entries (request slot, m0, n0, width); slot kTileNop / kTileStop
    const ResTileDesc *desc;   // res::kSlots
    unsigned *ctr;             // entry counters (res::kRingCap) then one per request slot
    const unsigned *heartbeat; // incremented by the SIMT worker for every entry a CTA passes
    res::Ctl *ctl;             // mapped control block (device address)
    unsigned long long start;  // first tile entry of this launch
};

__device__ __forceinline__ unsigned long long ld_acquire_sys64(const volatile unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_acquire_gpu32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys32(volatile unsigned *p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Persistent tensor-core worker of the resident loop: CTA c takes tile
// entries start + c, start + c + CTAs, ...  Its producer thread waits (bounded)
// for each entry's publication and for the request's split, then forwards the
// entry through a four-deep shared-memory queue to the MMA issuer and the
// epilogue warps (keep-alive entries too, so that no role's wait runs out
// while the server idles) and loads the tile as the grouped kernel does.
// The epilogue counts finished tiles; the warp that finishes a request
// writes its generation into the control block.
__global__ void __launch_bounds__(kThreads, 1) resident_tiles_kernel(const __grid_constant__ GMaps maps,
                                                                    const __grid_constant__ GArgs a,
                                                                    const __grid_constant__ ResTileArgs r) {
    uint64_t *xb = nullptr;
    Pipe pp = pipe_setup(&xb);
    uint64_t *qfull = xb, *qempty = xb + 4;
    int4 *tq = reinterpret_cast<int4 *>(xb + 8);
    if (threadIdx.x == 0) {
        for (int f = 0; f < 4; ++f) {
            bar_init(su32(&qfull[f]), 1);
            bar_init(su32(&qempty[f]), 1 + kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    fence_after();
    pp.tmem = *reinterpret_cast<uint32_t *>(pp.tempty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int loaded = 0, units_mma = 0;
    if (threadIdx.x == 0) r.ctl->alive[res::kMaxCtas + blockIdx.x] = 1u;
    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------- producer
        int it = 0;
        unsigned long long seen = 0, fi = 0;  // fi: entries forwarded to the queue
        auto forward = [&](int4 td) {
            const int f = (int)(fi & 3);
            if (fi >= 4 && !bar_wait(su32(&qempty[f]), (uint32_t)((fi >> 2) - 1) & 1, pp.abort_flag, a.err, 512u))
                return false;
            tq[f] = td;
            bar_arrive(su32(&qfull[f]));
            ++fi;
            return true;
        };
        for (unsigned long long i = 0;; ++i) {
            const unsigned long long t = r.start + blockIdx.x + i * gridDim.x;
            int4 td = make_int4(kTileStop, 0, 0, 0);
            bool ok = true;
            if (seen <= t) {
                const long long t0 = clock64();
                while ((seen = ld_acquire_sys64(&r.ctl->pub_tiles)) <= t) {
                    if (*pp.abort_flag || clock64() - t0 > kWaitLimit) {
                        *pp.abort_flag = 1;
                        atomicOr(a.err, 8u);
                        ok = false;
                        break;
                    }
                }
            }
            if (ok) {
                td = __ldcg(&r.ring[t % res::kRingCap]);
                r.ctl->tile_progress[blockIdx.x] = t + gridDim.x;  // this CTA's next entry
                if (td.x >= 0) {
                    // The request's digit slices must be complete before they
                    // are loaded (and seen by the async proxy).  Its split entry
                    // may wait behind other requests' SIMT work, so the bound
                    // is on the SIMT worker making no progress at all (its
                    // heartbeat counter), not on the time waited; meanwhile
                    // keep-alive markers keep the other roles' waits short.
                    const ResTileDesc &D = r.desc[td.x];
                    long long t0 = clock64(), tk = t0;
                    unsigned hb = ld_acquire_gpu32(r.heartbeat);
                    while ((int)(ld_acquire_gpu32(&r.ctr[D.split_ctr]) - D.split_target) < 0) {
                        const long long now = clock64();
                        const unsigned h = ld_acquire_gpu32(r.heartbeat);
                        if (h != hb) {
                            hb = h;
                            t0 = now;
                        }
                        if (*pp.abort_flag || now - t0 > kWaitLimit) {
                            *pp.abort_flag = 1;
                            atomicOr(a.err, 16u);
                            ok = false;
                            break;
                        }
                        if (now - tk > kWaitLimit / 8) {
                            if (!forward(make_int4(kTileNop, 0, 0, 0))) {
                                ok = false;
                                break;
                            }
                            tk = now;
                        }
                    }
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
            }
            if (!ok) td.x = kTileStop;
            // forward the entry to the MMA issuer and the epilogue
            if (!forward(td)) break;
            if (td.x == kTileStop) break;
            if (td.x < 0) continue;
            if (!produce_tile(maps, a, pp, r.desc[td.x].P, td, it, loaded)) break;
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------- MMA issuer
        int it = 0, gu = 0;
        for (unsigned long long i = 0;; ++i) {
            const int f = (int)(i & 3);
            if (!bar_wait(su32(&qfull[f]), (uint32_t)(i >> 2) & 1, pp.abort_flag, a.err, 128u)) break;
            const int4 td = tq[f];
            bar_arrive(su32(&qempty[f]));
            if (td.x == kTileStop) break;
            if (td.x < 0) continue;
            if (!mma_tile(a, pp, r.desc[td.x].P, td, it, gu, units_mma)) break;
        }
    } else if (warp >= 2) {
        // ---------------------------------------------------- epilogue
        float Sh[64], Sl[64];
        int gu = 0;
        for (unsigned long long i = 0;; ++i) {
            const int f = (int)(i & 3);
            if (!bar_wait(su32(&qfull[f]), (uint32_t)(i >> 2) & 1, pp.abort_flag, a.err, 256u)) break;
            const int4 td = tq[f];
            __syncwarp();
            if (lane == 0) bar_arrive(su32(&qempty[f]));
            if (td.x == kTileStop) break;
            if (td.x < 0) continue;
            const ResTileDesc &D = r.desc[td.x];
            if (!epilogue_tile(a, pp, D.P, td, gu, Sh, Sl)) break;
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                const unsigned old = atomicAdd(&r.ctr[D.done_ctr], 1u);
                if (old + 1u == D.done_target) {
                    __threadfence_system();
                    st_release_sys32(&r.ctl->done[D.slot], D.gen);
                }
            }
        }
    }
    pipe_teardown(pp, loaded, units_mma);
    if (threadIdx.x == 0 && *pp.abort_flag) r.ctl->fault = 1u;  // a wait ran out: the host stops serving
}

size_t smem_bytes() { return 1024 + (size_t)kStages * kStageBytes + 256; }

// ------------------------------------------------------------ scheme tables
// Pair scheme: products (p, q), p + q <= L, paired by p over consecutive q,
// smallest contributions first (the single-problem kernel's order).  Level
// schemes: unit = levels (s, s + 1), s = 2, 4, ..., terms A_p x [B_{s-p} |
// B_{s+1-p}] for p = 1 .. s (halves past level L or with q < 1 not fed),
// smallest levels first.  Slices 0-based in the table.
SchemeTab make_tab(int scheme, int k) {
    const eq::Shape e = eq::shape(scheme, k);
    SchemeTab T{};
    std::vector<std::vector<std::array<int, 3>>> units;
    std::vector<std::array<int, 2>> lv;  // 1-based levels of each unit's halves (0: none)
    if (scheme == eq::kSchemePairs) {
        struct U {
            int p, q1, q2;
        };
        std::vector<U> u;
        for (int p = 1; p <= e.slices; ++p)
            for (int q = 1; q <= e.levels - p; q += 2) u.push_back({p, q, q + 1 <= e.levels - p ? q + 1 : 0});
        std::stable_sort(u.begin(), u.end(), [](const U &x, const U &y) { return x.p + x.q1 > y.p + y.q1; });
        for (const U &x : u) {
            units.push_back({{x.p - 1, x.q1 - 1, x.q2 ? x.q2 - 1 : (int)kNone}});
            lv.push_back({x.p + x.q1, x.q2 ? x.p + x.q2 : 0});
        }
    } else {
        std::vector<std::vector<std::array<int, 3>>> us;
        for (int s = 2; s <= e.levels; s += 2) {
            std::vector<std::array<int, 3>> terms;
            const bool right = s + 1 <= e.levels;
            for (int p = 1; p <= s; ++p) {
                const int qL = s - p, qR = s + 1 - p;
                const bool fl = qL >= 1, fr = right && qR >= 1;
                if (!fl && !fr) continue;
                terms.push_back({p - 1, fl ? qL - 1 : (int)kNone, fr ? qR - 1 : (int)kNone});
            }
            units.insert(units.begin(), terms);  // smallest levels first
            lv.insert(lv.begin(), {s, right ? s + 1 : 0});
        }
    }
    OO_REQUIRE((int)units.size() <= kMaxUnits, OO_EINVAL, "too many accumulator units");
    T.nunits = (int)units.size();
    int nt = 0;
    for (size_t u = 0; u < units.size(); ++u) {
        // the first term of a unit must feed every half the unit uses (it
        // starts the accumulation)
        const auto &t0 = units[u][0];
        OO_REQUIRE(t0[1] != (int)kNone && (lv[u][1] == 0 || t0[2] != (int)kNone), OO_EINVAL, "bad unit order");
        T.ut0[u] = (unsigned char)nt;
        T.unt[u] = (unsigned char)units[u].size();
        for (const auto &x : units[u]) {
            OO_REQUIRE(nt < kMaxTerms, OO_EINVAL, "too many accumulator terms");
            T.tp[nt] = (unsigned char)x[0];
            T.tqL[nt] = (unsigned char)x[1];
            T.tqR[nt] = (unsigned char)x[2];
            ++nt;
        }
        T.usL[u] = std::ldexp(1.0f, -e.beta * lv[u][0]);
        T.usR[u] = lv[u][1] ? std::ldexp(1.0f, -e.beta * lv[u][1]) : 0.0f;
    }
    T.nterms = nt;
    return T;
}

int table_of(int scheme, int k) {
    if (scheme == eq::kSchemePairs) return eq::shape(scheme, k).beta == 8 ? 0 : 1;
    return scheme == eq::kSchemeLevel7 ? 2 : 3;
}
int scheme_of_table(int t) { return t <= 1 ? eq::kSchemePairs : (t == 2 ? eq::kSchemeLevel7 : eq::kSchemeLevel6); }

// 2D BF16 tensor map over rows x pitch (row-major, pitch a multiple of 64),
// box 64 K-elements x box_rows rows, 128-byte swizzle
void map_slices(CUtensorMap *m, const void *base, long long rows, long long pitch, int box_rows) {
    OO_REQUIRE(((uintptr_t)base & 15u) == 0, OO_EINVAL, "split operand must be 16-byte aligned");
    OO_REQUIRE(pitch % 64 == 0 && rows >= 1 && rows < (1ll << 31), OO_EINVAL, "bad split-operand shape");
    const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = encode_tiled()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims,
                                      strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    OO_REQUIRE(r == CUDA_SUCCESS, OO_ECUDA, "cuTensorMapEncodeTiled (grouped GEMM) failed: " + std::to_string((int)r));
}

GArgs make_args(unsigned *err) {
    GArgs a{};
    a.err = err;
    for (int t = 0; t < kTables; ++t) a.sch[t] = make_tab(scheme_of_table(t), t == 0 ? 256 : 4096);
    return a;
}

int pitch_class(int kp) {
    int c = 0;
    while (c < kClasses - 1 && kp > (64 << c)) ++c;
    return c;
}

int bucket_n(int n) {
    int b = 0;
    while (b < OO_TILE_NBUCKETS - 1 && n > (32 << b)) ++b;
    return b;
}
int bucket_k(int k) {
    int b = 0;
    while (b < OO_TILE_KBUCKETS - 1 && k > (64 << b)) ++b;
    return b;
}

// relative cost of a tile, for ordering the work list (largest first)
double tile_cost(const eq::Shape &e, int ksteps, int width) {
    return (double)width * ((double)ksteps * e.nprod + 8.0 * e.nkb * (e.scheme == eq::kSchemePairs
                                                                        ? (e.nprod + e.slices) / 2.0
                                                                        : (e.levels + 1) / 2.0));
}

}  // namespace

// The accumulation scheme of an FP64-equivalent product with inner
// dimension k: a fixed rule, so a problem gives the same bits alone and in a
// batch.  Measured on GB300 (grouped products of the batched workload):
// levels with 7-bit digits up to one 128-deep K-block, levels with 6-bit
// digits up to 512, the pair scheme beyond (long K: tensor-bound, fewer
// products win).
int eq_scheme_for(int k) {
    if (k <= 128) return eq::kSchemeLevel7;
    if (k <= 512) return eq::kSchemeLevel6;
    return eq::kSchemePairs;
}

// The built-in tile widths: the autotuner's choices on GB300, written by
// paper_2011_03602_gb300/tune_gemm_tiles.py (rows n <= 32 .. > 512, columns
// k <= 64 .. > 512).
int eq_default_width(int nb, int kb) {
    static const int table[OO_TILE_NBUCKETS][OO_TILE_KBUCKETS] = {
#include "eq_tile_table.inc"
    };
    if (nb < 0 || nb >= OO_TILE_NBUCKETS || kb < 0 || kb >= OO_TILE_KBUCKETS) return 128;
    return table[nb][kb];
}

int eq_tile_width(const int *widths, int n, int k) {
    const int w = widths ? widths[bucket_n(n) * OO_TILE_KBUCKETS + bucket_k(k)] : 0;
    return (w == 32 || w == 64 || w == 128) ? w : eq_default_width(bucket_n(n), bucket_k(k));
}

struct EqGroup {
    void *arena = nullptr;
    GMaps maps{};
    GArgs args{};
    GProb *d_probs = nullptr;
    int4 *d_tiles = nullptr;
    eq::GSplit *d_split = nullptr;
    int4 *d_jobs = nullptr;
    unsigned *d_err = nullptr;
    int ntiles = 0, njobs = 0, nrow_jobs = 0, grid = 1;
    double flops = 0;
};

EqGroup *eq_group_create(const std::vector<GemmDesc> &v, int num_sms, const int *widths) {
    OO_REQUIRE(!v.empty(), OO_EINVAL, "empty FP64-equivalent group");
    auto up = [](size_t x, size_t a) { return (x + a - 1) / a * a; };
    const size_t np = v.size();
    std::vector<eq::Shape> sh(np);
    std::vector<int> kp(np), cls(np), ra(np), rb(np), tab(np);
    long long rows_a[kClasses] = {0}, rows_b[kClasses] = {0};
    int KP[kClasses];
    for (int c = 0; c < kClasses; ++c) KP[c] = 64 << c;
    for (size_t i = 0; i < np; ++i) {
        const GemmDesc &d = v[i];
        OO_REQUIRE(d.m >= 1 && d.n >= 1 && d.k >= 1 && d.lda >= d.k && d.ldb >= d.n && d.ldc >= d.n, OO_EINVAL,
                   "bad GEMM in FP64-equivalent group");
        sh[i] = eq::shape(eq_scheme_for(d.k), d.k);
        tab[i] = table_of(sh[i].scheme, d.k);
        kp[i] = (d.k + kBK - 1) / kBK * kBK;
        cls[i] = pitch_class(kp[i]);
        if (cls[i] == kClasses - 1) KP[cls[i]] = std::max(KP[cls[i]], kp[i]);
        ra[i] = (int)rows_a[cls[i]];
        rb[i] = (int)rows_b[cls[i]];
        rows_a[cls[i]] += (long long)sh[i].slices * d.m;
        rows_b[cls[i]] += (long long)sh[i].slices * d.n;
        OO_REQUIRE(rows_a[cls[i]] < (1ll << 31) - kBM && rows_b[cls[i]] < (1ll << 31) - kBM, OO_EINVAL,
                   "FP64-equivalent group too large");
    }
    size_t at = 0;
    size_t off_a[kClasses], off_b[kClasses];
    for (int c = 0; c < kClasses; ++c) {
        off_a[c] = at;
        at += up((size_t)rows_a[c] * KP[c] * 2, 1024);
        off_b[c] = at;
        at += up((size_t)rows_b[c] * KP[c] * 2, 1024);
    }
    std::vector<size_t> off_ea(np), off_eb(np);
    for (size_t i = 0; i < np; ++i) {
        off_ea[i] = at;
        at += up((size_t)v[i].m * 4, 16);
        off_eb[i] = at;
        at += up((size_t)v[i].n * 4, 16);
    }
    at = up(at, 256);
    std::vector<int4> tiles, jobs, col_jobs;  // row jobs first, then column jobs
    std::vector<double> cost;
    double flops = 0;
    for (size_t i = 0; i < np; ++i) {
        const GemmDesc &d = v[i];
        flops += 2.0 * d.m * d.n * d.k;
        const int W = eq_tile_width(widths, d.n, d.k);
        for (int m0 = 0; m0 < d.m; m0 += kBM)
            for (int n0 = 0; n0 < d.n; n0 += W) {
                const int w = d.n - n0 >= W ? W : narrowest_width(d.n - n0);
                tiles.push_back(make_int4((int)i, m0, n0, w));
                cost.push_back(tile_cost(sh[i], kp[i] / kBK, w));
            }
        for (int r0 = 0; r0 < d.m; r0 += 8) jobs.push_back(make_int4(0, (int)i, r0, 0));
        for (int c0 = 0; c0 < d.n; c0 += 64) col_jobs.push_back(make_int4(1, (int)i, c0, 0));
    }
    const int nrow_jobs = (int)jobs.size();
    jobs.insert(jobs.end(), col_jobs.begin(), col_jobs.end());
    OO_REQUIRE(tiles.size() < (1u << 31) && jobs.size() < (1u << 31), OO_EINVAL, "too many tiles");
    std::vector<size_t> order(tiles.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<int4> sorted(tiles.size());
    for (size_t t = 0; t < order.size(); ++t) sorted[t] = tiles[order[t]];
    const size_t off_probs = at;
    at += up(np * sizeof(GProb), 256);
    const size_t off_split = at;
    at += up(np * sizeof(eq::GSplit), 256);
    const size_t off_tiles = at;
    at += up(sorted.size() * sizeof(int4), 256);
    const size_t off_jobs = at;
    at += up(jobs.size() * sizeof(int4), 256);
    const size_t off_err = at;
    at += 256;
    auto *g = new EqGroup();
    try {
        if (cudaMalloc(&g->arena, at) != cudaSuccess) {
            cudaGetLastError();
            g->arena = nullptr;
            throw Error{OO_ENOMEM, "FP64-equivalent group arena of " + std::to_string(at) + " bytes"};
        }
        char *base = static_cast<char *>(g->arena);
        for (int c = 0; c < kClasses; ++c) {
            if (rows_a[c] == 0) continue;
            map_slices(&g->maps.a[c], base + off_a[c], rows_a[c], KP[c], kBM);
            map_slices(&g->maps.b[c], base + off_b[c], rows_b[c], KP[c], kBRows);
        }
        std::vector<GProb> probs(np);
        std::vector<eq::GSplit> splits(np);
        for (size_t i = 0; i < np; ++i) {
            const GemmDesc &d = v[i];
            const eq::Shape &e = sh[i];
            int *ea = reinterpret_cast<int *>(base + off_ea[i]);
            int *eb = reinterpret_cast<int *>(base + off_eb[i]);
            GProb &P = probs[i];
            P.C = d.C;
            P.ea = ea;
            P.eb = eb;
            P.ldc = d.ldc;
            P.m = d.m;
            P.n = d.n;
            P.ksteps = kp[i] / kBK;
            P.kb_steps = e.kb / kBK;
            P.nkb = e.nkb;
            P.ra = ra[i];
            P.rb = rb[i];
            P.cls = cls[i];
            P.scheme = tab[i];
            auto *As = reinterpret_cast<__nv_bfloat16 *>(base + off_a[cls[i]]) + (size_t)ra[i] * KP[cls[i]];
            auto *Bs = reinterpret_cast<__nv_bfloat16 *>(base + off_b[cls[i]]) + (size_t)rb[i] * KP[cls[i]];
            splits[i] = eq::GSplit{d.A, d.B, d.lda, d.ldb, (long long)KP[cls[i]], d.m, d.n, d.k, kp[i], e.beta,
                               e.slices, As, Bs, ea, eb};
        }
        OO_CUDA_TRY(cudaMemcpy(base + off_probs, probs.data(), np * sizeof(GProb), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_split, splits.data(), np * sizeof(eq::GSplit), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_tiles, sorted.data(), sorted.size() * sizeof(int4), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_jobs, jobs.data(), jobs.size() * sizeof(int4), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemset(base + off_err, 0, 256));
        g->d_probs = reinterpret_cast<GProb *>(base + off_probs);
        g->d_split = reinterpret_cast<eq::GSplit *>(base + off_split);
        g->d_tiles = reinterpret_cast<int4 *>(base + off_tiles);
        g->d_jobs = reinterpret_cast<int4 *>(base + off_jobs);
        g->d_err = reinterpret_cast<unsigned *>(base + off_err);
        g->args = make_args(g->d_err);
        g->ntiles = (int)sorted.size();
        g->njobs = (int)jobs.size();
        g->nrow_jobs = nrow_jobs;
        g->grid = std::max(1, std::min(g->ntiles, num_sms));
        g->flops = flops;
    } catch (...) {
        if (g->arena) cudaFree(g->arena);
        delete g;
        throw;
    }
    return g;
}

void eq_group_launch(EqGroup *g, cudaStream_t s) {
    launch_eq_group_split(g->d_split, g->d_jobs, g->nrow_jobs, g->njobs - g->nrow_jobs, s);
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)gemm_eq_group_kernel, smem_bytes(), attr);
    gemm_eq_group_kernel<<<g->grid, kThreads, smem_bytes(), s>>>(g->maps, g->args, g->d_probs, g->d_tiles,
                                                                 g->ntiles);
    OO_CUDA_TRY(cudaGetLastError());
}

unsigned eq_group_check(EqGroup *g, cudaStream_t s) {
    unsigned e = 0;
    OO_CUDA_TRY(cudaMemcpyAsync(&e, g->d_err, 4, cudaMemcpyDeviceToHost, s));
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    if (e) OO_CUDA_TRY(cudaMemsetAsync(g->d_err, 0, 4, s));
    return e;
}

double eq_group_flops(const EqGroup *g) { return g->flops; }
int eq_group_tiles(const EqGroup *g) { return g->ntiles; }

void eq_group_destroy(EqGroup *g) {
    if (!g) return;
    if (g->arena) cudaFree(g->arena);
    delete g;
}

// One product in a level scheme, its operands already split into As (slice
// p at rows [p m, (p + 1) m), row pitch kp) and Bs (transposed, slice q at
// rows [q n, (q + 1) n)); tiles of `width` columns in grouped raster order.
void launch_gemm_eq_tiles(int m, int n, int k, const void *As, const void *Bs, const int *ea, const int *eb,
                          double *C, long long ldc, int width, unsigned *err, int num_sms, cudaStream_t s) {
    const eq::Shape e = eq::shape(eq_scheme_for(k), k);
    const int kp = (k + kBK - 1) / kBK * kBK;
    GMaps maps{};
    map_slices(&maps.a[0], As, (long long)e.slices * m, kp, kBM);
    map_slices(&maps.b[0], Bs, (long long)e.slices * n, kp, kBRows);
    GProb P{};
    P.C = C;
    P.ea = ea;
    P.eb = eb;
    P.ldc = ldc;
    P.m = m;
    P.n = n;
    P.ksteps = kp / kBK;
    P.kb_steps = e.kb / kBK;
    P.nkb = e.nkb;
    P.ra = 0;
    P.rb = 0;
    P.cls = 0;
    P.scheme = table_of(e.scheme, k);
    P.bn = (width == 32 || width == 64 || width == 128) ? width : 128;
    P.m_tiles = (m + kBM - 1) / kBM;
    P.n_tiles = (n + P.bn - 1) / P.bn;
    const long long tiles = (long long)P.m_tiles * P.n_tiles;
    OO_REQUIRE(tiles < (1ll << 31), OO_EINVAL, "too many tiles");
    const GArgs a = make_args(err);
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)gemm_eq_single_kernel, smem_bytes(), attr);
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, num_sms));
    gemm_eq_single_kernel<<<grid, kThreads, smem_bytes(), s>>>(maps, a, P);
    OO_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------- the autotuner
// For every (n, k) bucket: a fixed synthetic group of products drawn in the
// bucket (m log-uniform in [16, 512], n and k uniform in the bucket's range;
// zero inputs, the work does not depend on the values), timed with every
// tile width; the fastest width is kept in the context's table.
void tune_gemm_tiles(Ctx &c, double *ms_out) {
    static const int nlo[OO_TILE_NBUCKETS] = {16, 33, 65, 129, 257, 513};
    static const int nhi[OO_TILE_NBUCKETS] = {32, 64, 128, 256, 512, 1024};
    static const int klo[OO_TILE_KBUCKETS] = {16, 65, 129, 257, 513};
    static const int khi[OO_TILE_KBUCKETS] = {64, 128, 256, 512, 1024};
    static const int widths[3] = {32, 64, 128};
    constexpr int kProblems = 96, kReps = 3;
    cudaStream_t s = c.stream;
    uint64_t state = 0x2011036020113602ull;
    auto next = [&]() {  // splitmix64
        uint64_t z = (state += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    };
    auto uni = [&](int lo, int hi) { return lo + (int)(next() % (uint64_t)(hi - lo + 1)); };
    auto logu = [&](int lo, int hi) {
        const double u = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
        return std::min(hi, (int)std::floor(std::exp(std::log((double)lo) + u * (std::log(hi + 1.0) - std::log((double)lo)))));
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    OO_CUDA_TRY(cudaEventCreate(&e0));
    OO_CUDA_TRY(cudaEventCreate(&e1));
    void *buf = nullptr;
    EqGroup *g = nullptr;
    try {
        for (int nb = 0; nb < OO_TILE_NBUCKETS; ++nb)
            for (int kb = 0; kb < OO_TILE_KBUCKETS; ++kb) {
                std::vector<std::array<int, 3>> dims(kProblems);
                size_t elems = 0;
                for (auto &d : dims) {
                    d = {logu(16, 512), uni(nlo[nb], nhi[nb]), uni(klo[kb], khi[kb])};
                    elems += (size_t)d[0] * d[2] + (size_t)d[2] * d[1] + (size_t)d[0] * d[1] + 2;
                }
                OO_CUDA_TRY(cudaMalloc(&buf, elems * 8));
                OO_CUDA_TRY(cudaMemsetAsync(buf, 0, elems * 8, s));
                std::vector<GemmDesc> v;
                double *p = static_cast<double *>(buf);
                for (const auto &d : dims) {
                    const int m = d[0], n = d[1], k = d[2];
                    const double *A = p;
                    p += (size_t)m * k + 1;
                    const double *B = p;
                    p += (size_t)k * n + 1;
                    v.push_back(GemmDesc{m, n, k, A, k, B, n, p, n});
                    p += (size_t)m * n;
                }
                float best = 0.f;
                int best_w = 128;
                for (int wi = 0; wi < 3; ++wi) {
                    std::array<int, OO_TILE_NBUCKETS * OO_TILE_KBUCKETS> tab;
                    tab.fill(widths[wi]);
                    g = eq_group_create(v, c.num_sms, tab.data());
                    eq_group_launch(g, s);  // warm-up
                    OO_REQUIRE(eq_group_check(g, s) == 0, OO_ETIMEOUT, "pipeline wait ran out while tuning");
                    OO_CUDA_TRY(cudaEventRecord(e0, s));
                    for (int r = 0; r < kReps; ++r) eq_group_launch(g, s);
                    OO_CUDA_TRY(cudaEventRecord(e1, s));
                    OO_CUDA_TRY(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    OO_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                    ms /= kReps;
                    OO_REQUIRE(eq_group_check(g, s) == 0, OO_ETIMEOUT, "pipeline wait ran out while tuning");
                    eq_group_destroy(g);
                    g = nullptr;
                    if (ms_out) ms_out[(nb * OO_TILE_KBUCKETS + kb) * 3 + wi] = ms;
                    if (wi == 0 || ms < best) {
                        best = ms;
                        best_w = widths[wi];
                    }
                }
                OO_CUDA_TRY(cudaStreamSynchronize(s));
                OO_CUDA_TRY(cudaFree(buf));
                buf = nullptr;
                c.eq_widths[nb * OO_TILE_KBUCKETS + kb] = best_w;
            }
    } catch (...) {
        cudaStreamSynchronize(s);
        eq_group_destroy(g);
        if (buf) cudaFree(buf);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

// ------------------------------------------ resident loop: host-side parts
size_t res_tile_desc_bytes() { return sizeof(ResTileDesc); }

// The tile descriptor of one resident GEMM request: C (m x n, ldc), scale
// exponents ea / eb, digit slices at rows ra (A) and rb (B) of the slice
// region (row pitch res::kSlicePitch); its split entry's counter and target;
// its own completion counter, whose target is base + 8 x tiles.
void res_tile_desc_fill(void *dst, double *C, long long ldc, const int *ea, const int *eb, int m, int n, int k,
                        int ra, int rb, unsigned split_ctr, unsigned split_target, unsigned done_ctr,
                        unsigned done_target, unsigned gen, int slot) {
    const eq::Shape e = eq::shape(eq_scheme_for(k), k);
    const int kp = (k + kBK - 1) / kBK * kBK;
    OO_REQUIRE(kp <= res::kSlicePitch, OO_EINVAL, "inner dimension above the resident slice pitch");
    ResTileDesc D{};
    D.P.C = C;
    D.P.ea = ea;
    D.P.eb = eb;
    D.P.ldc = ldc;
    D.P.m = m;
    D.P.n = n;
    D.P.ksteps = kp / kBK;
    D.P.kb_steps = e.kb / kBK;
    D.P.nkb = e.nkb;
    D.P.ra = ra;
    D.P.rb = rb;
    D.P.cls = 0;
    D.P.scheme = table_of(e.scheme, k);
    D.split_ctr = split_ctr;
    D.split_target = split_target;
    D.done_ctr = done_ctr;
    D.done_target = done_target;
    D.gen = gen;
    D.slot = slot;
    std::memcpy(dst, &D, sizeof(D));
}

// The tile entries of one product (row blocks of 128, column tiles of the
// table's width for n and k, the last one the narrowest that covers it).
int res_tile_list(int m, int n, int k, const int *widths, int slot, std::vector<int4> &out) {
    const int W = eq_tile_width(widths, n, k);
    int count = 0;
    for (int m0 = 0; m0 < m; m0 += kBM)
        for (int n0 = 0; n0 < n; n0 += W) {
            out.push_back(make_int4(slot, m0, n0, n - n0 >= W ? W : narrowest_width(n - n0)));
            ++count;
        }
    return count;
}

void res_tile_marker(std::vector<int4> &out, bool stop) {
    out.push_back(make_int4(stop ? kTileStop : kTileNop, 0, 0, 0));
}

// Launch the resident tensor-core worker (ctas CTAs, one per SM) over the
// slice region (rows x res::kSlicePitch BF16, 16-byte aligned).
// Loads the tile worker and sets its shared-memory limit.  With lazy module
// loading a kernel is loaded at its first use, and loading can wait for the
// kernels already running on the device: the SIMT worker, which waits (with
// its bound) for entries that only come once the tile worker runs.  So both
// workers are loaded before either is launched.
void prepare_resident_tiles() {
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)resident_tiles_kernel, smem_bytes(), attr);
    cudaFuncAttributes fa{};
    OO_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void *)resident_tiles_kernel));
}

void launch_resident_tiles(const int4 *ring, const void *desc, unsigned *ctr, res::Ctl *ctl_dev,
                           unsigned long long start, const void *slices, long long slice_rows, unsigned *err,
                           int ctas, cudaStream_t s) {
    GMaps maps{};
    map_slices(&maps.a[0], slices, slice_rows, res::kSlicePitch, kBM);
    map_slices(&maps.b[0], slices, slice_rows, res::kSlicePitch, kBRows);
    const GArgs a = make_args(err);
    ResTileArgs r{};
    r.ring = ring;
    r.desc = static_cast<const ResTileDesc *>(desc);
    r.ctr = ctr;
    r.heartbeat = ctr + res::kRingCap + res::kSlots;
    r.ctl = ctl_dev;
    r.start = start;
    resident_tiles_kernel<<<ctas, kThreads, smem_bytes(), s>>>(maps, a, r);
    OO_CUDA_TRY(cudaGetLastError());
}

}  // namespace oo
