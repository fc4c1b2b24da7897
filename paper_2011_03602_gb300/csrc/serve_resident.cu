// Device-resident serving loop (oo_serve_start_resident): the same mixed
// GEMM / FFT / Jacobi service as the host-scheduled one (serve.cpp), with
// the request loop on the device.  Two persistent worker kernels are
// launched when serving starts and walk append-only rings of work entries
// (layout and protocol: resident.h):
//   - resident_simt_kernel (here, 512-thread CTAs): FP64-equivalent digit
//     splits, FFT passes (the grouped FFT's work items), Jacobi setup and
//     stencil sweeps (the per-point float-float arithmetic of the
//     cooperative Jacobi kernel, one chunk per CTA; p and wrk2 alternate
//     roles, which makes the copy-back nests' result without a copy);
//   - resident_tiles_kernel (gemm_eq_group.cu): the tensor-core tiles of the
//     FP64-equivalent products.
// The host scheduler thread admits the oldest waiting requests whose device
// footprint fits the free part of the device arena (and of the digit-slice
// region), uploads their inputs, descriptors and entries with copies,
// publishes the entries through the mapped control block once the copies
// have landed, watches the done flags the workers write, and copies the
// outputs back.  No kernel is launched per request.  Requests of different
// kinds and sizes overlap on the device: their entries interleave in the
// rings and every SM works on whatever is published.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unistd.h>
#include <vector>

#include "eq_digits.cuh"
#include "fft_device.cuh"
#include "jacobi_point.cuh"
#include "oo_internal.h"
#include "resident.h"

namespace oo {

// gemm_eq_group.cu
size_t res_tile_desc_bytes();
void res_tile_desc_fill(void *dst, double *C, long long ldc, const int *ea, const int *eb, int m, int n, int k,
                        int ra, int rb, unsigned split_ctr, unsigned split_target, unsigned done_ctr,
                        unsigned done_target, unsigned gen, int slot);
int res_tile_list(int m, int n, int k, const int *widths, int slot, std::vector<int4> &out);
void res_tile_marker(std::vector<int4> &out, bool stop);
void prepare_resident_tiles();
void launch_resident_tiles(const int4 *ring, const void *desc, unsigned *ctr, res::Ctl *ctl_dev,
                           unsigned long long start, const void *slices, long long slice_rows, unsigned *err,
                           int ctas, cudaStream_t s);

namespace {

using namespace res;

constexpr long long kResWait = 2000000000ll;  // clock64 ticks (~1 s)

// ----------------------------------------------------------- device side
__device__ __forceinline__ unsigned long long res_ld_acquire_sys64(const volatile unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned res_ld_acquire_gpu32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void res_st_release_sys32(volatile unsigned *p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct SimtArgs {
    const Entry *ring;
    unsigned *ctr;
    Ctl *ctl;
    unsigned *err;
    const eq::GSplit *split;  // kSlots
    const FftGroupReq *fft;   // kSlots
    int *expo;                // kSlots
    const int *tlist;         // kSlots: tlist[i] = i
    const JacDesc *jac;       // kSlots
    unsigned long long start;
};

// block-wide sum of v in a fixed order (warps by shuffle, then warp sums in
// warp order); the total is valid in thread 0
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// one item of an entry, by every thread of the CTA
__device__ __forceinline__ void run_item(const SimtArgs &a, const Entry &E, int i, float4 *sm, double *red,
                                         int *redi) {
    const int tid = threadIdx.x;
    if (E.type == kSplit) {
        // descriptors copied to registers: a reference into global memory
        // would be re-read after every store (the stores may alias it)
        const eq::GSplit G = a.split[E.slot];
        if (i < E.aux) {
            eq::split_rows_job(G, i * (kSimtThreads / 32));
        } else {
            double(*t)[65] = reinterpret_cast<double(*)[65]>(sm);
            int(*ri)[64] = reinterpret_cast<int(*)[64]>(reinterpret_cast<double *>(sm) + 64 * 65);
            eq::split_cols_job(G, (i - E.aux) * 64, t, ri);
        }
    } else if (E.type == kFftWhole || E.type == kFftCols || E.type == kFftRows) {
        const FftGroupReq &R = a.fft[E.slot];
        FftItem it{};
        it.first = E.slot;
        if (E.type == kFftWhole) {
            it.mode = 0;
            it.log2L = R.log2n;
            it.count = 1;
        } else if (E.type == kFftCols) {
            it.mode = 1;
            it.log2L = R.log2n1;
            it.c0 = i * (kFftElems >> R.log2n1);
        } else {
            it.mode = 2;
            it.log2L = R.log2n2;
            it.c0 = i * (kFftElems >> R.log2n2);
        }
        fft_group_item(it, a.fft, a.tlist, a.expo, sm, true);  // loads here bypass L1
    } else {
        const JacDesc J = a.jac[E.slot];
        const size_t sj = (size_t)J.pitch, si = (size_t)J.J * J.pitch;
        if (E.type == kJacSetup) {
            // N0 coefficients (constants) and N1 p = wrk2 = (k / (K - 1))^2,
            // the padding of each row zero, as the setup kernels write them
            const float val[NCOEF] = {1.0f, 1.0f, 1.0f, 1.0f / 6.0f, 0.0f, 0.0f, 0.0f, 1.0f, 1.0f, 1.0f, 1.0f, 0.0f};
            const int n4 = J.I * J.J * (J.pitch / 4), chunks = J.pitch / 4;
            const int x0 = i * J.chunk4, x1 = min(n4, x0 + J.chunk4);
            for (int x = x0 + tid; x < x1; x += kSimtThreads) {
#pragma unroll
                for (int q = 0; q < NCOEF; ++q)
                    reinterpret_cast<float4 *>(J.arr[q])[x] = make_float4(val[q], val[q], val[q], val[q]);
                const int k = (x % chunks) * 4;
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = (k + e < J.K) ? jacobi_face_value(k + e, J.K) : 0.0f;
                const float4 g4 = make_float4(v[0], v[1], v[2], v[3]);
                reinterpret_cast<float4 *>(J.arr[VAR_P])[x] = g4;
                reinterpret_cast<float4 *>(J.arr[VAR_WRK2])[x] = g4;
            }
        } else {  // kJacStencil
            // N2 of iteration E.aux.  p and wrk2 alternate roles (even
            // iterations read p and write wrk2, odd ones the reverse): both
            // hold the Dirichlet faces from the setup and the stencil writes
            // only the interior, so the array written is exactly p after the
            // copy-back nests N3-N5, and no copy is made.
            // Work unit: one (j, k) column over one of nseg slabs of planes;
            // a thread marches its column along i with the 3 x 3 windows of
            // planes i - 1, i, i + 1 in registers, reading one new window
            // (9 values) per point, the next one ahead of the arithmetic.
            const int Ji = J.J - 2, Ki = J.K - 2, ncols = Ji * Ki, np = J.I - 2;
            const int units = ncols * J.nseg;
            const int u0 = i * J.chunk, u1 = min(units, u0 + J.chunk);
            const bool odd = (E.aux & 1) != 0;  // selects, not an index: J stays in registers
            const float *pin = odd ? J.arr[VAR_WRK2] : J.arr[VAR_P];
            float *pout = odd ? J.arr[VAR_P] : J.arr[VAR_WRK2];
            float RH = 0.0f, RL = 0.0f;
            for (int u = u0 + tid; u < u1; u += kSimtThreads) {
                const int sg = u / ncols, col = u - sg * ncols;
                const int jr = col / Ki;
                const int j = 1 + jr, k = 1 + col - jr * Ki;
                const int ib = 1 + (int)((long long)np * sg / J.nseg);
                const int ie = 1 + (int)((long long)np * (sg + 1) / J.nseg);
                size_t c = (size_t)ib * si + (size_t)j * sj + k;
                PWin W, C, Ep;
                load_pwin(pin, c - si, sj, false, W);
                load_pwin(pin, c, sj, true, C);
                load_pwin(pin, c + si, sj, true, Ep);
                float cf[NCOEF];
#pragma unroll
                for (int q = 0; q < NCOEF; ++q) cf[q] = J.arr[q][c];
                for (int ii = ib; ii < ie; ++ii, c += si) {
                    // the next point's coefficients and window ahead of this one's arithmetic
                    const bool more = ii + 1 < ie;
                    float cn[NCOEF];
                    PWin Nx;
                    if (more) {
#pragma unroll
                        for (int q = 0; q < NCOEF; ++q) cn[q] = J.arr[q][c + si];
                        load_pwin(pin, c + 2 * si, sj, true, Nx);
                    }
                    pout[c] = stencil_point_core(cf, W, C, Ep, J.omega, RH, RL);
                    if (more) {
                        W = C;
                        C = Ep;
                        Ep = Nx;
#pragma unroll
                        for (int q = 0; q < NCOEF; ++q) cf[q] = cn[q];
                    }
                }
            }
            const double s = block_sum((double)RH + (double)RL, red);
            // two partial sets, by iteration parity: the next iteration's
            // items may start (its dependency is this entry's count) before
            // the CTA that completes this entry has summed this set; the one
            // after cannot start before that CTA has moved on
            if (tid == 0) J.partials[(E.aux & 1) * E.nitems + i] = s;
        }
    }
}

// Completion of an entry, by the first warp of the CTA whose item completed
// it (the other CTAs may already be on the next entry, so this is kept
// short): the Jacobi residual of the iteration -- the items' partials, each
// lane summing a fixed stride of them, then a fixed butterfly -- and the
// request's done flag.
__device__ __forceinline__ void finish_entry(const SimtArgs &a, const Entry &E) {
    const int lane = threadIdx.x & 31;
    if (E.type == kJacStencil) {
        const JacDesc &J = a.jac[E.slot];
        const double *part = J.partials + (E.aux & 1) * E.nitems;
        double s = 0.0;
        for (int q = lane; q < E.nitems; q += 32) s += __ldcg(&part[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) J.res[E.aux] = s;
    }
    if (lane == 0 && E.last) {
        __threadfence_system();
        res_st_release_sys32(&a.ctl->done[E.slot], E.gen);
    }
}

__global__ void __launch_bounds__(kSimtThreads, 1) resident_simt_kernel(const SimtArgs a) {
    extern __shared__ __align__(16) float4 rsm[];
    __shared__ __align__(16) Entry E;  // copied in as 16-byte words
    __shared__ int go, fin;
    __shared__ double red[kSimtThreads / 32];
    __shared__ int redi[kSimtThreads / 32];
    const int G = gridDim.x, me = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) a.ctl->alive[me] = 1u;
    unsigned long long seen = 0;
    for (unsigned long long e = a.start;; ++e) {
        if (tid == 0) {
            go = 1;
            if (seen <= e) {
                const long long t0 = clock64();
                while ((seen = res_ld_acquire_sys64(&a.ctl->pub_simt)) <= e) {
                    if (clock64() - t0 > kResWait) {
                        atomicOr(a.err, 32u);
                        a.ctl->stuck_at = e;
                        a.ctl->stuck_seen = seen;
                        a.ctl->fault = 1u;
                        go = -1;
                        break;
                    }
                }
            }
            if (go == 1) {
                const int4 *src = reinterpret_cast<const int4 *>(a.ring + e % kRingCap);
                int4 *dst = reinterpret_cast<int4 *>(&E);
#pragma unroll
                for (int w = 0; w < (int)(sizeof(Entry) / 16); ++w) dst[w] = __ldcg(src + w);
            }
        }
        __syncthreads();
        if (go < 0 || E.type == kStop) break;
        int i = (me - E.rot) % G;
        if (i < 0) i += G;
        bool waited = false;
        for (; i < E.nitems; i += G) {
            if (!waited) {
                if (tid == 0 && E.dep_ctr >= 0) {
                    const long long t0 = clock64();
                    while ((int)(res_ld_acquire_gpu32(&a.ctr[E.dep_ctr]) - E.dep_target) < 0) {
                        if (clock64() - t0 > kResWait) {
                            atomicOr(a.err, 64u);
                            a.ctl->fault = 1u;
                            go = -1;
                            break;
                        }
                    }
                }
                __syncthreads();
                if (go < 0) break;
                waited = true;
            }
            run_item(a, E, i, rsm, red, redi);
            __syncthreads();
            if (tid == 0) {
                __threadfence();  // this item's writes before its count
                const unsigned old = atomicAdd(&a.ctr[E.ctr], 1u);
                fin = old + 1u == E.target;
                if (fin) __threadfence();  // every item's writes before the completion's reads
            }
            __syncthreads();
            if (fin && tid < 32) finish_entry(a, E);
        }
        if (go < 0) break;
        if (tid == 0) {
            a.ctl->simt_progress[me] = e + 1;
            atomicAdd(a.ctr + kRingCap + kSlots, 1u);  // heartbeat: the tile worker's waits watch it
        }
        __syncthreads();  // E and go are rewritten for the next entry
    }
}

// FFT data (padded) + twiddles (up to 64 KB) + the columns' exponents
size_t simt_smem_bytes() { return (size_t)(kFftElemsPad + kFftElems) * sizeof(float4) + 16; }

// ------------------------------------------------------------- host side
using Clock = std::chrono::steady_clock;
double now_ms() { return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count(); }
size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// request states: queued; admitted, its inputs being copied in by an I/O
// thread; inputs on the device; entries being uploaded; published; its
// outputs being copied out by an I/O thread; done
enum { RS_QUEUED = 0, RS_INPUT = 1, RS_READY = 2, RS_UPLOAD = 3, RS_RUNNING = 4, RS_OUTPUT = 5, RS_DONE = 6 };

struct RReq {
    oo_serve_req r{};
    uint64_t ticket = 0;
    double t_submit = 0, t_done = 0;
    double t_admit = 0, t_ready = 0, t_pub = 0, t_dev = 0;  // stage boundaries
    int state = RS_QUEUED;
    oo_status status = OO_OK;
    std::string error;
    // pinned upload area (descriptors, entries) while the entries are staged
    size_t h_off = 0, h_bytes = 0;
    size_t d_off = 0, d_bytes = 0;     // device arena
    size_t row_off = 0, rows = 0;      // digit-slice rows (GEMM)
    int slot = -1;
    unsigned gen = 0;
    unsigned long long simt_end = 0, tile_end = 0;  // publish up to here once uploaded
    cudaEvent_t ev = nullptr;
    bool marker = false;  // keep-alive or stop entries, not a request
    int mark_slot = -1;   // its pinned upload slot
};
constexpr size_t kMarkBytes = sizeof(Entry) + (size_t)kMaxCtas * sizeof(int4);
constexpr int kIoThreads = 4;
constexpr int kMarkSlots = 64;

}  // namespace

struct Resident {
    Ctx *c = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    bool stop = false, failed = false;
    std::string fail_msg;
    std::deque<RReq *> queue, ready, uploading, running;
    // I/O threads: inputs copied from the caller's buffers to the device when
    // a request is admitted, outputs back into them when it is done, each
    // thread on its own stream (pageable copies block the thread issuing them)
    std::vector<std::thread> io;
    std::vector<cudaStream_t> io_streams;
    std::deque<RReq *> io_jobs;
    std::condition_variable cv_io;
    bool io_stop = false;
    int n_io_in = 0, n_io_out = 0;
    size_t queue_cap = 0;
    std::unordered_map<uint64_t, RReq *> reqs;
    uint64_t next_ticket = 1;
    Arena dev, host, rows;
    char *dev_base = nullptr, *host_base = nullptr;
    __nv_bfloat16 *slices = nullptr;
    long long slice_rows = 0;
    // device structures
    Entry *ring = nullptr;
    int4 *tiles = nullptr;
    unsigned *ctr = nullptr, *err = nullptr;
    eq::GSplit *split_desc = nullptr;
    char *tile_desc = nullptr;
    FftGroupReq *fft_desc = nullptr;
    int *expo = nullptr, *tlist = nullptr;
    JacDesc *jac_desc = nullptr;
    void *dev_misc = nullptr;
    Ctl *ctl = nullptr, *ctl_dev = nullptr;
    // host mirrors of the device protocol
    std::vector<unsigned> ctr_base;  // kRingCap entry counters, then kSlots GEMM completion counters
    unsigned long long simt_w = 0, tile_w = 0;  // entries written to the rings
    std::vector<int> free_slots;
    unsigned next_gen = 1;
    int simt_ctas = 0, tile_ctas = 0;
    cudaStream_t up = nullptr, down = nullptr, s_simt = nullptr, s_tiles = nullptr;
    std::vector<cudaEvent_t> event_pool;
    char *mark_pool = nullptr;  // pinned upload slots of keep-alive / stop entries
    std::vector<int> mark_free;
    double last_simt_pub = 0, last_tile_pub = 0, last_tile_round = 0;
    std::array<int, OO_TILE_NBUCKETS * OO_TILE_KBUCKETS> widths{};
    int inject_stall = 0;
    uint64_t n_submitted = 0, n_done = 0, n_busy = 0, n_failed = 0;
    double sum_ms[5] = {0, 0, 0, 0, 0};  // completed requests' stage times
    uint64_t n_timed = 0;
};

namespace {

unsigned long long min_progress(const volatile unsigned long long *p, int n) {
    unsigned long long m = ~0ull;
    for (int i = 0; i < n; ++i) {
        const unsigned long long v = p[i];
        m = v < m ? v : m;
    }
    return m;
}

cudaEvent_t take_event(Resident &S) {
    if (!S.event_pool.empty()) {
        cudaEvent_t e = S.event_pool.back();
        S.event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    OO_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return e;
}

// the device footprint of a request and the size of its upload area
struct Plan {
    size_t h_bytes;
    size_t d_bytes, rows;
    int n_simt, n_tiles;
};

// Jacobi items: one per SIMT CTA (fewer when a CTA would get under one
// unit per thread), equal chunks, so every entry is spread over the worker
void jac_split(long long units, int ctas, int &items, int &chunk) {
    items = (int)std::max<long long>(1, std::min<long long>(ctas, (units + kSimtThreads - 1) / kSimtThreads));
    chunk = (int)((units + items - 1) / items);
}

// Stencil work units: (j, k) columns x nseg slabs of planes, nseg chosen for
// the best share of busy threads (units / (threads x rounds)), discounted by
// the two planes each unit reads before its first point.
void jac_stencil_units(const JacobiDims &d, int ctas, int &nseg, int &items, int &chunk) {
    const long long ncols = (long long)(d.J - 2) * (d.K - 2), np = d.I - 2;
    const long long T = (long long)ctas * kSimtThreads;
    nseg = 1;
    double best = -1.0;
    for (long long ns = 1; ns <= std::max<long long>(1, std::min<long long>(np / 4, 64)); ++ns) {
        int it = 0, ch = 0;
        jac_split(ncols * ns, ctas, it, ch);
        const long long rounds = (ch + kSimtThreads - 1) / kSimtThreads;
        const double seg = (double)np / (double)ns;
        const double eff = (double)(ncols * ns) / (double)(T * rounds) * seg / (seg + 2.0);
        if (eff > best + 1e-9) {
            best = eff;
            nseg = (int)ns;
        }
    }
    jac_split(ncols * nseg, ctas, items, chunk);
}

Plan plan_request(Resident &S, const oo_serve_req &r) {
    Plan P{};
    if (r.kind == OO_BLOCK_GEMM) {
        const eq::Shape e = eq::shape(eq_scheme_for((int)r.k), (int)r.k);
        P.d_bytes = up256((size_t)r.m * r.k * 8) + up256((size_t)r.k * r.n * 8) + up256((size_t)r.m * r.n * 8) +
                    up256((size_t)r.m * 4) + up256((size_t)r.n * 4);
        P.rows = (size_t)e.slices * (r.m + r.n);
        P.n_simt = 1;
        P.n_tiles = (int)(((r.m + 127) / 128) * ((r.n + 31) / 32));  // upper bound (narrowest tiles)
    } else if (r.kind == OO_BLOCK_FFT) {
        // data, and for four-step lengths the intermediates and the first
        // pass's column exponents (at most 4096 of them)
        P.d_bytes = up256((size_t)r.n * 16) + (r.n > 4096 ? up256((size_t)r.n * 16) + up256(4096 * 4) : 0);
        P.n_simt = r.n > 4096 ? 3 : 2;
    } else {
        const JacobiDims d{(int)r.m, (int)r.n, (int)r.k, jacobi_pitch((int)r.k)};
        int nseg = 0, ns = 0, chunk = 0;
        jac_stencil_units(d, S.simt_ctas, nseg, ns, chunk);
        P.d_bytes = (size_t)NARR * up256(d.n_dev() * 4) + up256((size_t)std::max(1, r.iters) * 8) +
                    up256((size_t)2 * std::max(1, ns) * 8);
        P.n_simt = 1 + r.iters;
    }
    // upload area: the request's descriptors (first 1 KB) and entries
    P.h_bytes = up256(1024 + (size_t)P.n_simt * sizeof(Entry) + (size_t)P.n_tiles * sizeof(int4));
    return P;
}

void validate_resident(const oo_serve_req &r) {
    if (r.kind == OO_BLOCK_GEMM) {
        OO_REQUIRE(r.prec == OO_PREC_FP64EQ, OO_EINVAL,
                   "the device-resident loop serves FP64-equivalent GEMMs (OO_PREC_FP64EQ)");
        OO_REQUIRE(r.m >= 1 && r.n >= 1 && r.k >= 1 && r.m <= 65536 && r.n <= 65536 && r.k <= kSlicePitch,
                   OO_EINVAL, "bad GEMM dimensions (the device-resident loop takes k <= 2048)");
        OO_REQUIRE(r.in0 && r.in1 && r.out, OO_EINVAL, "null pointer");
    } else if (r.kind == OO_BLOCK_FFT) {
        OO_REQUIRE(r.n >= 1 && r.n <= (1 << 22) && (r.n & (r.n - 1)) == 0, OO_EINVAL,
                   "FFT length must be a power of two <= 2^22");
        OO_REQUIRE(r.dir == -1 || r.dir == 1, OO_EINVAL, "dir must be -1 or +1");
        OO_REQUIRE(r.in0 && r.out, OO_EINVAL, "null pointer");
    } else if (r.kind == OO_BLOCK_JACOBI) {
        OO_REQUIRE(r.m >= 3 && r.n >= 3 && r.k >= 3 && r.k <= 4096 && r.m * r.n * r.k < (1ll << 31), OO_EINVAL,
                   "bad Jacobi grid");
        OO_REQUIRE(r.iters >= 0 && r.iters <= 100000, OO_EINVAL, "bad iteration count");
        OO_REQUIRE(std::isfinite(r.omega), OO_EINVAL, "omega must be finite");
        OO_REQUIRE(r.out != nullptr, OO_EINVAL, "null pointer");
    } else {
        throw Error{OO_EINVAL, "unknown request kind"};
    }
}

// ring copies (the ring may wrap)
template <class T>
void upload_ring(T *ring, unsigned long long at, const T *src, size_t n, cudaStream_t s) {
    size_t done = 0;
    while (done < n) {
        const size_t pos = (size_t)((at + done) % kRingCap);
        const size_t cnt = std::min(n - done, (size_t)kRingCap - pos);
        OO_CUDA_TRY(cudaMemcpyAsync(ring + pos, src + done, cnt * sizeof(T), cudaMemcpyHostToDevice, s));
        done += cnt;
    }
}

// a new SIMT entry at ring position S.simt_w (+ index) with counter bases
Entry make_entry(Resident &S, unsigned long long pos, int type, int slot, int nitems, int aux, const Entry *dep) {
    Entry E{};
    E.type = type;
    E.slot = slot;
    E.nitems = nitems;
    E.rot = (int)(pos % (unsigned long long)S.simt_ctas);
    E.ctr = (unsigned)(pos % kRingCap);
    S.ctr_base[E.ctr] += (unsigned)nitems;
    E.target = S.ctr_base[E.ctr];
    E.dep_ctr = dep ? (int)dep->ctr : -1;
    E.dep_target = dep ? dep->target : 0u;
    E.aux = aux;
    return E;
}

// Stage a request whose inputs are on the device: descriptors and entries
// go to the device on the upload stream from the request's pinned upload
// area; an event marks when they have landed.  Returns false (nothing
// changed) when a ring has no room yet.
bool stage(Resident &S, RReq &q) {
    const oo_serve_req &r = q.r;
    char *dev = S.dev_base + q.d_off;
    char *upa = S.host_base + q.h_off;  // upload area
    std::vector<Entry> ents;
    std::vector<int4> tl;
    const unsigned long long s0 = S.simt_w, t0 = S.tile_w;
    auto pos = [&]() { return s0 + ents.size(); };
    cudaStream_t s = S.up;
    // room in the rings first: every CTA has passed the entries these
    // would overwrite
    size_t n_simt = 1;
    if (r.kind == OO_BLOCK_GEMM)
        res_tile_list((int)r.m, (int)r.n, (int)r.k, S.widths.data(), q.slot, tl);
    else if (r.kind == OO_BLOCK_FFT)
        n_simt = r.n > 4096 ? 3 : 2;
    else
        n_simt = 1 + (size_t)r.iters;
    {
        const unsigned long long ms = min_progress(S.ctl->simt_progress, S.simt_ctas);
        const unsigned long long mt = min_progress(S.ctl->tile_progress, S.tile_ctas);
        if (s0 + n_simt > ms + kRingCap - 16 || t0 + tl.size() > mt + kRingCap - (unsigned long long)S.tile_ctas)
            return false;
    }
    if (r.kind == OO_BLOCK_GEMM) {
        const int m = (int)r.m, n = (int)r.n, k = (int)r.k;
        const eq::Shape e = eq::shape(eq_scheme_for(k), k);
        double *A = reinterpret_cast<double *>(dev);
        double *B = reinterpret_cast<double *>(dev + up256((size_t)m * k * 8));
        double *C = reinterpret_cast<double *>(dev + up256((size_t)m * k * 8) + up256((size_t)k * n * 8));
        int *ea = reinterpret_cast<int *>(reinterpret_cast<char *>(C) + up256((size_t)m * n * 8));
        int *eb = reinterpret_cast<int *>(reinterpret_cast<char *>(ea) + up256((size_t)m * 4));
        const int na = (m + kSimtThreads / 32 - 1) / (kSimtThreads / 32), nb = (n + 63) / 64;
        ents.push_back(make_entry(S, pos(), kSplit, q.slot, na + nb, na, nullptr));
        const int ntile = (int)tl.size();
        const unsigned dctr = (unsigned)kRingCap + (unsigned)q.slot;
        S.ctr_base[dctr] += 8u * (unsigned)ntile;
        eq::GSplit G{};
        G.A = A;
        G.B = B;
        G.lda = k;
        G.ldb = n;
        G.pitch = kSlicePitch;
        G.m = m;
        G.n = n;
        G.k = k;
        G.kp = (k + 63) / 64 * 64;
        G.beta = e.beta;
        G.slices = e.slices;
        G.As = S.slices + q.row_off * kSlicePitch;
        G.Bs = G.As + (size_t)e.slices * m * kSlicePitch;
        G.ea = ea;
        G.eb = eb;
        std::memcpy(upa, &G, sizeof(G));
        res_tile_desc_fill(upa + 256, C, n, ea, eb, m, n, k, (int)q.row_off, (int)(q.row_off + (size_t)e.slices * m),
                           ents[0].ctr, ents[0].target, dctr, S.ctr_base[dctr], q.gen, q.slot);
        OO_CUDA_TRY(cudaMemcpyAsync(S.split_desc + q.slot, upa, sizeof(G), cudaMemcpyHostToDevice, s));
        OO_CUDA_TRY(cudaMemcpyAsync(S.tile_desc + (size_t)q.slot * res_tile_desc_bytes(), upa + 256,
                                    res_tile_desc_bytes(), cudaMemcpyHostToDevice, s));
        ents.back().last = 0;
    } else if (r.kind == OO_BLOCK_FFT) {
        const FftPlan *p = S.c->fft_plan(r.n);
        const int log2n = fft_plan_log2(p);
        double *x = reinterpret_cast<double *>(dev);
        float4 *mid = r.n > 4096 ? reinterpret_cast<float4 *>(dev + up256((size_t)r.n * 16)) : nullptr;
        int *colmax = r.n > 4096 ? reinterpret_cast<int *>(dev + 2 * up256((size_t)r.n * 16)) : nullptr;
        FftGroupReq R{};
        const void *tw[5];
        fft_plan_tables(p, &tw[0], &tw[1], &tw[2], &tw[3], &tw[4], &R.log2n, &R.log2n1, &R.log2n2);
        R.tw = static_cast<const float4 *>(tw[0]);
        R.tw_n1 = static_cast<const float4 *>(tw[1]);
        R.tw_n2 = static_cast<const float4 *>(tw[2]);
        R.tw_hi = static_cast<const float4 *>(tw[3]);
        R.tw_lo = static_cast<const float4 *>(tw[4]);
        R.in = x;
        R.out = x;
        R.mid = mid;
        R.colmax = colmax;
        R.inverse = r.dir > 0 ? 1 : 0;
        std::memcpy(upa, &R, sizeof(R));
        std::memset(upa + 512, 0, 4);  // the transform's exponent starts at zero (raised by the column pass)
        if (log2n <= 12) {
            ents.push_back(make_entry(S, pos(), kFftWhole, q.slot, 1, log2n, nullptr));
        } else {
            const int N1 = 1 << R.log2n1, N2 = 1 << R.log2n2;
            ents.push_back(make_entry(S, pos(), kFftCols, q.slot, N2 / (kFftElems / N1), R.log2n1, nullptr));
            ents.push_back(make_entry(S, pos(), kFftRows, q.slot, N1 / (kFftElems / N2), R.log2n2, &ents[0]));
        }
        OO_CUDA_TRY(cudaMemcpyAsync(S.fft_desc + q.slot, upa, sizeof(R), cudaMemcpyHostToDevice, s));
        OO_CUDA_TRY(cudaMemcpyAsync(S.expo + q.slot, upa + 512, 4, cudaMemcpyHostToDevice, s));
    } else {
        const JacobiDims d{(int)r.m, (int)r.n, (int)r.k, jacobi_pitch((int)r.k)};
        const size_t arr = up256(d.n_dev() * 4);
        JacDesc J{};
        for (int v = 0; v < NARR; ++v) J.arr[v] = reinterpret_cast<float *>(dev + (size_t)v * arr);
        J.res = reinterpret_cast<double *>(dev + (size_t)NARR * arr);
        J.partials = reinterpret_cast<double *>(dev + (size_t)NARR * arr + up256((size_t)std::max(1, r.iters) * 8));
        J.I = d.I;
        J.J = d.J;
        J.K = d.K;
        J.pitch = d.pitch;
        J.iters = r.iters;
        int n_setup = 0, n_st = 0;
        jac_split((long long)(d.n_dev() / 4), S.simt_ctas, n_setup, J.chunk4);
        jac_stencil_units(d, S.simt_ctas, J.nseg, n_st, J.chunk);
        J.omega = r.omega;
        std::memcpy(upa, &J, sizeof(J));
        ents.push_back(make_entry(S, pos(), kJacSetup, q.slot, n_setup, 0, nullptr));
        for (int it = 0; it < r.iters; ++it) {
            const Entry prev = ents.back();
            ents.push_back(make_entry(S, pos(), kJacStencil, q.slot, n_st, it, &prev));
        }
        OO_CUDA_TRY(cudaMemcpyAsync(S.jac_desc + q.slot, upa, sizeof(J), cudaMemcpyHostToDevice, s));
    }
    ents.back().last = r.kind == OO_BLOCK_GEMM ? 0 : 1;  // GEMMs finish in the tile epilogue
    ents.back().gen = q.gen;
    if (S.inject_stall) {
        // fault injection (tests): the request's first entry waits for its own
        // counter to pass its final value, which never happens
        ents[0].dep_ctr = (int)ents[0].ctr;
        ents[0].dep_target = ents[0].target + 1u;
        S.inject_stall = 0;
    }
    Entry *ue = reinterpret_cast<Entry *>(upa + 1024);
    std::memcpy(ue, ents.data(), ents.size() * sizeof(Entry));
    upload_ring(S.ring, s0, ue, ents.size(), s);
    if (!tl.empty()) {
        int4 *ut = reinterpret_cast<int4 *>(upa + 1024 + ents.size() * sizeof(Entry));
        std::memcpy(ut, tl.data(), tl.size() * sizeof(int4));
        upload_ring(S.tiles, t0, ut, tl.size(), s);
    }
    S.simt_w = s0 + ents.size();
    S.tile_w = t0 + tl.size();
    q.simt_end = S.simt_w;
    q.tile_end = S.tile_w;
    q.ev = take_event(S);
    OO_CUDA_TRY(cudaEventRecord(q.ev, s));
    return true;
}

// keep-alive (or stop) entries for every CTA of the SIMT worker and / or
// the tensor worker
RReq *stage_markers(Resident &S, bool stop, bool simt = true, bool tiles = true) {
    std::vector<Entry> ents(simt ? 1 : 0);
    if (simt) ents[0] = make_entry(S, S.simt_w, stop ? kStop : kNop, 0, 0, 0, nullptr);
    std::vector<int4> tl;
    if (tiles)
        for (int c = 0; c < S.tile_ctas; ++c) res_tile_marker(tl, stop);
    const unsigned long long ms = min_progress(S.ctl->simt_progress, S.simt_ctas);
    const unsigned long long mt = min_progress(S.ctl->tile_progress, S.tile_ctas);
    if (S.mark_free.empty() || S.simt_w + ents.size() > ms + kRingCap - 16 ||
        S.tile_w + tl.size() > mt + kRingCap - (unsigned long long)S.tile_ctas)
        return nullptr;
    auto *q = new RReq();
    q->marker = true;
    q->mark_slot = S.mark_free.back();
    S.mark_free.pop_back();
    char *buf = S.mark_pool + (size_t)q->mark_slot * kMarkBytes;
    if (!ents.empty()) {
        std::memcpy(buf, ents.data(), sizeof(Entry));
        upload_ring(S.ring, S.simt_w, reinterpret_cast<const Entry *>(buf), 1, S.up);
    }
    if (!tl.empty()) {
        std::memcpy(buf + sizeof(Entry), tl.data(), tl.size() * sizeof(int4));
        upload_ring(S.tiles, S.tile_w, reinterpret_cast<const int4 *>(buf + sizeof(Entry)), tl.size(), S.up);
    }
    S.simt_w += ents.size();
    S.tile_w += tl.size();
    q->simt_end = S.simt_w;
    q->tile_end = S.tile_w;
    q->ev = take_event(S);
    OO_CUDA_TRY(cudaEventRecord(q->ev, S.up));
    return q;
}

void fail_all(Resident &S, const std::string &why) {
    S.failed = true;
    S.fail_msg = why;
    auto fail = [&](RReq *q) {
        if (q->marker) {
            delete q;
            return;
        }
        q->status = OO_ETIMEOUT;
        q->error = why;
        q->state = RS_DONE;
        q->t_done = now_ms();
        ++S.n_failed;
        ++S.n_done;
    };
    // requests with an I/O thread finish there (inputs: failed; outputs:
    // the device had completed them)
    for (auto *dq : {&S.queue, &S.ready, &S.uploading, &S.running}) {
        for (RReq *q : *dq) fail(q);
        dq->clear();
    }
    S.cv_done.notify_all();
}

// device memory, digit-slice rows and descriptor slot back to the pools
void release(Resident &S, RReq *q) {
    S.dev.release(q->d_off, q->d_bytes);
    if (q->rows) S.rows.release(q->row_off, q->rows);
    S.free_slots.push_back(q->slot);
    if (q->ev) S.event_pool.push_back(q->ev);
    q->ev = nullptr;
}

// inputs from the caller's buffers to the request's device memory
void copy_in(Resident &S, const RReq &q, cudaStream_t s) {
    const oo_serve_req &r = q.r;
    char *dev = S.dev_base + q.d_off;
    if (r.kind == OO_BLOCK_GEMM) {
        OO_CUDA_TRY(cudaMemcpyAsync(dev, r.in0, (size_t)r.m * r.k * 8, cudaMemcpyHostToDevice, s));
        OO_CUDA_TRY(cudaMemcpyAsync(dev + up256((size_t)r.m * r.k * 8), r.in1, (size_t)r.k * r.n * 8,
                                    cudaMemcpyHostToDevice, s));
    } else if (r.kind == OO_BLOCK_FFT) {
        OO_CUDA_TRY(cudaMemcpyAsync(dev, r.in0, (size_t)r.n * 16, cudaMemcpyHostToDevice, s));
    }
    OO_CUDA_TRY(cudaStreamSynchronize(s));
}

// One write per page of a caller's output buffer, so that every page is
// mapped before the copy engine writes it: a copy into pages the process
// has never touched (a freshly allocated buffer) has the device fault them
// in one by one, which was measured to stall that copy and the copies
// queued behind it for tens of milliseconds; on the CPU the same pages are
// mapped at the cost of zero-filling them.
void touch_pages(void *p, size_t bytes) {
    static const size_t page = [] {
        const long v = sysconf(_SC_PAGESIZE);
        return v > 0 ? (size_t)v : (size_t)4096;
    }();
    if (!p || bytes == 0) return;
    volatile char *c = static_cast<volatile char *>(p);
    const size_t head = (page - ((uintptr_t)p % page)) % page;  // first page boundary inside
    c[0] = 0;
    for (size_t o = head; o < bytes; o += page) c[o] = 0;
    c[bytes - 1] = 0;
}

// outputs from the request's device memory to the caller's buffers
void copy_out(Resident &S, const RReq &q, cudaStream_t s) {
    const oo_serve_req &r = q.r;
    const char *dev = S.dev_base + q.d_off;
    if (r.kind == OO_BLOCK_GEMM)
        touch_pages(r.out, (size_t)r.m * r.n * 8);
    else if (r.kind == OO_BLOCK_FFT)
        touch_pages(r.out, (size_t)r.n * 16);
    else
        touch_pages(r.out, (size_t)r.m * r.n * r.k * 4);
    if (r.kind == OO_BLOCK_GEMM) {
        const char *C = dev + up256((size_t)r.m * r.k * 8) + up256((size_t)r.k * r.n * 8);
        OO_CUDA_TRY(cudaMemcpyAsync(r.out, C, (size_t)r.m * r.n * 8, cudaMemcpyDeviceToHost, s));
    } else if (r.kind == OO_BLOCK_FFT) {
        OO_CUDA_TRY(cudaMemcpyAsync(r.out, dev, (size_t)r.n * 16, cudaMemcpyDeviceToHost, s));
    } else {
        const JacobiDims d{(int)r.m, (int)r.n, (int)r.k, jacobi_pitch((int)r.k)};
        const size_t arr = up256(d.n_dev() * 4);
        const size_t wb = (size_t)d.K * 4;
        const int pv = r.iters % 2 ? VAR_WRK2 : VAR_P;  // the array the last sweep wrote
        OO_CUDA_TRY(cudaMemcpy2DAsync(r.out, wb, dev + (size_t)pv * arr, (size_t)d.pitch * 4, wb,
                                      (size_t)d.I * d.J, cudaMemcpyDeviceToHost, s));
        if (r.res && r.iters > 0)
            OO_CUDA_TRY(cudaMemcpyAsync(r.res, dev + (size_t)NARR * arr, (size_t)r.iters * 8,
                                        cudaMemcpyDeviceToHost, s));
    }
    OO_CUDA_TRY(cudaStreamSynchronize(s));
}

void io_worker(Resident *Sp, int idx) {
    Resident &S = *Sp;
    cudaSetDevice(S.c->device);
    cudaStream_t s = S.io_streams[(size_t)idx];
    std::unique_lock<std::mutex> lk(S.mu);
    while (true) {
        S.cv_io.wait(lk, [&] { return S.io_stop || !S.io_jobs.empty(); });
        if (S.io_jobs.empty()) break;  // stopping, nothing left
        RReq *q = S.io_jobs.front();
        S.io_jobs.pop_front();
        const bool in = q->state == RS_INPUT;
        lk.unlock();
        std::string err;
        try {
            if (in)
                copy_in(S, *q, s);
            else
                copy_out(S, *q, s);
        } catch (const Error &e) {
            err = e.msg;
        }
        lk.lock();
        if (in) {
            --S.n_io_in;
            if (err.empty() && !S.failed) {
                q->t_ready = now_ms();
                q->state = RS_READY;
                S.ready.push_back(q);
            } else {
                release(S, q);
                q->status = err.empty() ? OO_ETIMEOUT : OO_ECUDA;
                q->error = err.empty() ? S.fail_msg : "input copy: " + err;
                q->state = RS_DONE;
                q->t_done = now_ms();
                ++S.n_failed;
                ++S.n_done;
                S.cv_done.notify_all();
            }
        } else {
            --S.n_io_out;
            release(S, q);
            if (!err.empty()) {
                q->status = OO_ECUDA;
                q->error = "output copy: " + err;
                ++S.n_failed;
            }
            q->state = RS_DONE;
            q->t_done = now_ms();
            S.sum_ms[0] += q->t_admit - q->t_submit;
            S.sum_ms[1] += q->t_ready - q->t_admit;
            S.sum_ms[2] += q->t_pub - q->t_ready;
            S.sum_ms[3] += q->t_dev - q->t_pub;
            S.sum_ms[4] += q->t_done - q->t_dev;
            ++S.n_timed;
            ++S.n_done;
            S.cv_done.notify_all();
        }
        S.cv_sched.notify_one();
    }
}

void scheduler(Resident *Sp) {
    Resident &S = *Sp;
    cudaSetDevice(S.c->device);
    std::unique_lock<std::mutex> lk(S.mu);
    bool stop_sent = false;
    while (true) {
        bool progress = false;
        try {
            // ---- worker health: a worker that exits before the stop entries
            // has seen a bounded wait run out
            if (!S.failed && !stop_sent) {
                const cudaError_t a = cudaStreamQuery(S.s_simt), b = cudaStreamQuery(S.s_tiles);
                if (S.ctl->fault || a != cudaErrorNotReady || b != cudaErrorNotReady) {
                    // which wait: error bits of the workers (SIMT 32 publication, 64
                    // dependency; tensor 8 publication, 16 split, 512 / 128 / 256
                    // queue, 1 / 2 / 4 operand pipeline)
                    std::this_thread::sleep_for(std::chrono::milliseconds(5));
                    unsigned bits = 0;
                    cudaMemcpyAsync(&bits, S.err, 4, cudaMemcpyDeviceToHost, S.down);
                    cudaStreamSynchronize(S.down);
                    std::string why = "a bounded wait in the device-resident loop ran out (error bits " +
                                      std::to_string(bits) + (S.ctl->fault ? "" : ", a worker exited");
                    if (a != cudaErrorNotReady && a != cudaSuccess) why += std::string(", ") + cudaGetErrorString(a);
                    if (b != cudaErrorNotReady && b != cudaSuccess) why += std::string(", ") + cudaGetErrorString(b);
                    if (bits & 32u)
                        why += "; SIMT wait for entry " + std::to_string(S.ctl->stuck_at) + " saw publication " +
                               std::to_string(S.ctl->stuck_seen) + " of " + std::to_string(S.simt_w) + " written";
                    fail_all(S, why + "); the workers stop");
                }
            }
            // ---- finished on the device: an I/O thread copies the outputs back
            for (auto it = S.running.begin(); it != S.running.end();) {
                RReq *q = *it;
                if (S.ctl->done[q->slot] == q->gen) {
                    q->t_dev = now_ms();
                    q->state = RS_OUTPUT;
                    ++S.n_io_out;
                    S.io_jobs.push_back(q);
                    S.cv_io.notify_one();
                    it = S.running.erase(it);
                    progress = true;
                } else {
                    ++it;
                }
            }
            // ---- uploaded: publish in ring order
            while (!S.uploading.empty() && cudaEventQuery(S.uploading.front()->ev) == cudaSuccess) {
                RReq *q = S.uploading.front();
                S.uploading.pop_front();
                std::atomic_thread_fence(std::memory_order_release);
                const double t_pub = now_ms();
                if (q->simt_end > S.ctl->pub_simt) S.last_simt_pub = t_pub;
                if (q->tile_end > S.ctl->pub_tiles) S.last_tile_pub = t_pub;
                S.ctl->pub_simt = q->simt_end;
                S.ctl->pub_tiles = q->tile_end;
                progress = true;
                if (q->marker) {
                    S.event_pool.push_back(q->ev);
                    S.mark_free.push_back(q->mark_slot);
                    delete q;
                } else {
                    S.host.release(q->h_off, q->h_bytes);  // the upload area has been read
                    q->t_pub = t_pub;
                    q->state = RS_RUNNING;
                    S.running.push_back(q);
                }
            }
            // ---- admissions: oldest first, by free device memory (arena and
            // digit-slice rows) and a free descriptor slot; inputs go to an
            // I/O thread
            while (!S.failed && !S.queue.empty() && !S.free_slots.empty()) {
                RReq *q = S.queue.front();
                size_t off = 0, roff = 0;
                if (!S.dev.alloc(q->d_bytes, &off)) break;
                if (q->rows && !S.rows.alloc(q->rows, &roff)) {
                    S.dev.release(off, q->d_bytes);
                    break;
                }
                q->d_off = off;
                q->row_off = roff;
                q->slot = S.free_slots.back();
                S.free_slots.pop_back();
                q->gen = S.next_gen++;
                S.queue.pop_front();
                q->t_admit = now_ms();
                if (q->r.kind == OO_BLOCK_JACOBI) {  // no inputs
                    q->t_ready = q->t_admit;
                    q->state = RS_READY;
                    S.ready.push_back(q);
                } else {
                    q->state = RS_INPUT;
                    ++S.n_io_in;
                    S.io_jobs.push_back(q);
                    S.cv_io.notify_one();
                }
                progress = true;
            }
            // ---- inputs on the device: stage descriptors and entries, in the
            // order the inputs landed
            while (!S.failed && !S.ready.empty()) {
                RReq *q = S.ready.front();
                if (!S.host.alloc(q->h_bytes, &q->h_off)) break;
                if (!stage(S, *q)) {  // rings full: try again later
                    S.host.release(q->h_off, q->h_bytes);
                    break;
                }
                S.ready.pop_front();
                q->state = RS_UPLOAD;
                S.uploading.push_back(q);
                progress = true;
            }
            // ---- keep-alive / stop entries
            const bool idle_all = S.queue.empty() && S.ready.empty() && S.uploading.empty() && S.running.empty() &&
                                  S.n_io_in == 0 && S.n_io_out == 0;
            if (!S.failed && !stop_sent && S.stop && idle_all) {
                RReq *m = stage_markers(S, true);
                if (m) {
                    S.uploading.push_back(m);
                    stop_sent = true;
                }
            } else if (!S.failed && !stop_sent) {
                // Keep-alives, far inside the workers' one-second bound: every
                // SIMT CTA reads every entry, so one entry when nothing was
                // published for 20 ms; a tile CTA only sees every CTAs-th
                // entry, so a full round of markers (one per CTA) every 20 ms
                const double t = now_ms();
                bool in_flight_simt = false;
                for (RReq *u : S.uploading) in_flight_simt = in_flight_simt || u->simt_end > S.ctl->pub_simt;
                const bool ks = !in_flight_simt && t - S.last_simt_pub > 20.0;
                const bool kt = t - S.last_tile_round > 20.0;
                if (ks || kt) {
                    RReq *m = stage_markers(S, false, ks, kt);
                    if (m) {
                        S.uploading.push_back(m);
                        if (kt) S.last_tile_round = t;
                    }
                }
            }
            if (stop_sent && S.uploading.empty()) break;
            if (S.failed && S.stop && S.n_io_in == 0 && S.n_io_out == 0) break;
        } catch (const Error &e) {
            fail_all(S, e.msg);
        }
        if (!progress) {
            // work in flight: poll again at once (a timed wait sleeps tens of
            // microseconds past its deadline, at each stage of a request);
            // otherwise sleep until woken (a submission, an I/O thread), and
            // at least every millisecond for the keep-alives
            const bool busy = !S.uploading.empty() || !S.running.empty();
            if (busy) {
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                S.cv_sched.wait_for(lk, std::chrono::milliseconds(1));
            }
        }
    }
}

}  // namespace

void resident_stop(Resident *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_sched.notify_all();
    if (S->th.joinable()) S->th.join();
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->io_stop = true;
    }
    S->cv_io.notify_all();
    for (auto &t : S->io)
        if (t.joinable()) t.join();
    // the workers exit at the stop entries (or have exited after a bounded
    // wait ran out)
    if (S->s_simt) cudaStreamSynchronize(S->s_simt);
    if (S->s_tiles) cudaStreamSynchronize(S->s_tiles);
    if (S->up) cudaStreamSynchronize(S->up);
    if (S->down) cudaStreamSynchronize(S->down);
    for (auto &kv : S->reqs) delete kv.second;
    for (auto e : S->event_pool) cudaEventDestroy(e);
    for (cudaStream_t s : {S->up, S->down, S->s_simt, S->s_tiles})
        if (s) cudaStreamDestroy(s);
    for (cudaStream_t s : S->io_streams)
        if (s) cudaStreamDestroy(s);
    if (S->dev_misc) cudaFree(S->dev_misc);
    if (S->dev_base) cudaFree(S->dev_base);
    if (S->host_base) cudaFreeHost(S->host_base);
    if (S->ctl) cudaFreeHost(S->ctl);
    if (S->mark_pool) cudaFreeHost(S->mark_pool);
    delete S;
}

}  // namespace oo

using namespace oo;

namespace {
template <class F>
oo_status res_guard(Ctx &c, F &&f) {
    try {
        f();
        c.last_error.clear();
        return OO_OK;
    } catch (const Error &e) {
        c.last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        c.last_error = "host allocation failed";
        return OO_ENOMEM;
    } catch (...) {
        c.last_error = "unknown failure";
        return OO_ECUDA;
    }
}
}  // namespace

extern "C" oo_status oo_serve_start_resident(oo_ctx *ctx, uint64_t hbm_budget_bytes, int queue_cap,
                                              int tensor_ctas) {
    if (!ctx) return OO_EINVAL;
    Ctx &c = ctx_state(ctx);
    return res_guard(c, [&] {
        OO_REQUIRE(c.device >= 0, OO_ESTATE, "host-only context (device -1) cannot serve");
        OO_REQUIRE(c.server == nullptr && c.rserver == nullptr, OO_ESTATE, "the context is already serving");
        OO_REQUIRE(queue_cap >= 1, OO_EINVAL, "queue_cap must be >= 1");
        OO_REQUIRE(hbm_budget_bytes >= (64u << 20), OO_EINVAL, "device budget below 64 MiB");
        OO_CUDA_TRY(cudaSetDevice(c.device));
        const int sms = c.num_sms;
        // default split: an eighth of the SMs for the tensor tiles (served
        // mix of 50 % GEMM, 30 % FFT, 20 % Jacobi at saturation, 10 000 and
        // 20 000 req/s offered: 1026-1081 solves/s at 19 of 152 SMs,
        // 1012-1072 at 14, 1010-1062 at 10, 919-972 at 28, 925-973 at 38,
        // 857 at 57, 723 at 76; the Jacobi sweeps on the SIMT worker bound it)
        const int tc = tensor_ctas > 0 ? tensor_ctas : std::max(1, sms / 8);
        OO_REQUIRE(tc >= 1 && tc < sms && tc <= kMaxCtas && sms - tc <= kMaxCtas, OO_EINVAL,
                   "tensor_ctas must leave SMs for the SIMT worker");
        for (int e = 0; e <= 22; ++e) c.fft_plan(1ll << e);  // twiddle tables up front, before the workers
        OO_CUDA_TRY(cudaDeviceSynchronize());
        auto *S = new Resident();
        S->c = &c;
        S->queue_cap = (size_t)queue_cap;
        S->tile_ctas = tc;
        S->simt_ctas = sms - tc;
        S->widths = c.eq_widths;
        S->inject_stall = c.inject_wait == OO_INJECT_SERVE_STALL;
        if (S->inject_stall) c.inject_wait = OO_INJECT_NONE;
        try {
            // device budget: a quarter for the GEMM digit slices, the rest the arena
            const size_t budget = up256(hbm_budget_bytes);
            const size_t slice_bytes = budget / 4 / ((size_t)kSlicePitch * 2) * ((size_t)kSlicePitch * 2);
            const size_t arena = budget - slice_bytes;
            if (cudaMalloc(&S->dev_base, budget) != cudaSuccess) {
                cudaGetLastError();
                throw Error{OO_ENOMEM, "device budget of " + std::to_string(budget) + " bytes"};
            }
            S->dev.reset(arena);
            S->slices = reinterpret_cast<__nv_bfloat16 *>(S->dev_base + arena);
            S->slice_rows = (long long)(slice_bytes / ((size_t)kSlicePitch * 2));
            OO_REQUIRE(S->slice_rows > 2 * 128, OO_EINVAL, "device budget too small for the digit slices");
            S->rows.reset((size_t)S->slice_rows - 128);  // keep a box of rows past the end for TMA reads
            // pinned upload areas of the requests being staged (at most
            // ~4 MB each: their entries fit the rings)
            const size_t up_bytes = (size_t)64 << 20;
            if (cudaHostAlloc(&S->host_base, up_bytes, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                throw Error{OO_ENOMEM, "pinned upload areas of " + std::to_string(up_bytes) + " bytes"};
            }
            S->host.reset(up_bytes);
            if (cudaHostAlloc(&S->mark_pool, (size_t)kMarkSlots * kMarkBytes, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                S->mark_pool = nullptr;
                throw Error{OO_ENOMEM, "pinned marker slots"};
            }
            for (int i = kMarkSlots - 1; i >= 0; --i) S->mark_free.push_back(i);
            // rings, counters, descriptors
            size_t at = 0;
            auto put = [&](size_t b) {
                const size_t x = at;
                at += up256(b);
                return x;
            };
            const size_t o_ring = put((size_t)kRingCap * sizeof(Entry));
            const size_t o_tiles = put((size_t)kRingCap * sizeof(int4));
            const size_t o_ctr = put((size_t)(kRingCap + kSlots + 1) * 4);  // + the SIMT heartbeat
            const size_t o_err = put(4);
            const size_t o_split = put((size_t)kSlots * sizeof(eq::GSplit));
            const size_t o_tdesc = put((size_t)kSlots * res_tile_desc_bytes());
            const size_t o_fft = put((size_t)kSlots * sizeof(FftGroupReq));
            const size_t o_expo = put((size_t)kSlots * 4);
            const size_t o_tlist = put((size_t)kSlots * 4);
            const size_t o_jac = put((size_t)kSlots * sizeof(JacDesc));
            OO_CUDA_TRY(cudaMalloc(&S->dev_misc, at));
            char *b = static_cast<char *>(S->dev_misc);
            OO_CUDA_TRY(cudaMemset(b, 0, at));
            S->ring = reinterpret_cast<Entry *>(b + o_ring);
            S->tiles = reinterpret_cast<int4 *>(b + o_tiles);
            S->ctr = reinterpret_cast<unsigned *>(b + o_ctr);
            S->err = reinterpret_cast<unsigned *>(b + o_err);
            S->split_desc = reinterpret_cast<eq::GSplit *>(b + o_split);
            S->tile_desc = b + o_tdesc;
            S->fft_desc = reinterpret_cast<FftGroupReq *>(b + o_fft);
            S->expo = reinterpret_cast<int *>(b + o_expo);
            S->tlist = reinterpret_cast<int *>(b + o_tlist);
            S->jac_desc = reinterpret_cast<JacDesc *>(b + o_jac);
            std::vector<int> ident(kSlots);
            for (int i = 0; i < kSlots; ++i) ident[i] = i;
            OO_CUDA_TRY(cudaMemcpy(S->tlist, ident.data(), (size_t)kSlots * 4, cudaMemcpyHostToDevice));
            S->ctr_base.assign((size_t)kRingCap + kSlots, 0u);
            for (int i = kSlots - 1; i >= 0; --i) S->free_slots.push_back(i);
            // control block in mapped pinned host memory
            if (cudaHostAlloc(reinterpret_cast<void **>(&S->ctl), sizeof(Ctl), cudaHostAllocMapped) != cudaSuccess) {
                cudaGetLastError();
                S->ctl = nullptr;
                throw Error{OO_ENOMEM, "mapped control block"};
            }
            std::memset(const_cast<Ctl *>(S->ctl), 0, sizeof(Ctl));
            for (int i = 0; i < S->tile_ctas; ++i) S->ctl->tile_progress[i] = (unsigned long long)i;
            OO_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void **>(&S->ctl_dev), S->ctl, 0));
            for (cudaStream_t *s : {&S->up, &S->down, &S->s_simt, &S->s_tiles})
                OO_CUDA_TRY(cudaStreamCreateWithFlags(s, cudaStreamNonBlocking));
            // the workers: launched once, resident until the stop entries
            SimtArgs a{};
            a.ring = S->ring;
            a.ctr = S->ctr;
            a.ctl = S->ctl_dev;
            a.err = S->err;
            a.split = S->split_desc;
            a.fft = S->fft_desc;
            a.expo = S->expo;
            a.tlist = S->tlist;
            a.jac = S->jac_desc;
            a.start = 0;
            // both workers loaded before either runs (lazy loading of the
            // second could otherwise wait for the first to finish)
            static std::atomic<uint64_t> attr{0};
            set_smem_limit_once((const void *)resident_simt_kernel, simt_smem_bytes(), attr);
            cudaFuncAttributes fa{};
            OO_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void *)resident_simt_kernel));
            prepare_resident_tiles();
            resident_simt_kernel<<<S->simt_ctas, kSimtThreads, simt_smem_bytes(), S->s_simt>>>(a);
            OO_CUDA_TRY(cudaGetLastError());
            launch_resident_tiles(S->tiles, S->tile_desc, S->ctr, S->ctl_dev, 0, S->slices, S->slice_rows, S->err,
                                  S->tile_ctas, S->s_tiles);
            // every worker CTA must be resident (the static assignment of
            // items and tiles relies on it): wait, bounded, for all of them
            const double t0 = now_ms();
            while (true) {
                int up = 0;
                for (int i = 0; i < S->simt_ctas; ++i) up += S->ctl->alive[i] != 0;
                for (int i = 0; i < S->tile_ctas; ++i) up += S->ctl->alive[kMaxCtas + i] != 0;
                if (up == S->simt_ctas + S->tile_ctas) break;
                if (now_ms() - t0 > 5000.0)
                    throw Error{OO_ECUDA, "not every worker CTA of the device-resident loop became resident (" +
                                              std::to_string(up) + " of " +
                                              std::to_string(S->simt_ctas + S->tile_ctas) + ")"};
                std::this_thread::sleep_for(std::chrono::microseconds(200));
            }
            S->last_simt_pub = S->last_tile_pub = S->last_tile_round = now_ms();
            for (int i = 0; i < kIoThreads; ++i) {
                cudaStream_t st = nullptr;
                OO_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
                S->io_streams.push_back(st);
            }
            for (int i = 0; i < kIoThreads; ++i) S->io.emplace_back(io_worker, S, i);
            S->th = std::thread(scheduler, S);
        } catch (...) {
            {
                std::lock_guard<std::mutex> g(S->mu);
                S->stop = true;
                S->failed = true;
            }
            if (S->ctl && S->up && S->mark_pool) {
                // workers may be running: give them their stop entries
                RReq *m = stage_markers(*S, true);
                if (m) {
                    cudaEventSynchronize(m->ev);
                    S->ctl->pub_simt = m->simt_end;
                    S->ctl->pub_tiles = m->tile_end;
                    delete m;
                }
            }
            resident_stop(S);
            throw;
        }
        c.rserver = S;
    });
}

namespace oo {

oo_status resident_submit(Resident *S, const oo_serve_req *req, uint64_t *ticket) {
    auto *q = new (std::nothrow) RReq();
    if (!q) return OO_ENOMEM;
    try {
        validate_resident(*req);
        q->r = *req;
        std::lock_guard<std::mutex> g(S->mu);
        const Plan P = plan_request(*S, *req);
        q->h_bytes = P.h_bytes;
        q->d_bytes = P.d_bytes;
        q->rows = P.rows;
        if (q->d_bytes > S->dev.size() || q->rows > S->rows.size() || q->h_bytes > S->host.size() ||
            P.n_simt + 16 > kRingCap || P.n_tiles + 2 * S->tile_ctas > kRingCap) {
            delete q;
            return OO_EINVAL;  // can never be admitted
        }
        if (S->failed) {
            S->c->last_error = S->fail_msg;
            delete q;
            return OO_ESTATE;
        }
        if (S->stop || S->queue.size() >= S->queue_cap) {
            ++S->n_busy;
            delete q;
            return OO_EBUSY;
        }
        q->ticket = S->next_ticket++;
        q->t_submit = now_ms();
        S->reqs[q->ticket] = q;
        S->queue.push_back(q);
        ++S->n_submitted;
        *ticket = q->ticket;
    } catch (const Error &e) {
        delete q;
        return e.code;
    }
    S->cv_sched.notify_one();
    return OO_OK;
}

// The outputs are in the caller's buffers once the request is done (an I/O
// thread copied them there).
oo_status resident_wait(Ctx &c, Resident *S, uint64_t ticket, int timeout_ms, double *latency_ms) {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return OO_EINVAL;
    RReq *q = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    while (q->state != RS_DONE) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && q->state != RS_DONE)
            return OO_ETIMEOUT;
    }
    S->reqs.erase(ticket);
    const oo_status st = q->status;
    if (latency_ms) *latency_ms = q->t_done - q->t_submit;
    if (st != OO_OK) c.last_error = q->error;
    delete q;
    return st;
}

void resident_stats(Resident *S, oo_serve_stats_t *out) {
    std::lock_guard<std::mutex> g(S->mu);
    out->submitted = S->n_submitted;
    out->completed = S->n_done;
    out->rejected_busy = S->n_busy;
    out->failed = S->n_failed;
    out->queued = (uint64_t)S->queue.size();
    out->running = (uint64_t)(S->n_io_in + S->ready.size() + S->uploading.size() + S->running.size() + S->n_io_out);
    out->device_free_bytes = S->dev.free_bytes();
    out->device_budget_bytes = S->dev.size();
    const double n = S->n_timed ? (double)S->n_timed : 1.0;
    for (int i = 0; i < 5; ++i) out->stage_ms[i] = S->sum_ms[i] / n;
}

}  // namespace oo
