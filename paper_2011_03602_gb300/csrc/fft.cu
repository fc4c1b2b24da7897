// Fourier-transform function block (Sec. 3.2.2, Sec. 4.2.1): complex128 1D
// FFT, forward X_k = sum_n x_n e^{-2 pi i nk/N} and inverse with e^{+} and 1/N.
//
// GB300 design.  FP64 units run at 1/59 of FP32 on this part, so butterflies
// use float-float arithmetic (ff.cuh; ~47 significant bits, error ~ log2(N)
// * 2^-47 relative) and FP64 is used only to generate twiddle tables
// (sincospi) and to widen results back to double.  Inputs are scaled by
// powers of two (exact) before the split into float pairs, which keeps
// float-float's exponent range out of the way for any finite double input:
// each column of a CTA (a whole transform, or a four-step first-pass column)
// by the power that brings its own largest component into [1/2, 1), found
// from the values the CTA loads anyway; the second pass brings the columns
// to their transform's scale (fft_device.cuh).  No pass over the input
// precedes the transform.
//
// Structure: a CTA holds 4096 complex float-float values (64 KB) in shared
// memory and runs Stockham auto-sort stages -- a first stage of radix 2, 4
// or 8 (done in registers at load time where a thread holds whole
// butterflies of it), then radix-8 stages -- 512 threads x 8 values per
// stage, twiddles from a per-stage table (W_{8Ls}^{kq} for stage sub-length
// Ls) staged into shared memory; two CTAs per SM where the shared memory
// allows.  N <= 4096 runs in one pass
// (several transforms per CTA when N is small).  Larger N uses the four-step
// split N = N1 x N2: pass 1 does N2 column FFTs of length N1 and multiplies
// by W_N^{k1 n2} (two-level twiddle table), writing float-float
// intermediates; pass 2 does N1 row FFTs of length N2 and writes X[k1 + N1 k2]
// as doubles.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ff.cuh"
#include "fft_device.cuh"
#include "oo_internal.h"

namespace oo {

namespace {

struct FftArgs {
    int log2n, log2n1, log2n2;
    long long n;
    int batch;
    int inverse;
    const double *in_d;   // mode 0 / 1
    double *out_d;        // mode 0 / 2
    const float4 *in_ff;  // mode 2
    float4 *out_ff;       // mode 1
    const float4 *tw;     // W_L^t for the pass length L (table of L entries)
    const float4 *tw_hi;  // W_N^{m_hi * 2^kTwSplit}
    const float4 *tw_lo;  // W_N^{m_lo}
    int *expo;            // four-step, per transform: biased exponent of its largest component (zero first)
    int *colmax;          // four-step, per transform: the N2 first-pass columns' largest exponents
};

// The first stage (radix R, no twiddles) on the 8 values a thread has
// loaded (v[r] at shared-memory position dst[r] = column << log2L | t),
// stored in Stockham order: butterfly j's output p at column position
// j R + p.  COLFAST: value r of the thread is t0 + r L/8 of one column, so
// butterfly g takes r = g + m 8/R; otherwise value r = g R + m is
// tid + m 512 of column g (L = 512 R).
template <int R, bool COLFAST, class Pos>
__device__ __forceinline__ void first_stage_regs(float4 *sd, const float4 *v, const Pos &dst, int log2L, bool inv,
                                                 int ps) {
    static_assert(kFftElems / kFftThreads == 8, "eight values per thread");
    constexpr int G = 8 / R;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        cplx x[R];
#pragma unroll
        for (int m = 0; m < R; ++m) x[m] = ld_cplx(&v[COLFAST ? g + m * G : g * R + m]);
        const int r0 = COLFAST ? g : g * R;
        const int col = dst(r0) >> log2L, j = dst(r0) & ((1 << log2L) - 1);
        dft_small<R>(x, inv);
        const int o = (col << log2L) + j * R;
#pragma unroll
        for (int p = 0; p < R; ++p) st_cplx(sd + sp(o + p, ps), x[p]);
    }
}

// MODE 0: whole transforms of length L = n, several per CTA (double in/out)
// MODE 1: four-step pass 1: columns of length N1 (double in, ff out x twiddle)
// MODE 2: four-step pass 2: rows of length N2 (ff in, double out at k1 + N1 k2)
// Two CTAs per SM (64 registers, no spills; at most 96 KB of shared memory
// each, the 4096-point table being read in place), so one CTA's global loads
// and stores overlap the other's butterflies: 2^22 in 0.229 ms instead of
// 0.262 ms with one.  PAD: the padded shared-memory layout (every pass
// length but 2048, fft_padded), a template parameter so that the layout
// shift is a constant.
template <int MODE, bool PAD>
__global__ void __launch_bounds__(kFftThreads, 2) fft_pass_kernel(FftArgs a) {
    extern __shared__ __align__(16) float4 fsmem[];
    float4 *sd = fsmem;
    const int log2L = MODE == 0 ? a.log2n : (MODE == 1 ? a.log2n1 : a.log2n2);
    const int L = 1 << log2L;
    const int C = kFftElems >> log2L;  // columns (transforms / rows) in this CTA
    const bool inv = a.inverse != 0;
    const float4 *stw = a.tw;  // the 4096-point table is read in place
    if (twiddles_staged(log2L)) {
        float4 *t_s = fsmem + (PAD ? kFftElemsPad : kFftElems);
        for (int t = threadIdx.x; t < stage_table_count(log2L); t += kFftThreads) t_s[t] = a.tw[t];
        stw = t_s;
    }
    // the columns' largest exponents (modes 0, 1), after the staged table
    int *smax = reinterpret_cast<int *>(fsmem + (PAD ? kFftElemsPad : kFftElems) + (twiddles_staged(log2L) ? L : 0));
    constexpr int ps = PAD ? 3 : 30;  // data layout: fft_pad_shift(log2L)
    if (MODE != 2)
        for (int t = threadIdx.x; t < C; t += kFftThreads) smax[t] = 0;

    const long long n = a.n;
    const int N1 = 1 << a.log2n1, N2 = 1 << a.log2n2;
    int b = 0, c0 = 0;  // transform index, first column / row of this CTA
    if (MODE == 0) {
        c0 = blockIdx.x * C;
    } else {
        const int per = (MODE == 1 ? N2 : N1) / C;
        b = blockIdx.x / per;
        c0 = (blockIdx.x % per) * C;
    }

    // ---- load: all of this thread's 16-byte loads are issued before any is
    // used (eight in flight), then split and stored to shared memory -- after
    // the first stage, done in registers where this thread holds whole
    // butterflies of it: column-fastest loads (MODE 1) give it x[t0 + r L/8],
    // r < 8, of one column; row-fastest loads (MODE 0 / 2) give it, for
    // L = 1024, 2048, 4096, x[tid + m 512], m < L / 512 = the first radix, of
    // each of its columns
    constexpr int kPer = kFftElems / kFftThreads;
    const int b0 = first_radix_log2(log2L);
    const bool first_here = MODE == 1 ? log2L >= 3 : (log2L >= 10 && log2L <= 12);
    {
        // shared-memory position of value r of this thread: column c, element
        // t at (c << log2L) + t, which row-fastest is q itself
        auto dst = [&](int r) {
            const int q = threadIdx.x + r * kFftThreads;
            if (MODE == 1) return ((q & (C - 1)) << log2L) + (q >> (31 - __clz(C)));
            return q;
        };
        double2 raw[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int q = threadIdx.x + r * kFftThreads;
            int c, t;
            if (MODE == 1) {  // column-fastest for coalescing
                c = q & (C - 1);
                t = q >> (31 - __clz(C));
            } else {
                c = q >> log2L;
                t = q & (L - 1);
            }
            raw[r] = make_double2(0.0, 0.0);
            if (MODE == 0) {
                if (c0 + c < a.batch) raw[r] = reinterpret_cast<const double2 *>(a.in_d)[(long long)(c0 + c) * n + t];
            } else if (MODE == 1) {
                raw[r] = reinterpret_cast<const double2 *>(a.in_d)[(long long)b * n + (long long)t * N2 + c0 + c];
            } else {
                const float4 f = a.in_ff[(long long)b * n + (long long)(c0 + c) * N2 + t];
                raw[r] = make_double2(__hiloint2double(__float_as_int(f.y), __float_as_int(f.x)),
                                      __hiloint2double(__float_as_int(f.w), __float_as_int(f.z)));
            }
        }
        float4 v[kPer];
        if (MODE == 2) {
            // float-float intermediates: the 16 bytes as they were, brought
            // from their column's scale to the transform's
            const int em = a.expo[b];
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const float4 f = make_float4(__int_as_float(__double2loint(raw[r].x)),
                                             __int_as_float(__double2hiint(raw[r].x)),
                                             __int_as_float(__double2loint(raw[r].y)),
                                             __int_as_float(__double2hiint(raw[r].y)));
                const int t = dst(r) & (L - 1);
                v[r] = scale_down(f, col_shift(a.colmax[(long long)b * N2 + t], em));
            }
        } else {
            __syncthreads();  // smax cleared
            if (MODE == 1) {  // a thread's values are all of column tid mod C
                int m = 0;
#pragma unroll
                for (int r = 0; r < kPer; ++r) m = max(m, expo_of(raw[r]));
                colmax_warp(m, min(C, 32), false, smax, (int)threadIdx.x & (C - 1));
            } else {
#pragma unroll
                for (int r = 0; r < kPer; ++r) colmax_warp(expo_of(raw[r]), min(L, 32), true, smax, dst(r) >> log2L);
            }
            __syncthreads();
            if (MODE == 1 && (int)threadIdx.x < C) {
                const int m = smax[threadIdx.x];
                a.colmax[(long long)b * N2 + c0 + threadIdx.x] = m;
                if (m > 0) atomicMax(a.expo + b, m);
            }
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const int S = scale_from(smax[dst(r) >> log2L]);
                split_scaled(raw[r].x, S, v[r].x, v[r].y);
                split_scaled(raw[r].y, S, v[r].z, v[r].w);
            }
        }
        if (first_here) {
            if (b0 == 1)
                first_stage_regs<2, MODE == 1>(sd, v, dst, log2L, inv, ps);
            else if (b0 == 2)
                first_stage_regs<4, MODE == 1>(sd, v, dst, log2L, inv, ps);
            else
                first_stage_regs<8, MODE == 1>(sd, v, dst, log2L, inv, ps);
        } else {
#pragma unroll
            for (int r = 0; r < kPer; ++r) sd[sp(dst(r), ps)] = v[r];
        }
    }
    __syncthreads();

    if (first_here)
        fft_in_smem_after_first(sd, stw, log2L, inv, ps);
    else
        fft_in_smem(sd, stw, log2L, inv, ps);

    // ---- store
    for (int q = threadIdx.x; q < kFftElems; q += kFftThreads) {
        int c, t;
        if (MODE == 0) {
            c = q >> log2L;
            t = q & (L - 1);
        } else {  // column / row index fastest
            c = q & (C - 1);
            t = q >> (31 - __clz(C));
        }
        cplx v = ld_cplx(sd + sp((c << log2L) + t, ps));
        if (MODE == 1) {
            // W_N^{k1 n2}, k1 = t, n2 = c0 + c; m < N so no reduction needed
            const long long m = (long long)t * (c0 + c);
            const int mh = (int)(m >> kTwSplit), ml = (int)(m & ((1 << kTwSplit) - 1));
            cplx w = ff::cmul_lazy(ld_cplx(a.tw_hi + mh), ld_cplx(a.tw_lo + ml));
            if (inv) w = ff::conj(w);
            v = ff::cmul_lazy(v, w);  // pass 2 takes lazy pairs
            st_cplx(a.out_ff + (long long)b * n + (long long)t * N2 + c0 + c, v);
        } else {
            const int tb = MODE == 0 ? c0 + c : b;
            if (MODE == 0 && tb >= a.batch) continue;
            const int e = MODE == 0 ? smax[c] : a.expo[b];  // the transform's (mode 0: the column's) exponent
            const int S = scale_from(e) - (inv ? a.log2n : 0);
            const double re = widen_scaled(v.rh, v.rl, S), im = widen_scaled(v.ih, v.il, S);
            const long long idx = MODE == 0 ? (long long)tb * n + t
                                            : (long long)b * n + (c0 + c) + (long long)N1 * t;
            reinterpret_cast<double2 *>(a.out_d)[idx] = e == kNonFiniteExpo ? nan2() : make_double2(re, im);
        }
    }
}

// table[t] = W_M^{t * stride} = exp(-2 pi i t stride / M), t < count, in FP64, split to float pairs
__global__ void fft_twiddle_kernel(float4 *table, int count, long long stride, int log2M) {
    const long long M = 1ll << log2M;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const long long m = ((long long)t * stride) & (M - 1);
        double s, c;
        sincospi(ldexp((double)(2 * m), -log2M), &s, &c);  // angle 2 pi m / M
        const double re = c, im = -s;
        const float rh = (float)re, ih = (float)im;
        table[t] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
    }
}

// per-stage twiddle table of a length-2^log2L transform: for each radix-8
// stage after the first (in execution order), 7 Ls entries W_{8Ls}^{k q},
// q = 1..7, k < Ls, computed in FP64 and split to float pairs
__global__ void fft_stage_twiddle_kernel(float4 *table, int log2L) {
    const int count = stage_table_count(log2L);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        int lg = first_radix_log2(log2L), Ls = 1 << lg, off = 0;  // lg = log2 Ls
        while (t >= off + 7 * Ls) {
            off += 7 * Ls;
            Ls *= 8;
            lg += 3;
        }
        const int r = t - off, q = r / Ls + 1, k = r % Ls;
        const long long m = ((long long)k * q) & ((8ll << lg) - 1);  // W_{8Ls}^m, 8Ls = 2^(lg + 3)
        double sn, cs;
        sincospi(ldexp((double)(2 * m), -(lg + 3)), &sn, &cs);    // angle 2 pi m / (8 Ls)
        const double re = cs, im = -sn;
        const float rh = (float)re, ih = (float)im;
        table[t] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
    }
}

__global__ void __launch_bounds__(kFftThreads, 2)
    fft_group_kernel(const FftItem *items, int nitems, const FftGroupReq *reqs, const int *tlist, int *expo) {
    extern __shared__ __align__(16) float4 fsmem[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const FftItem item = items[it];
        fft_group_item(item, reqs, tlist, expo, fsmem, false);
    }
}

}  // namespace

// ------------------------------------------------------------------ plans
struct FftPlan {
    int log2n = -1, log2n1 = 0, log2n2 = 0;
    float4 *tables = nullptr;   // tw for each pass length, tw_hi, tw_lo
    const float4 *tw_single = nullptr, *tw_n1 = nullptr, *tw_n2 = nullptr, *tw_hi = nullptr,
                 *tw_lo = nullptr;
};

static int ilog2_exact(long long n) {
    int k = 0;
    while ((1ll << k) < n) ++k;
    return (1ll << k) == n ? k : -1;
}

FftPlan *fft_plan_create(long long n) {
    const int k = ilog2_exact(n);
    OO_REQUIRE(k >= 0 && k <= 24, OO_EINVAL, "FFT length must be a power of two, 1 .. 2^24");
    auto p = new FftPlan();
    p->log2n = k;
    const int four_step = k > 12;
    p->log2n1 = four_step ? k / 2 : k;
    p->log2n2 = four_step ? k - k / 2 : 0;
    OO_REQUIRE(p->log2n2 <= 12, OO_EINVAL, "FFT length above 2^24 not supported");
    size_t count = 0;
    if (!four_step) {
        count = (size_t)1 << k;
    } else {
        count = ((size_t)1 << p->log2n1) + ((size_t)1 << p->log2n2) + ((size_t)1 << (k - kTwSplit > 0 ? k - kTwSplit : 0)) +
                ((size_t)1 << kTwSplit);
    }
    try {
        OO_CUDA_TRY(cudaMalloc(&p->tables, std::max<size_t>(count, 1) * sizeof(float4)));
        float4 *t = p->tables;
        auto gen = [&](int cnt, long long stride, int log2M) {
            fft_twiddle_kernel<<<std::max(1, std::min(1024, (cnt + 255) / 256)), 256>>>(t, cnt, stride, log2M);
            OO_CUDA_TRY(cudaGetLastError());
            const float4 *r = t;
            t += cnt;
            return r;
        };
        auto gen_stages = [&](int lg) {
            const int cnt = stage_table_count(lg);
            if (cnt > 0) {
                fft_stage_twiddle_kernel<<<std::max(1, std::min(1024, (cnt + 255) / 256)), 256>>>(t, lg);
                OO_CUDA_TRY(cudaGetLastError());
            }
            const float4 *r = t;
            t += (size_t)1 << lg;  // a table slot of 2^lg entries (count < 2^lg)
            return r;
        };
        if (!four_step) {
            p->tw_single = gen_stages(k);
        } else {
            p->tw_n1 = gen_stages(p->log2n1);
            p->tw_n2 = gen_stages(p->log2n2);
            p->tw_hi = gen(1 << std::max(0, k - kTwSplit), 1ll << kTwSplit, k);
            p->tw_lo = gen(1 << kTwSplit, 1, k);
        }
        OO_CUDA_TRY(cudaDeviceSynchronize());
    } catch (...) {
        if (p->tables) cudaFree(p->tables);
        delete p;
        throw;
    }
    return p;
}

int fft_plan_log2(const FftPlan *p) { return p->log2n; }

void fft_plan_tables(const FftPlan *p, const void **tw, const void **tw_n1, const void **tw_n2, const void **tw_hi,
                     const void **tw_lo, int *log2n, int *log2n1, int *log2n2) {
    *tw = p->tw_single;
    *tw_n1 = p->tw_n1;
    *tw_n2 = p->tw_n2;
    *tw_hi = p->tw_hi;
    *tw_lo = p->tw_lo;
    *log2n = p->log2n;
    *log2n1 = p->log2n1;
    *log2n2 = p->log2n2;
}

void fft_plan_destroy(FftPlan *p) {
    if (!p) return;
    if (p->tables) cudaFree(p->tables);
    delete p;
}

size_t fft_scratch_bytes(const FftPlan *p, int batch) {
    const size_t n = (size_t)1 << p->log2n;
    if (p->log2n <= 12) return 256;  // one pass: nothing beyond the CTAs' shared memory
    // four-step: the intermediates, each transform's exponent and its
    // first-pass columns' exponents
    return n * (size_t)batch * sizeof(float4) + (size_t)batch * sizeof(int) * (1 + ((size_t)1 << p->log2n2)) + 256;
}

void launch_fft(const FftPlan *p, int batch, int dir, const double *in, double *out, void *scratch,
                cudaStream_t s) {
    OO_REQUIRE(batch >= 1, OO_EINVAL, "batch must be >= 1");
    OO_REQUIRE(dir == -1 || dir == 1, OO_EINVAL, "dir must be -1 (forward) or +1 (inverse)");
    const long long n = 1ll << p->log2n;
    const bool four_step = p->log2n > 12;
    if (n == 1) {  // the length-1 transform (either direction) is the identity, exactly
        if (in != out)
            OO_CUDA_TRY(cudaMemcpyAsync(out, in, (size_t)batch * 16, cudaMemcpyDeviceToDevice, s));
        return;
    }
    FftArgs a{};
    if (four_step) {
        float4 *mid = reinterpret_cast<float4 *>(scratch);
        a.expo = reinterpret_cast<int *>(reinterpret_cast<char *>(scratch) + (size_t)n * batch * sizeof(float4));
        a.colmax = a.expo + batch;
        a.out_ff = mid;
        a.in_ff = mid;
        OO_CUDA_TRY(cudaMemsetAsync(a.expo, 0, (size_t)batch * sizeof(int), s));
    }
    a.log2n = p->log2n;
    a.log2n1 = p->log2n1;
    a.log2n2 = p->log2n2;
    a.n = n;
    a.batch = batch;
    a.inverse = dir > 0 ? 1 : 0;
    static std::atomic<uint64_t> attr_done[6];
    auto smem_for = [&](int log2L) { return fft_smem_bytes(log2L); };
    // the pass kernel of a mode in the layout of a pass length, its shared-
    // memory limit raised once per device
    auto pick = [&](int mode, int log2L) {
        const bool pad = fft_padded(log2L);
        const void *fn = mode == 0 ? (pad ? (const void *)fft_pass_kernel<0, true> : (const void *)fft_pass_kernel<0, false>)
                       : mode == 1 ? (pad ? (const void *)fft_pass_kernel<1, true> : (const void *)fft_pass_kernel<1, false>)
                                   : (pad ? (const void *)fft_pass_kernel<2, true> : (const void *)fft_pass_kernel<2, false>);
        set_smem_limit_once(fn, kFftSmemMax, attr_done[2 * mode + (pad ? 1 : 0)]);
        return fn;
    };
    auto launch = [&](const void *fn, long long grid, size_t smem) {
        void *args[] = {&a};
        OO_CUDA_TRY(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kFftThreads), args, smem, s));
    };
    if (!four_step) {
        const int C = kFftElems >> p->log2n;
        const int grid = (int)((batch + C - 1) / C);
        a.in_d = in;
        a.out_d = out;
        a.tw = p->tw_single;
        launch(pick(0, p->log2n), grid, smem_for(p->log2n));
        return;
    }
    const int N1 = 1 << p->log2n1, N2 = 1 << p->log2n2;
    a.tw_hi = p->tw_hi;
    a.tw_lo = p->tw_lo;
    {
        a.in_d = in;
        a.tw = p->tw_n1;
        const int C = kFftElems / N1;
        const long long grid = (long long)batch * (N2 / C);
        launch(pick(1, p->log2n1), grid, smem_for(p->log2n1));
    }
    {
        a.out_d = out;
        a.tw = p->tw_n2;
        const int R = kFftElems / N2;
        const long long grid = (long long)batch * (N1 / R);
        launch(pick(2, p->log2n2), grid, smem_for(p->log2n2));
    }
}

// ------------------------------------------------------------ group plans
struct FftGroup {
    void *arena = nullptr;
    FftItem *d_items = nullptr;
    FftGroupReq *d_reqs = nullptr;
    int *d_tlist = nullptr, *d_expo = nullptr;
    // three launches: [0] whole transforms and column passes with L <= 2048,
    // [1] whole transforms of 4096 points (a 64 KB twiddle table: one CTA per
    // SM), [2] row passes (after every column pass); items stored in that order
    int n_items[3] = {0, 0, 0}, grid[3] = {1, 1, 1};
    size_t smem[3] = {0, 0, 0};
    int nreq = 0;
    double elems = 0;
};

FftGroup *fft_group_create(const std::vector<FftDesc> &v, const std::vector<const FftPlan *> &plans, int num_sms) {
    OO_REQUIRE(!v.empty() && v.size() == plans.size(), OO_EINVAL, "empty FFT group");
    OO_REQUIRE(v.size() <= 65535, OO_EINVAL, "at most 65535 transforms in a group");
    auto up = [](size_t x, size_t a) { return (x + a - 1) / a * a; };
    size_t at = 0;
    std::vector<size_t> off_mid(v.size(), 0), off_colmax(v.size(), 0);
    for (size_t i = 0; i < v.size(); ++i) {
        OO_REQUIRE(v[i].dir == -1 || v[i].dir == 1, OO_EINVAL, "dir must be -1 or +1");
        OO_REQUIRE((((uintptr_t)v[i].in) & 15u) == 0 && (((uintptr_t)v[i].out) & 15u) == 0, OO_EINVAL,
                   "FFT buffers must be 16-byte aligned");
        if (plans[i]->log2n > 12) {
            off_mid[i] = at;
            at += up(((size_t)1 << plans[i]->log2n) * sizeof(float4), 256);
            off_colmax[i] = at;  // the first pass's column exponents
            at += up(((size_t)1 << plans[i]->log2n2) * sizeof(int), 256);
        }
    }
    // items: whole transforms grouped by (length, direction); then the passes
    std::vector<FftItem> items_a, items_b;
    std::vector<int> tlist;
    std::vector<std::pair<std::pair<int, int>, int>> small;
    for (size_t i = 0; i < v.size(); ++i)
        if (plans[i]->log2n <= 12) small.push_back({{plans[i]->log2n, v[i].dir}, (int)i});
    std::stable_sort(small.begin(), small.end(),
                     [](const std::pair<std::pair<int, int>, int> &x, const std::pair<std::pair<int, int>, int> &y) {
                         return x.first < y.first;
                     });
    for (size_t a = 0; a < small.size();) {
        size_t b = a;
        while (b < small.size() && small[b].first == small[a].first) ++b;
        const int log2L = small[a].first.first, C = kFftElems >> log2L;
        for (size_t c = a; c < b; c += C) {
            const int cnt = (int)std::min<size_t>(C, b - c);
            items_a.push_back(FftItem{0, log2L, (int)tlist.size(), cnt, 0, 0, 0, 0});
            for (int x = 0; x < cnt; ++x) tlist.push_back(small[c + x].second);
        }
        a = b;
    }
    for (size_t i = 0; i < v.size(); ++i) {
        const FftPlan *p = plans[i];
        if (p->log2n <= 12) continue;
        const int N1 = 1 << p->log2n1, N2 = 1 << p->log2n2;
        const int C1 = kFftElems / N1, C2 = kFftElems / N2;
        for (int c0 = 0; c0 < N2; c0 += C1) items_a.push_back(FftItem{1, p->log2n1, (int)i, 0, c0, 0, 0, 0});
        for (int r0 = 0; r0 < N1; r0 += C2) items_b.push_back(FftItem{2, p->log2n2, (int)i, 0, r0, 0, 0, 0});
    }
    at = up(at, 256);
    const size_t off_items = at; at += up((items_a.size() + items_b.size()) * sizeof(FftItem), 256);
    const size_t off_reqs = at; at += up(v.size() * sizeof(FftGroupReq), 256);
    const size_t off_tlist = at; at += up(std::max<size_t>(tlist.size(), 1) * 4, 256);
    const size_t off_expo = at; at += up(v.size() * 4, 256);
    auto *g = new FftGroup();
    try {
        if (cudaMalloc(&g->arena, at) != cudaSuccess) {
            cudaGetLastError();
            throw Error{OO_ENOMEM, "FFT group arena of " + std::to_string(at) + " bytes"};
        }
        char *base = static_cast<char *>(g->arena);
        std::vector<FftGroupReq> reqs(v.size());
        double elems = 0;
        for (size_t i = 0; i < v.size(); ++i) {
            const FftPlan *p = plans[i];
            reqs[i] = FftGroupReq{v[i].in, v[i].out,
                                  p->log2n > 12 ? reinterpret_cast<float4 *>(base + off_mid[i]) : nullptr,
                                  p->tw_single, p->tw_n1, p->tw_n2, p->tw_hi, p->tw_lo,
                                  p->log2n > 12 ? reinterpret_cast<int *>(base + off_colmax[i]) : nullptr,
                                  p->log2n, p->log2n1, p->log2n2, v[i].dir > 0 ? 1 : 0};
            elems += (double)(1ll << p->log2n);
        }
        std::vector<FftItem> part[3];
        for (const FftItem &it : items_a) part[it.log2L == 12 ? 1 : 0].push_back(it);
        part[2] = items_b;
        std::vector<FftItem> all;
        for (int q = 0; q < 3; ++q) {
            all.insert(all.end(), part[q].begin(), part[q].end());
            g->n_items[q] = (int)part[q].size();
            // data + the largest per-stage twiddle table staged in this launch
            size_t smem = fft_smem_bytes(0);
            for (const FftItem &it : part[q]) smem = std::max(smem, fft_smem_bytes(it.log2L));
            g->smem[q] = smem;
            const int per_sm = g->smem[q] <= (size_t)110 * 1024 ? 2 : 1;
            g->grid[q] = std::max(1, std::min(g->n_items[q], num_sms * per_sm));
        }
        OO_CUDA_TRY(cudaMemcpy(base + off_items, all.data(), all.size() * sizeof(FftItem), cudaMemcpyHostToDevice));
        OO_CUDA_TRY(cudaMemcpy(base + off_reqs, reqs.data(), reqs.size() * sizeof(FftGroupReq), cudaMemcpyHostToDevice));
        if (!tlist.empty())
            OO_CUDA_TRY(cudaMemcpy(base + off_tlist, tlist.data(), tlist.size() * 4, cudaMemcpyHostToDevice));
        g->d_items = reinterpret_cast<FftItem *>(base + off_items);
        g->d_reqs = reinterpret_cast<FftGroupReq *>(base + off_reqs);
        g->d_tlist = reinterpret_cast<int *>(base + off_tlist);
        g->d_expo = reinterpret_cast<int *>(base + off_expo);
        g->nreq = (int)v.size();
        g->elems = elems;
    } catch (...) {
        if (g->arena) cudaFree(g->arena);
        delete g;
        throw;
    }
    return g;
}

void fft_group_launch(FftGroup *g, cudaStream_t s) {
    OO_CUDA_TRY(cudaMemsetAsync(g->d_expo, 0, (size_t)g->nreq * 4, s));  // raised by the column passes
    static std::atomic<uint64_t> attr{0};
    set_smem_limit_once((const void *)fft_group_kernel, kFftSmemMax, attr);
    int first = 0;
    for (int q = 0; q < 3; ++q) {
        if (g->n_items[q] > 0) {
            fft_group_kernel<<<g->grid[q], kFftThreads, g->smem[q], s>>>(g->d_items + first, g->n_items[q],
                                                                          g->d_reqs, g->d_tlist, g->d_expo);
            OO_CUDA_TRY(cudaGetLastError());
        }
        first += g->n_items[q];
    }
}

double fft_group_elements(const FftGroup *g) { return g->elems; }

void fft_group_destroy(FftGroup *g) {
    if (!g) return;
    if (g->arena) cudaFree(g->arena);
    delete g;
}

}  // namespace oo
