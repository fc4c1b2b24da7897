// GPU nests of the Jacobi program (sm_103a).
//
// The six loop nests a gene can place on the GPU (Sec. 3.2.1, Sec. 4.2.2):
//   N0 coef      fill the twelve coefficient arrays           (write stream)
//   N1 pinit     p = wrk2 = (k/(K-1))^2                        (write stream)
//   N2 stencil   19-point update + FP64 residual               (HBM bound)
//   N3 copyback  p = wrk2 on the interior                      (copy)
//   N4 bc_ij     Dirichlet faces i, j                          (tiny)
//   N5 bc_k      Dirichlet faces k                             (tiny)
// When N3, N4 and N5 all run on the GPU with no copy between them, one pass
// (copyback_faces_kernel) writes what the three leave; on small grids with
// every iteration nest on the GPU, one cooperative kernel runs all
// iterations (jacobi_fused_kernel).
//
// Device layout: each array is I x J x pitch floats, k fastest, pitch a
// multiple of 32 floats (128-byte rows) so every row starts on a TMA- and
// float4-aligned address.
//
// N2 is a persistent, warp-specialised kernel.  One producer thread streams
// tiles with TMA (cp.async.bulk.tensor) into shared memory: for every plane i
// of a work unit, the twelve coefficient tiles (TK x TJ) and one p tile with
// a one-point halo in j and a 4-float-aligned halo in k.  Consumer warps
// march i through the unit with the three p planes i-1, i, i+1 resident in a
// ring, compute the update in float-float arithmetic (error-free sums and
// FMA products, about 44 significant bits, rounded once at the store), and
// accumulate ss^2 in float-float per thread and in FP64 per warp and unit.
// Every unit's partial residuals go to scratch; the last CTA to finish sums
// them in unit order, so the residual is deterministic.  Five tile variants
// (tile shape, consumer warps, points per thread, CTAs per SM) compute the
// same values; a rule by row length picks one unless a plan is given one
// (the autotuner, oo_tune_stencil).  Every mbarrier wait is bounded; a wait that runs out
// sets an error word the host reads, drains the copies in flight and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "ff.cuh"
#include "jacobi_point.cuh"
#include "oo_internal.h"

namespace oo {

// ===================================================================== helpers
namespace {

constexpr long long kWaitLimitCycles = 2000000000ll;  // ~1 s at 2 GHz

__device__ __forceinline__ float dirichlet_dev(int k, int K) {
    return __fdiv_rn((float)(k * k), (float)((K - 1) * (K - 1)));
}

using ff::two_prod;
using ff::two_sum;
// (H, L) += (th, tl)
__device__ __forceinline__ void ff_acc(float &H, float &L, float th, float tl) { ff::acc(H, L, th, tl); }

// -------- mbarrier / TMA (inline PTX)
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            bar),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait.  Returns false when the CTA aborted or the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned *err, unsigned code) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitLimitCycles) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint32_t bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar), "l"(policy)
        : "memory");
}

}  // namespace

// ============================================================ simple nests
namespace {

__global__ void coef_kernel(float *base, size_t stride, size_t n4) {
    const float val[NCOEF] = {1.0f, 1.0f, 1.0f, 1.0f / 6.0f, 0.0f, 0.0f,
                              0.0f, 1.0f, 1.0f, 1.0f,        1.0f, 0.0f};
    const size_t step = (size_t)gridDim.x * blockDim.x;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n4; x += step) {
#pragma unroll
        for (int a = 0; a < NCOEF; ++a) {
            const float v = val[a];
            reinterpret_cast<float4 *>(base + a * stride)[x] = make_float4(v, v, v, v);
        }
    }
}

// rows = I*J, each `pitch` floats; thread handles float4 chunk c of row r.
__global__ void pinit_kernel(float *p, float *wrk2, int rows, int pitch, int K) {
    const unsigned chunks = (unsigned)pitch / 4u;
    const size_t total = (size_t)rows * chunks;
    const size_t step = (size_t)gridDim.x * blockDim.x;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += step) {
        const int k = (int)(x % chunks) * 4;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = (k + e < K) ? dirichlet_dev(k + e, K) : 0.0f;
        const float4 q = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4 *>(p)[x] = q;
        reinterpret_cast<float4 *>(wrk2)[x] = q;
    }
}

// One warp per interior row (i, j): its lanes copy the row's float4 chunks
// (k in [0, 4 ceil((K-1)/4))), interior k only; one division per row.
__global__ void copyback_kernel(float *__restrict__ p, const float *__restrict__ wrk2, int I, int J, int K,
                                int pitch) {
    const long long jr = J - 2, rows = (long long)(I - 2) * jr;
    const int chunks = (K - 1 + 3) / 4;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (long long r = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (long long)gridDim.x * wpb) {
        const long long i = 1 + r / jr, j = 1 + r % jr;
        const size_t off = ((size_t)i * J + (size_t)j) * pitch;
        const float4 *src = reinterpret_cast<const float4 *>(wrk2 + off);
        float4 *dst = reinterpret_cast<float4 *>(p + off);
#pragma unroll 4
        for (int c = lane; c < chunks; c += 32) {
            const int k = 4 * c;
            if (k >= 1 && k + 3 <= K - 2) {
                dst[c] = src[c];
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (k + e >= 1 && k + e <= K - 2) p[off + k + e] = wrk2[off + k + e];
            }
        }
    }
}

// N3, N4 and N5 in one pass, for patterns that run all three on the GPU
// with no copy between them: one warp per (i, j) row of p; an interior row
// takes wrk2 on 1 <= k <= K-2 and g(0), g(K-1) at its ends, a face row g(k)
// everywhere.  Every element is written once, with the values the three
// nests leave in sequence (interior copy, then the i / j faces, then the k
// faces, which all hold g).
__global__ void copyback_faces_kernel(float *__restrict__ p, const float *__restrict__ wrk2, int I, int J, int K,
                                      int pitch) {
    const long long rows = (long long)I * J;
    const int chunks = (K + 3) / 4;
    const float g0 = dirichlet_dev(0, K), g1 = dirichlet_dev(K - 1, K);
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (long long r = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (long long)gridDim.x * wpb) {
        const int i = (int)(r / J), j = (int)(r % J);
        const size_t off = (size_t)r * pitch;
        float4 *dst = reinterpret_cast<float4 *>(p + off);
        if (i == 0 || i == I - 1 || j == 0 || j == J - 1) {
            for (int c = lane; c < chunks; c += 32) {
                const int k = 4 * c;
                if (k + 3 < K) {
                    dst[c] = make_float4(dirichlet_dev(k, K), dirichlet_dev(k + 1, K), dirichlet_dev(k + 2, K),
                                         dirichlet_dev(k + 3, K));
                } else {
                    for (int e = 0; e < 4 && k + e < K; ++e) p[off + k + e] = dirichlet_dev(k + e, K);
                }
            }
            continue;
        }
        const float4 *src = reinterpret_cast<const float4 *>(wrk2 + off);
#pragma unroll 4
        for (int c = lane; c < chunks; c += 32) {
            const int k = 4 * c;
            if (k + 3 < K) {
                float4 v = src[c];
                if (k == 0) v.x = g0;
                if (k + 3 == K - 1) v.w = g1;
                dst[c] = v;
            } else {
                for (int e = 0; e < 4 && k + e < K; ++e) {
                    const int kk = k + e;
                    p[off + kk] = kk == 0 ? g0 : (kk == K - 1 ? g1 : wrk2[off + kk]);
                }
            }
        }
    }
}

__global__ void bc_ij_kernel(float *p, int I, int J, int K, int pitch) {
    const unsigned chunks = (unsigned)(K + 3) / 4u;
    const unsigned face_rows = 2u * J + 2u * (I - 2);
    const size_t total = (size_t)face_rows * chunks;
    const size_t step = (size_t)gridDim.x * blockDim.x;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += step) {
        const unsigned c = (unsigned)(x % chunks);
        const unsigned r = (unsigned)(x / chunks);
        int i, j;
        if (r < 2u * J) {
            i = (r < (unsigned)J) ? 0 : I - 1;
            j = (int)(r % (unsigned)J);
        } else {
            const unsigned q = r - 2u * J;
            i = 1 + (int)(q / 2u);
            j = (q % 2u) ? J - 1 : 0;
        }
        const size_t off = ((size_t)i * J + j) * pitch + 4u * c;
        const int k = 4 * (int)c;
        if (k + 3 < K) {
            reinterpret_cast<float4 *>(p + off)[0] =
                make_float4(dirichlet_dev(k, K), dirichlet_dev(k + 1, K), dirichlet_dev(k + 2, K),
                            dirichlet_dev(k + 3, K));
        } else {
            for (int e = 0; e < 4 && k + e < K; ++e) p[off + e] = dirichlet_dev(k + e, K);
        }
    }
}

__global__ void bc_k_kernel(float *p, int rows, int K, int pitch) {
    const float g0 = dirichlet_dev(0, K), g1 = dirichlet_dev(K - 1, K);
    const int step = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += step) {
        p[(size_t)r * pitch] = g0;
        p[(size_t)r * pitch + K - 1] = g1;
    }
}

int grid_for(size_t work, int threads, int max_blocks) {
    const size_t b = (work + threads - 1) / threads;
    return (int)std::max<size_t>(1, std::min<size_t>(b, (size_t)max_blocks));
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return n;
}

}  // namespace

void launch_coef(const JacobiDims &d, float *const coef[NCOEF], cudaStream_t s) {
    const size_t stride = (size_t)(coef[1] - coef[0]);
    for (int a = 1; a < NCOEF; ++a)
        OO_REQUIRE((size_t)(coef[a] - coef[a - 1]) == stride, OO_EINVAL,
                   "coefficient arrays must be equally spaced");
    const size_t n4 = d.n_dev() / 4;
    coef_kernel<<<grid_for(n4, 256, sm_count() * 8), 256, 0, s>>>(coef[0], stride, n4);
    OO_CUDA_TRY(cudaGetLastError());
}

void launch_pinit(const JacobiDims &d, float *p, float *wrk2, cudaStream_t s) {
    const size_t n4 = d.n_dev() / 4;
    pinit_kernel<<<grid_for(n4, 256, sm_count() * 8), 256, 0, s>>>(p, wrk2, d.I * d.J, d.pitch, d.K);
    OO_CUDA_TRY(cudaGetLastError());
}

void launch_copyback(const JacobiDims &d, float *p, const float *wrk2, cudaStream_t s) {
    const size_t rows = (size_t)(d.I - 2) * (d.J - 2);  // one warp each, 8 warps per block
    copyback_kernel<<<grid_for(rows, 8, sm_count() * 16), 256, 0, s>>>(p, wrk2, d.I, d.J, d.K, d.pitch);
    OO_CUDA_TRY(cudaGetLastError());
}

void launch_copyback_faces(const JacobiDims &d, float *p, const float *wrk2, cudaStream_t s) {
    const size_t rows = (size_t)d.I * d.J;  // one warp each, 8 warps per block
    copyback_faces_kernel<<<grid_for(rows, 8, sm_count() * 16), 256, 0, s>>>(p, wrk2, d.I, d.J, d.K, d.pitch);
    OO_CUDA_TRY(cudaGetLastError());
}

void launch_bc_ij(const JacobiDims &d, float *p, cudaStream_t s) {
    const size_t work = (size_t)(2 * d.J + 2 * (d.I - 2)) * ((d.K + 3) / 4);
    bc_ij_kernel<<<grid_for(work, 256, sm_count() * 4), 256, 0, s>>>(p, d.I, d.J, d.K, d.pitch);
    OO_CUDA_TRY(cudaGetLastError());
}

void launch_bc_k(const JacobiDims &d, float *p, cudaStream_t s) {
    const int rows = d.I * d.J;
    bc_k_kernel<<<grid_for(rows, 256, sm_count() * 4), 256, 0, s>>>(p, rows, d.K, d.pitch);
    OO_CUDA_TRY(cudaGetLastError());
}

// ======================================================= fused iterations
// All iterations of the all-GPU iteration nests (N2 stencil, N3 copy-back,
// N4 / N5 boundary) in one cooperative launch, for grids small enough that
// launch latency, not HBM, bounds the separate kernels.  Per iteration:
// the stencil over the interior (each thread a strided set of points, the
// same float-float arithmetic as the tiled kernel, term by term), a grid
// barrier, block 0 sums the per-block FP64 residual partials in block
// order, every point of p is rewritten (interior = wrk2, faces = g(k), i.e.
// N3, N4 and N5), a second grid barrier.  Barrier waits are bounded: a wait
// that runs out sets the error word and every block leaves at its next
// barrier.
namespace {

struct FusedArgs {
    const float *coef[NCOEF];
    float *p, *wrk2;
    double *res;
    double *partials;       // gridDim.x
    unsigned *ctl;          // [0] arrivals, [1] generation, [2] error
    int I, J, K, pitch, iters;
    float omega;
    unsigned barrier_extra;  // fault injection: arrivals awaited beyond the grid (0 in normal runs)
};

__device__ __forceinline__ bool fused_grid_barrier(unsigned *ctl, unsigned extra) {
    __syncthreads();
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = ctl + 1, *err = ctl + 2;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(ctl, 1u) == gridDim.x - 1 + extra) {
            atomicExch(ctl, 0u);
            __threadfence();
            atomicAdd(ctl + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (*err) break;
                if (clock64() - t0 > kWaitLimitCycles) {
                    atomicOr(ctl + 2, 1u);
                    break;
                }
            }
        }
        __threadfence();
        ok_s = *err == 0;
    }
    __syncthreads();
    return ok_s != 0;
}

__global__ void __launch_bounds__(512, 1) jacobi_fused_kernel(FusedArgs a) {
    __shared__ double red[16];
    const int I = a.I, J = a.J, K = a.K, Ji = J - 2, Ki = K - 2;
    const int nint = (I - 2) * Ji * Ki, nall = I * J * K;
    const int stride = gridDim.x * blockDim.x, tid0 = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t sj = a.pitch, si = (size_t)J * a.pitch;
    const float omega = a.omega;
    for (int it = 0; it < a.iters; ++it) {
        // ---- N2: stencil on the interior
        float RH = 0.0f, RL = 0.0f;
        for (int x = tid0; x < nint; x += stride) {
            const int k = 1 + x % Ki, r = x / Ki, j = 1 + r % Ji, i = 1 + r / Ji;
            stencil_point_ff(a.coef, a.p, (size_t)i * si + (size_t)j * sj + k, si, sj, omega, a.wrk2, RH, RL);
        }
        double v = (double)RH + (double)RL;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
            a.partials[blockIdx.x] = b;
        }
        if (!fused_grid_barrier(a.ctl, a.barrier_extra)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double sum = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) sum += __ldcg(&a.partials[b]);
            a.res[it] = sum;
        }
        // ---- N3 copy-back (interior), N4 / N5 faces = g(k)
        for (int x = tid0; x < nall; x += stride) {
            const int k = x % K, r = x / K, j = r % J, i = r / J;
            const size_t c = (size_t)i * si + (size_t)j * sj + k;
            const bool interior = i >= 1 && i <= I - 2 && j >= 1 && j <= J - 2 && k >= 1 && k <= K - 2;
            a.p[c] = interior ? __ldcg(&a.wrk2[c]) : dirichlet_dev(k, K);
        }
        if (!fused_grid_barrier(a.ctl, a.barrier_extra)) return;
    }
}

}  // namespace

size_t jacobi_fused_ctl_bytes() { return 256 + (size_t)sm_count() * 8; }

bool jacobi_fused_eligible(const JacobiDims &d, int option) {
    if (option == 0) return false;
    const long long nall = (long long)d.I * d.J * d.K;
    if (option == 1) return nall < (1ll << 31);
    // measured (all iteration nests, 100 iterations): fused 0.74 vs 1.17 ms at
    // 33 x 33 x 65, 2.73 vs 2.87 ms at 65 x 65 x 129, but 5.36 vs 4.83 ms at
    // 97 x 97 x 193, where the tiled kernels' bandwidth wins
    return nall <= (1ll << 20);
}

void launch_jacobi_fused(const JacobiDims &d, const float *const coef[NCOEF], float *p, float *wrk2, float omega,
                         int iters, double *res_dev, void *ctl, cudaStream_t s, bool inject_timeout) {
    OO_REQUIRE((long long)d.I * d.J * d.K < (1ll << 31), OO_EINVAL, "grid too large for the fused iterations");
    if (iters <= 0) return;
    // one 512-thread block per SM: every grid barrier is sm_count() arrivals
    // on one counter (thousands of small blocks made the barriers the cost)
    static std::atomic<int> fits{-1};
    if (fits.load() < 0) {
        int b = 0;
        OO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, jacobi_fused_kernel, 512, 0));
        fits.store(b >= 1 ? 1 : 0);
    }
    OO_REQUIRE(fits.load() == 1, OO_ECUDA, "fused Jacobi kernel does not fit an SM");
    const long long nall = (long long)d.I * d.J * d.K;
    const int grid = (int)std::max<long long>(1, std::min<long long>(sm_count(), (nall + 511) / 512));
    FusedArgs a{};
    for (int q = 0; q < NCOEF; ++q) a.coef[q] = coef[q];
    a.p = p;
    a.wrk2 = wrk2;
    a.res = res_dev;
    a.ctl = static_cast<unsigned *>(ctl);
    a.partials = reinterpret_cast<double *>(static_cast<char *>(ctl) + 256);
    a.I = d.I;
    a.J = d.J;
    a.K = d.K;
    a.pitch = d.pitch;
    a.iters = iters;
    a.omega = omega;
    a.barrier_extra = inject_timeout ? 1u : 0u;  // one arrival that never comes
    OO_CUDA_TRY(cudaMemsetAsync(ctl, 0, 16, s));
    void *args[] = {&a};
    OO_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)jacobi_fused_kernel, dim3(grid), dim3(512), args, 0, s));
}

unsigned jacobi_fused_check(void *ctl, cudaStream_t s) {
    unsigned e = 0;
    OO_CUDA_TRY(cudaMemcpyAsync(&e, static_cast<char *>(ctl) + 8, 4, cudaMemcpyDeviceToHost, s));
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    return e;
}

// ================================================================== stencil
struct StencilMaps {
    CUtensorMap coef[NCOEF];
    CUtensorMap p;
};

struct StencilArgs {
    int I, J, K, pitch;
    int n_kt, n_jt, n_seg, n_units;
    float omega;
    float *wrk2;
    double *partials;   // n_units
    unsigned *counter;  // CTAs finished (reset by the last one)
    unsigned *err;      // error bits
    double *res;        // FP64 residual of this sweep
};

namespace {

// residual partial slots per work unit in the scratch array: one per
// consumer warp, so no variant may have more consumer warps than this
constexpr int kMaxConsumerWarps = 16;

template <int TK, int TJ>
struct Tile {
    static constexpr int PW = TK + 8;                   // p tile row: k0-4 .. k0+TK+3
    static constexpr int PH = TJ + 2;                   // p tile rows: j0-1 .. j0+TJ
    static constexpr int PSLOT = (PW * PH + 31) / 32 * 32;  // floats, 128-byte multiple
    static constexpr int CTILE = TK * TJ;               // floats per coefficient tile
    static constexpr uint32_t PBYTES = PW * PH * 4;
    static constexpr uint32_t CBYTES = NCOEF * CTILE * 4;
};

__device__ __forceinline__ void decode_unit(const StencilArgs &a, int u, int I, int TK, int TJ,
                                            int &k0, int &j0, int &ib, int &ie) {
    const int kt = u % a.n_kt;
    const int jt = (u / a.n_kt) % a.n_jt;
    const int sg = u / (a.n_kt * a.n_jt);
    k0 = kt * TK;
    j0 = 1 + jt * TJ;
    const long long span = I - 2;
    ib = 1 + (int)(span * sg / a.n_seg);
    ie = 1 + (int)(span * (sg + 1) / a.n_seg);
}

// INJ (tests of the bounded waits only): the producer never issues its first
// p-tile copy, so the consumers' wait for it runs out; a separate
// instantiation, so the kernel that runs normally carries no trace of it.
template <int TK, int TJ, int NCW, int DC, int DP, int PPT, int MINB, bool INJ>
__global__ void __launch_bounds__((NCW + 1) * 32, MINB)
    stencil_kernel(const __grid_constant__ StencilMaps maps, const StencilArgs a) {
    using T = Tile<TK, TJ>;
    static_assert(NCW <= kMaxConsumerWarps, "more consumer warps than partial slots per unit");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations need 128-byte alignment; the launch adds 128 bytes of slack
    unsigned char *smem_base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    float *coef_s = reinterpret_cast<float *>(smem_base);
    float *p_s = coef_s + (size_t)DC * NCOEF * T::CTILE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(p_s + (size_t)DP * T::PSLOT);
    uint64_t *full_c = bars, *empty_c = bars + DC, *full_p = bars + 2 * DC,
             *empty_p = bars + 2 * DC + DP;
    double *red = reinterpret_cast<double *>(bars + 2 * (DC + DP));  // 32 doubles
    volatile int *abort_flag = reinterpret_cast<volatile int *>(red + 32);
    int *last_flag = const_cast<int *>(reinterpret_cast<volatile int *>(abort_flag + 1));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int c = 0; c < DC; ++c) {
            mbar_init(smem_u32(&full_c[c]), 1);
            mbar_init(smem_u32(&empty_c[c]), NCW);
        }
        for (int q = 0; q < DP; ++q) {
            mbar_init(smem_u32(&full_p[q]), 1);
            mbar_init(smem_u32(&empty_p[q]), NCW);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    const int I = a.I, J = a.J, K = a.K;

    if (warp == NCW) {
        // ------------------------------------------------------ producer
        if (lane == 0) {
            const uint64_t pol_stream = policy_evict_first();
            const uint64_t pol_p = policy_evict_last();
            uint32_t cfill = 0, pfill = 0;
            bool ok = true;
            for (int u = blockIdx.x; ok && u < a.n_units; u += gridDim.x) {
                int k0, j0, ib, ie;
                decode_unit(a, u, I, TK, TJ, k0, j0, ib, ie);
                for (int q = ib - 1; q <= ie; ++q) {
                    {
                        const uint32_t slot = pfill % DP, use = pfill / DP;
                        if (use > 0 &&
                            !mbar_wait(smem_u32(&empty_p[slot]), (use - 1) & 1, abort_flag, a.err, 1u)) {
                            ok = false;
                            break;
                        }
                        const uint32_t bar = smem_u32(&full_p[slot]);
                        if (!(INJ && pfill == 0)) {
                            mbar_expect_tx(bar, T::PBYTES);
                            tma_load_3d(smem_u32(p_s + (size_t)slot * T::PSLOT), &maps.p, k0 - 4, j0 - 1, q,
                                        bar, pol_p);
                        }
                        ++pfill;
                    }
                    if (q >= ib + 1) {
                        const uint32_t slot = cfill % DC, use = cfill / DC;
                        if (use > 0 &&
                            !mbar_wait(smem_u32(&empty_c[slot]), (use - 1) & 1, abort_flag, a.err, 2u)) {
                            ok = false;
                            break;
                        }
                        const uint32_t bar = smem_u32(&full_c[slot]);
                        mbar_expect_tx(bar, T::CBYTES);
                        float *dst = coef_s + (size_t)slot * NCOEF * T::CTILE;
#pragma unroll
                        for (int c = 0; c < NCOEF; ++c)
                            tma_load_3d(smem_u32(dst + c * T::CTILE), &maps.coef[c], k0, j0, q - 1, bar,
                                        pol_stream);
                        ++cfill;
                    }
                }
            }
            if (!ok) {
                // drain: wait (bounded) for the last fill of every slot to land
                for (int s = 0; s < DP; ++s) {
                    const uint32_t n = pfill > (uint32_t)s ? (pfill - 1 - s) / DP : 0;
                    if (pfill > (uint32_t)s) {
                        const long long t0 = clock64();
                        while (!mbar_try(smem_u32(&full_p[s]), n & 1) && clock64() - t0 < kWaitLimitCycles) {
                        }
                    }
                }
                for (int s = 0; s < DC; ++s) {
                    const uint32_t n = cfill > (uint32_t)s ? (cfill - 1 - s) / DC : 0;
                    if (cfill > (uint32_t)s) {
                        const long long t0 = clock64();
                        while (!mbar_try(smem_u32(&full_c[s]), n & 1) && clock64() - t0 < kWaitLimitCycles) {
                        }
                    }
                }
            }
        }
    } else {
        // ------------------------------------------------------ consumers
        // Each thread owns PPT consecutive k points of one tile row and marches
        // them through the unit's planes.  Carried in registers from plane to
        // plane: the row-(j) window of planes i-1 and i, the j+-1 centres of
        // plane i, D = p(j+1) - p(j-1) on plane i (exact two-sum pairs, all
        // window positions) and its centres on plane i-1.  Per plane only the
        // three rows of plane i+1 are read from shared memory, and every cross
        // difference is one float-float subtraction of carried exact pairs:
        //   Xij = D(i+1) - D(i-1),  Xjk = D(i)(k+1) - D(i)(k-1),
        //   Xik = F(k+1) - F(k-1)  with  F = p(i+1) - p(i-1)  on row j.
        constexpr int QR = TK / PPT;                     // point groups per tile row
        static_assert(TJ * QR == NCW * 32, "one point group per consumer thread");
        static_assert(PPT == 2 || PPT == 4, "2 or 4 points per group");
        constexpr int W = PPT + 2;                       // window: k-1 .. k+PPT
        using VecT = typename std::conditional<PPT == 4, float4, float2>::type;
        const float omega = a.omega;
        const int r = (warp * 32 + lane) / QR, cg = (warp * 32 + lane) % QR;
        const int cc = PPT * cg + 4;                     // p-tile column of the group's first k
        auto winw = [&](const float *P, int row, float w[W]) {
            const float *base = P + row * T::PW + cc;
            const VecT v = *reinterpret_cast<const VecT *>(base);
            const float *vf = reinterpret_cast<const float *>(&v);
            w[0] = base[-1];
#pragma unroll
            for (int e = 0; e < PPT; ++e) w[e + 1] = vf[e];
            w[PPT + 1] = base[PPT];
        };
        auto winc = [&](const float *P, int row, float w[PPT]) {
            const VecT v = *reinterpret_cast<const VecT *>(P + row * T::PW + cc);
            const float *vf = reinterpret_cast<const float *>(&v);
#pragma unroll
            for (int e = 0; e < PPT; ++e) w[e] = vf[e];
        };
        // float-float difference (ah + al) - (bh + bl), unnormalised
        auto ffsub = [](float ah, float al, float bh, float bl, float &h, float &l) {
            float e;
            two_sum(ah, -bh, h, e);
            l = __fadd_rn(e, __fsub_rn(al, bl));
        };
        uint32_t cuse = 0, pseq = 0;
        bool ok = true;
        for (int u = blockIdx.x; ok && u < a.n_units; u += gridDim.x) {
            int k0, j0, ib, ie;
            decode_unit(a, u, I, TK, TJ, k0, j0, ib, ie);
            const int j = j0 + r, kb = k0 + PPT * cg;
            const bool row_in = (j <= J - 2);
            float RH = 0.0f, RL = 0.0f;  // this thread's ss^2 sum over the unit (float-float)
            const uint32_t pbase = pseq;
            for (uint32_t s = pbase; s < pbase + 2; ++s)
                if (!mbar_wait(smem_u32(&full_p[s % DP]), (s / DP) & 1, abort_flag, a.err, 4u)) {
                    ok = false;
                    break;
                }
            if (!ok) break;
            // prologue: planes ib-1 and ib
            float Ww[W], Cw[W], Nc[PPT], Sc[PPT];
            float Dh[W], Dl[W], Gh[PPT], Gl[PPT];
            {
                const float *P0 = p_s + (size_t)(pbase % DP) * T::PSLOT;
                const float *P1 = p_s + (size_t)((pbase + 1) % DP) * T::PSLOT;
                float t0[PPT], t1[PPT], n6[W], s6[W];
                winw(P0, r + 1, Ww);
                winc(P0, r + 2, t0);
                winc(P0, r, t1);
#pragma unroll
                for (int e = 0; e < PPT; ++e) two_sum(t0[e], -t1[e], Gh[e], Gl[e]);
                winw(P1, r + 1, Cw);
                winw(P1, r + 2, n6);
                winw(P1, r, s6);
#pragma unroll
                for (int x = 0; x < W; ++x) two_sum(n6[x], -s6[x], Dh[x], Dl[x]);
#pragma unroll
                for (int e = 0; e < PPT; ++e) {
                    Nc[e] = n6[e + 1];
                    Sc[e] = s6[e + 1];
                }
            }
            // unrolled by two: the compiler renames the plane windows instead
            // of moving them every plane (0.8 % faster at 257 x 257 x 513;
            // by three is slower)
#pragma unroll 2
            for (int i = ib; ok && i < ie; ++i) {
                const uint32_t sprev = pbase + (uint32_t)(i - ib);
                const uint32_t snext = sprev + 2;
                if (!mbar_wait(smem_u32(&full_p[snext % DP]), (snext / DP) & 1, abort_flag, a.err, 4u) ||
                    !mbar_wait(smem_u32(&full_c[cuse % DC]), (cuse / DC) & 1, abort_flag, a.err, 8u)) {
                    ok = false;
                    break;
                }
                const float *P2 = p_s + (size_t)(snext % DP) * T::PSLOT;
                const float *CS = coef_s + (size_t)(cuse % DC) * NCOEF * T::CTILE;
                float Ew[W], ENw[W], ESw[W];
                winw(P2, r + 1, Ew);
                winw(P2, r + 2, ENw);
                winw(P2, r, ESw);
                float cf[NCOEF][PPT];
#pragma unroll
                for (int c = 0; c < NCOEF; ++c) {
                    const VecT v = *reinterpret_cast<const VecT *>(CS + c * T::CTILE + r * TK + PPT * cg);
                    const float *vf = reinterpret_cast<const float *>(&v);
#pragma unroll
                    for (int e = 0; e < PPT; ++e) cf[c][e] = vf[e];
                }
                __syncwarp();
                if (lane == 0) {
                    // all shared-memory reads of this plane are in registers
                    mbar_arrive(smem_u32(&empty_c[cuse % DC]));
                    mbar_arrive(smem_u32(&empty_p[sprev % DP]));
                }
                ++cuse;
                float DNh[W], DNl[W], Fh[W], Fl[W];
#pragma unroll
                for (int x = 0; x < W; ++x) {
                    two_sum(ENw[x], -ESw[x], DNh[x], DNl[x]);  // D on plane i+1
                    two_sum(Ew[x], -Ww[x], Fh[x], Fl[x]);      // F on row j
                }
                float out[PPT];
                bool inside[PPT];
                bool all_in = row_in;
#pragma unroll
                for (int e = 0; e < PPT; ++e) {
                    const int k = kb + e;
                    inside[e] = row_in && k >= 1 && k <= K - 2;
                    all_in = all_in && inside[e];
                    float H, L, th, tl, xh, xl, t1;
                    two_prod(cf[0][e], Ew[e + 1], H, L);                         // a0 p[i+1]
                    two_prod(cf[1][e], Nc[e], th, tl); ff_acc(H, L, th, tl);     // a1 p[j+1]
                    two_prod(cf[2][e], Cw[e + 2], th, tl); ff_acc(H, L, th, tl); // a2 p[k+1]
                    ffsub(DNh[e + 1], DNl[e + 1], Gh[e], Gl[e], xh, xl);        // b0 Xij
                    two_prod(cf[4][e], xh, th, t1);
                    tl = __fmaf_rn(cf[4][e], xl, t1);
                    ff_acc(H, L, th, tl);
                    ffsub(Dh[e + 2], Dl[e + 2], Dh[e], Dl[e], xh, xl);          // b1 Xjk
                    two_prod(cf[5][e], xh, th, t1);
                    tl = __fmaf_rn(cf[5][e], xl, t1);
                    ff_acc(H, L, th, tl);
                    ffsub(Fh[e + 2], Fl[e + 2], Fh[e], Fl[e], xh, xl);          // b2 Xik
                    two_prod(cf[6][e], xh, th, t1);
                    tl = __fmaf_rn(cf[6][e], xl, t1);
                    ff_acc(H, L, th, tl);
                    two_prod(cf[7][e], Ww[e + 1], th, tl); ff_acc(H, L, th, tl); // c0 p[i-1]
                    two_prod(cf[8][e], Sc[e], th, tl); ff_acc(H, L, th, tl);     // c1 p[j-1]
                    two_prod(cf[9][e], Cw[e], th, tl); ff_acc(H, L, th, tl);     // c2 p[k-1]
                    ff_acc(H, L, cf[11][e], 0.0f);                               // wrk1
                    // ss = (s0 * a3 - p) * bnd
                    const float pc = Cw[e + 1];
                    float dh, dl, e1, sh, s1;
                    two_prod(H, cf[3][e], th, t1);
                    tl = __fmaf_rn(L, cf[3][e], t1);
                    two_sum(th, -pc, dh, e1);
                    dl = __fadd_rn(e1, tl);
                    two_prod(dh, cf[10][e], sh, s1);
                    const float sl = __fmaf_rn(dl, cf[10][e], s1);
                    // wrk2 = p + omega * ss, rounded once
                    float wh, w1, yh, e2;
                    two_prod(omega, sh, wh, w1);
                    const float wl = __fmaf_rn(omega, sl, w1);
                    two_sum(pc, wh, yh, e2);
                    out[e] = __fadd_rn(yh, __fadd_rn(e2, wl));
                    // ss^2 from the renormalised pair: on smooth fields ss is nearly the
                    // same at every point, so rounding it to float first would bias the
                    // residual by up to 2^-24; sl can be ~1% of sh when ss cancels deeply
                    float nh, nl, qh, q1;
                    two_sum(sh, sl, nh, nl);
                    two_prod(nh, nh, qh, q1);
                    const float ql = __fmaf_rn(__fadd_rn(nh, nh), nl, q1);
                    ff_acc(RH, RL, inside[e] ? qh : 0.0f, inside[e] ? ql : 0.0f);
                }
                if (row_in) {
                    float *dst = a.wrk2 + ((size_t)i * J + j) * a.pitch + kb;
                    if (all_in) {
                        VecT v;
                        float *vf = reinterpret_cast<float *>(&v);
#pragma unroll
                        for (int e = 0; e < PPT; ++e) vf[e] = out[e];
                        *reinterpret_cast<VecT *>(dst) = v;
                    } else {
#pragma unroll
                        for (int e = 0; e < PPT; ++e)
                            if (inside[e]) dst[e] = out[e];
                    }
                }
                // march: plane i+1 becomes the centre plane
#pragma unroll
                for (int e = 0; e < PPT; ++e) {
                    Gh[e] = Dh[e + 1];
                    Gl[e] = Dl[e + 1];
                    Nc[e] = ENw[e + 1];
                    Sc[e] = ESw[e + 1];
                }
#pragma unroll
                for (int x = 0; x < W; ++x) {
                    Ww[x] = Cw[x];
                    Cw[x] = Ew[x];
                    Dh[x] = DNh[x];
                    Dl[x] = DNl[x];
                }
            }
            if (!ok) break;
            // release the unit's last two planes
            __syncwarp();
            if (lane == 0) {
                const uint32_t s1 = pbase + (uint32_t)(ie - ib);
                mbar_arrive(smem_u32(&empty_p[s1 % DP]));
                mbar_arrive(smem_u32(&empty_p[(s1 + 1) % DP]));
            }
            pseq = pbase + (uint32_t)(ie - ib + 2);
            // unit partial residual of this warp in FP64 (no cross-warp
            // barrier, so an aborting warp can never leave another waiting)
            double racc = (double)RH + (double)RL;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) racc += __shfl_xor_sync(0xffffffffu, racc, o);
            if (lane == 0) a.partials[(size_t)u * NCW + warp] = racc;
        }
        if (lane == 0) __threadfence();  // partials visible before the CTA is counted
    }
    __syncthreads();

    // ------------------------------------------ last CTA sums the partials
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(a.counter, 1u);
        *last_flag = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (*last_flag) {
        __threadfence();
        const int np = a.n_units * NCW;
        double s = 0.0;
        for (int u = threadIdx.x; u < np; u += blockDim.x) s += __ldcg(&a.partials[u]);
        // fixed-shape tree: within warps, then warp sums in warp order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
            *a.res = tot;
            *a.counter = 0u;
        }
    }
}

// variants: (TK, TJ, NCW, DC, DP, PPT, MINB)
struct VariantInfo {
    int TK, TJ, ctas_per_sm, ncw;
    void (*launch)(int grid, const StencilMaps &m, const StencilArgs &a, cudaStream_t s, bool inject);
};

template <int TK, int TJ, int NCW, int DC, int DP, int PPT, int MINB>
struct Variant {
    using T = Tile<TK, TJ>;
    static constexpr int kThreads = (NCW + 1) * 32;
    static size_t smem_bytes() {
        return 128 + (size_t)DC * NCOEF * T::CTILE * 4 + (size_t)DP * T::PSLOT * 4 +
               2 * (DC + DP) * 8 + 32 * 8 + 16;
    }
    static void launch(int grid, const StencilMaps &m, const StencilArgs &a, cudaStream_t s, bool inject) {
        static std::atomic<uint64_t> done{0}, done_inj{0};
        if (inject) {
            set_smem_limit_once((const void *)stencil_kernel<TK, TJ, NCW, DC, DP, PPT, MINB, true>, smem_bytes(),
                                done_inj);
            stencil_kernel<TK, TJ, NCW, DC, DP, PPT, MINB, true><<<grid, kThreads, smem_bytes(), s>>>(m, a);
        } else {
            set_smem_limit_once((const void *)stencil_kernel<TK, TJ, NCW, DC, DP, PPT, MINB, false>, smem_bytes(),
                                done);
            stencil_kernel<TK, TJ, NCW, DC, DP, PPT, MINB, false><<<grid, kThreads, smem_bytes(), s>>>(m, a);
        }
        OO_CUDA_TRY(cudaGetLastError());
    }
    static VariantInfo info() { return VariantInfo{TK, TJ, MINB, NCW, &launch}; }
};

// 0: 128x8 tile, 8 consumer warps x 4 points, 1 CTA/SM
// 1: 128x8 tile, 16 consumer warps x 2 points, 1 CTA/SM
// 2: 128x4 tile, 8 consumer warps x 2 points, 2 CTAs/SM
// 3: 64x8 tile, 4 consumer warps x 4 points (short rows, K <= 65)
// 4: 64x8 tile, 8 consumer warps x 2 points, 2 CTAs/SM (short rows)
const VariantInfo &variant(int v) {
    static const VariantInfo table[] = {
        Variant<128, 8, 8, 3, 5, 4, 1>::info(),
        Variant<128, 8, 16, 3, 5, 2, 1>::info(),
        Variant<128, 4, 8, 3, 5, 2, 2>::info(),
        Variant<64, 8, 4, 3, 5, 4, 1>::info(),
        Variant<64, 8, 8, 3, 5, 2, 2>::info(),
    };
    constexpr int n = sizeof(table) / sizeof(table[0]);
    return table[(v >= 0 && v < n) ? v : 0];
}
constexpr int kNumVariants = 5;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        OO_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q));
        OO_REQUIRE(q == cudaDriverEntryPointSuccess && p != nullptr, OO_ECUDA,
                   "driver has no cuTensorMapEncodeTiled");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

void make_map(CUtensorMap *m, const float *base, const JacobiDims &d, uint32_t bx, uint32_t by) {
    OO_REQUIRE(((uintptr_t)base & 15u) == 0, OO_EINVAL, "array base must be 16-byte aligned");
    const cuuint64_t dims[3] = {(cuuint64_t)d.pitch, (cuuint64_t)d.J, (cuuint64_t)d.I};
    const cuuint64_t strides[2] = {(cuuint64_t)d.pitch * 4, (cuuint64_t)d.pitch * d.J * 4};
    const cuuint32_t box[3] = {bx, by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims,
                                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    OO_REQUIRE(r == CUDA_SUCCESS, OO_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

}  // namespace

struct StencilPlan {
    JacobiDims d{};
    int variant = -1;  // tile variant; -1 on creation: the default rule picks
    int TK = 128, TJ = 8;
    StencilMaps maps;
    StencilArgs args{};
    int grid = 0;
    void *scratch = nullptr;
    bool own_scratch = true;
};

namespace {
// tensor maps, tile shape and the i-segment split of a plan (no scratch yet)
// max_slots > 0 caps the partial-residual slots (units x consumer warps)
// the i-segment split may use
void fill_stencil_plan(StencilPlan *sp, const JacobiDims &d, const float *const coef[NCOEF], const float *p,
                       float *wrk2, int num_sms, long long max_slots = 0) {
    sp->d = d;
    // default tile shape by row length (16 consumer warps x 2 points measured
    // ~0.6 % faster than 8 x 4 at 257 x 257 x 513) unless the caller chose
    // one (a tuned choice or the context's option)
    if (sp->variant < 0 || sp->variant >= kNumVariants) sp->variant = stencil_default_variant(d);
    sp->TK = variant(sp->variant).TK;
    sp->TJ = variant(sp->variant).TJ;
    for (int c = 0; c < NCOEF; ++c) make_map(&sp->maps.coef[c], coef[c], d, sp->TK, sp->TJ);
    make_map(&sp->maps.p, p, d, sp->TK + 8, sp->TJ + 2);
    StencilArgs &a = sp->args;
    a.I = d.I;
    a.J = d.J;
    a.K = d.K;
    a.pitch = d.pitch;
    a.n_kt = (d.K - 1 + sp->TK - 1) / sp->TK;
    a.n_jt = (d.J - 2 + sp->TJ - 1) / sp->TJ;
    const int cols = a.n_kt * a.n_jt;
    const int span = d.I - 2;
    // segments of the i range: balance units over one CTA per SM, with a
    // charge for the two halo planes and the prologue every unit pays
    const int G = std::max(1, num_sms * variant(sp->variant).ctas_per_sm);
    const int ncw = variant(sp->variant).ncw;
    OO_REQUIRE(max_slots <= 0 || (long long)cols * ncw <= max_slots, OO_EINVAL,
               "grid too large for the static scratch: ceil((K-1)/tile_k) * ceil((J-2)/tile_j) * consumer warps "
               "must be <= " + std::to_string(max_slots));
    double best = 1e300;
    int best_seg = 1;
    for (int ns = 1; ns <= span; ++ns) {
        if (max_slots > 0 && (long long)cols * ns * ncw > max_slots) break;
        const int smax = (span + ns - 1) / ns;
        const long long units = (long long)cols * ns;
        const long long rounds = (units + G - 1) / G;
        const double cost = (double)rounds * (smax + 0.6);
        if (cost < best - 1e-9) {
            best = cost;
            best_seg = ns;
        }
    }
    a.n_seg = best_seg;
    a.n_units = cols * best_seg;
    sp->grid = std::min(a.n_units, G);
    a.wrk2 = wrk2;
}
void attach_scratch(StencilPlan *sp, void *scratch) {
    StencilArgs &a = sp->args;
    sp->scratch = scratch;
    a.partials = reinterpret_cast<double *>(scratch);
    a.counter = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(scratch) +
                                             (size_t)a.n_units * kMaxConsumerWarps * 8);
    a.err = a.counter + 1;
}
size_t plan_scratch_bytes(const StencilPlan *sp) {
    return (size_t)sp->args.n_units * kMaxConsumerWarps * 8 + 256;
}
}  // namespace

size_t stencil_scratch_bytes(const JacobiDims &d, int num_sms) {
    // upper bound over the tile variants (smallest tile 64 x 4) and every
    // i-segment split (at most one unit per plane)
    (void)num_sms;
    const long long kt = (d.K - 1 + 63) / 64, jt = (d.J - 2 + 3) / 4;
    return (size_t)(kt * jt * std::max(1, d.I - 2)) * kMaxConsumerWarps * 8 + 256;
}

StencilPlan *stencil_plan_create_ext(const JacobiDims &d, const float *const coef[NCOEF], const float *p, float *wrk2,
                                     int num_sms, void *scratch, size_t scratch_bytes, cudaStream_t s, int variant) {
    OO_REQUIRE(d.I >= 3 && d.J >= 3 && d.K >= 3, OO_EINVAL, "grid must be at least 3 x 3 x 3");
    OO_REQUIRE(d.pitch >= d.K && d.pitch % 4 == 0, OO_EINVAL, "pitch must be >= K and a multiple of 4");
    OO_REQUIRE(((uintptr_t)wrk2 & 15u) == 0 && ((uintptr_t)scratch & 15u) == 0, OO_EINVAL,
               "wrk2 and scratch must be 16-byte aligned");
    auto sp = new StencilPlan();
    sp->variant = variant;
    try {
        fill_stencil_plan(sp, d, coef, p, wrk2, num_sms);
        OO_REQUIRE(plan_scratch_bytes(sp) <= scratch_bytes, OO_EINVAL, "stencil scratch too small");
        attach_scratch(sp, scratch);
        sp->own_scratch = false;
        OO_CUDA_TRY(cudaMemsetAsync(sp->args.counter, 0, 8, s));
    } catch (...) {
        delete sp;
        throw;
    }
    return sp;
}

StencilPlan *stencil_plan_create(const JacobiDims &d, const float *const coef[NCOEF], const float *p,
                                 float *wrk2, int num_sms, int variant) {
    OO_REQUIRE(d.I >= 3 && d.J >= 3 && d.K >= 3, OO_EINVAL, "grid must be at least 3 x 3 x 3");
    OO_REQUIRE(d.pitch >= d.K && d.pitch % 4 == 0, OO_EINVAL, "pitch must be >= K and a multiple of 4");
    OO_REQUIRE(((uintptr_t)wrk2 & 15u) == 0, OO_EINVAL, "wrk2 must be 16-byte aligned");
    auto sp = new StencilPlan();
    sp->variant = variant;
    try {
        fill_stencil_plan(sp, d, coef, p, wrk2, num_sms);
        const size_t bytes = plan_scratch_bytes(sp);  // up to 16 consumer warps
        void *scr = nullptr;
        OO_CUDA_TRY(cudaMalloc(&scr, bytes));
        attach_scratch(sp, scr);
        OO_CUDA_TRY(cudaMemset(sp->scratch, 0, bytes));
    } catch (...) {
        if (sp->scratch) cudaFree(sp->scratch);
        delete sp;
        throw;
    }
    return sp;
}

int stencil_plan_variant(const StencilPlan *sp) { return sp->variant; }
int stencil_variant_count() { return kNumVariants; }
int stencil_default_variant(const JacobiDims &d) { return d.K - 1 > 64 ? 1 : 4; }

void stencil_plan_destroy(StencilPlan *sp) {
    if (!sp) return;
    if (sp->scratch && sp->own_scratch) cudaFree(sp->scratch);
    delete sp;
}

void launch_stencil(StencilPlan *sp, float omega, double *res_dev, cudaStream_t s, bool inject_timeout) {
    sp->args.omega = omega;
    sp->args.res = res_dev;
    variant(sp->variant).launch(sp->grid, sp->maps, sp->args, s, inject_timeout);
}

const unsigned *stencil_plan_err_ptr(const StencilPlan *sp) { return sp->args.err; }

unsigned stencil_plan_check(StencilPlan *sp, cudaStream_t s) {
    unsigned e = 0;
    OO_CUDA_TRY(cudaMemcpyAsync(&e, sp->args.err, 4, cudaMemcpyDeviceToHost, s));
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    if (e) OO_CUDA_TRY(cudaMemsetAsync(sp->args.err, 0, 4, s));
    return e;
}

// ======================================= allocation-free stencil entry point
// Some callers cannot allocate device memory when they call in: a serving
// loop with a fixed device-memory budget handed out by its own pool, or a
// language runtime that owns every allocation on the device.  For them the stencil
// sweep below keeps its scratch (per-warp partial residuals, the CTA-done
// counter and the error word) in one static device array instead of
// cudaMalloc'd memory.  The caller still passes every input and output.
namespace {

constexpr int kStaticPartials = 65536;  // doubles: 512 KB of partial residuals
constexpr size_t kStaticScratchBytes = (size_t)kStaticPartials * 8 + 256;
constexpr int kMaxDevices = 64;

// Held by every device that loads the library until the process exits.  In
// host code this name is only a stand-in for the device symbol: its device
// address is looked up with cudaGetSymbolAddress per device below.
static __device__ __align__(256) unsigned char g_stencil_scratch[kStaticScratchBytes];

// The device address of g_stencil_scratch on `device`, looked up once per
// device (with that device current) under a lock, so host threads making
// their first calls at the same time agree.  The cached address belongs to
// the device's primary context: a device reset between calls invalidates it.
void *static_scratch_ptr(int device) {
    static std::mutex mu;
    static void *addr[kMaxDevices] = {nullptr};
    OO_REQUIRE(device >= 0 && device < kMaxDevices, OO_EINVAL, "device index beyond the static table");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        OO_CUDA_TRY(cudaGetSymbolAddress(&p, g_stencil_scratch));
        addr[device] = p;
    }
    return addr[device];
}

}  // namespace

}  // namespace oo

extern "C" oo_status oo_stencil_noalloc_dev(oo_ctx *ctx, int I, int J, int K, int pitch,
                                            const float *const *coef, const float *p, float omega,
                                            float *wrk2, double *res_dev) {
    using namespace oo;
    if (!ctx) return OO_EINVAL;
    Ctx &c = ctx_state(ctx);
    try {
        OO_REQUIRE(c.device >= 0, OO_ESTATE, "host-only context (device -1) cannot run GPU work");
        OO_REQUIRE(coef && p && wrk2 && res_dev, OO_EINVAL, "null pointer");
        for (int a = 0; a < NCOEF; ++a) OO_REQUIRE(coef[a] != nullptr, OO_EINVAL, "null coefficient array");
        OO_REQUIRE(I >= 3 && J >= 3 && K >= 3 && K <= 4096, OO_EINVAL, "bad grid");
        OO_REQUIRE(pitch >= K && pitch % 4 == 0, OO_EINVAL, "pitch must be >= K and a multiple of 4");
        OO_REQUIRE(((uintptr_t)wrk2 & 15u) == 0, OO_EINVAL, "wrk2 must be 16-byte aligned");
        OO_REQUIRE(std::isfinite(omega), OO_EINVAL, "omega must be finite");
        OO_CUDA_TRY(cudaSetDevice(c.device));
        // the plan lives on the host stack: tile variant and i-segment split
        // as oo_stencil_dev chooses them (the context's option or tuned
        // choice, else the default rule), the split capped at the static
        // array's slots
        StencilPlan sp;
        sp.variant = c.stencil_variant_for(I, J, K);
        fill_stencil_plan(&sp, JacobiDims{I, J, K, pitch}, coef, p, wrk2, c.num_sms, kStaticPartials);
        char *scratch = static_cast<char *>(static_scratch_ptr(c.device));
        StencilArgs &sa = sp.args;
        sa.partials = reinterpret_cast<double *>(scratch);
        sa.counter = reinterpret_cast<unsigned *>(scratch + (size_t)kStaticPartials * 8);
        sa.err = sa.counter + 1;
        sa.omega = omega;
        sa.res = res_dev;
        // the array keeps the previous call's contents: the CTA counter and
        // the error word must start at zero
        OO_CUDA_TRY(cudaMemsetAsync(sa.counter, 0, 8, c.stream));
        const bool inject = c.inject_wait == OO_INJECT_STENCIL_LOAD;
        if (inject) c.inject_wait = OO_INJECT_NONE;
        variant(sp.variant).launch(sp.grid, sp.maps, sa, c.stream, inject);
        OO_CUDA_TRY(cudaGetLastError());
        c.last_error.clear();
        return OO_OK;
    } catch (const Error &e) {
        c.last_error = e.msg;
        return e.code;
    } catch (...) {
        c.last_error = "unknown failure";
        return OO_ECUDA;
    }
}

// Completion check of oo_stencil_noalloc_dev: the error word sits in the
// static array, so reading it allocates nothing either.
extern "C" oo_status oo_stencil_noalloc_check(oo_ctx *ctx) {
    using namespace oo;
    if (!ctx) return OO_EINVAL;
    Ctx &c = ctx_state(ctx);
    try {
        OO_REQUIRE(c.device >= 0, OO_ESTATE, "host-only context (device -1) cannot run GPU work");
        OO_CUDA_TRY(cudaSetDevice(c.device));
        unsigned *err = reinterpret_cast<unsigned *>(static_cast<char *>(static_scratch_ptr(c.device)) +
                                                     (size_t)kStaticPartials * 8) + 1;
        unsigned e = 0;
        OO_CUDA_TRY(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, c.stream));
        OO_CUDA_TRY(cudaStreamSynchronize(c.stream));
        if (e) {
            OO_CUDA_TRY(cudaMemsetAsync(err, 0, 4, c.stream));
            OO_CUDA_TRY(cudaStreamSynchronize(c.stream));
            throw Error{OO_ETIMEOUT, "stencil pipeline wait ran out (error bits " + std::to_string(e) +
                                         "); wrk2 and the residual of that sweep are incomplete"};
        }
        c.last_error.clear();
        return OO_OK;
    } catch (const Error &e) {
        c.last_error = e.msg;
        return e.code;
    } catch (...) {
        c.last_error = "unknown failure";
        return OO_ECUDA;
    }
}
