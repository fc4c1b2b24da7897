// Blackwell (sm_103a) building blocks shared by the tensor-core kernels:
// mbarrier waits with an iteration bound, 2D TMA tile loads, shared-memory
// matrix descriptors for 128-byte-swizzled K-major BF16 tiles, tcgen05.mma
// (kind::f16, cta_group::1), commits, fences, and tensor-memory loads /
// stores.  Every wait is bounded: on time-out it raises the CTA's abort
// flag and an error bit that the host reads after the launch.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ff.cuh"
#include "oo_internal.h"

namespace oo {
namespace tc {

constexpr long long kWaitLimit = 2000000000ll;  // clock64 ticks (~1 s)

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t b, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(c) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t b, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(b),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(b) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t b, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(b), "r"(par)
        : "memory");
    return ok != 0;
}
// Wait for phase `par` of barrier b; false if another role aborted or this
// wait ran out (then the abort flag and error bit `code` are set).
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t par, volatile int *abort_flag, unsigned *err,
                                         unsigned code) {
    if (bar_try(b, par)) return true;
    const long long t0 = clock64();
    while (true) {
        if (bar_try(b, par)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitLimit) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}
// bounded wait used only while draining after an abort
__device__ __forceinline__ void bar_drain(uint32_t b, uint32_t par) {
    const long long t0 = clock64();
    while (!bar_try(b, par) && clock64() - t0 < kWaitLimit) {
    }
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand tile stored as rows of
// 128 bytes (64 BF16) with the 128-byte swizzle that TMA SWIZZLE_128B writes;
// 8-row core groups 1024 bytes apart (SBO); LBO unused for this layout.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (encoded 16 B; ignored)
    d |= (uint64_t)(1024u >> 4) << 32;      // SBO = 1024 B
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32 (format code 2),
// both K-major; an MMA covers K = 8 TF32 values (32 bytes of each row, as
// K = 16 BF16 values do)
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
template <uint32_t IDESC>
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}

template <uint32_t IDESC>
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
// ---- CTA pairs (cta_group::2).  The two CTAs of a 2-CTA cluster run one
// M = 256 MMA together: each holds 128 rows of A and half of B's N columns
// in its own shared memory (at the same offsets) and 128 rows of the
// accumulator in its own tensor memory; the even CTA (rank 0) issues the
// MMAs.  A kernel that uses these uses no cta_group::1 instruction.
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared-memory location in CTA `rank`
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// every thread of both CTAs
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void bar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// try_wait that also orders after arrivals made by the other CTA
__device__ __forceinline__ bool bar_try_cluster(uint32_t b, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(b), "r"(par)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait_cluster(uint32_t b, uint32_t par, volatile int *abort_flag, unsigned *err,
                                                 unsigned code) {
    if (bar_try_cluster(b, par)) return true;
    const long long t0 = clock64();
    while (true) {
        if (bar_try_cluster(b, par)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitLimit) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}
// 2D tile load into this CTA's shared memory whose completion is counted on
// a barrier of either CTA of the pair (bar: shared::cluster address)
__device__ __forceinline__ void tma_2d_pair(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                              uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// arrive on the barrier at this offset in every CTA of `mask` once the
// MMAs issued so far are complete
__device__ __forceinline__ void mma_commit_pair(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"(mask)
        : "memory");
}
// executed by one warp of each CTA of the pair
__device__ __forceinline__ void tmem_alloc_pair(uint32_t slot_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Non-finite inputs of the matrix products.  The exponent passes over A's
// rows and B's columns report a row / column holding a NaN or an infinity
// as this biased exponent (above every finite one), so its scale exponent
// is 2^20: the split then flushes every entry of that row / column to zero
// (the products stay finite), and the epilogue writes NaN wherever the
// row's and column's scales add up to more than any finite pair can
// (|S| <= 1024 each).  A compensated FP64 dot product that meets an
// infinite or NaN term gives NaN, and so does this product.
constexpr int kNonFiniteExp = (1 << 20) + 1022;
__device__ __forceinline__ int biased_exp_or_flag(unsigned long long bits) {
    const int e = (int)((bits >> 52) & 0x7ff);
    return e == 0x7ff ? kNonFiniteExp : e;
}
__device__ __forceinline__ double nan_or_scaled(double v, int S) {
    return S > 4096 ? __longlong_as_double(0x7ff8000000000000ll) : ff::scale_pow2(v, S);
}

}  // namespace tc
}  // namespace oo

// 32 consecutive TMEM columns of this warp's 32 lanes -> r[0..31] (one
// column per register); lane l reads TMEM lane (taddr >> 16) + l.
#define OO_TMEM_LD32(taddr, r)                                                                              \
    asm volatile(                                                                                           \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"   \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                           \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),   \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),          \
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),        \
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),        \
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                                             \
        : "r"(taddr))

// r[0..31] -> 32 consecutive TMEM columns of this warp's 32 lanes
#define OO_TMEM_ST32(taddr, r)                                                                              \
    asm volatile(                                                                                           \
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),                \
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),  \
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),      \
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),     \
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])                  \
        : "memory")

namespace oo {
namespace tc {

inline PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        OO_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        OO_REQUIRE(q == cudaDriverEntryPointSuccess && p != nullptr, OO_ECUDA, "driver has no cuTensorMapEncodeTiled");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2D BF16 tensor map over a rows x kp row-major array (kp a multiple of
// 64), box = 64 K-elements x box_rows rows, 128-byte swizzle; rows outside
// the array read as zero.
inline void map_bf16(CUtensorMap *m, const void *base, long long rows, int kp, int box_rows) {
    OO_REQUIRE(((uintptr_t)base & 15u) == 0, OO_EINVAL, "split operand must be 16-byte aligned");
    OO_REQUIRE(kp % 64 == 0 && rows >= 1 && rows < (1ll << 31), OO_EINVAL, "bad split-operand shape");
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = encode_tiled()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims,
                                      strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    OO_REQUIRE(r == CUDA_SUCCESS, OO_ECUDA, "cuTensorMapEncodeTiled (GEMM) failed: " + std::to_string((int)r));
}

// FP32 (TF32-rounded) split operand: rows x kp floats, K-major, 128-byte
// swizzle, boxes of 32 floats (one 128-byte row) x box_rows
inline void map_f32(CUtensorMap *m, const void *base, long long rows, int kp, int box_rows) {
    OO_REQUIRE(((uintptr_t)base & 15u) == 0, OO_EINVAL, "split operand must be 16-byte aligned");
    OO_REQUIRE(kp % 32 == 0 && rows >= 1 && rows < (1ll << 31), OO_EINVAL, "bad split-operand shape");
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 4};
    const cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = encode_tiled()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims,
                                      strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    OO_REQUIRE(r == CUDA_SUCCESS, OO_ECUDA, "cuTensorMapEncodeTiled (GEMM, FP32) failed: " + std::to_string((int)r));
}

}  // namespace tc
}  // namespace oo
