// Internal declarations of liboo: context, workspaces, kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <map>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/oo.h"

namespace oo {

// ------------------------------------------------------------ error helpers
struct Error {
    oo_status code;
    std::string msg;
};

#define OO_CUDA_TRY(expr)                                                        \
    do {                                                                         \
        cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess)                                                   \
            throw ::oo::Error{OO_ECUDA, std::string(#expr) + ": " +              \
                                            cudaGetErrorString(e_)};             \
    } while (0)

#define OO_REQUIRE(cond, code, text)                                             \
    do {                                                                         \
        if (!(cond)) throw ::oo::Error{(code), (text)};                          \
    } while (0)

// ------------------------------------------------------------- nest tables
struct NestTable {
    struct Var {
        std::string name;
        uint64_t bytes;
    };
    struct Nest {
        std::string name;
        int level;
        int parallelisable;
        uint64_t reads, writes, partial;
    };
    std::vector<Var> vars;
    std::vector<Nest> nests;
    uint64_t outputs = 0;
    int gene_len() const;
    // placement[n] = 1 when nest n runs on the GPU under `gene`
    std::vector<int> placement(uint64_t gene) const;
};

void validate_table(const NestTable &t);
NestTable jacobi_table(int I, int J, int K, int iters);

// The coherence walk of the transfer rules; returns the ordered copy list.
std::vector<oo_xfer> make_plan(const NestTable &t, uint64_t gene, int hoist, int iters,
                               uint64_t *h2d, uint64_t *d2h);

// ------------------------------------------------------------------ Jacobi
enum { NCOEF = 12, NARR = 14, VAR_P = 12, VAR_WRK2 = 13, VAR_RES = 14 };

struct JacobiDims {
    int I, J, K, pitch;
    size_t n_host() const { return (size_t)I * J * K; }
    size_t n_dev() const { return (size_t)I * J * pitch; }
};

int jacobi_pitch(int K);

// Opaque per-(I,J,K) stencil launch state (tensor maps, work split, scratch).
struct StencilPlan;

// Device + pinned host workspace of the Jacobi program for one grid size.
struct JacobiWork {
    JacobiDims d{};
    int iters_cap = 0;
    float *dev = nullptr;             // NARR arrays, each n_dev() floats
    size_t dev_stride = 0;            // floats between arrays
    double *res_dev = nullptr;        // iters_cap doubles
    float *host = nullptr;            // NARR arrays, each n_host() floats (pinned)
    double *res_host = nullptr;       // iters_cap doubles (pinned)
    StencilPlan *splan = nullptr;
    void *fused_ctl = nullptr;        // fused-iteration barrier words + residual partials
    float *dptr(int v) const { return dev + (size_t)v * dev_stride; }
    float *hptr(int v) const { return host + (size_t)v * d.n_host(); }
};

// -------------------------------------------------------------------- FFT
struct FftPlan;
FftPlan *fft_plan_create(long long n);
void fft_plan_destroy(FftPlan *p);
size_t fft_scratch_bytes(const FftPlan *p, int batch);
// Serving works on a (thread-safe) context-owned plan cache; see Ctx::fft_plan.
// batch transforms of length n (contiguous, interleaved complex128); dir -1
// forward, +1 inverse (1/n scaled); in may equal out; async on s
void launch_fft(const FftPlan *p, int batch, int dir, const double *in, double *out, void *scratch,
                cudaStream_t s);

// ------------------------------------------------------------------- GEMM
size_t gemm_scratch_bytes(int m, int n, int k);
// C = A B (FP64, row-major) via split BF16 tensor-core products; async on s.
// pair: 0 = 128 x 128 tiles on single CTAs; 1 = 256-row tiles on CTA pairs
// (cta_group::2), width chosen per problem; 160, 192, 224 or 256 = CTA pairs
// with that tile width.  The same products in the same order in every case.
void launch_gemm_split3(int m, int n, int k, const double *A, long long lda, const double *B, long long ldb,
                        double *C, long long ldc, void *scratch, cudaStream_t s, int pair = 1);
// reads and clears the kernel's error word (0 = fine); synchronises s
unsigned gemm_check_error(void *scratch, int m, int n, int k, cudaStream_t s);
// the kernel's device error word inside its scratch (for asynchronous reads)
unsigned *gemm_error_word(void *scratch, int m, int n, int k);
// the same products with TF32 hi / lo operands (kind::tf32); scratch and
// error word laid out by gemm_tf32_scratch_bytes / gemm_tf32_error_word
size_t gemm_tf32_scratch_bytes(int m, int n, int k);
void launch_gemm_split3_tf32(int m, int n, int k, const double *A, long long lda, const double *B, long long ldb,
                             double *C, long long ldc, void *scratch, cudaStream_t s);
unsigned *gemm_tf32_error_word(void *scratch, int m, int n, int k);
// FP64-equivalent mode (gemm_fp64eq.cu): Ozaki-type BF16 digit slices
size_t gemm_fp64eq_scratch_bytes(int m, int n, int k);
int gemm_fp64eq_products(int k);
void gemm_fp64eq_shape(int k, int *beta, int *levels, int *k_block);
// width: tile width (32, 64 or 128) for the products of a level scheme;
// pair: the pair scheme's products on CTA pairs (256 x 128 tiles,
// cta_group::2), else on single CTAs (128 x 128); the same bits either way
void launch_gemm_fp64eq(int m, int n, int k, const double *A, long long lda, const double *B, long long ldb,
                        double *C, long long ldc, void *scratch, cudaStream_t s, int width, bool pair = true);
unsigned gemm_fp64eq_check_error(void *scratch, cudaStream_t s);
unsigned *gemm_fp64eq_error_word(void *scratch);

// FP64-equivalent accumulation scheme for inner dimension k (eq_digits.cuh:
// 0 pairs, 1 levels with 7-bit digits, 2 levels with 6-bit digits)
int eq_scheme_for(int k);
// tile width of a problem's full tiles from a context's table (nullptr: the
// built-in table)
int eq_tile_width(const int *widths, int n, int k);
int eq_default_width(int nb, int kb);
// Grouped FFTs (batched function blocks): transforms of different lengths
// and directions in two persistent launches.
struct FftDesc {
    long long n;
    int dir;
    const double *in;
    double *out;
};
struct FftGroup;
FftGroup *fft_group_create(const std::vector<FftDesc> &v, const std::vector<const FftPlan *> &plans, int num_sms);
void fft_group_launch(FftGroup *g, cudaStream_t s);
double fft_group_elements(const FftGroup *g);
void fft_group_destroy(FftGroup *g);

// Grouped GEMMs (batched function blocks): one split pass and one persistent
// tensor-core kernel over the tiles of every problem.
struct GemmDesc {
    int m, n, k;
    const double *A;
    long long lda;
    const double *B;
    long long ldb;
    double *C;
    long long ldc;
};
struct GemmGroup;
GemmGroup *gemm_group_create(const std::vector<GemmDesc> &v, int num_sms);
void gemm_group_launch(GemmGroup *g, cudaStream_t s);
unsigned gemm_group_check(GemmGroup *g, cudaStream_t s);
double gemm_group_flops(const GemmGroup *g);
void gemm_group_destroy(GemmGroup *g);

// a single product of a level scheme on split operands (gemm_eq_group.cu)
void launch_gemm_eq_tiles(int m, int n, int k, const void *As, const void *Bs, const int *ea,
                          const int *eb, double *C, long long ldc, int width, unsigned *err, int num_sms,
                          cudaStream_t s);
// Grouped FP64-equivalent products: one split launch and one persistent
// tensor-core launch over the tiles of every problem.
struct EqGroup;
EqGroup *eq_group_create(const std::vector<GemmDesc> &v, int num_sms, const int *widths);
void eq_group_launch(EqGroup *g, cudaStream_t s);
namespace eq {
struct GSplit;
}
// the grouped products' digit split (gemm_fp64eq.cu): njobs jobs of eight A
// rows or 64 B columns
void launch_eq_group_split(const eq::GSplit *gs, const int4 *jobs, int nrow_jobs, int ncol_jobs, cudaStream_t s);
unsigned eq_group_check(EqGroup *g, cudaStream_t s);
double eq_group_flops(const EqGroup *g);
int eq_group_tiles(const EqGroup *g);
void eq_group_destroy(EqGroup *g);


// Raise a kernel's dynamic shared-memory limit on the current device once
// (the attribute is per device and a process may drive several; `done`
// holds one bit per device and is safe to share between threads).
inline void set_smem_limit_once(const void *fn, size_t bytes, std::atomic<uint64_t> &done) {
    int dev = 0;
    OO_CUDA_TRY(cudaGetDevice(&dev));
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    OO_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.fetch_or(bit, std::memory_order_acq_rel);
}

// Grow-only device buffer owned by a context.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    void *get(size_t want) {
        if (want <= bytes) return ptr;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        if (cudaMalloc(&ptr, want) != cudaSuccess) {
            cudaGetLastError();
            throw Error{OO_ENOMEM, "device scratch of " + std::to_string(want) + " bytes"};
        }
        bytes = want;
        return ptr;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
};

// Serving loop state (serve.cpp: host-scheduled; serve_resident.cu: the
// request loop resident on the device).
struct Server;
void server_stop(Server *S);
struct Resident;
void resident_stop(Resident *S);
oo_status resident_submit(Resident *S, const oo_serve_req *req, uint64_t *ticket);
struct Ctx;
oo_status resident_wait(Ctx &c, Resident *S, uint64_t ticket, int timeout_ms, double *latency_ms);
void resident_stats(Resident *S, oo_serve_stats_t *out);

// first-fit allocator over [0, size) with 256-byte granules
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        free_[0] = size;
        size_ = size;
        free_bytes_ = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (std::max<size_t>(bytes, 256) + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                free_bytes_ -= bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (std::max<size_t>(bytes, 256) + 255) / 256 * 256;
        free_bytes_ += bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t free_bytes() const { return free_bytes_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, free_bytes_ = 0;
};


// --------------------------------------------------------------- context
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    std::string last_error;
    NestTable table;
    bool have_table = false;
    JacobiWork *jw = nullptr;
    // correctness references for the GA gate: all-CPU residuals per problem
    struct Ref {
        int I, J, K, iters;
        float omega;
        std::vector<double> res;
        std::vector<float> p;
    };
    std::vector<Ref> refs;
    // function blocks
    std::vector<std::pair<long long, FftPlan *>> fft_plans;
    DevBuf fft_scratch, stage_a, stage_b, stage_c, gemm_scratch;
    Server *server = nullptr;
    Resident *rserver = nullptr;
    // fault injection armed by oo_inject_wait_timeout (one-shot; 0 = none)
    int inject_wait = 0;
    // options set by oo_set_option: OO_OPT_JACOBI_FUSED (-1 default rule,
    // 0 never, 1 whenever the placement allows) and OO_OPT_STENCIL_VARIANT
    // (-1 tuned choice or default rule, else that variant for every grid)
    int opt_fused = -1;
    int opt_stencil_variant = -1;
    int opt_gemm_pair = 1;  // split-BF16 kernel: 0 single CTAs, 1 CTA pairs, 160..256 CTA pairs of that width
    // tile widths of the FP64-equivalent products by (n, k) bucket
    // (oo_tune_gemm_tiles / oo_set_gemm_tiles; 0 = the built-in choice)
    std::array<int, OO_TILE_NBUCKETS * OO_TILE_KBUCKETS> eq_widths{};
    // stencil tile variant chosen by oo_tune_stencil per grid: {I, J, K, variant}
    std::vector<std::array<int, 4>> stencil_choice;
    // the variant a stencil plan for this grid should use (-1: default rule)
    int stencil_variant_for(int I, int J, int K) const {
        if (opt_stencil_variant >= 0) return opt_stencil_variant;
        for (const auto &x : stencil_choice)
            if (x[0] == I && x[1] == J && x[2] == K) return x[3];
        return -1;
    }
    FftPlan *fft_plan(long long n) {
        for (auto &kv : fft_plans)
            if (kv.first == n) return kv.second;
        FftPlan *p = fft_plan_create(n);
        fft_plans.push_back({n, p});
        return p;
    }
};

// The library state behind a C-ABI context handle (api.cpp).
Ctx &ctx_state(oo_ctx *ctx);

// FFT plan accessors for the device-resident loop (fft.cu)
int fft_plan_log2(const FftPlan *p);
void fft_plan_tables(const FftPlan *p, const void **tw, const void **tw_n1, const void **tw_n2, const void **tw_hi,
                     const void **tw_lo, int *log2n, int *log2n1, int *log2n2);

// Kernel launchers (jacobi.cu).  All asynchronous on `s`.
void launch_coef(const JacobiDims &d, float *const coef[NCOEF], cudaStream_t s);
void launch_pinit(const JacobiDims &d, float *p, float *wrk2, cudaStream_t s);
void launch_copyback(const JacobiDims &d, float *p, const float *wrk2, cudaStream_t s);
// N3 + N4 + N5 in one pass (all three on the GPU, no copy between them)
void launch_copyback_faces(const JacobiDims &d, float *p, const float *wrk2, cudaStream_t s);
void launch_bc_ij(const JacobiDims &d, float *p, cudaStream_t s);
void launch_bc_k(const JacobiDims &d, float *p, cudaStream_t s);

// variant: tile variant to use (0 .. stencil_variant_count() - 1), or -1
// for the default rule by row length
StencilPlan *stencil_plan_create(const JacobiDims &d, const float *const coef[NCOEF],
                                 const float *p, float *wrk2, int num_sms, int variant = -1);
int stencil_plan_variant(const StencilPlan *sp);
int stencil_variant_count();
// the variant a plan takes when none is chosen (by row length)
int stencil_default_variant(const JacobiDims &d);
// A plan whose scratch (partial residuals, counter, error word) lives in
// caller-provided device memory of at least stencil_scratch_bytes(d, sms).
StencilPlan *stencil_plan_create_ext(const JacobiDims &d, const float *const coef[NCOEF], const float *p, float *wrk2,
                                     int num_sms, void *scratch, size_t scratch_bytes, cudaStream_t s,
                                     int variant = -1);
size_t stencil_scratch_bytes(const JacobiDims &d, int num_sms);
void stencil_plan_destroy(StencilPlan *sp);
// One stencil sweep; the residual (FP64) lands in *res_dev.
// inject_timeout: fault injection for tests -- the producer never issues the
// first p-tile fill, so the consumers' bounded wait runs out (~1 s) and the
// sweep reports an error bit instead of a result
void launch_stencil(StencilPlan *sp, float omega, double *res_dev, cudaStream_t s, bool inject_timeout = false);
// All iterations of the all-GPU iteration nests in one cooperative launch
// (small grids): ctl is jacobi_fused_ctl_bytes() of device scratch.
size_t jacobi_fused_ctl_bytes();
// option: -1 the size rule (at most 2^20 points), 0 never, 1 always
bool jacobi_fused_eligible(const JacobiDims &d, int option);
void launch_jacobi_fused(const JacobiDims &d, const float *const coef[NCOEF], float *p, float *wrk2, float omega,
                         int iters, double *res_dev, void *ctl, cudaStream_t s,
                         bool inject_timeout = false);
unsigned jacobi_fused_check(void *ctl, cudaStream_t s);
// Device address of the plan's error word (0 = fine).
const unsigned *stencil_plan_err_ptr(const StencilPlan *sp);
// Reads and clears the device-side error word of the plan (0 = fine).
unsigned stencil_plan_check(StencilPlan *sp, cudaStream_t s);

// Host nests (host_nests.cpp), on unpadded I x J x K arrays.
void host_coef(const JacobiDims &d, float *const coef[NCOEF]);
void host_pinit(const JacobiDims &d, float *p, float *wrk2);
double host_stencil(const JacobiDims &d, const float *const coef[NCOEF], const float *p,
                    float omega, float *wrk2);
void host_copyback(const JacobiDims &d, float *p, const float *wrk2);
void host_bc_ij(const JacobiDims &d, float *p);
void host_bc_k(const JacobiDims &d, float *p);

// Pattern execution (pattern.cpp).
// time every stencil tile variant for an I x J x K grid on the context's
// workspace; the fastest is kept for the grid and returned (ms_out: one entry
// per variant, may be null)
int tune_stencil(Ctx &c, int I, int J, int K, double *ms_out);
// time every tile width of the grouped FP64-equivalent product for every
// (n, k) bucket and keep the fastest in c.eq_widths (ms_out: buckets x 3,
// may be null); gemm_eq_group.cu
void tune_gemm_tiles(Ctx &c, double *ms_out);
void run_pattern(Ctx &c, uint64_t gene, int hoist, const oo_jacobi &prob, float *p_out,
                 double *res_out, bool out_on_device, oo_run_stats *stats,
                 double abort_after_ms = 0.0, bool *aborted = nullptr);
void jacobi_work_free(JacobiWork *w);

// GA (ga.cpp).
struct Rng {
    uint64_t s[4];
    void seed(uint64_t seed);
    uint64_t next();
    double uniform();
    int randint(int n);
};
uint64_t splitmix64(uint64_t &state);

struct GaResult {
    uint64_t best_gene = 0;
    double best_time = 0;
    std::vector<uint64_t> history;
};
// time_of(gene) returns the gene's time (infinity = failed the gate)
GaResult ga_run(int L, int pop, int gens, double pc, double pm, uint64_t seed,
                const std::function<double(uint64_t)> &time_of);

// Generic loop programs (program.cpp).
void run_program(Ctx &c, uint64_t gene, int hoist, int iters, oo_nest_fn fn, void *user, void *const *host_vars,
                 void *const *dev_vars, oo_run_stats *stats);
GaResult ga_program(Ctx &c, int hoist, int iters, oo_nest_fn fn, oo_check_fn check, void *user,
                    void *const *host_vars, void *const *dev_vars, int pop, int gens, double pc, double pm,
                    uint64_t seed, std::vector<double> *gene_ms);

// Function-block lookup (blocks.cpp).
int lookup_block(const char *callee, int lang);

// Function-block trial (fb_search.cpp): per-combination wall times of the
// known sites (infinity where a result fails the tolerance or the mask
// offloads an unknown site) and the decision on such a table.
using FbGpu = std::function<void(int prec, int block, const oo_fb_site &, const double *a, const double *b,
                                 double *out)>;
void fb_trial(const oo_fb_site *sites, int n_sites, int prec, double tol, uint64_t seed,
              std::vector<double> &mask_ms, std::vector<int> &block_ids, const FbGpu &gpu);
uint32_t fb_best(const double *mask_ms, int n_sites, double *best_ms);

}  // namespace oo
