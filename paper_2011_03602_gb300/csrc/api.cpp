// C ABI of liboo: argument checks, error translation, context lifetime.
#include <cmath>
#include <cstring>
#include <limits>
#include <map>

#include "oo_internal.h"

using namespace oo;

struct oo_ctx {
    Ctx c;
    // cached stencil launch state for oo_stencil_dev (keyed by its arguments)
    StencilPlan *user_plan = nullptr;
    std::vector<const void *> user_key;
    int gemm_prec = -1;  // precision pattern of the last GEMM launch
};

namespace oo {
Ctx &ctx_state(oo_ctx *ctx) { return ctx->c; }
}  // namespace oo

namespace {

thread_local std::string g_last_error;

template <class F>
oo_status guarded(oo_ctx *ctx, F &&f) {
    try {
        f();
        if (ctx) ctx->c.last_error.clear();
        return OO_OK;
    } catch (const Error &e) {
        if (ctx) ctx->c.last_error = e.msg;
        g_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        if (ctx) ctx->c.last_error = "host allocation failed";
        return OO_ENOMEM;
    } catch (const std::exception &e) {
        if (ctx) ctx->c.last_error = e.what();
        return OO_EINVAL;
    } catch (...) {
        if (ctx) ctx->c.last_error = "unknown failure";
        return OO_ECUDA;
    }
}

// GPU work of a context.  While the device-resident serving loop runs, its
// persistent workers hold the device: a kernel that is loaded lazily at its
// first launch could wait for them, so the context's other GPU calls are
// refused until oo_serve_stop.
void use_device(Ctx &c, bool compute = true) {
    OO_REQUIRE(c.device >= 0, OO_ESTATE, "host-only context (device -1) cannot run GPU work");
    OO_REQUIRE(!compute || c.rserver == nullptr, OO_ESTATE,
               "the device-resident serving loop runs on this context: oo_serve_stop it first");
    OO_CUDA_TRY(cudaSetDevice(c.device));
}

const Ctx::Ref &cpu_reference(Ctx &c, const oo_jacobi &prob) {
    for (const auto &r : c.refs)
        if (r.I == prob.I && r.J == prob.J && r.K == prob.K && r.iters == prob.iters &&
            r.omega == prob.omega)
            return r;
    Ctx::Ref r{prob.I, prob.J, prob.K, prob.iters, prob.omega, {}, {}};
    r.res.resize((size_t)prob.iters);
    r.p.resize((size_t)prob.I * prob.J * prob.K);
    oo_jacobi q = prob;
    q.timing = 0;
    run_pattern(c, 0, 1, q, r.p.data(), r.res.data(), false, nullptr);
    c.refs.push_back(std::move(r));
    return c.refs.back();
}

}  // namespace

extern "C" {

const char *oo_status_str(oo_status s) {
    switch (s) {
        case OO_OK: return "ok";
        case OO_EINVAL: return "invalid argument";
        case OO_ENOMEM: return "out of memory";
        case OO_ECUDA: return "CUDA failure";
        case OO_ETIMEOUT: return "timed out";
        case OO_ETOLERANCE: return "result outside tolerance";
        case OO_EBUSY: return "busy";
        case OO_ENOTFOUND: return "not found";
        case OO_ESTATE: return "invalid state";
        case OO_EUSER: return "nest function failed";
        default: return "unknown status";
    }
}

const char *oo_last_error(const oo_ctx *ctx) {
    return ctx ? ctx->c.last_error.c_str() : g_last_error.c_str();
}

oo_status oo_create(int device, void *cuda_stream, oo_ctx **out) {
    if (!out) return OO_EINVAL;
    *out = nullptr;
    oo_ctx *ctx = new (std::nothrow) oo_ctx();
    if (!ctx) return OO_ENOMEM;
    if (device == -1) {  // host-only context: tables, plans, table-driven GA
        ctx->c.device = -1;
        *out = ctx;
        return OO_OK;
    }
    const oo_status st = guarded(nullptr, [&] {
        int n = 0;
        OO_CUDA_TRY(cudaGetDeviceCount(&n));
        OO_REQUIRE(device >= 0 && device < n, OO_EINVAL, "no such CUDA device");
        ctx->c.device = device;
        OO_CUDA_TRY(cudaSetDevice(device));
        OO_CUDA_TRY(cudaDeviceGetAttribute(&ctx->c.num_sms, cudaDevAttrMultiProcessorCount, device));
        if (cuda_stream) {
            ctx->c.stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            OO_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->c.stream, cudaStreamNonBlocking));
            ctx->c.own_stream = true;
        }
    });
    if (st != OO_OK) {
        delete ctx;
        return st;
    }
    *out = ctx;
    return OO_OK;
}

void oo_destroy(oo_ctx *ctx) {
    if (!ctx) return;
    if (ctx->c.device < 0) {
        delete ctx;
        return;
    }
    cudaSetDevice(ctx->c.device);
    if (ctx->c.server) {
        server_stop(ctx->c.server);
        ctx->c.server = nullptr;
    }
    if (ctx->c.rserver) {
        resident_stop(ctx->c.rserver);
        ctx->c.rserver = nullptr;
    }
    if (ctx->c.stream) cudaStreamSynchronize(ctx->c.stream);
    stencil_plan_destroy(ctx->user_plan);
    jacobi_work_free(ctx->c.jw);
    for (auto &kv : ctx->c.fft_plans) fft_plan_destroy(kv.second);
    ctx->c.fft_scratch.release();
    ctx->c.stage_a.release();
    ctx->c.stage_b.release();
    ctx->c.stage_c.release();
    ctx->c.gemm_scratch.release();
    if (ctx->c.own_stream && ctx->c.stream) cudaStreamDestroy(ctx->c.stream);
    delete ctx;
}

oo_status oo_sync(oo_ctx *ctx) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        use_device(ctx->c, false);
        OO_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
    });
}

oo_status oo_tune_stencil(oo_ctx *ctx, int I, int J, int K, int *variant, double *ms_per_variant) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(I >= 3 && J >= 3 && K >= 3 && K <= 4096 && (long long)I * J * K < (1ll << 31), OO_EINVAL,
                   "bad grid");
        use_device(ctx->c);
        const int v = tune_stencil(ctx->c, I, J, K, ms_per_variant);
        if (variant) *variant = v;
    });
}

oo_status oo_inject_wait_timeout(oo_ctx *ctx, int what) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(what == OO_INJECT_NONE || what == OO_INJECT_STENCIL_LOAD || what == OO_INJECT_FUSED_BARRIER ||
                       what == OO_INJECT_SERVE_STALL,
                   OO_EINVAL, "unknown fault injection " + std::to_string(what));
        ctx->c.inject_wait = what;
    });
}

oo_status oo_load_nests(oo_ctx *ctx, const oo_nest *nests, int n_nests, const oo_var *vars,
                        int n_vars, uint64_t outputs, int *gene_len_out) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(nests && vars && n_nests > 0 && n_vars > 0, OO_EINVAL, "empty table");
        NestTable t;
        for (int v = 0; v < n_vars; ++v) t.vars.push_back({vars[v].name ? vars[v].name : "", vars[v].bytes});
        for (int n = 0; n < n_nests; ++n)
            t.nests.push_back({nests[n].name ? nests[n].name : "", nests[n].level,
                               nests[n].parallelisable ? 1 : 0, nests[n].reads, nests[n].writes,
                               nests[n].partial});
        t.outputs = outputs;
        validate_table(t);
        ctx->c.table = std::move(t);
        ctx->c.have_table = true;
        if (gene_len_out) *gene_len_out = ctx->c.table.gene_len();
    });
}

oo_status oo_load_jacobi_nests(oo_ctx *ctx, int I, int J, int K, int iters, int *gene_len_out) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(I >= 3 && J >= 3 && K >= 3 && iters >= 0, OO_EINVAL, "bad Jacobi problem");
        ctx->c.table = jacobi_table(I, J, K, iters);
        ctx->c.have_table = true;
        if (gene_len_out) *gene_len_out = ctx->c.table.gene_len();
    });
}

oo_status oo_transfer_plan(oo_ctx *ctx, uint64_t gene, int hoist, int iters, oo_xfer *out, int cap,
                           int *n_out, uint64_t *h2d, uint64_t *d2h) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(ctx->c.have_table, OO_ESTATE, "no loop-nest table loaded");
        OO_REQUIRE(hoist == 0 || hoist == 1, OO_EINVAL, "hoist must be 0 or 1");
        OO_REQUIRE(cap >= 0 && (cap == 0 || out), OO_EINVAL, "bad output buffer");
        const auto plan = make_plan(ctx->c.table, gene, hoist, iters, h2d, d2h);
        const size_t n = std::min(plan.size(), (size_t)cap);
        if (n) std::memcpy(out, plan.data(), n * sizeof(oo_xfer));
        if (n_out) *n_out = (int)plan.size();
    });
}

int oo_jacobi_pitch(int K) { return jacobi_pitch(K); }

oo_status oo_run_pattern(oo_ctx *ctx, uint64_t gene, int hoist, const oo_jacobi *prob, float *p_out,
                         double *res_out, oo_run_stats *stats) {
    if (!ctx || !prob) return OO_EINVAL;
    return guarded(ctx, [&] {
        use_device(ctx->c);
        run_pattern(ctx->c, gene, hoist, *prob, p_out, res_out, false, stats);
    });
}

oo_status oo_run_pattern_dev(oo_ctx *ctx, uint64_t gene, int hoist, const oo_jacobi *prob, float *p_dev,
                             double *res_dev, oo_run_stats *stats) {
    if (!ctx || !prob) return OO_EINVAL;
    return guarded(ctx, [&] {
        use_device(ctx->c);
        run_pattern(ctx->c, gene, hoist, *prob, p_dev, res_dev, true, stats);
    });
}

oo_status oo_stencil_dev(oo_ctx *ctx, int I, int J, int K, int pitch, const float *const *coef,
                         const float *p, float omega, float *wrk2, double *res_dev) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(coef && p && wrk2 && res_dev, OO_EINVAL, "null pointer");
        for (int a = 0; a < NCOEF; ++a) OO_REQUIRE(coef[a] != nullptr, OO_EINVAL, "null coefficient array");
        OO_REQUIRE(I >= 3 && J >= 3 && K >= 3 && K <= 4096, OO_EINVAL, "bad grid");
        OO_REQUIRE(pitch >= K && pitch % 4 == 0, OO_EINVAL, "pitch must be >= K and a multiple of 4");
        OO_REQUIRE(std::isfinite(omega), OO_EINVAL, "omega must be finite");
        use_device(ctx->c);
        std::vector<const void *> key(coef, coef + NCOEF);
        key.push_back(p);
        key.push_back(wrk2);
        key.push_back(reinterpret_cast<const void *>((uintptr_t)I));
        key.push_back(reinterpret_cast<const void *>((uintptr_t)J));
        key.push_back(reinterpret_cast<const void *>((uintptr_t)K));
        key.push_back(reinterpret_cast<const void *>((uintptr_t)pitch));
        const int want = ctx->c.stencil_variant_for(I, J, K);
        key.push_back(reinterpret_cast<const void *>((intptr_t)want));
        if (!ctx->user_plan || ctx->user_key != key) {
            if (ctx->user_plan) {
                OO_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
                stencil_plan_destroy(ctx->user_plan);
                ctx->user_plan = nullptr;
            }
            ctx->user_plan = stencil_plan_create(JacobiDims{I, J, K, pitch}, coef, p, wrk2, ctx->c.num_sms, want);
            ctx->user_key = key;
        }
        const bool inject = ctx->c.inject_wait == OO_INJECT_STENCIL_LOAD;
        if (inject) ctx->c.inject_wait = OO_INJECT_NONE;
        launch_stencil(ctx->user_plan, omega, res_dev, ctx->c.stream, inject);
    });
}

oo_status oo_stencil_check(oo_ctx *ctx) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        use_device(ctx->c, false);
        OO_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
        if (!ctx->user_plan) return;
        const unsigned e = stencil_plan_check(ctx->user_plan, ctx->c.stream);
        OO_REQUIRE(e == 0, OO_ETIMEOUT, "stencil pipeline wait ran out (error bits " + std::to_string(e) +
                                            "); wrk2 and the residual of that sweep are incomplete");
    });
}

oo_status oo_set_option(oo_ctx *ctx, int option, int value) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        if (option == OO_OPT_JACOBI_FUSED) {
            OO_REQUIRE(value >= -1 && value <= 1, OO_EINVAL, "OO_OPT_JACOBI_FUSED takes -1, 0 or 1");
            ctx->c.opt_fused = value;
        } else if (option == OO_OPT_STENCIL_VARIANT) {
            OO_REQUIRE(value >= -1 && value < OO_STENCIL_VARIANTS, OO_EINVAL,
                       "OO_OPT_STENCIL_VARIANT takes -1 or a variant below OO_STENCIL_VARIANTS");
            ctx->c.opt_stencil_variant = value;
        } else if (option == OO_OPT_GEMM_PAIR) {
            OO_REQUIRE(value == 0 || value == 1 || value == 160 || value == 192 || value == 224 || value == 256,
                       OO_EINVAL, "OO_OPT_GEMM_PAIR takes 0, 1, 160, 192, 224 or 256");
            ctx->c.opt_gemm_pair = value;
        } else {
            throw Error{OO_EINVAL, "unknown option " + std::to_string(option)};
        }
    });
}

oo_status oo_get_option(oo_ctx *ctx, int option, int *value) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(value, OO_EINVAL, "null pointer");
        if (option == OO_OPT_JACOBI_FUSED)
            *value = ctx->c.opt_fused;
        else if (option == OO_OPT_STENCIL_VARIANT)
            *value = ctx->c.opt_stencil_variant;
        else if (option == OO_OPT_GEMM_PAIR)
            *value = ctx->c.opt_gemm_pair;
        else
            throw Error{OO_EINVAL, "unknown option " + std::to_string(option)};
    });
}

oo_status oo_ga_table(int L, int pop, int gens, double pc, double pm, uint64_t seed,
                      const double *time_of_gene, uint64_t *history, uint64_t *best_gene,
                      double *best_time) {
    return guarded(nullptr, [&] {
        OO_REQUIRE(L >= 1 && L <= 20, OO_EINVAL, "table GA needs 1 <= L <= 20");
        OO_REQUIRE(time_of_gene && best_gene && best_time, OO_EINVAL, "null pointer");
        const GaResult r = ga_run(L, pop, gens, pc, pm, seed,
                                  [&](uint64_t g) { return time_of_gene[g]; });
        if (history) std::memcpy(history, r.history.data(), r.history.size() * 8);
        *best_gene = r.best_gene;
        *best_time = r.best_time;
    });
}

namespace {
// Sec. 4.2.2 GA over measured patterns; known_ms (2^6 entries, NaN =
// not known) seeds the per-gene memo, so a search can resume from a saved
// table: genes with a known time are not measured again, and with the same
// seed and times the GA makes the same choices.
oo_status ga_search(oo_ctx *ctx, const oo_jacobi *prob, int hoist, int pop, int gens, double pc, double pm,
                    uint64_t seed, double eval_timeout_ms, const double *known_ms, uint64_t *best_gene,
                    double *best_ms, uint64_t *history, double *gene_ms) {
    if (!ctx || !prob) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(best_gene && best_ms, OO_EINVAL, "null pointer");
        const int L = 6;
        std::map<uint64_t, double> memo;
        if (known_ms)
            for (int g = 0; g < (1 << L); ++g)
                if (!std::isnan(known_ms[g])) {
                    OO_REQUIRE(known_ms[g] > 0.0, OO_EINVAL, "known times must be positive, INFINITY or NaN");
                    memo[(uint64_t)g] = known_ms[g];
                }
        std::vector<float> p;
        std::vector<double> res;
        auto measure = [&](uint64_t g) -> double {
            auto it = memo.find(g);
            if (it != memo.end()) return it->second;
            use_device(ctx->c);
            const Ctx::Ref &ref = cpu_reference(ctx->c, *prob);
            p.resize((size_t)prob->I * prob->J * prob->K);
            res.resize((size_t)prob->iters);
            oo_run_stats st{};
            bool aborted = false;
            oo_jacobi q = *prob;
            q.timing = 0;
            run_pattern(ctx->c, g, hoist, q, p.data(), res.data(), false, &st, eval_timeout_ms, &aborted);
            double t = aborted ? INFINITY : st.wall_ms;
            if (!aborted) {
                // Sec. 4.2.2: a result that differs from the original beyond
                // tolerance counts as infinitely slow
                for (size_t x = 0; x < res.size(); ++x)
                    if (!(std::fabs(res[x] - ref.res[x]) <= 1e-5 * std::fabs(ref.res[x]))) t = INFINITY;
                for (size_t x = 0; x < p.size() && std::isfinite(t); ++x)
                    if (!(std::fabs(p[x] - ref.p[x]) <= 1e-5f)) t = INFINITY;
            }
            memo[g] = t;
            return t;
        };
        const GaResult r = ga_run(L, pop, gens, pc, pm, seed, measure);
        if (history) std::memcpy(history, r.history.data(), r.history.size() * 8);
        if (gene_ms) {
            for (int g = 0; g < (1 << L); ++g) gene_ms[g] = INFINITY;
            for (const auto &kv : memo) gene_ms[kv.first] = kv.second;
        }
        *best_gene = r.best_gene;
        *best_ms = r.best_time;
    });
}
}  // namespace

oo_status oo_ga_search(oo_ctx *ctx, const oo_jacobi *prob, int hoist, int pop, int gens, double pc, double pm,
                       uint64_t seed, double eval_timeout_ms, uint64_t *best_gene, double *best_ms,
                       uint64_t *history, double *gene_ms) {
    return ga_search(ctx, prob, hoist, pop, gens, pc, pm, seed, eval_timeout_ms, nullptr, best_gene, best_ms,
                     history, gene_ms);
}

oo_status oo_ga_search_resume(oo_ctx *ctx, const oo_jacobi *prob, int hoist, int pop, int gens, double pc,
                              double pm, uint64_t seed, double eval_timeout_ms, const double *known_ms,
                              uint64_t *best_gene, double *best_ms, uint64_t *history, double *gene_ms) {
    if (!known_ms) return OO_EINVAL;
    return ga_search(ctx, prob, hoist, pop, gens, pc, pm, seed, eval_timeout_ms, known_ms, best_gene, best_ms,
                     history, gene_ms);
}

oo_status oo_fft_c128_dev(oo_ctx *ctx, int64_t n, int batch, int dir, const double *din, double *dout) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(din && dout, OO_EINVAL, "null pointer");
        OO_REQUIRE((((uintptr_t)din) & 15u) == 0 && (((uintptr_t)dout) & 15u) == 0, OO_EINVAL,
                   "FFT buffers must be 16-byte aligned");
        use_device(ctx->c);
        FftPlan *p = ctx->c.fft_plan(n);
        void *scratch = ctx->c.fft_scratch.get(fft_scratch_bytes(p, batch));
        launch_fft(p, batch, dir, din, dout, scratch, ctx->c.stream);
    });
}

namespace {
// host buffers in / out through the context's staging buffers, synchronous
void fft_host(oo_ctx *ctx, int64_t n, int dir, const double *in, double *out) {
    FftPlan *p = ctx->c.fft_plan(n);
    const size_t bytes = (size_t)n * 16;
    double *d = static_cast<double *>(ctx->c.stage_a.get(bytes));
    void *scratch = ctx->c.fft_scratch.get(fft_scratch_bytes(p, 1));
    OO_CUDA_TRY(cudaMemcpyAsync(d, in, bytes, cudaMemcpyHostToDevice, ctx->c.stream));
    launch_fft(p, 1, dir, d, d, scratch, ctx->c.stream);
    OO_CUDA_TRY(cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, ctx->c.stream));
    OO_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
}
}  // namespace

oo_status oo_fft_c128(oo_ctx *ctx, int64_t n, int dir, const double *in, double *out) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(in && out, OO_EINVAL, "null pointer");
        use_device(ctx->c);
        fft_host(ctx, n, dir, in, out);
    });
}

namespace {
void gemm_checks(int prec, int m, int n, int k, int lda, int ldb, int ldc) {
    OO_REQUIRE(prec == OO_PREC_SPLIT3_BF16 || prec == OO_PREC_SPLIT3_TF32 || prec == OO_PREC_FP64EQ, OO_EINVAL,
               "unsupported precision pattern");
    OO_REQUIRE(m >= 1 && n >= 1 && k >= 1, OO_EINVAL, "m, n, k must be >= 1");
    OO_REQUIRE(m <= (1 << 20) && n <= (1 << 20) && k <= (1 << 21), OO_EINVAL, "matrix too large");
    OO_REQUIRE(lda >= k && ldb >= n && ldc >= n, OO_EINVAL, "leading dimension too small");
}
size_t gemm_scratch(int prec, int m, int n, int k) {
    if (prec == OO_PREC_FP64EQ) return gemm_fp64eq_scratch_bytes(m, n, k);
    return prec == OO_PREC_SPLIT3_TF32 ? gemm_tf32_scratch_bytes(m, n, k) : gemm_scratch_bytes(m, n, k);
}
void gemm_launch(oo_ctx *ctx, int prec, int m, int n, int k, const double *dA, long long lda, const double *dB,
                 long long ldb, double *dC, long long ldc, cudaStream_t s) {
    void *scratch = ctx->c.gemm_scratch.get(gemm_scratch(prec, m, n, k));
    ctx->gemm_prec = prec;
    if (prec == OO_PREC_FP64EQ)
        launch_gemm_fp64eq(m, n, k, dA, lda, dB, ldb, dC, ldc, scratch, s,
                           eq_tile_width(ctx->c.eq_widths.data(), n, k), ctx->c.opt_gemm_pair != 0);
    else if (prec == OO_PREC_SPLIT3_TF32)
        launch_gemm_split3_tf32(m, n, k, dA, lda, dB, ldb, dC, ldc, scratch, s);
    else
        launch_gemm_split3(m, n, k, dA, lda, dB, ldb, dC, ldc, scratch, s, ctx->c.opt_gemm_pair);
}
unsigned gemm_error(oo_ctx *ctx, int m, int n, int k) {
    void *scratch = ctx->c.gemm_scratch.ptr;
    if (ctx->gemm_prec == OO_PREC_FP64EQ) return gemm_fp64eq_check_error(scratch, ctx->c.stream);
    if (ctx->gemm_prec == OO_PREC_SPLIT3_TF32) {
        unsigned *err = gemm_tf32_error_word(scratch, m, n, k);
        unsigned e = 0;
        OO_CUDA_TRY(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, ctx->c.stream));
        OO_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
        if (e) OO_CUDA_TRY(cudaMemsetAsync(err, 0, 4, ctx->c.stream));
        return e;
    }
    return gemm_check_error(scratch, m, n, k, ctx->c.stream);
}
}  // namespace

oo_status oo_gemm_f64_dev(oo_ctx *ctx, int prec, int m, int n, int k, const double *dA, int lda,
                          const double *dB, int ldb, double *dC, int ldc) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(dA && dB && dC, OO_EINVAL, "null pointer");
        gemm_checks(prec, m, n, k, lda, ldb, ldc);
        use_device(ctx->c);
        gemm_launch(ctx, prec, m, n, k, dA, lda, dB, ldb, dC, ldc, ctx->c.stream);
    });
}

namespace {
void gemm_host(oo_ctx *ctx, int prec, int m, int n, int k, const double *A, int lda, const double *B, int ldb,
               double *C, int ldc) {
    cudaStream_t s = ctx->c.stream;
    double *dA = static_cast<double *>(ctx->c.stage_a.get((size_t)m * k * 8));
    double *dB = static_cast<double *>(ctx->c.stage_b.get((size_t)k * n * 8));
    double *dC = static_cast<double *>(ctx->c.stage_c.get((size_t)m * n * 8));
    OO_CUDA_TRY(cudaMemcpy2DAsync(dA, (size_t)k * 8, A, (size_t)lda * 8, (size_t)k * 8, m, cudaMemcpyHostToDevice, s));
    OO_CUDA_TRY(cudaMemcpy2DAsync(dB, (size_t)n * 8, B, (size_t)ldb * 8, (size_t)n * 8, k, cudaMemcpyHostToDevice, s));
    gemm_launch(ctx, prec, m, n, k, dA, k, dB, n, dC, n, s);
    OO_CUDA_TRY(cudaMemcpy2DAsync(C, (size_t)ldc * 8, dC, (size_t)n * 8, (size_t)n * 8, m, cudaMemcpyDeviceToHost, s));
    const unsigned e = gemm_error(ctx, m, n, k);
    OO_REQUIRE(e == 0, OO_ETIMEOUT, "GEMM pipeline wait ran out (error bits " + std::to_string(e) + ")");
}
}  // namespace

namespace {
// the offloaded form of a function-block site (host buffers, synchronous)
FbGpu fb_gpu(oo_ctx *ctx) {
    return [ctx](int prec, int block, const oo_fb_site &s, const double *a, const double *b, double *out) {
        if (block == OO_BLOCK_GEMM)
            gemm_host(ctx, prec, (int)s.m, (int)s.n, (int)s.k, a, (int)s.k, b, (int)s.n, out, (int)s.n);
        else
            fft_host(ctx, s.n, -1, a, out);
    };
}
}  // namespace

oo_status oo_gemm_f64(oo_ctx *ctx, int prec, int m, int n, int k, const double *A, int lda, const double *B,
                      int ldb, double *C, int ldc) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(A && B && C, OO_EINVAL, "null pointer");
        gemm_checks(prec, m, n, k, lda, ldb, ldc);
        use_device(ctx->c);
        gemm_host(ctx, prec, m, n, k, A, lda, B, ldb, C, ldc);
    });
}

oo_status oo_gemm_check(oo_ctx *ctx, int m, int n, int k) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        use_device(ctx->c);
        OO_REQUIRE(ctx->gemm_prec >= 0 && ctx->c.gemm_scratch.ptr &&
                       ctx->c.gemm_scratch.bytes >= gemm_scratch(ctx->gemm_prec, m, n, k),
                   OO_ESTATE, "no GEMM of that shape has run on this context");
        const unsigned e = gemm_error(ctx, m, n, k);
        OO_REQUIRE(e == 0, OO_ETIMEOUT, "GEMM pipeline wait ran out (error bits " + std::to_string(e) + ")");
    });
}

oo_status oo_gemm_plan(int prec, int k, int *products, int *beta, int *levels, int *k_block) {
    return guarded(nullptr, [&] {
        OO_REQUIRE(prec == OO_PREC_SPLIT3_BF16 || prec == OO_PREC_SPLIT3_TF32 || prec == OO_PREC_FP64EQ, OO_EINVAL,
                   "unsupported precision pattern");
        OO_REQUIRE(k >= 1 && k <= (1 << 21), OO_EINVAL, "k out of range");
        int pr = 3, b = 0, l = 0, kb = 0;
        if (prec == OO_PREC_FP64EQ) {
            pr = gemm_fp64eq_products(k);
            gemm_fp64eq_shape(k, &b, &l, &kb);
        }
        if (products) *products = pr;
        if (beta) *beta = b;
        if (levels) *levels = l;
        if (k_block) *k_block = kb;
    });
}

oo_status oo_gemm_scheme(int k, int *scheme, int *per_accumulator) {
    return guarded(nullptr, [&] {
        OO_REQUIRE(k >= 1 && k <= (1 << 21), OO_EINVAL, "k out of range");
        const int s = eq_scheme_for(k);
        int L = 0;
        gemm_fp64eq_shape(k, nullptr, &L, nullptr);
        if (scheme) *scheme = s == 0 ? OO_EQ_PAIRS : OO_EQ_LEVELS;
        if (per_accumulator) *per_accumulator = s == 0 ? 1 : L - 1;
    });
}

oo_status oo_get_gemm_tiles(oo_ctx *ctx, int *widths) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(widths, OO_EINVAL, "null pointer");
        for (int nb = 0; nb < OO_TILE_NBUCKETS; ++nb)
            for (int kb = 0; kb < OO_TILE_KBUCKETS; ++kb) {
                const int i = nb * OO_TILE_KBUCKETS + kb;
                widths[i] = ctx->c.eq_widths[i] ? ctx->c.eq_widths[i] : eq_default_width(nb, kb);
            }
    });
}

oo_status oo_set_gemm_tiles(oo_ctx *ctx, const int *widths) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(widths, OO_EINVAL, "null pointer");
        for (int i = 0; i < OO_TILE_NBUCKETS * OO_TILE_KBUCKETS; ++i)
            OO_REQUIRE(widths[i] == 32 || widths[i] == 64 || widths[i] == 128, OO_EINVAL,
                       "tile widths must be 32, 64 or 128");
        for (int i = 0; i < OO_TILE_NBUCKETS * OO_TILE_KBUCKETS; ++i) ctx->c.eq_widths[i] = widths[i];
    });
}

oo_status oo_tune_gemm_tiles(oo_ctx *ctx, int *widths, double *ms) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        use_device(ctx->c);
        tune_gemm_tiles(ctx->c, ms);
        if (widths)
            for (int nb = 0; nb < OO_TILE_NBUCKETS; ++nb)
                for (int kb = 0; kb < OO_TILE_KBUCKETS; ++kb) {
                    const int i = nb * OO_TILE_KBUCKETS + kb;
                    widths[i] = ctx->c.eq_widths[i];
                }
    });
}

oo_status oo_lookup_block(const char *callee, int lang, int *block_id) {
    return guarded(nullptr, [&] {
        OO_REQUIRE(callee && block_id, OO_EINVAL, "null pointer");
        OO_REQUIRE(lang >= OO_LANG_C && lang <= OO_LANG_JAVA, OO_EINVAL, "unknown language");
        const int b = lookup_block(callee, lang);
        OO_REQUIRE(b != 0, OO_ENOTFOUND, std::string("no code pattern for ") + callee);
        *block_id = b;
    });
}

oo_status oo_fb_search(oo_ctx *ctx, const oo_fb_site *sites, int n_sites, int prec, double tol, uint64_t seed,
                       int32_t *block_ids, double *mask_ms, uint32_t *best_mask, double *best_ms) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(best_mask && best_ms, OO_EINVAL, "null pointer");
        OO_REQUIRE(prec == OO_PREC_SPLIT3_BF16 || prec == OO_PREC_FP64EQ, OO_EINVAL, "unsupported precision pattern");
        use_device(ctx->c);
        std::vector<double> ms;
        std::vector<int> ids;
        fb_trial(sites, n_sites, prec, tol, seed, ms, ids, fb_gpu(ctx));
        if (block_ids)
            for (int i = 0; i < n_sites; ++i) block_ids[i] = ids[i];
        if (mask_ms) std::memcpy(mask_ms, ms.data(), ms.size() * sizeof(double));
        *best_mask = fb_best(ms.data(), n_sites, best_ms);
    });
}

oo_status oo_fb_best(int n_sites, const double *mask_ms, uint32_t *best_mask, double *best_ms) {
    return guarded(nullptr, [&] {
        OO_REQUIRE(n_sites >= 1 && n_sites <= 12, OO_EINVAL, "1..12 function-block sites");
        OO_REQUIRE(mask_ms && best_mask, OO_EINVAL, "null pointer");
        for (uint32_t m = 0; m < (1u << n_sites); ++m)
            OO_REQUIRE(!std::isnan(mask_ms[m]), OO_EINVAL, "NaN in the time table");
        *best_mask = fb_best(mask_ms, n_sites, best_ms);
    });
}

oo_status oo_offload_search(oo_ctx *ctx, const oo_fb_site *sites, int n_sites, int prec, double tol,
                            uint64_t seed, const oo_jacobi *prob, int hoist, int pop, int gens, double pc,
                            double pm, uint64_t ga_seed, double eval_timeout_ms, uint32_t *best_mask,
                            uint64_t *best_gene, double *fb_ms, double *loop_ms) {
    if (!ctx || !prob) return OO_EINVAL;
    // Sec. 4.2: function blocks first ...
    oo_status st = OO_OK;
    if (n_sites > 0) {
        st = oo_fb_search(ctx, sites, n_sites, prec, tol, seed, nullptr, nullptr, best_mask, fb_ms);
        if (st != OO_OK) return st;
    } else {
        if (!best_mask || !fb_ms) return OO_EINVAL;
        *best_mask = 0;
        *fb_ms = 0.0;
    }
    // ... then the loop GA on the code outside them (the program's loop
    // nests are not part of any library call site)
    return oo_ga_search(ctx, prob, hoist, pop, gens, pc, pm, ga_seed, eval_timeout_ms, best_gene, loop_ms, nullptr,
                        nullptr);
}

oo_status oo_run_program(oo_ctx *ctx, uint64_t gene, int hoist, int iters, oo_nest_fn fn, void *user,
                         void *const *host_vars, void *const *dev_vars, oo_run_stats *stats) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        use_device(ctx->c);
        run_program(ctx->c, gene, hoist, iters, fn, user, host_vars, dev_vars, stats);
    });
}

oo_status oo_ga_program(oo_ctx *ctx, int hoist, int iters, oo_nest_fn fn, oo_check_fn check, void *user,
                        void *const *host_vars, void *const *dev_vars, int pop, int gens, double pc,
                        double pm, uint64_t seed, uint64_t *best_gene, double *best_ms, uint64_t *history,
                        double *gene_ms) {
    if (!ctx) return OO_EINVAL;
    return guarded(ctx, [&] {
        OO_REQUIRE(best_gene && best_ms, OO_EINVAL, "null pointer");
        use_device(ctx->c);
        std::vector<double> gm;
        const GaResult r = ga_program(ctx->c, hoist, iters, fn, check, user, host_vars, dev_vars, pop, gens, pc,
                                      pm, seed, gene_ms ? &gm : nullptr);
        if (history) std::memcpy(history, r.history.data(), r.history.size() * 8);
        if (gene_ms) std::memcpy(gene_ms, gm.data(), gm.size() * sizeof(double));
        *best_gene = r.best_gene;
        *best_ms = r.best_time;
    });
}

}  // extern "C"
