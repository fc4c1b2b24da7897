// Execution of an offload pattern of the Jacobi program.
//
// Sec. 3.2.1 / Sec. 4.2.2: the gene places each parallelisable nest on the
// GPU (1) or CPU (0); the transfer plan for the placement (hoisted or not)
// says which variables cross between host and device before which nest.
// This file walks the program order, issues the planned copies on the
// context's stream, launches GPU nests there and runs CPU nests on the host
// after synchronising, then delivers the outputs p and res.  Host arrays are
// the library's pinned buffers (unpadded, k fastest); device arrays use the
// padded row pitch the kernels want; copies between the two are 2D.
// Adjacent GPU nests with no copy between them share launches: N3 + N4 + N5
// in one pass, and on small grids every iteration in one cooperative kernel
// (per-nest timing keeps all nests apart).
#include <chrono>
#include <cmath>
#include <cstring>

#include "oo_internal.h"

namespace oo {

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

void free_work(JacobiWork *w) {
    if (!w) return;
    stencil_plan_destroy(w->splan);
    if (w->fused_ctl) cudaFree(w->fused_ctl);
    if (w->dev) cudaFree(w->dev);
    if (w->res_dev) cudaFree(w->res_dev);
    if (w->host) cudaFreeHost(w->host);
    if (w->res_host) cudaFreeHost(w->res_host);
    delete w;
}

JacobiWork *ensure_work(Ctx &c, int I, int J, int K, int iters) {
    JacobiWork *w = c.jw;
    if (w && w->d.I == I && w->d.J == J && w->d.K == K) {
        // the plan follows the context's current variant choice
        int want = c.stencil_variant_for(I, J, K);
        if (want < 0 || want >= stencil_variant_count()) want = stencil_default_variant(w->d);
        if (stencil_plan_variant(w->splan) != want) {
            OO_CUDA_TRY(cudaStreamSynchronize(c.stream));
            const float *coef[NCOEF];
            for (int a = 0; a < NCOEF; ++a) coef[a] = w->dptr(a);
            StencilPlan *np = stencil_plan_create(w->d, coef, w->dptr(VAR_P), w->dptr(VAR_WRK2), c.num_sms, want);
            stencil_plan_destroy(w->splan);
            w->splan = np;
        }
    }
    if (w && w->d.I == I && w->d.J == J && w->d.K == K && w->iters_cap >= std::max(iters, 1)) return w;
    if (w && w->d.I == I && w->d.J == J && w->d.K == K) {
        // only the residual buffers are too small
        const int cap = std::max(iters, 1);
        double *rd = nullptr, *rh = nullptr;
        OO_CUDA_TRY(cudaMalloc(&rd, (size_t)cap * 8));
        if (cudaHostAlloc(&rh, (size_t)cap * 8, cudaHostAllocDefault) != cudaSuccess) {
            cudaFree(rd);
            throw Error{OO_ENOMEM, "pinned residual buffer"};
        }
        cudaFree(w->res_dev);
        cudaFreeHost(w->res_host);
        w->res_dev = rd;
        w->res_host = rh;
        w->iters_cap = cap;
        return w;
    }
    free_work(w);
    c.jw = nullptr;
    w = new JacobiWork();
    try {
        w->d = JacobiDims{I, J, K, jacobi_pitch(K)};
        w->iters_cap = std::max(iters, 1);
        w->dev_stride = (w->d.n_dev() + 63) / 64 * 64;
        if (cudaMalloc(&w->dev, (size_t)NARR * w->dev_stride * 4) != cudaSuccess) {
            cudaGetLastError();
            throw Error{OO_ENOMEM, "device arrays of the Jacobi program"};
        }
        OO_CUDA_TRY(cudaMalloc(&w->res_dev, (size_t)w->iters_cap * 8));
        if (cudaHostAlloc(&w->host, (size_t)NARR * w->d.n_host() * 4, cudaHostAllocDefault) !=
            cudaSuccess) {
            cudaGetLastError();
            throw Error{OO_ENOMEM, "pinned host arrays of the Jacobi program"};
        }
        OO_CUDA_TRY(cudaHostAlloc(&w->res_host, (size_t)w->iters_cap * 8, cudaHostAllocDefault));
        const float *coef[NCOEF];
        for (int a = 0; a < NCOEF; ++a) coef[a] = w->dptr(a);
        w->splan = stencil_plan_create(w->d, coef, w->dptr(VAR_P), w->dptr(VAR_WRK2), c.num_sms,
                                       c.stencil_variant_for(I, J, K));
        OO_CUDA_TRY(cudaMalloc(&w->fused_ctl, jacobi_fused_ctl_bytes()));
    } catch (...) {
        free_work(w);
        throw;
    }
    c.jw = w;
    return w;
}

// Copy variable v between the host workspace and the device workspace.
void copy_var(JacobiWork &w, int v, int dir, int iters, cudaStream_t s) {
    if (v == VAR_RES) {
        const size_t bytes = (size_t)iters * 8;
        if (bytes == 0) return;
        if (dir > 0)
            OO_CUDA_TRY(cudaMemcpyAsync(w.res_dev, w.res_host, bytes, cudaMemcpyHostToDevice, s));
        else
            OO_CUDA_TRY(cudaMemcpyAsync(w.res_host, w.res_dev, bytes, cudaMemcpyDeviceToHost, s));
        return;
    }
    const size_t wb = (size_t)w.d.K * 4, rows = (size_t)w.d.I * w.d.J;
    if (dir > 0)
        OO_CUDA_TRY(cudaMemcpy2DAsync(w.dptr(v), (size_t)w.d.pitch * 4, w.hptr(v), wb, wb, rows,
                                      cudaMemcpyHostToDevice, s));
    else
        OO_CUDA_TRY(cudaMemcpy2DAsync(w.hptr(v), wb, w.dptr(v), (size_t)w.d.pitch * 4, wb, rows,
                                      cudaMemcpyDeviceToHost, s));
}

}  // namespace

void jacobi_work_free(JacobiWork *w) { free_work(w); }

// Time every stencil tile variant on the context's workspace for this grid
// (its arrays hold whatever the last run left; every pattern run rewrites
// them with its setup nests, and the variants' timing does not depend on the
// values) and keep the fastest for the grid: the workspace's plan is remade
// with it now, and any later workspace for the grid uses it too.
int tune_stencil(Ctx &c, int I, int J, int K, double *ms_out) {
    JacobiWork &w = *ensure_work(c, I, J, K, 1);
    cudaStream_t s = c.stream;
    const float *coef[NCOEF];
    for (int a = 0; a < NCOEF; ++a) coef[a] = w.dptr(a);
    const int nv = stencil_variant_count();
    OO_REQUIRE(nv == OO_STENCIL_VARIANTS, OO_ESTATE, "stencil variant table and OO_STENCIL_VARIANTS disagree");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    OO_CUDA_TRY(cudaEventCreate(&e0));
    OO_CUDA_TRY(cudaEventCreate(&e1));
    int best = -1;
    float best_ms = 0.f;
    try {
        for (int v = 0; v < nv; ++v) {
            StencilPlan *sp = stencil_plan_create(w.d, coef, w.dptr(VAR_P), w.dptr(VAR_WRK2), c.num_sms, v);
            float ms = 0.f;
            try {
                launch_stencil(sp, 0.8f, w.res_dev, s);  // warm-up (kernel attributes, caches)
                const unsigned e = stencil_plan_check(sp, s);
                OO_REQUIRE(e == 0, OO_ETIMEOUT, "stencil pipeline wait ran out while tuning variant " +
                                                   std::to_string(v));
                constexpr int kReps = 3;
                OO_CUDA_TRY(cudaEventRecord(e0, s));
                for (int r = 0; r < kReps; ++r) launch_stencil(sp, 0.8f, w.res_dev, s);
                OO_CUDA_TRY(cudaEventRecord(e1, s));
                OO_CUDA_TRY(cudaEventSynchronize(e1));
                OO_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                ms /= kReps;
                const unsigned e2 = stencil_plan_check(sp, s);
                OO_REQUIRE(e2 == 0, OO_ETIMEOUT, "stencil pipeline wait ran out while tuning variant " +
                                                    std::to_string(v));
            } catch (...) {
                stencil_plan_destroy(sp);
                throw;
            }
            stencil_plan_destroy(sp);
            if (ms_out) ms_out[v] = ms;
            if (best < 0 || ms < best_ms) {
                best = v;
                best_ms = ms;
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bool found = false;
    for (auto &x : c.stencil_choice)
        if (x[0] == I && x[1] == J && x[2] == K) {
            x[3] = best;
            found = true;
        }
    if (!found) c.stencil_choice.push_back({I, J, K, best});
    StencilPlan *np = stencil_plan_create(w.d, coef, w.dptr(VAR_P), w.dptr(VAR_WRK2), c.num_sms, best);
    stencil_plan_destroy(w.splan);
    w.splan = np;
    return best;
}

void run_pattern(Ctx &c, uint64_t gene, int hoist, const oo_jacobi &prob, float *p_out,
                 double *res_out, bool out_on_device, oo_run_stats *stats, double abort_after_ms,
                 bool *aborted) {
    OO_REQUIRE(prob.I >= 3 && prob.J >= 3 && prob.K >= 3, OO_EINVAL, "grid must be at least 3 x 3 x 3");
    OO_REQUIRE(prob.K <= 4096 && prob.iters >= 0, OO_EINVAL, "K must be <= 4096 and iters >= 0");
    OO_REQUIRE((size_t)prob.I * prob.J * prob.K < (1ull << 34), OO_EINVAL, "grid too large");
    OO_REQUIRE(hoist == 0 || hoist == 1, OO_EINVAL, "hoist must be 0 or 1");
    OO_REQUIRE(std::isfinite(prob.omega), OO_EINVAL, "omega must be finite");
    const int iters = prob.iters;
    const NestTable t = jacobi_table(prob.I, prob.J, prob.K, iters);
    OO_REQUIRE((gene >> 6) == 0, OO_EINVAL, "the Jacobi program has a 6-bit gene");
    uint64_t h2d = 0, d2h = 0;
    const std::vector<oo_xfer> plan = make_plan(t, gene, hoist, iters, &h2d, &d2h);
    const std::vector<int> gpu = t.placement(gene);
    JacobiWork &w = *ensure_work(c, prob.I, prob.J, prob.K, iters);
    const JacobiDims &d = w.d;
    cudaStream_t s = c.stream;
    if (aborted) *aborted = false;

    float *hc[NCOEF];
    float *dc[NCOEF];
    for (int a = 0; a < NCOEF; ++a) {
        hc[a] = w.hptr(a);
        dc[a] = w.dptr(a);
    }
    const bool timing = prob.timing != 0;
    std::vector<cudaEvent_t> evs;
    std::vector<int> ev_nest;
    double nest_ms[6] = {0, 0, 0, 0, 0, 0};
    double xfer_ms = 0.0;
    int launches = 0;
    bool stencil_on_gpu = false;

    OO_CUDA_TRY(cudaStreamSynchronize(s));
    const Clock::time_point t0 = Clock::now();

    const int n_points = 2 + 4 * iters;
    size_t xi = 0;
    auto run_transfers = [&](int point) {
        while (xi < plan.size() && plan[xi].point == point) {
            if (point == n_points) break;  // outputs are delivered below
            copy_var(w, plan[xi].var, plan[xi].dir, iters, s);
            ++xi;
        }
    };
    auto run_nest = [&](int n, int it) {
        if (gpu[n]) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (timing) {
                OO_CUDA_TRY(cudaEventCreate(&e0));
                OO_CUDA_TRY(cudaEventCreate(&e1));
                OO_CUDA_TRY(cudaEventRecord(e0, s));
            }
            switch (n) {
                case 0: launch_coef(d, dc, s); break;
                case 1: launch_pinit(d, w.dptr(VAR_P), w.dptr(VAR_WRK2), s); break;
                case 2: {
                    // a fault injection armed on the context (one-shot)
                    // applies to the next stencil sweep launched
                    const bool inject = c.inject_wait == OO_INJECT_STENCIL_LOAD;
                    if (inject) c.inject_wait = OO_INJECT_NONE;
                    launch_stencil(w.splan, prob.omega, w.res_dev + it, s, inject);
                    if (!stencil_on_gpu) {
                        // a pipeline wait that ran out would repeat in every
                        // sweep: check the first one before queueing the rest
                        const unsigned e = stencil_plan_check(w.splan, s);
                        OO_REQUIRE(e == 0, OO_ETIMEOUT,
                                   "stencil kernel pipeline wait ran out (error bits " +
                                       std::to_string(e) + ")");
                    }
                    stencil_on_gpu = true;
                    break;
                }
                case 3: launch_copyback(d, w.dptr(VAR_P), w.dptr(VAR_WRK2), s); break;
                case 4: launch_bc_ij(d, w.dptr(VAR_P), s); break;
                case 5: launch_bc_k(d, w.dptr(VAR_P), s); break;
            }
            ++launches;
            if (timing) {
                OO_CUDA_TRY(cudaEventRecord(e1, s));
                evs.push_back(e0);
                evs.push_back(e1);
                ev_nest.push_back(n);
            }
        } else {
            const Clock::time_point ts = Clock::now();
            OO_CUDA_TRY(cudaStreamSynchronize(s));
            const Clock::time_point th = Clock::now();
            xfer_ms += std::chrono::duration<double, std::milli>(th - ts).count();
            switch (n) {
                case 0: host_coef(d, hc); break;
                case 1: host_pinit(d, w.hptr(VAR_P), w.hptr(VAR_WRK2)); break;
                case 2: w.res_host[it] = host_stencil(d, hc, w.hptr(VAR_P), prob.omega, w.hptr(VAR_WRK2)); break;
                case 3: host_copyback(d, w.hptr(VAR_P), w.hptr(VAR_WRK2)); break;
                case 4: host_bc_ij(d, w.hptr(VAR_P)); break;
                case 5: host_bc_k(d, w.hptr(VAR_P)); break;
            }
            nest_ms[n] += ms_since(th);
        }
    };

    int point = 0;
    bool stop = false;
    for (int n = 0; n < 2; ++n) {
        run_transfers(point++);
        run_nest(n, 0);
    }
    // All four iteration nests on the GPU with no copy inside the loop (the
    // hoisted plan): small grids run every iteration in one cooperative
    // launch instead of 4 x iters launches (per-nest timing keeps the
    // separate kernels).
    bool fused = false;
    if (!timing && iters > 0 && gpu[2] && gpu[3] && gpu[4] && gpu[5] && jacobi_fused_eligible(d, c.opt_fused)) {
        fused = true;
        for (const auto &x : plan)
            if (x.point > 2 && x.point < n_points) fused = false;
    }
    if (fused) {
        run_transfers(point);
        const bool inject = c.inject_wait == OO_INJECT_FUSED_BARRIER;
        if (inject) c.inject_wait = OO_INJECT_NONE;
        launch_jacobi_fused(d, dc, w.dptr(VAR_P), w.dptr(VAR_WRK2), prob.omega, iters, w.res_dev, w.fused_ctl, s,
                            inject);
        ++launches;
        point = n_points;
        // one launch holds every iteration, so an evaluation time limit can
        // only be measured as a whole
        if (abort_after_ms > 0.0) {
            OO_CUDA_TRY(cudaStreamSynchronize(s));
            if (ms_since(t0) > abort_after_ms) stop = true;
        }
    }
    // N3, N4 and N5 on the GPU with no copy between them: one pass writes
    // what the three leave (interior from wrk2, faces g), instead of three
    // launches; per-nest timing keeps them apart
    std::vector<char> xfer_at((size_t)n_points + 1, 0);
    for (const auto &x : plan)
        if (x.point >= 0 && x.point <= n_points) xfer_at[x.point] = 1;
    const bool tail_on_gpu = !timing && gpu[3] && gpu[4] && gpu[5];
    for (int it = 0; it < iters && !stop && !fused; ++it) {
        for (int n = 2; n < 6; ++n) {
            if (n == 3 && tail_on_gpu && !xfer_at[point + 1] && !xfer_at[point + 2]) {
                run_transfers(point);
                launch_copyback_faces(d, w.dptr(VAR_P), w.dptr(VAR_WRK2), s);
                ++launches;
                point += 3;
                break;
            }
            run_transfers(point++);
            run_nest(n, it);
        }
        if (abort_after_ms > 0.0 && ms_since(t0) > abort_after_ms) stop = true;
    }
    if (stop) {
        OO_CUDA_TRY(cudaStreamSynchronize(s));
        for (auto e : evs) cudaEventDestroy(e);
        if (aborted) *aborted = true;
        if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            stats->wall_ms = INFINITY;
        }
        return;
    }

    // deliver the outputs: the end-of-program copies land directly in the
    // caller's buffers; outputs already current on the host are copied there
    const size_t wb = (size_t)d.K * 4, rows = (size_t)d.I * d.J;
    bool p_dev_valid = false, res_dev_valid = false;
    for (size_t x = xi; x < plan.size(); ++x) {
        if (plan[x].point != n_points) continue;
        if (plan[x].var == VAR_P) p_dev_valid = true;
        if (plan[x].var == VAR_RES) res_dev_valid = true;
    }
    const cudaMemcpyKind from_dev = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind from_host = out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    if ((p_out && !p_dev_valid) || (res_out && !res_dev_valid))
        OO_CUDA_TRY(cudaStreamSynchronize(s));  // host copies must be complete
    if (p_out) {
        if (p_dev_valid)
            OO_CUDA_TRY(cudaMemcpy2DAsync(p_out, wb, w.dptr(VAR_P), (size_t)d.pitch * 4, wb, rows, from_dev, s));
        else if (out_on_device)
            OO_CUDA_TRY(cudaMemcpyAsync(p_out, w.hptr(VAR_P), wb * rows, from_host, s));
        else
            std::memcpy(p_out, w.hptr(VAR_P), wb * rows);
    }
    if (res_out && iters > 0) {
        if (res_dev_valid)
            OO_CUDA_TRY(cudaMemcpyAsync(res_out, w.res_dev, (size_t)iters * 8, from_dev, s));
        else if (out_on_device)
            OO_CUDA_TRY(cudaMemcpyAsync(res_out, w.res_host, (size_t)iters * 8, from_host, s));
        else
            std::memcpy(res_out, w.res_host, (size_t)iters * 8);
    }
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    const double wall = ms_since(t0);
    if (stencil_on_gpu) {
        const unsigned e = stencil_plan_check(w.splan, s);
        OO_REQUIRE(e == 0, OO_ETIMEOUT,
                   "stencil kernel pipeline wait ran out (error bits " + std::to_string(e) + ")");
    }
    if (fused) {
        const unsigned e = jacobi_fused_check(w.fused_ctl, s);
        OO_REQUIRE(e == 0, OO_ETIMEOUT, "fused Jacobi iterations: a grid barrier wait ran out");
    }
    OO_CUDA_TRY(cudaGetLastError());
    if (timing) {
        for (size_t x = 0; x < ev_nest.size(); ++x) {
            float ms = 0.f;
            OO_CUDA_TRY(cudaEventElapsedTime(&ms, evs[2 * x], evs[2 * x + 1]));
            nest_ms[ev_nest[x]] += ms;
        }
    }
    for (auto e : evs) cudaEventDestroy(e);
    if (stats) {
        stats->wall_ms = wall;
        for (int n = 0; n < 6; ++n) stats->nest_ms[n] = nest_ms[n];
        stats->xfer_ms = xfer_ms;
        stats->h2d_bytes = h2d;
        stats->d2h_bytes = d2h;
        stats->n_xfers = (int32_t)plan.size();
        stats->n_launches = launches;
    }
}

}  // namespace oo
