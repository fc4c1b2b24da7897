// Serving loop: mixed GEMM / FFT / Jacobi requests from any number of client
// threads (the C, Python and Java front-ends all call oo_submit / oo_wait),
// continuously admitted onto the GPU.
//
//  - oo_submit (client thread): validates the request, copies its inputs into
//    a pinned staging pool and queues it; a full queue or pool answers
//    OO_EBUSY (back-pressure), a request larger than the device budget
//    OO_EINVAL.
//  - the scheduler thread: whenever a slot (CUDA stream) is free, admits the
//    oldest waiting requests whose device footprint fits the free part of the
//    device arena ("admission by free HBM"; a request older than 50 ms at
//    the head of the queue stops later ones from overtaking it), enqueues
//    copy-in, the block's kernels and copy-out on the slot's stream, and
//    polls completion events.  Requests admitted while others run overlap on
//    the device; device state (inputs, workspaces, results) stays resident
//    until the copy-out.
//  - oo_wait (client thread): waits for the ticket, copies the result from
//    staging into the caller's buffer and returns the request's latency
//    (submission to completion observed by the scheduler).
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "oo_internal.h"

namespace oo {

namespace {

using Clock = std::chrono::steady_clock;
double now_ms() {
    return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}
size_t up256(size_t x) { return (x + 255) / 256 * 256; }

enum { ST_QUEUED = 0, ST_RUNNING = 1, ST_DONE = 2 };

struct SReq {
    oo_serve_req r{};
    uint64_t ticket = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int state = ST_QUEUED;
    oo_status status = OO_OK;
    std::string error;
    // pinned staging: inputs, outputs, 16-byte error word
    size_t h_off = 0, h_bytes = 0, h_in0 = 0, h_in1 = 0, h_out = 0, h_res = 0, h_err = 0;
    // device block
    size_t d_off = 0, d_bytes = 0;
    int slot = -1;
    StencilPlan *splan = nullptr;
    const FftPlan *fplan = nullptr;
};

}  // namespace

struct Server {
    Ctx *c = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    bool stop = false;
    std::deque<SReq *> queue;
    size_t queue_cap = 0;
    std::unordered_map<uint64_t, SReq *> reqs;
    uint64_t next_ticket = 1;
    Arena dev, host;
    char *dev_base = nullptr, *host_base = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<SReq *> slot_req;
    uint64_t n_submitted = 0, n_done = 0, n_busy = 0, n_failed = 0;
    double busy_since = 0;
    double sum_queued_ms = 0, sum_slot_ms = 0;  // completed requests: queued, then on a slot
};

namespace {

// device footprint and staging layout of a request
void plan_sizes(Server &S, SReq &q) {
    const oo_serve_req &r = q.r;
    size_t h = 0, d = 0;
    auto hput = [&](size_t bytes) {
        const size_t at = h;
        h += up256(bytes);
        return at;
    };
    if (r.kind == OO_BLOCK_GEMM) {
        q.h_in0 = hput((size_t)r.m * r.k * 8);
        q.h_in1 = hput((size_t)r.k * r.n * 8);
        q.h_out = hput((size_t)r.m * r.n * 8);
        d = up256((size_t)r.m * r.k * 8) + up256((size_t)r.k * r.n * 8) + up256((size_t)r.m * r.n * 8) +
            up256(r.prec == OO_PREC_FP64EQ ? gemm_fp64eq_scratch_bytes((int)r.m, (int)r.n, (int)r.k)
                                           : gemm_scratch_bytes((int)r.m, (int)r.n, (int)r.k));
    } else if (r.kind == OO_BLOCK_FFT) {
        q.h_in0 = hput((size_t)r.n * 16);
        q.h_out = hput((size_t)r.n * 16);
        q.fplan = S.c->fft_plan(r.n);
        d = up256((size_t)r.n * 16) + up256(fft_scratch_bytes(q.fplan, 1));
    } else {
        const JacobiDims jd{(int)r.m, (int)r.n, (int)r.k, jacobi_pitch((int)r.k)};
        q.h_out = hput(jd.n_host() * 4);
        q.h_res = hput((size_t)std::max(1, r.iters) * 8);
        d = (size_t)NARR * up256(jd.n_dev() * 4) + up256((size_t)std::max(1, r.iters) * 8) +
            up256(stencil_scratch_bytes(jd, S.c->num_sms));
    }
    q.h_err = hput(16);
    q.h_bytes = h;
    q.d_bytes = d;
}

void validate(const oo_serve_req &r) {
    if (r.kind == OO_BLOCK_GEMM) {
        OO_REQUIRE(r.prec == OO_PREC_SPLIT3_BF16 || r.prec == OO_PREC_FP64EQ, OO_EINVAL,
                   "unsupported precision pattern");
        OO_REQUIRE(r.m >= 1 && r.n >= 1 && r.k >= 1 && r.m <= 65536 && r.n <= 65536 && r.k <= 65536, OO_EINVAL,
                   "bad GEMM dimensions");
        OO_REQUIRE(r.in0 && r.in1 && r.out, OO_EINVAL, "null pointer");
    } else if (r.kind == OO_BLOCK_FFT) {
        OO_REQUIRE(r.n >= 1 && r.n <= (1 << 24) && (r.n & (r.n - 1)) == 0, OO_EINVAL,
                   "FFT length must be a power of two <= 2^24");
        OO_REQUIRE(r.dir == -1 || r.dir == 1, OO_EINVAL, "dir must be -1 or +1");
        OO_REQUIRE(r.in0 && r.out, OO_EINVAL, "null pointer");
    } else if (r.kind == OO_BLOCK_JACOBI) {
        OO_REQUIRE(r.m >= 3 && r.n >= 3 && r.k >= 3 && r.k <= 4096 && r.m * r.n * r.k < (1ll << 31), OO_EINVAL,
                   "bad Jacobi grid");
        OO_REQUIRE(r.iters >= 0 && r.iters <= 1000000, OO_EINVAL, "bad iteration count");
        OO_REQUIRE(std::isfinite(r.omega), OO_EINVAL, "omega must be finite");
        OO_REQUIRE(r.out != nullptr, OO_EINVAL, "null pointer");
    } else {
        throw Error{OO_EINVAL, "unknown request kind"};
    }
}

// enqueue a request's copy-in, kernels and copy-out on its slot stream
void start(Server &S, SReq &q) {
    const Ctx &c = *S.c;
    cudaStream_t s = S.streams[q.slot];
    char *dev = S.dev_base + q.d_off;
    char *hst = S.host_base + q.h_off;
    const oo_serve_req &r = q.r;
    unsigned *err_h = reinterpret_cast<unsigned *>(hst + q.h_err);
    *err_h = 0;
    if (r.kind == OO_BLOCK_GEMM) {
        const size_t a = up256((size_t)r.m * r.k * 8), b = up256((size_t)r.k * r.n * 8), cc = up256((size_t)r.m * r.n * 8);
        double *dA = reinterpret_cast<double *>(dev), *dB = reinterpret_cast<double *>(dev + a),
               *dC = reinterpret_cast<double *>(dev + a + b);
        void *scratch = dev + a + b + cc;
        OO_CUDA_TRY(cudaMemcpyAsync(dA, hst + q.h_in0, (size_t)r.m * r.k * 8, cudaMemcpyHostToDevice, s));
        OO_CUDA_TRY(cudaMemcpyAsync(dB, hst + q.h_in1, (size_t)r.k * r.n * 8, cudaMemcpyHostToDevice, s));
        const unsigned *err_d;
        if (r.prec == OO_PREC_FP64EQ) {
            launch_gemm_fp64eq((int)r.m, (int)r.n, (int)r.k, dA, r.k, dB, r.n, dC, r.n, scratch, s,
                               eq_tile_width(c.eq_widths.data(), (int)r.n, (int)r.k));
            err_d = gemm_fp64eq_error_word(scratch);
        } else {
            launch_gemm_split3((int)r.m, (int)r.n, (int)r.k, dA, r.k, dB, r.n, dC, r.n, scratch, s);
            err_d = gemm_error_word(scratch, (int)r.m, (int)r.n, (int)r.k);
        }
        OO_CUDA_TRY(cudaMemcpyAsync(hst + q.h_out, dC, (size_t)r.m * r.n * 8, cudaMemcpyDeviceToHost, s));
        OO_CUDA_TRY(cudaMemcpyAsync(err_h, err_d, 4, cudaMemcpyDeviceToHost, s));
    } else if (r.kind == OO_BLOCK_FFT) {
        double *dx = reinterpret_cast<double *>(dev);
        void *scratch = dev + up256((size_t)r.n * 16);
        OO_CUDA_TRY(cudaMemcpyAsync(dx, hst + q.h_in0, (size_t)r.n * 16, cudaMemcpyHostToDevice, s));
        launch_fft(q.fplan, 1, r.dir, dx, dx, scratch, s);
        OO_CUDA_TRY(cudaMemcpyAsync(hst + q.h_out, dx, (size_t)r.n * 16, cudaMemcpyDeviceToHost, s));
    } else {
        const JacobiDims d{(int)r.m, (int)r.n, (int)r.k, jacobi_pitch((int)r.k)};
        const size_t arr = up256(d.n_dev() * 4);
        float *a[NARR];
        for (int v = 0; v < NARR; ++v) a[v] = reinterpret_cast<float *>(dev + (size_t)v * arr);
        double *res = reinterpret_cast<double *>(dev + (size_t)NARR * arr);
        char *scr = dev + (size_t)NARR * arr + up256((size_t)std::max(1, r.iters) * 8);
        const float *coef[NCOEF];
        float *coefw[NCOEF];
        for (int v = 0; v < NCOEF; ++v) {
            coef[v] = a[v];
            coefw[v] = a[v];
        }
        (void)c;
        // a tile variant tuned for this grid on the context (oo_tune_stencil
        // before oo_serve_start) applies here too
        q.splan = stencil_plan_create_ext(d, coef, a[VAR_P], a[VAR_WRK2], c.num_sms, scr,
                                          stencil_scratch_bytes(d, c.num_sms), s,
                                          c.stencil_variant_for((int)r.m, (int)r.n, (int)r.k));
        // the offload pattern with every nest on the GPU and hoisted copies:
        // nothing crosses until the final p and res
        launch_coef(d, coefw, s);
        launch_pinit(d, a[VAR_P], a[VAR_WRK2], s);
        for (int it = 0; it < r.iters; ++it) {
            launch_stencil(q.splan, r.omega, res + it, s);
            launch_copyback_faces(d, a[VAR_P], a[VAR_WRK2], s);  // N3 + N4 + N5
        }
        const size_t wb = (size_t)d.K * 4;
        OO_CUDA_TRY(cudaMemcpy2DAsync(hst + q.h_out, wb, a[VAR_P], (size_t)d.pitch * 4, wb, (size_t)d.I * d.J,
                                      cudaMemcpyDeviceToHost, s));
        if (r.iters > 0)
            OO_CUDA_TRY(cudaMemcpyAsync(hst + q.h_res, res, (size_t)r.iters * 8, cudaMemcpyDeviceToHost, s));
        OO_CUDA_TRY(cudaMemcpyAsync(err_h, stencil_plan_err_ptr(q.splan), 4, cudaMemcpyDeviceToHost, s));
    }
    OO_CUDA_TRY(cudaEventRecord(S.events[q.slot], s));
}

void scheduler(Server *Sp) {
    Server &S = *Sp;
    cudaSetDevice(S.c->device);
    std::unique_lock<std::mutex> lk(S.mu);
    while (true) {
        bool progress = false;
        // ---- completions
        for (size_t s = 0; s < S.slot_req.size(); ++s) {
            SReq *q = S.slot_req[s];
            if (!q) continue;
            const cudaError_t e = cudaEventQuery(S.events[s]);
            if (e == cudaErrorNotReady) continue;
            q->t_done = now_ms();
            S.sum_queued_ms += q->t_start - q->t_submit;
            S.sum_slot_ms += q->t_done - q->t_start;
            if (e != cudaSuccess) {
                q->status = OO_ECUDA;
                q->error = cudaGetErrorString(e);
            } else if (*reinterpret_cast<unsigned *>(S.host_base + q->h_off + q->h_err) != 0) {
                q->status = OO_ETIMEOUT;
                q->error = "a bounded pipeline wait in a kernel ran out";
            }
            if (q->status != OO_OK) ++S.n_failed;
            stencil_plan_destroy(q->splan);
            q->splan = nullptr;
            S.dev.release(q->d_off, q->d_bytes);
            q->state = ST_DONE;
            S.slot_req[s] = nullptr;
            ++S.n_done;
            progress = true;
            S.cv_done.notify_all();
        }
        // ---- admissions: oldest first, by free slot and free device memory.
        // Chosen under the lock, started after releasing it (client threads
        // keep queueing meanwhile, so no queue iterator survives the unlock).
        const double t = now_ms();
        std::vector<SReq *> to_start;
        for (auto it = S.queue.begin(); it != S.queue.end();) {
            int slot = -1;
            for (size_t s = 0; s < S.slot_req.size(); ++s)
                if (!S.slot_req[s]) {
                    slot = (int)s;
                    break;
                }
            if (slot < 0) break;
            SReq *q = *it;
            size_t off = 0;
            if (!S.dev.alloc(q->d_bytes, &off)) {
                if (it == S.queue.begin() && t - q->t_submit > 50.0) break;  // no overtaking a starved head
                ++it;
                continue;
            }
            q->d_off = off;
            q->slot = slot;
            q->state = ST_RUNNING;
            q->t_start = t;
            S.slot_req[slot] = q;
            it = S.queue.erase(it);
            to_start.push_back(q);
        }
        if (!to_start.empty()) {
            progress = true;
            lk.unlock();
            for (SReq *q : to_start) {
                try {
                    start(S, *q);
                } catch (const Error &e) {
                    // only this thread touches a running request; the
                    // completion pass reports the status once the event fires
                    q->status = e.code;
                    q->error = e.msg;
                    cudaEventRecord(S.events[q->slot], S.streams[q->slot]);
                }
            }
            lk.lock();
        }
        if (S.stop && S.queue.empty()) {
            bool idle = true;
            for (SReq *q : S.slot_req) idle = idle && q == nullptr;
            if (idle) break;
        }
        if (!progress) S.cv_sched.wait_for(lk, std::chrono::microseconds(20));
    }
}

}  // namespace

void server_stop(Server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_sched.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto &kv : S->reqs) delete kv.second;
    for (auto s : S->streams) cudaStreamDestroy(s);
    for (auto e : S->events) cudaEventDestroy(e);
    if (S->dev_base) cudaFree(S->dev_base);
    if (S->host_base) cudaFreeHost(S->host_base);
    delete S;
}

}  // namespace oo

using namespace oo;

extern "C" {

oo_status oo_serve_start(oo_ctx *ctx, int slots, uint64_t hbm_budget_bytes, int queue_cap) {
    if (!ctx) return OO_EINVAL;
    Ctx &c = ctx_state(ctx);
    try {
        OO_REQUIRE(c.device >= 0, OO_ESTATE, "host-only context (device -1) cannot serve");
        OO_REQUIRE(c.server == nullptr && c.rserver == nullptr, OO_ESTATE, "the context is already serving");
        OO_REQUIRE(slots >= 1 && slots <= 256, OO_EINVAL, "slots must be 1..256");
        OO_REQUIRE(queue_cap >= 1, OO_EINVAL, "queue_cap must be >= 1");
        OO_REQUIRE(hbm_budget_bytes >= (1u << 20), OO_EINVAL, "device budget below 1 MiB");
        OO_CUDA_TRY(cudaSetDevice(c.device));
        auto *S = new Server();
        S->c = &c;
        try {
            S->queue_cap = (size_t)queue_cap;
            const size_t db = up256(hbm_budget_bytes);
            if (cudaMalloc(&S->dev_base, db) != cudaSuccess) {
                cudaGetLastError();
                throw Error{OO_ENOMEM, "device budget of " + std::to_string(db) + " bytes"};
            }
            S->dev.reset(db);
            if (cudaHostAlloc(&S->host_base, db, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                throw Error{OO_ENOMEM, "pinned staging of " + std::to_string(db) + " bytes"};
            }
            S->host.reset(db);
            for (int i = 0; i < slots; ++i) {
                cudaStream_t s = nullptr;
                cudaEvent_t e = nullptr;
                OO_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
                OO_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                S->streams.push_back(s);
                S->events.push_back(e);
            }
            S->slot_req.assign(slots, nullptr);
            for (int e = 0; e <= 22; ++e) c.fft_plan(1ll << e);  // twiddle tables up front
            S->th = std::thread(scheduler, S);
        } catch (...) {
            server_stop(S);
            throw;
        }
        c.server = S;
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

oo_status oo_submit(oo_ctx *ctx, const oo_serve_req *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return OO_EINVAL;
    Ctx &c = ctx_state(ctx);
    if (c.rserver) return resident_submit(c.rserver, req, ticket);
    Server *S = c.server;
    if (!S) return OO_ESTATE;
    auto *q = new (std::nothrow) SReq();
    if (!q) return OO_ENOMEM;
    try {
        validate(*req);
        q->r = *req;
        {
            std::lock_guard<std::mutex> g(S->mu);
            plan_sizes(*S, *q);  // may create an FFT plan (table generation) under the lock
        }
        if (q->d_bytes > S->dev.size()) {
            delete q;
            return OO_EINVAL;  // can never be admitted
        }
        {
            std::lock_guard<std::mutex> g(S->mu);
            if (S->stop || S->queue.size() >= S->queue_cap || !S->host.alloc(q->h_bytes, &q->h_off)) {
                ++S->n_busy;
                delete q;
                return OO_EBUSY;
            }
        }
        char *h = S->host_base + q->h_off;
        if (req->kind == OO_BLOCK_GEMM) {
            std::memcpy(h + q->h_in0, req->in0, (size_t)req->m * req->k * 8);
            std::memcpy(h + q->h_in1, req->in1, (size_t)req->k * req->n * 8);
        } else if (req->kind == OO_BLOCK_FFT) {
            std::memcpy(h + q->h_in0, req->in0, (size_t)req->n * 16);
        }
        std::lock_guard<std::mutex> g(S->mu);
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

oo_status oo_wait(oo_ctx *ctx, uint64_t ticket, int timeout_ms, double *latency_ms) {
    if (!ctx) return OO_EINVAL;
    Ctx &c = ctx_state(ctx);
    if (c.rserver) return resident_wait(c, c.rserver, ticket, timeout_ms, latency_ms);
    Server *S = c.server;
    if (!S) return OO_ESTATE;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return OO_EINVAL;
    SReq *q = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    while (q->state != ST_DONE) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && q->state != ST_DONE)
            return OO_ETIMEOUT;
    }
    // submissions may have rehashed the table while this thread waited: erase
    // by key, never through the iterator found before the wait
    S->reqs.erase(ticket);
    lk.unlock();
    const oo_status st = q->status;
    if (st == OO_OK) {
        const char *h = S->host_base + q->h_off;
        const oo_serve_req &r = q->r;
        if (r.kind == OO_BLOCK_GEMM) {
            std::memcpy(r.out, h + q->h_out, (size_t)r.m * r.n * 8);
        } else if (r.kind == OO_BLOCK_FFT) {
            std::memcpy(r.out, h + q->h_out, (size_t)r.n * 16);
        } else {
            std::memcpy(r.out, h + q->h_out, (size_t)r.m * r.n * r.k * 4);
            if (r.res && r.iters > 0) std::memcpy(r.res, h + q->h_res, (size_t)r.iters * 8);
        }
    }
    if (latency_ms) *latency_ms = q->t_done - q->t_submit;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->host.release(q->h_off, q->h_bytes);
        if (st != OO_OK) c.last_error = q->error;
    }
    delete q;
    return st;
}

oo_status oo_serve_stats(oo_ctx *ctx, oo_serve_stats_t *out) {
    if (!ctx || !out) return OO_EINVAL;
    Ctx &c = ctx_state(ctx);
    if (c.rserver) {
        resident_stats(c.rserver, out);
        return OO_OK;
    }
    Server *S = c.server;
    if (!S) return OO_ESTATE;
    std::lock_guard<std::mutex> g(S->mu);
    out->submitted = S->n_submitted;
    out->completed = S->n_done;
    out->rejected_busy = S->n_busy;
    out->failed = S->n_failed;
    out->queued = (uint64_t)S->queue.size();
    uint64_t running = 0;
    for (SReq *q : S->slot_req) running += q != nullptr;
    out->running = running;
    out->device_free_bytes = S->dev.free_bytes();
    out->device_budget_bytes = S->dev.size();
    const double n = S->n_done ? (double)S->n_done : 1.0;
    for (double &v : out->stage_ms) v = 0.0;
    out->stage_ms[0] = S->sum_queued_ms / n;
    out->stage_ms[3] = S->sum_slot_ms / n;
    return OO_OK;
}

oo_status oo_serve_stop(oo_ctx *ctx) {
    if (!ctx) return OO_EINVAL;
    Ctx &c = ctx_state(ctx);
    if (c.rserver) {
        resident_stop(c.rserver);
        c.rserver = nullptr;
        return OO_OK;
    }
    if (!c.server) return OO_ESTATE;
    server_stop(c.server);
    c.server = nullptr;
    return OO_OK;
}

}  // extern "C"
