// Serving replicas: requests routed over several serving contexts (one per
// GPU, or several loops on one device) by free device memory.  The method
// itself targets whichever destination is free (Sec. 3); on a node with
// several GPUs every one serves the same mix, so requests are independent
// and the replicas share nothing: a request goes to the replica whose
// arena has the most free bytes among those with room for its footprint
// (ties: fewer requests waiting or running there, then the lower index),
// and to the replica with the fewest requests in flight when none has room
// (it queues there).  The decision is a pure function of the replicas'
// (free bytes, requests in flight), so processes that hold one replica each
// reach the same decision from the same gathered figures (oo_route_batch).
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "oo_internal.h"

using namespace oo;

namespace {

// device bytes a request occupies while it runs (the serving loops' own
// accounting differs in alignment and scratch; this is the routing estimate)
uint64_t footprint(const oo_serve_req &r) {
    if (r.kind == OO_BLOCK_GEMM) {
        const uint64_t m = (uint64_t)std::max<int64_t>(r.m, 0), n = (uint64_t)std::max<int64_t>(r.n, 0),
                       k = (uint64_t)std::max<int64_t>(r.k, 0);
        const uint64_t kp = (k + 63) / 64 * 64;
        // operands and result in FP64, plus up to 8 BF16 digit slices of A and B
        return 8 * (m * k + k * n + m * n) + (r.prec == OO_PREC_FP64EQ ? 8 * 2 * kp * (m + n) : 0);
    }
    if (r.kind == OO_BLOCK_FFT) return 32 * (uint64_t)std::max<int64_t>(r.n, 0);
    if (r.kind == OO_BLOCK_JACOBI) {
        const uint64_t I = (uint64_t)std::max<int64_t>(r.m, 0), J = (uint64_t)std::max<int64_t>(r.n, 0);
        const int K = (int)std::max<int64_t>(r.k, 3);
        return (uint64_t)NARR * I * J * (uint64_t)jacobi_pitch(K) * 4;
    }
    return 0;
}

int pick(const uint64_t *free_bytes, const uint64_t *queued, int n, uint64_t need) {
    int best = -1;
    for (int i = 0; i < n; ++i) {
        if (free_bytes[i] < need) continue;
        if (best < 0 || free_bytes[i] > free_bytes[best] ||
            (free_bytes[i] == free_bytes[best] && queued[i] < queued[best]))
            best = i;
    }
    if (best >= 0) return best;
    best = 0;
    for (int i = 1; i < n; ++i)
        if (queued[i] < queued[best]) best = i;
    return best;
}

}  // namespace

struct oo_router {
    std::vector<oo_ctx *> ctxs;
    // bytes of the requests routed to each replica and not yet waited for:
    // a replica's queue does not show in its arena's free bytes until the
    // requests start, so the router charges them itself
    std::vector<std::unordered_map<uint64_t, uint64_t>> routed;
    std::vector<uint64_t> routed_bytes;
    std::mutex mu;  // one routing decision at a time: it reads every replica's figures
};

extern "C" {

oo_status oo_route_pick(const uint64_t *free_bytes, const uint64_t *queued, int n, uint64_t need, int *replica) {
    if (!free_bytes || !queued || !replica || n < 1) return OO_EINVAL;
    *replica = pick(free_bytes, queued, n, need);
    return OO_OK;
}

oo_status oo_route_batch(const uint64_t *free_bytes, const uint64_t *queued, int n, const uint64_t *needs, int m,
                         int *replicas) {
    if (!free_bytes || !queued || n < 1 || m < 0 || (m > 0 && (!needs || !replicas))) return OO_EINVAL;
    std::vector<uint64_t> f(free_bytes, free_bytes + n), q(queued, queued + n);
    for (int j = 0; j < m; ++j) {
        const int r = pick(f.data(), q.data(), n, needs[j]);
        replicas[j] = r;
        f[r] = f[r] >= needs[j] ? f[r] - needs[j] : 0;
        ++q[r];
    }
    return OO_OK;
}

oo_status oo_serve_footprint(const oo_serve_req *req, uint64_t *bytes) {
    if (!req || !bytes) return OO_EINVAL;
    if (req->kind != OO_BLOCK_GEMM && req->kind != OO_BLOCK_FFT && req->kind != OO_BLOCK_JACOBI) return OO_EINVAL;
    *bytes = footprint(*req);
    return OO_OK;
}

oo_status oo_router_create(oo_ctx *const *ctxs, int n, oo_router **out) {
    if (!ctxs || !out || n < 1) return OO_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return OO_EINVAL;
    auto *r = new (std::nothrow) oo_router();
    if (!r) return OO_ENOMEM;
    r->ctxs.assign(ctxs, ctxs + n);
    r->routed.resize((size_t)n);
    r->routed_bytes.assign((size_t)n, 0);
    *out = r;
    return OO_OK;
}

oo_status oo_router_submit(oo_router *r, const oo_serve_req *req, int *replica, uint64_t *ticket) {
    if (!r || !req || !replica || !ticket) return OO_EINVAL;
    std::lock_guard<std::mutex> g(r->mu);
    const int n = (int)r->ctxs.size();
    std::vector<uint64_t> f((size_t)n), q((size_t)n);
    std::vector<int> ok((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        oo_serve_stats_t st{};
        if (oo_serve_stats(r->ctxs[(size_t)i], &st) != OO_OK) continue;  // not serving
        // free bytes: the arena's, but at most the budget less the
        // footprints this router sent there and has not seen waited for
        const uint64_t by_budget = st.device_budget_bytes > r->routed_bytes[(size_t)i]
                                       ? st.device_budget_bytes - r->routed_bytes[(size_t)i]
                                       : 0;
        f[(size_t)i] = std::min<uint64_t>(st.device_free_bytes, by_budget);
        q[(size_t)i] = st.queued + st.running;
        ok[(size_t)i] = 1;
    }
    const uint64_t need = footprint(*req);
    // best replica first; on back-pressure the next best, and so on
    oo_status last = OO_ESTATE;
    for (int tries = 0; tries < n; ++tries) {
        std::vector<uint64_t> fa, qa;
        std::vector<int> idx;
        for (int i = 0; i < n; ++i)
            if (ok[(size_t)i]) {
                fa.push_back(f[(size_t)i]);
                qa.push_back(q[(size_t)i]);
                idx.push_back(i);
            }
        if (idx.empty()) break;
        const int c = idx[(size_t)pick(fa.data(), qa.data(), (int)idx.size(), need)];
        last = oo_submit(r->ctxs[(size_t)c], req, ticket);
        if (last == OO_OK) {
            *replica = c;
            r->routed[(size_t)c][*ticket] = need;
            r->routed_bytes[(size_t)c] += need;
            return OO_OK;
        }
        if (last != OO_EBUSY && last != OO_ESTATE) return last;  // malformed: every replica would refuse it
        ok[(size_t)c] = 0;
    }
    return last;
}

oo_status oo_router_wait(oo_router *r, int replica, uint64_t ticket, int timeout_ms, double *latency_ms) {
    if (!r || replica < 0 || replica >= (int)r->ctxs.size()) return OO_EINVAL;
    const oo_status st = oo_wait(r->ctxs[(size_t)replica], ticket, timeout_ms, latency_ms);
    if (st != OO_ETIMEOUT) {  // the ticket is finished with (a timed-out wait keeps it)
        std::lock_guard<std::mutex> g(r->mu);
        auto &m = r->routed[(size_t)replica];
        auto it = m.find(ticket);
        if (it != m.end()) {
            r->routed_bytes[(size_t)replica] -= it->second;
            m.erase(it);
        }
    }
    return st;
}

void oo_router_destroy(oo_router *r) { delete r; }

}  // extern "C"
