// Generic loop programs: the method applied to a program other than the
// built-in Jacobi solver.
//
// Sec. 4.3 keeps the loop and variable information of any source program in
// a language-independent table; the gene, the transfer rules and the GA are
// defined on that table alone (Sec. 4.2.2).  Here the caller loads such a
// table (oo_load_nests) and supplies the nests' bodies as one callback that
// runs a nest on the CPU (host copies of the variables) or on the GPU
// (device copies, work enqueued on the context's stream).  The executor
// walks the program order -- setup nests once, then the iteration nests
// `iters` times -- performs the copies the planner puts before each program
// point, and calls each nest on the side its gene bit chooses.  The GA
// searches genes of such a program with the same operators as for Jacobi,
// fitness from the measured wall time and a caller-supplied result check.
#include <chrono>
#include <cmath>
#include <map>
#include <vector>

#include "oo_internal.h"

namespace oo {

namespace {
double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

void run_program(Ctx &c, uint64_t gene, int hoist, int iters, oo_nest_fn fn, void *user,
                 void *const *host_vars, void *const *dev_vars, oo_run_stats *stats) {
    OO_REQUIRE(c.have_table, OO_ESTATE, "no loop-nest table loaded");
    OO_REQUIRE(fn != nullptr && host_vars != nullptr && dev_vars != nullptr, OO_EINVAL, "null pointer");
    const NestTable &t = c.table;
    uint64_t h2d = 0, d2h = 0;
    const std::vector<oo_xfer> plan = make_plan(t, gene, hoist, iters, &h2d, &d2h);
    const std::vector<int> gpu = t.placement(gene);
    const int nv = (int)t.vars.size();
    // every variable a copy names needs both buffers; a GPU nest needs the
    // device buffers of what it touches
    for (const auto &x : plan)
        OO_REQUIRE(host_vars[x.var] && dev_vars[x.var], OO_EINVAL, "variable " + t.vars[x.var].name +
                                                                      " is copied but has no host or device buffer");
    for (size_t n = 0; n < t.nests.size(); ++n) {
        const auto &ns = t.nests[n];
        const uint64_t touched = ns.reads | ns.writes;
        for (int v = 0; v < nv; ++v)
            if ((touched >> v) & 1u)
                OO_REQUIRE(gpu[n] ? dev_vars[v] != nullptr : host_vars[v] != nullptr, OO_EINVAL,
                           "nest " + ns.name + " uses " + t.vars[v].name + " without a buffer on its side");
    }
    std::vector<int> order, loop;
    for (size_t n = 0; n < t.nests.size(); ++n) (t.nests[n].level == 0 ? order : loop).push_back((int)n);

    cudaStream_t s = c.stream;
    size_t next = 0;        // next planned copy
    bool pending = false;   // device work or copies enqueued since the last synchronisation
    int launches = 0;
    auto copies_before = [&](int point) {
        for (; next < plan.size() && plan[next].point == point; ++next) {
            const oo_xfer &x = plan[next];
            if (x.dir > 0)
                OO_CUDA_TRY(cudaMemcpyAsync(dev_vars[x.var], host_vars[x.var], x.bytes, cudaMemcpyHostToDevice, s));
            else
                OO_CUDA_TRY(cudaMemcpyAsync(host_vars[x.var], dev_vars[x.var], x.bytes, cudaMemcpyDeviceToHost, s));
            pending = true;
        }
    };
    auto call = [&](int n, long long it) {
        if (gpu[n]) {
            const int rc = fn(user, n, 1, it, dev_vars, (void *)s);
            OO_REQUIRE(rc == 0, OO_EUSER, "nest " + t.nests[n].name + " (GPU) returned " + std::to_string(rc));
            pending = true;
            ++launches;
        } else {
            if (pending) {
                OO_CUDA_TRY(cudaStreamSynchronize(s));
                pending = false;
            }
            const int rc = fn(user, n, 0, it, host_vars, nullptr);
            OO_REQUIRE(rc == 0, OO_EUSER, "nest " + t.nests[n].name + " (CPU) returned " + std::to_string(rc));
        }
    };
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    const double t0 = now_ms();
    int point = 0;
    for (int n : order) {
        copies_before(point);
        call(n, -1);
        ++point;
    }
    for (int it = 0; it < iters; ++it)
        for (int n : loop) {
            copies_before(point);
            call(n, it);
            ++point;
        }
    copies_before(point);
    OO_CUDA_TRY(cudaStreamSynchronize(s));
    OO_CUDA_TRY(cudaGetLastError());
    const double t1 = now_ms();
    OO_REQUIRE(next == plan.size(), OO_ESTATE, "transfer plan not fully executed");
    if (stats) {
        *stats = oo_run_stats{};
        stats->wall_ms = t1 - t0;
        stats->h2d_bytes = h2d;
        stats->d2h_bytes = d2h;
        stats->n_xfers = (int32_t)plan.size();
        stats->n_launches = launches;
    }
}

GaResult ga_program(Ctx &c, int hoist, int iters, oo_nest_fn fn, oo_check_fn check, void *user,
                    void *const *host_vars, void *const *dev_vars, int pop, int gens, double pc, double pm,
                    uint64_t seed, std::vector<double> *gene_ms) {
    OO_REQUIRE(c.have_table, OO_ESTATE, "no loop-nest table loaded");
    const int L = c.table.gene_len();
    OO_REQUIRE(L >= 1 && L <= 20, OO_EINVAL, "gene length must be 1..20 for the GA");
    std::map<uint64_t, double> memo;
    auto measure = [&](uint64_t g) -> double {
        auto it = memo.find(g);
        if (it != memo.end()) return it->second;
        oo_run_stats st{};
        run_program(c, g, hoist, iters, fn, user, host_vars, dev_vars, &st);
        // Sec. 4.2.2: a result that fails the check counts as infinitely slow
        double t = st.wall_ms;
        if (check && check(user, host_vars) != 0) t = INFINITY;
        memo[g] = t;
        return t;
    };
    GaResult r = ga_run(L, pop, gens, pc, pm, seed, measure);
    if (gene_ms) {
        gene_ms->assign((size_t)1 << L, INFINITY);
        for (const auto &kv : memo) (*gene_ms)[kv.first] = kv.second;
    }
    return r;
}

}  // namespace oo
