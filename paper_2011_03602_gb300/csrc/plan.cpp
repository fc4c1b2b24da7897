// Loop/variable tables, gene decoding and the transfer planner.
//
// Sec. 4.3 keeps loops and variables in a language-independent table; the
// gene has one bit per parallelisable nest (Sec. 4.2.2).  The planner
// applies the Sec. 4.2.2 transfer rules -- a variable set on one side and
// referenced on the other must be copied across -- and the Sec. 3.2.1
// hoisting rule -- copy once at the outermost level the variable allows
// rather than at every inner invocation.  Hoisting is realised as a lazy
// coherence walk over the program order with a per-side validity bit per
// variable; without hoisting each GPU nest copies its inputs in and its
// outputs out around every invocation.
#include "oo_internal.h"

namespace oo {

int NestTable::gene_len() const {
    int g = 0;
    for (const auto &n : nests) g += n.parallelisable ? 1 : 0;
    return g;
}

std::vector<int> NestTable::placement(uint64_t gene) const {
    std::vector<int> on_gpu(nests.size(), 0);
    int bit = 0;
    for (size_t n = 0; n < nests.size(); ++n) {
        if (!nests[n].parallelisable) continue;
        on_gpu[n] = (int)((gene >> bit) & 1u);
        ++bit;
    }
    return on_gpu;
}

void validate_table(const NestTable &t) {
    OO_REQUIRE(!t.vars.empty() && t.vars.size() <= 64, OO_EINVAL, "1..64 variables required");
    OO_REQUIRE(!t.nests.empty() && t.nests.size() <= 64, OO_EINVAL, "1..64 nests required");
    const uint64_t all = t.vars.size() == 64 ? ~0ull : ((1ull << t.vars.size()) - 1);
    for (const auto &n : t.nests) {
        OO_REQUIRE(n.level == 0 || n.level == 1, OO_EINVAL, "nest level must be 0 or 1: " + n.name);
        OO_REQUIRE(((n.reads | n.writes | n.partial) & ~all) == 0, OO_EINVAL,
                   "nest names a variable outside the table: " + n.name);
        OO_REQUIRE((n.partial & ~n.writes) == 0, OO_EINVAL,
                   "partial writes must be a subset of writes: " + n.name);
    }
    OO_REQUIRE((t.outputs & ~all) == 0, OO_EINVAL, "outputs name a variable outside the table");
}

NestTable jacobi_table(int I, int J, int K, int iters) {
    static const char *names[15] = {"a0", "a1", "a2", "a3", "b0", "b1", "b2", "c0",
                                    "c1", "c2", "bnd", "wrk1", "p", "wrk2", "res"};
    NestTable t;
    const uint64_t arr = 4ull * (uint64_t)I * (uint64_t)J * (uint64_t)K;
    for (int v = 0; v < 15; ++v) t.vars.push_back({names[v], v < 14 ? arr : 8ull * (uint64_t)iters});
    const uint64_t coef = (1ull << NCOEF) - 1, p = 1ull << VAR_P, w = 1ull << VAR_WRK2,
                   r = 1ull << VAR_RES;
    t.nests = {
        {"coef", 0, 1, 0, coef, 0},
        {"pinit", 0, 1, 0, p | w, 0},
        {"stencil", 1, 1, coef | p, w | r, w},
        {"copyback", 1, 1, w, p, p},
        {"bc_ij", 1, 1, 0, p, p},
        {"bc_k", 1, 1, 0, p, p},
    };
    t.outputs = p | r;
    return t;
}

std::vector<oo_xfer> make_plan(const NestTable &t, uint64_t gene, int hoist, int iters,
                               uint64_t *h2d, uint64_t *d2h) {
    OO_REQUIRE(iters >= 0, OO_EINVAL, "iters must be >= 0");
    const int L = t.gene_len();
    OO_REQUIRE(L == 64 || (gene >> L) == 0, OO_EINVAL, "gene has bits beyond the gene length");
    const std::vector<int> gpu = t.placement(gene);
    const int nv = (int)t.vars.size();
    std::vector<char> host_ok(nv, 1), dev_ok(nv, 0);
    std::vector<oo_xfer> out;
    uint64_t in_bytes = 0, out_bytes = 0;
    auto push = [&](int point, int v, int dir) {
        oo_xfer x{};
        x.point = point;
        x.var = v;
        x.dir = dir;
        x.bytes = t.vars[v].bytes;
        out.push_back(x);
        (dir > 0 ? in_bytes : out_bytes) += x.bytes;
    };
    // program order: level-0 nests once, then `iters` rounds of level-1 nests
    std::vector<int> order;
    for (size_t n = 0; n < t.nests.size(); ++n)
        if (t.nests[n].level == 0) order.push_back((int)n);
    std::vector<int> loop;
    for (size_t n = 0; n < t.nests.size(); ++n)
        if (t.nests[n].level == 1) loop.push_back((int)n);
    int point = 0;
    auto visit = [&](int n) {
        const auto &ns = t.nests[n];
        const uint64_t need = ns.reads | ns.partial;
        if (hoist) {
            std::vector<char> &mine = gpu[n] ? dev_ok : host_ok;
            std::vector<char> &other = gpu[n] ? host_ok : dev_ok;
            for (int v = 0; v < nv; ++v)
                if (((need >> v) & 1u) && !mine[v]) {
                    push(point, v, gpu[n] ? +1 : -1);
                    mine[v] = 1;
                }
            for (int v = 0; v < nv; ++v)
                if ((ns.writes >> v) & 1u) {
                    mine[v] = 1;
                    other[v] = 0;
                }
        } else if (gpu[n]) {
            for (int v = 0; v < nv; ++v)
                if ((need >> v) & 1u) push(point, v, +1);
            for (int v = 0; v < nv; ++v)
                if ((ns.writes >> v) & 1u) push(point + 1, v, -1);
        }
        ++point;
    };
    for (int n : order) visit(n);
    for (int it = 0; it < iters; ++it)
        for (int n : loop) visit(n);
    if (hoist)
        for (int v = 0; v < nv; ++v)
            if (((t.outputs >> v) & 1u) && !host_ok[v]) {
                push(point, v, -1);
                host_ok[v] = 1;
            }
    if (h2d) *h2d = in_bytes;
    if (d2h) *d2h = out_bytes;
    return out;
}

int jacobi_pitch(int K) { return (K + 31) / 32 * 32; }

}  // namespace oo
