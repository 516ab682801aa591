// Host planner: graphical model (Section 3.A), elimination order and slices
// (Sections 3.B.1-3.B.3), the pairwise contraction program and its device image.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <functional>
#include <system_error>
#include <thread>
#include <numeric>
#include <unordered_map>

#include "plan.h"

namespace qvx {
namespace {

// ---------------------------------------------------------------- gate matrices [out][in]
bool gate_matrix(const qvx_gate &g, cplx m[2][2]) {
    const double r = 1.0 / std::sqrt(2.0);
    switch (g.kind) {
    case QVX_GATE_H:
        m[0][0] = r; m[0][1] = r; m[1][0] = r; m[1][1] = -r;
        return true;
    case QVX_GATE_SQRT_X:
        m[0][0] = cplx(0.5, 0.5); m[0][1] = cplx(0.5, -0.5);
        m[1][0] = cplx(0.5, -0.5); m[1][1] = cplx(0.5, 0.5);
        return true;
    case QVX_GATE_SQRT_Y:
        m[0][0] = cplx(0.5, 0.5); m[0][1] = cplx(-0.5, -0.5);
        m[1][0] = cplx(0.5, 0.5); m[1][1] = cplx(0.5, 0.5);
        return true;
    case QVX_GATE_RXY: {
        // cos(t/2) I - i sin(t/2) [[0, e^{-i phi}], [e^{i phi}, 0]]
        const double c = std::cos(g.theta / 2), s = std::sin(g.theta / 2);
        m[0][0] = c; m[1][1] = c;
        m[0][1] = cplx(0, -s) * std::polar(1.0, -g.phi);
        m[1][0] = cplx(0, -s) * std::polar(1.0, g.phi);
        return true;
    }
    case QVX_GATE_U1:
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) m[i][j] = cplx(g.u[2 * (2 * i + j)], g.u[2 * (2 * i + j) + 1]);
        return true;
    default:
        return false;
    }
}

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int find_pos(const std::vector<int> &v, int x) {
    for (size_t i = 0; i < v.size(); i++)
        if (v[i] == x) return (int)i;
    return -1;
}

// S *= T broadcast over S's modes (T's modes are a subset of S's).
void absorb_into(HostTensor &S, const HostTensor &T) {
    std::vector<int> pos(T.modes.size());
    for (size_t j = 0; j < T.modes.size(); j++) pos[j] = find_pos(S.modes, T.modes[j]);
    for (size_t i = 0; i < S.data.size(); i++) {
        size_t t = 0;
        for (size_t j = 0; j < pos.size(); j++) t |= ((i >> pos[j]) & 1u) << j;
        S.data[i] *= T.data[t];
    }
}

bool is_subset(const std::vector<int> &a, const std::vector<int> &b) {
    for (int x : a)
        if (find_pos(b, x) < 0) return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------- graphical model
bool build_model(const qvx_circuit *c, Model *m, std::string *err, bool keep_params) {
    if (!c || c->n_qubits < 1 || c->n_qubits > 128 || c->n_gates < 0 || (c->n_gates > 0 && !c->gates)) {
        *err = "circuit: need 1 <= n_qubits <= 128 and a gate array";
        return false;
    }
    const int n = c->n_qubits;
    std::vector<int> cur(n, 0);
    struct Raw {
        std::vector<std::pair<int, int>> keys;   // (qubit, ordinal); bit j of an index <-> keys[j]
        std::vector<cplx> data;
        int param = -1;
        double theta = 0, phi = 0;
    };
    std::vector<Raw> raw;
    raw.reserve((size_t)c->n_gates);
    for (int64_t i = 0; i < c->n_gates; i++) {
        const qvx_gate &g = c->gates[i];
        if (g.q0 < 0 || g.q0 >= n) { *err = "gate " + std::to_string(i) + ": qubit out of range"; return false; }
        Raw r;
        if (g.kind == QVX_GATE_CZ) {
            if (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0) { *err = "gate " + std::to_string(i) + ": bad CZ pair"; return false; }
            r.keys = {{g.q0, cur[g.q0]}, {g.q1, cur[g.q1]}};
            r.data = {1.0, 1.0, 1.0, -1.0};
        } else if (g.kind == QVX_GATE_T) {
            r.keys = {{g.q0, cur[g.q0]}};
            r.data = {1.0, std::polar(1.0, M_PI / 4)};
        } else {
            cplx u[2][2];
            if (!gate_matrix(g, u)) { *err = "gate " + std::to_string(i) + ": unknown kind"; return false; }
            // rank-2 tensor tau[i, j] = U[j, i] between the old and the new variable (Fig. 3)
            r.keys = {{g.q0, cur[g.q0]}, {g.q0, cur[g.q0] + 1}};
            r.data.resize(4);
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) r.data[a | (b << 1)] = u[b][a];
            if (keep_params && g.kind == QVX_GATE_RXY && g.param_index >= 0) {
                r.param = g.param_index;
                r.theta = g.theta;
                r.phi = g.phi;
            }
            cur[g.q0]++;
        }
        raw.push_back(std::move(r));
    }
    m->n_qubits = n;
    m->var_qubit.clear();
    m->var_ordinal.clear();
    std::vector<int> first_id(n, 0);
    for (int q = 0; q < n; q++) {
        first_id[q] = (int)m->var_qubit.size();
        for (int j = 1; j < cur[q]; j++) {
            m->var_qubit.push_back(q);
            m->var_ordinal.push_back(j);
        }
    }
    m->n_vars = (int)m->var_qubit.size();
    m->zero_mask[0] = m->zero_mask[1] = 0;
    for (int q = 0; q < n; q++)
        if (cur[q] == 0) m->zero_mask[q >> 6] |= 1ull << (q & 63);
    m->scalar = 1.0;
    m->tensors.clear();
    // key -> id: input (q, 0) is fixed to 0 (-1 here); summed (q, j) -> canonical id;
    // output (q, last) -> n_vars + q
    auto id_of = [&](int q, int j) -> int {
        if (j == 0) return -1;
        if (j == cur[q]) return m->n_vars + q;
        return first_id[q] + j - 1;
    };
    m->cz_count.assign(m->n_vars, 0);
    for (Raw &r : raw) {
        if (r.keys.size() == 2 && r.keys[0].first != r.keys[1].first)   // a CZ between two qubits
            for (auto &k : r.keys) {
                const int id = id_of(k.first, k.second);
                if (id >= 0 && id < m->n_vars) m->cz_count[id]++;
            }
    }
    for (Raw &r : raw) {
        HostTensor t;
        std::vector<int> keep;
        for (size_t j = 0; j < r.keys.size(); j++) {
            int id = id_of(r.keys[j].first, r.keys[j].second);
            if (id >= 0) { t.modes.push_back(id); keep.push_back((int)j); }
        }
        t.data.resize(size_t(1) << t.modes.size());
        t.param = r.param;
        t.theta = r.theta;
        t.phi = r.phi;
        for (size_t e = 0; e < t.data.size(); e++) {
            size_t src = 0;  // fixed inputs take value 0
            for (size_t j = 0; j < keep.size(); j++) src |= ((e >> j) & 1u) << keep[j];
            t.data[e] = r.data[src];
            if (t.param >= 0) t.code.push_back((uint8_t)src);   // raw index a | b << 1 = element [b][a]
        }
        if (t.modes.empty()) m->scalar *= t.data[0];
        else m->tensors.push_back(std::move(t));
    }
    // absorb every tensor whose modes are a subset of another's (rank-1 gates into their
    // neighbours, parallel rank-2 tensors into one); the graph is unchanged by this
    std::vector<int> idx(m->tensors.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return m->tensors[a].modes.size() < m->tensors[b].modes.size();
    });
    std::vector<int> rank_pos(idx.size());
    for (size_t i = 0; i < idx.size(); i++) rank_pos[idx[i]] = (int)i;
    std::unordered_map<int, std::vector<int>> by_mode;
    for (size_t t = 0; t < m->tensors.size(); t++)
        for (int v : m->tensors[t].modes) by_mode[v].push_back((int)t);
    std::vector<char> dead(m->tensors.size(), 0);
    for (size_t i = 0; i < idx.size(); i++) {
        int t = idx[i];
        const HostTensor &T = m->tensors[t];
        if (T.param >= 0) continue;                 // parametrised gates stay tensors of their own
        int best = -1;
        for (int s : by_mode[T.modes[0]]) {
            if (s == t || dead[s] || rank_pos[s] < (int)i || m->tensors[s].param >= 0) continue;
            if (m->tensors[s].modes.size() < T.modes.size()) continue;
            if (!is_subset(T.modes, m->tensors[s].modes)) continue;
            if (best < 0 || rank_pos[s] < rank_pos[best]) best = s;
        }
        if (best >= 0) {
            absorb_into(m->tensors[best], T);
            dead[t] = 1;
        }
    }
    std::vector<HostTensor> kept;
    for (size_t t = 0; t < m->tensors.size(); t++)
        if (!dead[t]) kept.push_back(std::move(m->tensors[t]));
    m->tensors = std::move(kept);
    // edges between summed variables sharing a tensor
    std::vector<std::pair<int, int>> es;
    for (const HostTensor &t : m->tensors)
        for (size_t a = 0; a < t.modes.size(); a++)
            for (size_t b = a + 1; b < t.modes.size(); b++) {
                int u = t.modes[a], v = t.modes[b];
                if (u >= m->n_vars || v >= m->n_vars) continue;
                es.push_back({std::min(u, v), std::max(u, v)});
            }
    std::sort(es.begin(), es.end());
    es.erase(std::unique(es.begin(), es.end()), es.end());
    m->edges = std::move(es);
    return true;
}

// ---------------------------------------------------------------- orderings
namespace {

struct Graph {
    int n = 0, W = 0;
    std::vector<uint64_t> bits;  // n rows of W words
    uint64_t *row(int v) { return &bits[(size_t)v * W]; }
    const uint64_t *row(int v) const { return &bits[(size_t)v * W]; }
    void init(int n_, const std::vector<std::pair<int, int>> &es) {
        n = n_;
        W = (n + 63) / 64;
        if (W == 0) W = 1;
        bits.assign((size_t)n * W, 0);
        for (auto &e : es) {
            row(e.first)[e.second >> 6] |= 1ull << (e.second & 63);
            row(e.second)[e.first >> 6] |= 1ull << (e.first & 63);
        }
    }
    int degree(int v) const {
        int d = 0;
        for (int w = 0; w < W; w++) d += __builtin_popcountll(row(v)[w]);
        return d;
    }
    // Section 3.B.1 step 4: join every two neighbours of v, then remove v.
    void eliminate(int v) {
        uint64_t *rv = row(v);
        for (int w = 0; w < W; w++) {
            uint64_t m = rv[w];
            while (m) {
                int u = w * 64 + __builtin_ctzll(m);
                m &= m - 1;
                uint64_t *ru = row(u);
                for (int x = 0; x < W; x++) ru[x] |= rv[x];
                ru[u >> 6] &= ~(1ull << (u & 63));
                ru[v >> 6] &= ~(1ull << (v & 63));
            }
        }
        std::fill(rv, rv + W, 0ull);
    }
    // Fixing v (Section 3.B.2) removes the vertex and its edges.
    void remove(int v) {
        uint64_t *rv = row(v);
        for (int w = 0; w < W; w++) {
            uint64_t m = rv[w];
            while (m) {
                int u = w * 64 + __builtin_ctzll(m);
                m &= m - 1;
                row(u)[v >> 6] &= ~(1ull << (v & 63));
            }
        }
        std::fill(rv, rv + W, 0ull);
    }
};

// Cost of an order (sum of 2^deg(v), Section 3.B.1) with `removed` vertices fixed first.
double order_cost(const Graph &g0, const std::vector<int> &order, const std::vector<char> &removed,
                  int *width) {
    Graph g = g0;
    for (int v = 0; v < g.n; v++)
        if (removed[v]) g.remove(v);
    double cost = 0;
    int wd = 0;
    for (int v : order) {
        if (removed[v]) continue;
        int d = g.degree(v);
        cost += std::ldexp(1.0, d);
        wd = std::max(wd, d);
        g.eliminate(v);
    }
    if (width) *width = wd;
    return cost;
}

// Greedy min-fill elimination order with random tie-breaks (stand-in for QuickBB's
// min-fill branching, Section 3.B.3). Each vertex's fill-in (pairs of its neighbours not yet
// joined) and degree are cached; eliminating v changes them only for v's neighbours (their
// neighbourhoods change) and for the neighbours of those (edges appear among v's
// neighbours), so only that two-hop set is recomputed.
double minfill_order(const Graph &g0, const std::vector<char> &removed, uint64_t seed,
                     std::vector<int> *order, int *width) {
    Graph g = g0;
    std::vector<int> alive;
    for (int v = 0; v < g.n; v++) {
        if (removed[v]) g.remove(v);
    }
    for (int v = 0; v < g.n; v++)
        if (!removed[v]) alive.push_back(v);
    auto fill_of = [&](int v) {
        const uint64_t *rv = g.row(v);
        long fill = 0;
        for (int w = 0; w < g.W; w++) {
            uint64_t m = rv[w];
            while (m) {
                int u = w * 64 + __builtin_ctzll(m);
                m &= m - 1;
                const uint64_t *ru = g.row(u);
                for (int x = 0; x < g.W; x++) fill += __builtin_popcountll(rv[x] & ~ru[x]);
                fill -= 1;  // u itself
            }
        }
        return fill / 2;
    };
    std::vector<long> fill(g.n, 0);
    std::vector<int> deg(g.n, 0);
    for (int v : alive) {
        fill[v] = fill_of(v);
        deg[v] = g.degree(v);
    }
    order->clear();
    double cost = 0;
    int wd = 0;
    uint64_t rng = seed;
    std::vector<int> ties;
    std::vector<uint64_t> touched(g.W);
    while (!alive.empty()) {
        long best_fill = -1;
        int best_deg = 0;
        ties.clear();
        for (int v : alive) {
            if (best_fill < 0 || fill[v] < best_fill || (fill[v] == best_fill && deg[v] < best_deg)) {
                best_fill = fill[v];
                best_deg = deg[v];
                ties.clear();
                ties.push_back(v);
            } else if (fill[v] == best_fill && deg[v] == best_deg) {
                ties.push_back(v);
            }
        }
        int pick = ties[splitmix64(rng) % ties.size()];
        int d = deg[pick];
        cost += std::ldexp(1.0, d);
        wd = std::max(wd, d);
        // the two-hop set of pick (before its removal the neighbours are its row)
        std::fill(touched.begin(), touched.end(), 0ull);
        const uint64_t *rp = g.row(pick);
        for (int w = 0; w < g.W; w++) {
            uint64_t m = rp[w];
            touched[w] |= m;
            while (m) {
                int u = w * 64 + __builtin_ctzll(m);
                m &= m - 1;
                const uint64_t *ru = g.row(u);
                for (int x = 0; x < g.W; x++) touched[x] |= ru[x];
            }
        }
        g.eliminate(pick);
        order->push_back(pick);
        alive.erase(std::find(alive.begin(), alive.end(), pick));
        touched[pick >> 6] &= ~(1ull << (pick & 63));
        // neighbours of the neighbours after the join: the join adds no vertex outside the
        // set above, since every new edge joins two former neighbours of pick
        for (int w = 0; w < g.W; w++) {
            uint64_t m = touched[w];
            while (m) {
                int u = w * 64 + __builtin_ctzll(m);
                m &= m - 1;
                fill[u] = fill_of(u);
                deg[u] = g.degree(u);
            }
        }
    }
    if (width) *width = wd;
    return cost;
}

double best_order(const Graph &g, const std::vector<char> &removed, const qvx_plan_opts &o,
                  uint64_t salt, std::vector<int> *order, int *width) {
    double best = -1;
    std::vector<int> cand;
    int w = 0;
    uint64_t s = o.order_seed ^ (salt * 0x9E3779B97F4A7C15ull);
    for (int r = 0; r < std::max(1, o.order_restarts); r++) {
        uint64_t seed = splitmix64(s);
        double cst = minfill_order(g, removed, seed, &cand, &w);
        if (best < 0 || cst < best) {
            best = cst;
            *order = cand;
            *width = w;
        }
    }
    return best;
}

}  // namespace

// ---------------------------------------------------------------- program construction
namespace {

constexpr int kMergedOnHost = -2;     // consumer id of a leaf folded into a bigger leaf

// out[R] = sum over the `dead` variables of A * B, in FP64 (A, B, out over their modes).
HostTensor host_contract(const HostTensor &A, const HostTensor &B, const std::vector<int> &R,
                         const std::vector<int> &dead) {
    HostTensor out;
    out.modes = R;
    out.data.assign(size_t(1) << R.size(), 0.0);
    std::vector<int> all = R;
    all.insert(all.end(), dead.begin(), dead.end());
    std::vector<int> pa(A.modes.size()), pb(B.modes.size());
    for (size_t j = 0; j < A.modes.size(); j++) pa[j] = find_pos(all, A.modes[j]);
    for (size_t j = 0; j < B.modes.size(); j++) pb[j] = find_pos(all, B.modes[j]);
    for (size_t full = 0; full < (size_t(1) << all.size()); full++) {
        size_t ia = 0, ib = 0;
        for (size_t j = 0; j < pa.size(); j++) ia |= ((full >> pa[j]) & 1u) << j;
        for (size_t j = 0; j < pb.size(); j++) ib |= ((full >> pb[j]) & 1u) << j;
        out.data[full & ((size_t(1) << R.size()) - 1)] += A.data[ia] * B.data[ib];
    }
    return out;
}

struct ProgramBuilder {
    Plan &p;
    const Model &m;
    int n_ids;                          // variable id space: summed + outputs
    std::vector<char> open;             // inner sliced variables
    std::vector<char> fixed;            // outer sliced variables and outputs
    std::vector<int> cnt;               // live pool tensors holding each variable
    std::vector<char> summed;
    std::vector<int> pool;
    cplx factor = 1.0;
    std::string err;

    ProgramBuilder(Plan &p_, const Model &m_) : p(p_), m(m_) {
        n_ids = m.n_vars + m.n_qubits;
        open.assign(n_ids, 0);
        fixed.assign(n_ids, 0);
        cnt.assign(n_ids, 0);
        summed.assign(n_ids, 0);
        for (int v = m.n_vars; v < n_ids; v++) fixed[v] = 1;
        for (int qb : p.open_qubits) {   // open outputs: never fixed, never summed
            fixed[m.n_vars + qb] = 0;
            open[m.n_vars + qb] = 1;
        }
        for (size_t i = 0; i < p.slices.size(); i++) {
            if ((int)i < p.n_inner) open[p.slices[i]] = 1;
            else fixed[p.slices[i]] = 1;
        }
    }

    int new_tensor(std::vector<int> modes) {
        PTensor t;
        t.modes = std::move(modes);
        p.tensors.push_back(std::move(t));
        return (int)p.tensors.size() - 1;
    }

    bool add_leaves() {
        for (size_t i = 0; i < m.tensors.size(); i++) {
            const HostTensor &h = m.tensors[i];
            std::vector<int> modes;
            for (int v : h.modes)
                if (!fixed[v]) modes.push_back(v);
            p.leaves.push_back(h);
            int t = new_tensor(modes);
            p.tensors[t].leaf = (int)p.leaves.size() - 1;
            for (int v : modes) cnt[v]++;
            pool.push_back(t);
        }
        return true;
    }

    bool summable(int v) const { return v < m.n_vars && !open[v] && !fixed[v]; }

    // pairwise contraction of pool tensors a and b; every variable held by no other live
    // tensor is summed here
    int contract(int a, int b) {
        const std::vector<int> A = p.tensors[a].modes, B = p.tensors[b].modes;
        std::vector<int> U = A;
        for (int v : B)
            if (find_pos(U, v) < 0) U.push_back(v);
        PStep s;
        s.a = a;
        s.b = b;
        std::vector<int> C;
        for (int v : U) {
            bool ia = find_pos(A, v) >= 0, ib = find_pos(B, v) >= 0;
            bool dead = summable(v) && cnt[v] == (int)ia + (int)ib;
            if (!dead) C.push_back(v);
            else if (ia && ib) s.k_ab.push_back(v);
            else if (ia) s.k_a.push_back(v);
            else s.k_b.push_back(v);
        }
        for (int v : A) cnt[v]--;
        for (int v : B) cnt[v]--;
        for (int v : C) cnt[v]++;
        for (int v : s.k_ab) summed[v] = 1;
        for (int v : s.k_a) summed[v] = 1;
        for (int v : s.k_b) summed[v] = 1;
        const int la = p.tensors[a].leaf, lb = p.tensors[b].leaf;
        if (la >= 0 && lb >= 0 && p.leaves[la].param < 0 && p.leaves[lb].param < 0) {
            // two leaves: contract them here, in FP64, when the result stays small; the
            // result keeps the modes fixed per work item, so it serves every item
            std::vector<int> dead = s.k_ab;
            dead.insert(dead.end(), s.k_a.begin(), s.k_a.end());
            dead.insert(dead.end(), s.k_b.begin(), s.k_b.end());
            const HostTensor &LA = p.leaves[la], &LB = p.leaves[lb];
            std::vector<int> R;
            for (int v : LA.modes)
                if (find_pos(dead, v) < 0) R.push_back(v);
            for (int v : LB.modes)
                if (find_pos(dead, v) < 0 && find_pos(R, v) < 0) R.push_back(v);
            if ((int)R.size() <= p.opts.host_merge_rank) {
                p.leaves.push_back(host_contract(LA, LB, R, dead));
                int c = new_tensor(C);
                p.tensors[c].leaf = (int)p.leaves.size() - 1;
                p.tensors[a].consumer = kMergedOnHost;
                p.tensors[b].consumer = kMergedOnHost;
                pool.erase(std::find(pool.begin(), pool.end(), a));
                pool.erase(std::find(pool.begin(), pool.end(), b));
                pool.push_back(c);
                return c;
            }
        }
        int c = new_tensor(C);
        s.c = c;
        int sid = (int)p.steps.size();
        p.tensors[a].consumer = sid;
        p.tensors[b].consumer = sid;
        p.tensors[c].producer = sid;
        p.steps.push_back(s);
        pool.erase(std::find(pool.begin(), pool.end(), a));
        pool.erase(std::find(pool.begin(), pool.end(), b));
        pool.push_back(c);
        return c;
    }

    // Two consecutive steps C = sum_S X Y and D = sum_S2 C Z, where Y and Z are leaves and C
    // feeds only the second, equal D = sum_{(S u S2) n X} X W with the leaf
    // W = sum_{(S u S2) \ X} Y Z (Z holds no mode of S, which C no longer has). W is contracted
    // here in FP64 when it stays within host_merge_rank modes (modes fixed per work item
    // included) and the new step costs no more flops than the two it replaces; C is never
    // written and one pass over the large operand is saved. Applied along chains of leaves.
    void absorb_leaf_chains() {
        std::vector<char> gone(p.steps.size(), 0);
        auto dev_modes = [&](const std::vector<int> &full) {
            std::vector<int> r;
            for (int v : full)
                if (!fixed[v]) r.push_back(v);
            return r;
        };
        auto union_size = [](const std::vector<int> &A, const std::vector<int> &B) {
            size_t n = A.size();
            for (int v : B) n += find_pos(A, v) < 0 ? 1 : 0;
            return n;
        };
        for (size_t s = 0; s < p.steps.size(); s++) {
            if (gone[s] || p.steps[s].b < 0) continue;
            const int c = p.steps[s].c, s2 = p.tensors[c].consumer;
            if (s2 < 0 || p.steps[s2].b < 0) continue;
            const PStep st = p.steps[s], st2 = p.steps[s2];
            const int z = st2.a == c ? st2.b : st2.a;
            const int lz = p.tensors[z].leaf;
            if (lz < 0 || p.leaves[lz].param >= 0) continue;
            std::vector<int> S = st.k_ab, S2 = st2.k_ab;
            S.insert(S.end(), st.k_a.begin(), st.k_a.end());
            S.insert(S.end(), st.k_b.begin(), st.k_b.end());
            S2.insert(S2.end(), st2.k_a.begin(), st2.k_a.end());
            S2.insert(S2.end(), st2.k_b.begin(), st2.k_b.end());
            std::vector<int> SS = S;
            for (int v : S2) SS.push_back(v);
            int best_y = -1;
            HostTensor best_w;
            std::vector<int> best_wdev;
            for (int y : {st.a, st.b}) {
                const int x = y == st.a ? st.b : st.a;
                const int ly = p.tensors[y].leaf;
                if (ly < 0 || p.leaves[ly].param >= 0) continue;
                const std::vector<int> &X = p.tensors[x].modes;
                const HostTensor &Y = p.leaves[ly], &Z = p.leaves[lz];
                std::vector<int> dead, R;
                for (int v : SS)
                    if (find_pos(X, v) < 0) dead.push_back(v);
                for (const std::vector<int> *M : {&Y.modes, &Z.modes})
                    for (int v : *M)
                        if (find_pos(dead, v) < 0 && find_pos(R, v) < 0) R.push_back(v);
                if ((int)R.size() > p.opts.host_merge_rank) continue;
                const std::vector<int> wdev = dev_modes(R);
                const double before = std::ldexp(1.0, (int)union_size(X, p.tensors[y].modes)) +
                                      std::ldexp(1.0, (int)union_size(p.tensors[c].modes, p.tensors[z].modes));
                const double after = std::ldexp(1.0, (int)union_size(X, wdev));
                if (after > before) continue;
                if (best_y < 0 || wdev.size() < best_wdev.size()) {
                    best_y = y;
                    best_w = host_contract(Y, Z, R, dead);
                    best_wdev = wdev;
                }
            }
            if (best_y < 0) continue;
            const int x = best_y == st.a ? st.b : st.a;
            p.leaves.push_back(best_w);
            const int w = new_tensor(best_wdev);
            p.tensors[w].leaf = (int)p.leaves.size() - 1;
            PStep ns;
            ns.a = x;
            ns.b = w;
            ns.c = st2.c;
            for (int v : SS) {
                if (find_pos(p.tensors[x].modes, v) < 0) continue;
                if (find_pos(best_wdev, v) >= 0) ns.k_ab.push_back(v);
                else ns.k_a.push_back(v);
            }
            p.steps[s2] = ns;
            gone[s] = 1;
            p.tensors[x].consumer = s2;
            p.tensors[w].consumer = s2;
            p.tensors[best_y].consumer = kMergedOnHost;
            p.tensors[z].consumer = kMergedOnHost;
            p.tensors[c].producer = -1;
            p.tensors[c].consumer = kMergedOnHost;
        }
        // drop the absorbed steps and renumber producers and consumers
        std::vector<int> new_id(p.steps.size(), -1);
        std::vector<PStep> kept;
        for (size_t s = 0; s < p.steps.size(); s++)
            if (!gone[s]) { new_id[s] = (int)kept.size(); kept.push_back(p.steps[s]); }
        for (PTensor &t : p.tensors) {
            if (t.producer >= 0) t.producer = new_id[t.producer];
            if (t.consumer >= 0) t.consumer = new_id[t.consumer];
        }
        p.steps = std::move(kept);
    }

    int reduce(int a) {
        const std::vector<int> A = p.tensors[a].modes;
        PStep s;
        s.a = a;
        std::vector<int> C;
        for (int v : A) {
            if (summable(v) && cnt[v] == 1) s.k_a.push_back(v);
            else C.push_back(v);
        }
        for (int v : A) cnt[v]--;
        for (int v : C) cnt[v]++;
        for (int v : s.k_a) summed[v] = 1;
        int c = new_tensor(C);
        s.c = c;
        int sid = (int)p.steps.size();
        p.tensors[a].consumer = sid;
        p.tensors[c].producer = sid;
        p.steps.push_back(s);
        pool.erase(std::find(pool.begin(), pool.end(), a));
        pool.push_back(c);
        return c;
    }

    size_t union_rank(int a, int b, bool drop_dead) const {
        const auto &A = p.tensors[a].modes, &B = p.tensors[b].modes;
        size_t r = 0;
        std::vector<int> U = A;
        for (int v : B)
            if (find_pos(U, v) < 0) U.push_back(v);
        for (int v : U) {
            bool ia = find_pos(A, v) >= 0, ib = find_pos(B, v) >= 0;
            bool dead = summable(v) && cnt[v] == (int)ia + (int)ib;
            if (!drop_dead || !dead) r++;
        }
        return r;
    }

    // multiply a set of tensors pairwise, the pair with the smallest result first
    // (small inputs first, the large tensor last: Section 3.B.1)
    void combine(std::vector<int> bucket) {
        while (bucket.size() > 1) {
            size_t bi = 0, bj = 1, best = SIZE_MAX, best_in = SIZE_MAX;
            for (size_t i = 0; i < bucket.size(); i++)
                for (size_t j = i + 1; j < bucket.size(); j++) {
                    size_t r = union_rank(bucket[i], bucket[j], true);
                    size_t in = std::max(p.tensors[bucket[i]].modes.size(), p.tensors[bucket[j]].modes.size());
                    if (r < best || (r == best && in < best_in)) {
                        best = r; best_in = in; bi = i; bj = j;
                    }
                }
            int c = contract(bucket[bi], bucket[bj]);
            bucket.erase(bucket.begin() + bj);
            bucket[bi] = c;
        }
    }

    bool run() {
        add_leaves();
        for (int v : p.order) {
            if (summed[v]) continue;            // already summed with a pair that held it last
            std::vector<int> bucket;
            for (int t : pool)
                if (find_pos(p.tensors[t].modes, v) >= 0) bucket.push_back(t);
            if (bucket.empty()) {               // v is in no tensor: sum over v of 1
                factor *= 2.0;
                summed[v] = 1;
                continue;
            }
            if (bucket.size() == 1) reduce(bucket[0]);
            else combine(bucket);
            if (!summed[v]) { err = "internal: variable not summed"; return false; }
        }
        for (int t : pool)
            for (int v : p.tensors[t].modes)
                if (!open[v]) { err = "internal: variable left in the final tensors"; return false; }
        if (pool.empty()) {                     // nothing at all: the constant 1
            HostTensor one;
            one.data = {1.0};
            p.leaves.push_back(one);
            int t = new_tensor({});
            p.tensors[t].leaf = (int)p.leaves.size() - 1;
            pool.push_back(t);
        }
        combine(pool);
        int fin = pool[0];
        if (p.tensors[fin].leaf >= 0) fin = reduce(fin);   // the final tensor lives in the arena
        p.final_tensor = fin;
        if (p.opts.host_merge_rank > 0) absorb_leaf_chains();
        return true;
    }
};

void assign_layouts(Plan &p) {
    // the final tensor: inner slice modes in slice-number bit order, then the open outputs
    PTensor &f = p.tensors[p.final_tensor];
    std::vector<int> fin;
    for (int i = 0; i < p.n_inner; i++)
        if (find_pos(f.modes, p.slices[i]) >= 0) fin.push_back(p.slices[i]);
    for (int qb : p.open_qubits)
        if (find_pos(f.modes, p.model.n_vars + qb) >= 0) fin.push_back(p.model.n_vars + qb);
    f.modes = fin;
    // every operand takes its consumer's order: output modes first (in the output's
    // order), then the summed modes
    for (int s = (int)p.steps.size() - 1; s >= 0; s--) {
        const PStep &st = p.steps[s];
        const std::vector<int> C = p.tensors[st.c].modes;
        auto lay = [&](int t, const std::vector<int> &own) {
            std::vector<int> old = p.tensors[t].modes, L;
            for (int v : C)
                if (find_pos(old, v) >= 0) L.push_back(v);
            for (int v : st.k_ab) L.push_back(v);
            for (int v : own) L.push_back(v);
            p.tensors[t].modes = L;
        };
        lay(st.a, st.k_a);
        if (st.b >= 0) lay(st.b, st.k_b);
    }
}

// Every step output in a region of its own, 128-byte aligned: the persistent engine reads
// tensors written by other SMs of the same launch through their L1 caches, which is safe
// only if no cache line ever held other data.
int64_t allocate_arena_unique(Plan &p) {
    int64_t off = 0;
    for (const PStep &st : p.steps) {
        p.tensors[st.c].offset = off;
        const int64_t len = int64_t(1) << p.tensors[st.c].modes.size();
        off += (len + 15) & ~int64_t(15);
    }
    return off;
}

// First-fit arena allocation of the step outputs over their lifetimes.
int64_t allocate_arena(Plan &p) {
    struct Block { int64_t off, len; int t; };
    std::vector<Block> live;
    int64_t peak = 0;
    auto alloc = [&](int t) {
        int64_t len = int64_t(1) << p.tensors[t].modes.size();
        len = (len + 3) & ~int64_t(3);            // 32-byte granules
        std::sort(live.begin(), live.end(), [](const Block &a, const Block &b) { return a.off < b.off; });
        int64_t at = 0;
        for (const Block &b : live) {
            if (b.off - at >= len) break;
            at = std::max(at, b.off + b.len);
        }
        live.push_back({at, len, t});
        p.tensors[t].offset = at;
        peak = std::max(peak, at + len);
    };
    auto release = [&](int t) {
        for (size_t i = 0; i < live.size(); i++)
            if (live[i].t == t) { live.erase(live.begin() + i); return; }
    };
    // steps of one phase run concurrently: their outputs are placed while every operand of
    // the phase is still live, and the operands are released after the phase
    for (const auto &ph : p.phases) {
        for (int s = ph.first; s < ph.second; s++) alloc(p.steps[s].c);
        for (int s = ph.first; s < ph.second; s++) {
            const PStep &st = p.steps[s];
            if (p.tensors[st.a].leaf < 0) release(st.a);
            if (st.b >= 0 && p.tensors[st.b].leaf < 0) release(st.b);
        }
    }
    return peak;
}

// Orders the steps by level (1 + the deepest level among the steps producing their
// operands) and groups each level into a phase of mutually independent steps.
void schedule_levels(Plan &p) {
    const size_t ns = p.steps.size();
    std::vector<int> level(ns, 0);
    for (size_t s = 0; s < ns; s++) {
        const PStep &st = p.steps[s];
        int lv = 0;
        for (int t : {st.a, st.b})
            if (t >= 0 && p.tensors[t].producer >= 0) lv = std::max(lv, level[p.tensors[t].producer] + 1);
        level[s] = lv;
    }
    std::vector<int> idx(ns);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return level[x] < level[y]; });
    std::vector<PStep> sorted(ns);
    for (size_t i = 0; i < ns; i++) {
        sorted[i] = p.steps[idx[i]];
        p.tensors[sorted[i].c].producer = (int)i;
        p.tensors[sorted[i].a].consumer = (int)i;
        if (sorted[i].b >= 0) p.tensors[sorted[i].b].consumer = (int)i;
    }
    p.steps = std::move(sorted);
    p.phases.clear();
    for (size_t i = 0; i < ns;) {
        size_t j = i;
        while (j < ns && level[idx[j]] == level[idx[i]]) j++;
        p.phases.push_back({(int)i, (int)j});
        i = j;
    }
}

// Algorithmic work of one step of one work item: real flops (8 per complex multiply-add,
// 2 per complex add of a one-operand sum) and complex64 bytes (operands read once, output
// written once).
void step_work(const Plan &p, const PStep &s, double *fl, double *by) {
    const auto &A = p.tensors[s.a].modes;
    const auto &C = p.tensors[s.c].modes;
    if (s.b < 0) {
        *fl = 2.0 * std::ldexp(1.0, (int)A.size());
        *by = 8.0 * (std::ldexp(1.0, (int)A.size()) + std::ldexp(1.0, (int)C.size()));
    } else {
        const auto &B = p.tensors[s.b].modes;
        const int u = (int)(C.size() + s.k_ab.size() + s.k_a.size() + s.k_b.size());
        *fl = 8.0 * std::ldexp(1.0, u);
        *by = 8.0 * (std::ldexp(1.0, (int)A.size()) + std::ldexp(1.0, (int)B.size()) +
                     std::ldexp(1.0, (int)C.size()));
    }
}

void program_stats(Plan &p) {
    double fl = 0, by = 0;
    int mr = 0;
    for (const PStep &s : p.steps) {
        double f, b;
        step_work(p, s, &f, &b);
        fl += f;
        by += b;
        mr = std::max(mr, (int)p.tensors[s.c].modes.size());
    }
    p.flops_per_item = fl;
    p.bytes_per_item = by;
    p.max_rank = mr;
}

bool make_runs(const std::vector<int> &C, const std::vector<int> &X, DevRun *runs, uint8_t *n_runs,
               uint8_t *n_cb) {
    int nr = 0, dst = 0;
    size_t j = 0;
    while (j < C.size()) {
        if (find_pos(X, C[j]) < 0) { j++; continue; }
        size_t k = j;
        while (k < C.size() && find_pos(X, C[k]) >= 0) k++;
        if (nr >= kMaxRuns) return false;
        runs[nr].src = (uint8_t)j;
        runs[nr].len = (uint8_t)(k - j);
        runs[nr].dst = (uint8_t)dst;
        runs[nr].pad = 0;
        dst += (int)(k - j);
        nr++;
        j = k;
    }
    *n_runs = (uint8_t)nr;
    *n_cb = (uint8_t)dst;
    return true;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Runs that move the bits of an index laid out as `src` (bit j <-> src[j]) to the
// positions of the same modes in `dst`; modes of src absent from dst contribute nothing.
bool map_runs(const std::vector<int> &src, const std::vector<int> &dst, DevRun *runs, uint8_t *n) {
    int nr = 0;
    size_t j = 0;
    while (j < src.size()) {
        const int pj = find_pos(dst, src[j]);
        if (pj < 0) { j++; continue; }
        size_t k = j + 1;
        while (k < src.size() && find_pos(dst, src[k]) == pj + (int)(k - j)) k++;
        if (nr >= kMaxRuns) return false;
        runs[nr].src = (uint8_t)j;
        runs[nr].len = (uint8_t)(k - j);
        runs[nr].dst = (uint8_t)pj;
        runs[nr].pad = 0;
        nr++;
        j = k;
    }
    *n = (uint8_t)nr;
    return true;
}

// Reverse-mode program over the pairwise contractions. Every forward output keeps its own
// arena slot; for a step C = contract(A, B) the adjoint of A is contract(adj C, B) over
// the modes of C and B that A lacks (and symmetrically for B); the adjoint of the final
// tensor is the constant 2^(inner slice modes it lacks). Each parametrised leaf then gets
// d alpha / d theta = sum over its entries of adj(leaf) * dU/dtheta (a rank-0 step).
// First-fit placement of tensors with lifetimes in phases: tensor i (size[i] entries) is
// written in phase birth[i] and last read in phase death[i]. The outputs of a phase are
// placed while every tensor read in that phase is still live, and released after their last
// reading phase, so no phase writes over anything it, or a later phase, reads.
int64_t place_by_phases(const std::vector<int64_t> &size, const std::vector<int> &birth,
                        const std::vector<int> &death, int n_phases, std::vector<int64_t> *off) {
    struct Block { int64_t off, len; int id; };
    std::vector<Block> live;
    std::vector<std::vector<int>> born(n_phases + 1), dies(n_phases + 1);
    off->assign(size.size(), -1);
    for (size_t i = 0; i < size.size(); i++) {
        if (birth[i] < 0) continue;
        born[birth[i]].push_back((int)i);
        const int d = std::max(death[i], birth[i]);
        if (d < n_phases) dies[d].push_back((int)i);
    }
    int64_t peak = 0;
    for (int ph = 0; ph < n_phases; ph++) {
        for (int id : born[ph]) {
            const int64_t len = (size[id] + 3) & ~int64_t(3);   // 32-byte granules
            std::sort(live.begin(), live.end(), [](const Block &x, const Block &y) { return x.off < y.off; });
            int64_t at = 0;
            for (const Block &bl : live) {
                if (bl.off - at >= len) break;
                at = std::max(at, bl.off + bl.len);
            }
            live.push_back({at, len, id});
            (*off)[id] = at;
            peak = std::max(peak, at + len);
        }
        for (int id : dies[ph])
            for (size_t j = 0; j < live.size(); j++)
                if (live[j].id == id) { live.erase(live.begin() + j); break; }
    }
    return peak;
}

// keep[t] = 0: the forward value of tensor t is not kept for the backward pass; each
// backward level that reads it recomputes it (and, first, any operand of it that is not kept
// either) in phases of its own just before the level's adjoint steps (checkpointing: the
// kept tensors are the checkpoints).
bool build_grad_program(Plan &p, const std::vector<int> &dev_leaf, const std::vector<char> &keep, std::string *err) {
    const size_t nt = p.tensors.size();
    std::vector<char> need(nt, 0);
    for (size_t t = 0; t < nt; t++) {
        const PTensor &T = p.tensors[t];
        if (T.leaf >= 0 && T.consumer >= 0 && p.leaves[T.leaf].param >= 0) need[t] = 1;
    }
    for (const PStep &st : p.steps) need[st.c] = need[st.a] || (st.b >= 0 && need[st.b]);
    // arena tensors by id: forward output of tensor t = t, adjoint of t = nt + t, the
    // derivative slots = 2 nt; steps are emitted with ids as offsets, placed afterwards
    std::vector<int64_t> fo(nt, -1), ao(nt, -1);
    for (const PStep &st : p.steps) fo[st.c] = st.c;
    std::vector<int> pl;   // parametrised leaf tensors
    for (size_t t = 0; t < nt; t++) {
        if (!need[t]) continue;
        ao[t] = (int64_t)(nt + t);
        if (p.tensors[t].leaf >= 0) pl.push_back((int)t);
    }
    const int64_t gslot = (int64_t)(2 * nt);
    int64_t next_id = gslot + 1;    // recomputed forward values get ids from here on
    std::vector<int64_t> rsize;     // their sizes (entries), by id - next_id's start
    std::vector<int64_t> out_rel;   // per gradient step: entry offset inside its output tensor
    p.grad_steps.clear();
    std::vector<int64_t> cur_fwd = fo;   // where a forward value is read from right now
    auto operand = [&](GenOperand &o, int t, bool adj, const std::vector<int> &out, const std::vector<int> &S) {
        std::memset(&o, 0, sizeof(o));
        if (t < 0) { o.kind = kOpOne; return true; }
        const PTensor &T = p.tensors[t];
        if (adj) { o.kind = kOpArena; o.off = (uint64_t)ao[t]; }
        else if (T.leaf >= 0) { o.kind = kOpLeaf; o.off = (uint64_t)dev_leaf[T.leaf]; }
        else { o.kind = kOpArena; o.off = (uint64_t)cur_fwd[t]; }
        return map_runs(out, T.modes, o.oruns, &o.n_oruns) && map_runs(S, T.modes, o.kruns, &o.n_kruns);
    };
    p.grad_flops_per_item = 0;
    p.grad_bytes_per_item = 0;
    auto emit = [&](int64_t out_off, const std::vector<int> &out, int x, bool xadj, int y, bool yadj,
                    const std::vector<int> &S) {
        p.grad_flops_per_item += 8.0 * std::ldexp(1.0, (int)(out.size() + S.size()));
        p.grad_bytes_per_item += 8.0 * std::ldexp(1.0, (int)out.size());
        for (int t : {x, y})
            if (t >= 0) p.grad_bytes_per_item += 8.0 * std::ldexp(1.0, (int)p.tensors[t].modes.size());
        GenStep g;
        std::memset(&g, 0, sizeof(g));
        g.out_off = (uint64_t)out_off;
        g.ro = (uint32_t)out.size();
        g.nk = (uint32_t)S.size();
        if (!operand(g.x, x, xadj, out, S) || !operand(g.y, y, yadj, out, S)) return false;
        p.grad_steps.push_back(g);
        out_rel.push_back(0);
        return true;
    };
    auto minus = [](const std::vector<int> &u, const std::vector<int> &w, const std::vector<int> &drop) {
        std::vector<int> r;
        for (const std::vector<int> *v : {&u, &w})
            for (int m : *v)
                if (find_pos(drop, m) < 0 && find_pos(r, m) < 0) r.push_back(m);
        return r;
    };
    const std::string runs_err = "gradient program: address map needs too many runs";
    p.grad_phase_first.clear();
    for (const auto &ph : p.phases) p.grad_phase_first.push_back((uint32_t)ph.first);   // forward levels
    for (const PStep &st : p.steps) {   // forward, every output kept
        std::vector<int> S = st.k_ab;
        S.insert(S.end(), st.k_a.begin(), st.k_a.end());
        S.insert(S.end(), st.k_b.begin(), st.k_b.end());
        if (!emit(fo[st.c], p.tensors[st.c].modes, st.a, false, st.b, false, S)) { *err = runs_err; return false; }
    }
    const int F = p.final_tensor;
    p.grad_phase_first.push_back((uint32_t)p.grad_steps.size());   // the adjoint of the final tensor
    if (need[F]) {
        std::vector<int> absent;   // inner slice modes the final tensor lacks: dummy summed modes
        for (int i = 0; i < p.n_inner; i++)
            if (find_pos(p.tensors[F].modes, p.slices[i]) < 0) absent.push_back(-1 - i);
        if (!emit(ao[F], p.tensors[F].modes, -1, false, -1, false, absent)) { *err = runs_err; return false; }
    }
    // backward, level by level from the last: the adjoints of a level's operands depend only
    // on adjoints of later levels
    auto summed_of = [](const PStep &st) {
        std::vector<int> S = st.k_ab;
        S.insert(S.end(), st.k_a.begin(), st.k_a.end());
        S.insert(S.end(), st.k_b.begin(), st.k_b.end());
        return S;
    };
    auto dropped = [&](int t) { return t >= 0 && p.tensors[t].leaf < 0 && !keep[t]; };
    p.grad_recomputed = 0;
    for (int l = (int)p.phases.size() - 1; l >= 0; l--) {
        // forward values this level reads that were not kept, with the not-kept operands they
        // are recomputed from, by depth (depth 0: computed from kept values and leaves only)
        std::vector<int> depth(nt, -1), order;
        std::function<int(int)> visit = [&](int t) -> int {
            if (depth[t] >= 0) return depth[t];
            const PStep &pr = p.steps[p.tensors[t].producer];
            int d = 0;
            for (int u : {pr.a, pr.b})
                if (dropped(u)) d = std::max(d, visit(u) + 1);
            depth[t] = d;
            order.push_back(t);
            return d;
        };
        for (int s = p.phases[l].second - 1; s >= p.phases[l].first; s--) {
            const PStep &st = p.steps[s];
            if (!need[st.c]) continue;
            if (need[st.a] && dropped(st.b)) visit(st.b);
            if (st.b >= 0 && need[st.b] && dropped(st.a)) visit(st.a);
        }
        int max_depth = -1;
        for (int t : order) max_depth = std::max(max_depth, depth[t]);
        for (int t : order) {
            cur_fwd[t] = next_id++;
            rsize.push_back(int64_t(1) << p.tensors[t].modes.size());
        }
        for (int d = 0; d <= max_depth; d++) {
            p.grad_phase_first.push_back((uint32_t)p.grad_steps.size());
            for (int t : order) {
                if (depth[t] != d) continue;
                const PStep &pr = p.steps[p.tensors[t].producer];
                if (!emit(cur_fwd[t], p.tensors[t].modes, pr.a, false, pr.b, false, summed_of(pr))) {
                    *err = runs_err;
                    return false;
                }
                p.grad_recomputed++;
            }
        }
        p.grad_phase_first.push_back((uint32_t)p.grad_steps.size());
        for (int s = p.phases[l].second - 1; s >= p.phases[l].first; s--) {
            const PStep &st = p.steps[s];
            if (!need[st.c]) continue;
            const std::vector<int> &LC = p.tensors[st.c].modes, &LA = p.tensors[st.a].modes;
            if (need[st.a]) {
                const std::vector<int> none;
                const std::vector<int> &LB = st.b >= 0 ? p.tensors[st.b].modes : none;
                if (!emit(ao[st.a], LA, st.c, true, st.b, false, minus(LC, LB, LA))) { *err = runs_err; return false; }
            }
            if (st.b >= 0 && need[st.b]) {
                const std::vector<int> &LB = p.tensors[st.b].modes;
                if (!emit(ao[st.b], LB, st.c, true, st.a, false, minus(LC, LA, LB))) { *err = runs_err; return false; }
            }
        }
        for (int t : order) cur_fwd[t] = fo[t];
    }
    p.grad_param_leaves.clear();
    p.grad_phase_first.push_back((uint32_t)p.grad_steps.size());   // the dot products
    for (size_t i = 0; i < pl.size(); i++) {   // d alpha / d theta per parametrised leaf
        const int t = pl[i];
        GenStep g;
        std::memset(&g, 0, sizeof(g));
        g.out_off = (uint64_t)gslot;
        g.ro = 0;
        g.nk = (uint32_t)p.tensors[t].modes.size();
        const std::vector<int> none;
        if (!operand(g.x, t, true, none, p.tensors[t].modes) || !operand(g.y, t, false, none, p.tensors[t].modes)) {
            *err = runs_err;
            return false;
        }
        g.y.kind = kOpDeriv;
        p.grad_flops_per_item += 8.0 * std::ldexp(1.0, (int)g.nk);
        p.grad_bytes_per_item += 16.0 * std::ldexp(1.0, (int)g.nk) + 8.0;
        p.grad_steps.push_back(g);
        out_rel.push_back((int64_t)i);
        p.grad_param_leaves.push_back(p.tensors[t].leaf);
    }
    p.grad_phase_first.push_back((uint32_t)p.grad_steps.size());
    // drop empty phases; element offsets of each step inside its phase
    std::vector<uint32_t> firsts;
    for (size_t i = 0; i + 1 < p.grad_phase_first.size(); i++)
        if (p.grad_phase_first[i] < p.grad_phase_first[i + 1]) firsts.push_back(p.grad_phase_first[i]);
    firsts.push_back((uint32_t)p.grad_steps.size());
    p.grad_phase_first = firsts;
    p.grad_elem_off.assign(p.grad_steps.size(), 0);
    for (size_t i = 0; i + 1 < firsts.size(); i++) {
        uint64_t acc = 0;
        for (uint32_t g = firsts[i]; g < firsts[i + 1]; g++) {
            if (acc > 0xffffffffull) { *err = "gradient program: phase too large"; return false; }
            p.grad_elem_off[g] = (uint32_t)acc;
            acc += uint64_t(1) << p.grad_steps[g].ro;
        }
    }
    // lifetimes of the arena tensors in phases, then their places
    const int n_ph = (int)firsts.size() - 1;
    const size_t n_ids = (size_t)next_id;
    std::vector<int64_t> size(n_ids, 0);
    std::vector<int> birth(n_ids, -1), death(n_ids, -1);
    for (size_t t = 0; t < nt; t++) size[t] = size[nt + t] = int64_t(1) << p.tensors[t].modes.size();
    size[gslot] = std::max<int64_t>((int64_t)pl.size(), 1);
    for (size_t i = 0; i < rsize.size(); i++) size[gslot + 1 + i] = rsize[i];
    for (int ph = 0; ph < n_ph; ph++)
        for (uint32_t gi = firsts[ph]; gi < firsts[ph + 1]; gi++) {
            const GenStep &g = p.grad_steps[gi];
            if (birth[g.out_off] < 0) birth[g.out_off] = ph;
            for (const GenOperand *o : {&g.x, &g.y})
                if (o->kind == kOpArena) death[o->off] = std::max(death[o->off], ph);
        }
    if (fo[F] >= 0) death[fo[F]] = n_ph;    // read by the amplitude partial after the last phase
    death[gslot] = n_ph;    // read by the derivative partials
    std::vector<int64_t> place;
    p.grad_arena_elems = place_by_phases(size, birth, death, n_ph, &place);
    for (size_t gi = 0; gi < p.grad_steps.size(); gi++) {
        GenStep &g = p.grad_steps[gi];
        g.out_off = (uint64_t)(place[g.out_off] + out_rel[gi]);
        for (GenOperand *o : {&g.x, &g.y})
            if (o->kind == kOpArena) o->off = (uint64_t)place[o->off];
    }
    p.grad_final_off = fo[F] >= 0 ? place[fo[F]] : -1;
    p.grad_gslot_off = place[gslot];
    return true;
}

// Moves bit runs of v: sum of ((v >> src) & (2^len - 1)) << dst over the runs.
uint32_t move_runs(uint32_t v, const DevRun *runs, int n) {
    uint32_t r = 0;
    for (int i = 0; i < n; i++) r |= ((v >> runs[i].src) & ((1u << runs[i].len) - 1u)) << runs[i].dst;
    return r;
}

// The gradient program as one record per output entry (GradEntry) plus a table of summed-
// index offsets; false if an offset does not fit 16 bits (the global-memory kernel runs).
bool build_grad_tables(const Plan &p, std::vector<GradEntry> *ent, std::vector<uint32_t> *ktab,
                       std::vector<uint32_t> *phase_entry) {
    ent->clear();
    ktab->clear();
    phase_entry->clear();
    if (p.grad_arena_elems > 65536) return false;
    std::vector<uint32_t> first(p.grad_steps.size() + 1, 0);
    for (size_t s = 0; s < p.grad_steps.size(); s++) {
        const GenStep &g = p.grad_steps[s];
        first[s] = (uint32_t)ent->size();
        if (g.ro > 16 || g.nk > 15) return false;
        auto ref = [](const GenOperand &op) { return op.kind == kOpOne ? uint64_t(0) : op.off; };
        if (ref(g.x) > 65535 || ref(g.y) > 65535) return false;
        uint32_t k1 = 0;
        auto koff = [&](uint32_t k) -> int64_t {
            const uint32_t kx = g.x.kind == kOpOne ? 0u : move_runs(k, g.x.kruns, g.x.n_kruns);
            const uint32_t ky = g.y.kind == kOpOne ? 0u : move_runs(k, g.y.kruns, g.y.n_kruns);
            if (kx > 65535 || ky > 65535) return -1;
            return (int64_t)(kx | (ky << 16));
        };
        if (g.nk == 1) {
            const int64_t v = koff(1);
            if (v < 0) return false;
            k1 = (uint32_t)v;
        } else if (g.nk >= 2) {
            k1 = (uint32_t)ktab->size();
            for (uint32_t k = 1; k < (1u << g.nk); k++) {
                const int64_t v = koff(k);
                if (v < 0) return false;
                ktab->push_back((uint32_t)v);
            }
        }
        for (uint32_t oi = 0; oi < (1u << g.ro); oi++) {
            GradEntry e;
            const uint64_t c = g.out_off + oi;
            const uint32_t xo = g.x.kind == kOpOne ? 0u : move_runs(oi, g.x.oruns, g.x.n_oruns);
            const uint32_t yo = g.y.kind == kOpOne ? 0u : move_runs(oi, g.y.oruns, g.y.n_oruns);
            if (c > 65535 || xo > 65535 || yo > 65535) return false;
            e.c = (uint16_t)c;
            e.meta = (uint16_t)(g.x.kind | (g.y.kind << 2) | (g.nk << 4));
            e.xr = (uint16_t)ref(g.x);
            e.xo = (uint16_t)xo;
            e.yr = (uint16_t)ref(g.y);
            e.yo = (uint16_t)yo;
            e.k1 = k1;
            ent->push_back(e);
        }
    }
    first[p.grad_steps.size()] = (uint32_t)ent->size();
    for (uint32_t s : p.grad_phase_first) phase_entry->push_back(first[s]);
    return true;
}

bool serialize(Plan &p, std::string *err) {
    const Model &m = p.model;
    // leaf element maps and stored data
    // only leaves that a step reads are stored; dev_leaf maps leaf index -> device index
    std::vector<int> leaf_tensor(p.leaves.size(), -1), dev_leaf(p.leaves.size(), -1), live;
    for (size_t t = 0; t < p.tensors.size(); t++)
        if (p.tensors[t].leaf >= 0 && p.tensors[t].consumer >= 0) leaf_tensor[p.tensors[t].leaf] = (int)t;
    for (size_t l = 0; l < p.leaves.size(); l++)
        if (leaf_tensor[l] >= 0) { dev_leaf[l] = (int)live.size(); live.push_back((int)l); }
    std::vector<DevLeaf> dl(live.size());
    std::vector<float> ldata;
    std::vector<ParamLeaf> pls;
    std::vector<uint8_t> codes;
    std::vector<int> pleaf_of_leaf(p.leaves.size(), -1);
    for (size_t di = 0; di < live.size(); di++) {
        const int l = live[di];
        const HostTensor &h = p.leaves[l];
        const std::vector<int> &P = p.tensors[leaf_tensor[l]].modes;
        DevLeaf &d = dl[di];
        std::memset(&d, 0, sizeof(d));
        d.data_off = (uint32_t)(ldata.size() / 2);
        d.n_elem = 1u << P.size();
        // stored order: the consumer's modes, then the fixed modes
        std::vector<int> stored = P;
        for (size_t j = 0; j < h.modes.size(); j++) {
            int v = h.modes[j];
            if (find_pos(P, v) >= 0) continue;
            if ((int)d.n_fixed >= kMaxFixed) { *err = "a leaf has too many fixed modes"; return false; }
            uint8_t src;
            if (v >= m.n_vars) src = (uint8_t)(v - m.n_vars);
            else {
                int si = find_pos(p.slices, v);
                if (si < p.n_inner) { *err = "internal: leaf mode neither kept nor fixed"; return false; }
                if (si - p.n_inner >= 64) { *err = "more than 64 outer sliced variables"; return false; }
                src = (uint8_t)(128 + (si - p.n_inner));
            }
            d.fixed_src[d.n_fixed] = src;
            d.fixed_pos[d.n_fixed] = (uint8_t)stored.size();
            d.n_fixed++;
            stored.push_back(v);
        }
        std::vector<int> pos(stored.size());
        for (size_t j = 0; j < stored.size(); j++) pos[j] = find_pos(h.modes, stored[j]);
        if (h.param >= 0) {
            ParamLeaf pl;
            std::memset(&pl, 0, sizeof(pl));
            pl.leaf = (uint32_t)di;
            pl.param = (uint32_t)h.param;
            pl.n_stored = 1u << stored.size();
            pl.code_off = (uint32_t)codes.size();
            pl.phi = h.phi;
            pleaf_of_leaf[l] = (int)pls.size();
            pls.push_back(pl);
        }
        for (size_t e = 0; e < (size_t(1) << stored.size()); e++) {
            size_t src = 0;
            for (size_t j = 0; j < stored.size(); j++) src |= ((e >> j) & 1u) << pos[j];
            ldata.push_back((float)h.data[src].real());
            ldata.push_back((float)h.data[src].imag());
            if (h.param >= 0) codes.push_back(h.code[src]);
        }
    }
    std::vector<DevStep> ds(p.steps.size());
    for (size_t s = 0; s < p.steps.size(); s++) {
        const PStep &st = p.steps[s];
        DevStep &d = ds[s];
        std::memset(&d, 0, sizeof(d));
        const PTensor &A = p.tensors[st.a], &C = p.tensors[st.c];
        d.rc = (uint8_t)C.modes.size();
        d.nk_ab = (uint8_t)st.k_ab.size();
        d.nk_a = (uint8_t)st.k_a.size();
        d.nk_b = (uint8_t)st.k_b.size();
        d.c_off = (uint64_t)C.offset;
        if (A.leaf >= 0) { d.flags |= kStepALeaf; d.a_off = (uint64_t)dev_leaf[A.leaf]; }
        else d.a_off = (uint64_t)A.offset;
        if (!make_runs(C.modes, A.modes, d.runs_a, &d.na_runs, &d.a_cb)) { *err = "address map needs too many runs"; return false; }
        if (st.b < 0) {
            d.flags |= kStepUnary;
        } else {
            const PTensor &B = p.tensors[st.b];
            if (B.leaf >= 0) { d.flags |= kStepBLeaf; d.b_off = (uint64_t)dev_leaf[B.leaf]; }
            else d.b_off = (uint64_t)B.offset;
            if (!make_runs(C.modes, B.modes, d.runs_b, &d.nb_runs, &d.b_cb)) { *err = "address map needs too many runs"; return false; }
        }
    }
    // register-tiled form of the two-operand steps (global-arena engines): up to two output
    // modes held by A alone and two held by B alone, all above C's five lowest bits (a
    // warp's 32 lanes run along those, so its loads and stores stay coalesced), become a
    // per-thread tile of 2^rm x 2^rn entries. Compute-bound steps (16 or more flops per
    // algorithmic byte, above the FP32 ridge of about 12; at least 2^12 threads per work
    // item) take up to three of each: an 8 x 8 tile does 16 FMAs per loaded 8-byte entry where
    // a 4 x 4 tile does 8, which halves the L1 traffic that bounds the smaller tile there. On
    // output-bound steps the wide tile's 8 warps per SM issue too few stores (2.8 TB/s on a
    // 7-flop/B step), so they keep the 4 x 4 tile
    std::vector<RegTileStep> rts;
    if (p.engine != QVX_ENGINE_FUSED) {
        rts.assign(ds.size(), RegTileStep{});
        for (size_t s = 0; s < p.steps.size(); s++) {
            const PStep &st = p.steps[s];
            RegTileStep &r = rts[s];
            std::memset(&r, 0, sizeof(r));
            if (st.b < 0 || ds[s].rc < 6) continue;
            const std::vector<int> &LA = p.tensors[st.a].modes, &LB = p.tensors[st.b].modes, &LC = p.tensors[st.c].modes;
            double fl = 0, by = 0;
            step_work(p, st, &fl, &by);
            const size_t max_bits = fl >= 16.0 * by && LC.size() >= 18 ? 3 : 2;
            std::vector<int> tm, tn;   // tile bits: positions in C
            for (int j = 5; j < (int)LC.size(); j++) {
                const bool ia = find_pos(LA, LC[j]) >= 0, ib = find_pos(LB, LC[j]) >= 0;
                if (ia && !ib && tm.size() < max_bits) tm.push_back(j);
                if (ib && !ia && tn.size() < max_bits) tn.push_back(j);
            }
            if (tm.empty() && tn.empty()) continue;
            const DevStep &d = ds[s];
            r.a_off = d.a_off;
            r.b_off = d.b_off;
            r.c_off = d.c_off;
            r.flags = d.flags;
            r.rc = d.rc;
            r.rm = (uint8_t)tm.size();
            r.rn = (uint8_t)tn.size();
            r.nt = (uint8_t)(d.rc - r.rm - r.rn);
            r.nk_ab = d.nk_ab;
            r.nk_a = d.nk_a;
            r.nk_b = d.nk_b;
            r.a_cb = d.a_cb;
            r.b_cb = d.b_cb;
            r.na_runs = d.na_runs;
            r.nb_runs = d.nb_runs;
            for (int i = 0; i < kMaxRuns; i++) { r.runs_a[i] = d.runs_a[i]; r.runs_b[i] = d.runs_b[i]; }
            // free bits of C in increasing order, as runs from the thread index
            int nf = 0, tb = 0;
            for (int j = 0; j < (int)LC.size();) {
                if (find_pos(tm, j) >= 0 || find_pos(tn, j) >= 0) { j++; continue; }
                int k = j + 1;
                while (k < (int)LC.size() && find_pos(tm, k) < 0 && find_pos(tn, k) < 0) k++;
                r.free_runs[nf].src = (uint8_t)tb;
                r.free_runs[nf].len = (uint8_t)(k - j);
                r.free_runs[nf].dst = (uint8_t)j;
                nf++;
                tb += k - j;
                j = k;
            }
            r.n_free = (uint8_t)nf;
            for (int i = 0; i < (1 << r.rm); i++)
                for (int q = 0; q < r.rm; q++)
                    if ((i >> q) & 1) {
                        r.a_m[i] += 1u << find_pos(LA, LC[tm[q]]);
                        r.c_m[i] += 1u << tm[q];
                    }
            for (int i = 0; i < (1 << r.rn); i++)
                for (int q = 0; q < r.rn; q++)
                    if ((i >> q) & 1) {
                        r.b_n[i] += 1u << find_pos(LB, LC[tn[q]]);
                        r.c_n[i] += 1u << tn[q];
                    }
        }
    }
    // tensor-core form of the dense contractions (stepwise engine, opts.tensor_cores): every
    // summed mode in both operands, 8 to 1024 summed entries (K) and an arithmetic intensity
    // of at least 5 flops per byte: from there the register-tiled SIMT form is issue-bound
    // (about four instructions per complex multiply-add; 1.9 TB/s on a 16-entry step at 10.7
    // flop/B, under 3.5 TB/s on 8-entry steps), while the tensor cores run such output-bound
    // steps near the rate of their epilogue's stores (5 to 6 TB/s). The GEMM's row role goes to
    // the operand that holds C's lowest mode (its unit stride) alone: a tile's 128 rows then
    // sit in consecutive tensor-memory lanes and the epilogue's stores of each column are
    // consecutive in C. That operand needs 128 output entries of its own, the other 8; a step
    // whose lowest output mode is held by both operands (a batch mode) keeps its SIMT form.
    // Complex products commute, so the step's B may take the row role.
    std::vector<GemmStep> gms;
    if (p.engine == QVX_ENGINE_STEPWISE && p.opts.tensor_cores) {
        gms.assign(ds.size(), GemmStep{});
        for (size_t s = 0; s < p.steps.size(); s++) {
            const PStep &st = p.steps[s];
            GemmStep &g = gms[s];
            std::memset(&g, 0, sizeof(g));
            if (st.b < 0 || !st.k_a.empty() || !st.k_b.empty() || st.k_ab.size() < 3 || st.k_ab.size() > 10) continue;
            if (p.tensors[st.c].modes.empty()) continue;
            const int low = p.tensors[st.c].modes[0];
            const bool low_a = find_pos(p.tensors[st.a].modes, low) >= 0;
            const bool low_b = find_pos(p.tensors[st.b].modes, low) >= 0;
            if (low_a == low_b) continue;   // a batch mode
            const bool swap = low_b;
            std::vector<int> gb, gm, gn;
            {
                const std::vector<int> &LA = p.tensors[swap ? st.b : st.a].modes;
                const std::vector<int> &LB = p.tensors[swap ? st.a : st.b].modes;
                for (int v : p.tensors[st.c].modes) {
                    const bool ia = find_pos(LA, v) >= 0, ib = find_pos(LB, v) >= 0;
                    if (ia && ib) gb.push_back(v);
                    else if (ia) gm.push_back(v);
                    else gn.push_back(v);
                }
            }
            if (gm.size() < 7 || gn.size() < 3) continue;
            const std::vector<int> &LA = p.tensors[swap ? st.b : st.a].modes;
            const std::vector<int> &LB = p.tensors[swap ? st.a : st.b].modes, &LC = p.tensors[st.c].modes;
            const double flops = 8.0 * std::ldexp(1.0, (int)(LC.size() + st.k_ab.size()));
            const double bytes = 8.0 * (std::ldexp(1.0, (int)LA.size()) + std::ldexp(1.0, (int)LB.size()) +
                                        std::ldexp(1.0, (int)LC.size()));
            if (flops < 5.0 * bytes) continue;
            bool ok = true;
            auto gmap = [&](const std::vector<int> &grp, const std::vector<int> &L, DevRun *runs, uint8_t *n) {
                DevRun r[kMaxRuns];
                uint8_t nr = 0;
                if (!map_runs(grp, L, r, &nr) || nr > kGroupRuns) { ok = false; return; }
                for (int i = 0; i < nr; i++) runs[i] = r[i];
                *n = nr;
            };
            gmap(gb, LA, g.ab, &g.n_ab); gmap(gm, LA, g.am, &g.n_am); gmap(st.k_ab, LA, g.ak, &g.n_ak);
            gmap(gb, LB, g.bb, &g.n_bb); gmap(gn, LB, g.bn, &g.n_bn); gmap(st.k_ab, LB, g.bk, &g.n_bk);
            gmap(gb, LC, g.cb, &g.n_cb); gmap(gm, LC, g.cm, &g.n_cm); gmap(gn, LC, g.cn, &g.n_cn);
            if (!ok) { std::memset(&g, 0, sizeof(g)); continue; }
            g.a_off = swap ? ds[s].b_off : ds[s].a_off;
            g.b_off = swap ? ds[s].a_off : ds[s].b_off;
            g.c_off = ds[s].c_off;
            g.flags = ds[s].flags & ~(kStepALeaf | kStepBLeaf);
            if (ds[s].flags & (swap ? kStepBLeaf : kStepALeaf)) g.flags |= kStepALeaf;
            if (ds[s].flags & (swap ? kStepALeaf : kStepBLeaf)) g.flags |= kStepBLeaf;
            g.nb = (uint8_t)gb.size();
            g.nm = (uint8_t)gm.size();
            g.nn = (uint8_t)gn.size();
            g.nk = (uint8_t)st.k_ab.size();
        }
    }
    // fused form: per-step tables of pext(c) for both operands (16-bit offsets), and per
    // phase a map from each lane of a work item's group to the step it works on
    std::vector<FusedStep> fs(ds.size());
    std::vector<uint32_t> tab, lane_map;
    bool fused_ok = p.arena_elems <= 65536 && ds.size() <= 4096;
    for (size_t s = 0; s < ds.size() && fused_ok; s++) {
        const DevStep &d = ds[s];
        FusedStep &f = fs[s];
        std::memset(&f, 0, sizeof(f));
        f.a_off = (uint32_t)d.a_off;
        f.b_off = (uint32_t)d.b_off;
        f.c_off = (uint32_t)d.c_off;
        f.flags = d.flags;
        f.rc = d.rc;
        f.nk_ab = d.nk_ab;
        f.nk_a = d.nk_a;
        f.nk_b = d.nk_b;
        f.a_cb = d.a_cb;
        f.b_cb = d.b_cb;
        f.nk = (uint8_t)(d.nk_ab + d.nk_a + d.nk_b);
        for (uint32_t k = 0; k < 8 && k < (1u << f.nk); k++) {
            const uint32_t ka = k & ((1u << (d.nk_ab + d.nk_a)) - 1u);
            const uint32_t kb = (k & ((1u << d.nk_ab) - 1u)) | ((k >> (d.nk_ab + d.nk_a)) << d.nk_ab);
            f.koff_a[k] = (uint16_t)(ka << d.a_cb);
            f.koff_b[k] = (uint16_t)(kb << d.b_cb);
        }
        f.tab_off = (uint32_t)tab.size();
        if (d.rc > 16 || d.a_cb + d.nk_ab + d.nk_a > 16 || d.b_cb + d.nk_ab + d.nk_b > 16) { fused_ok = false; break; }
        for (uint32_t c = 0; c < (1u << d.rc); c++) {
            uint32_t ia = 0, ib = 0;
            for (int r = 0; r < d.na_runs; r++)
                ia |= ((c >> d.runs_a[r].src) & ((1u << d.runs_a[r].len) - 1u)) << d.runs_a[r].dst;
            for (int r = 0; r < d.nb_runs; r++)
                ib |= ((c >> d.runs_b[r].src) & ((1u << d.runs_b[r].len) - 1u)) << d.runs_b[r].dst;
            tab.push_back(ia | (ib << 16));
        }
    }
    // lanes per phase: at least one per step, the rest in proportion to the steps' work,
    // never more than a step has output entries; a phase with more steps than lanes is
    // split into several
    const int lanes = 32 * p.warps_per_item;
    int n_phases = 0;
    for (const auto &ph : p.phases) {
        if (!fused_ok) break;
        for (int b0 = ph.first; b0 < ph.second; b0 += lanes) {
            const int b1 = std::min(ph.second, b0 + lanes);
            const int n = b1 - b0;
            std::vector<int> cnt(n, 1);
            std::vector<double> work(n);
            for (int i = 0; i < n; i++) work[i] = std::ldexp(1.0, ds[b0 + i].rc + ds[b0 + i].nk_ab + ds[b0 + i].nk_a + ds[b0 + i].nk_b);
            for (int left = lanes - n; left > 0; left--) {
                int best = -1;
                for (int i = 0; i < n; i++) {
                    if (cnt[i] >= (1 << ds[b0 + i].rc) || cnt[i] >= 1023) continue;
                    if (best < 0 || work[i] / cnt[i] > work[best] / cnt[best]) best = i;
                }
                if (best < 0) break;
                cnt[best]++;
            }
            // lanes of steps of the same kind (summed entries, one or two operands) are
            // adjacent, so fewer warps mix the kernel's per-kind code paths
            std::vector<int> by_kind(n);
            std::iota(by_kind.begin(), by_kind.end(), 0);
            auto kind = [&](int i) {
                const DevStep &d = ds[b0 + i];
                return ((d.flags & kStepUnary) ? 16 : 0) + d.nk_ab + d.nk_a + d.nk_b;
            };
            std::stable_sort(by_kind.begin(), by_kind.end(), [&](int x, int y) { return kind(x) < kind(y); });
            std::vector<uint32_t> row(lanes, 0xffffffffu);
            int lane = 0;
            for (int i : by_kind)
                for (int j = 0; j < cnt[i]; j++, lane++)
                    row[lane] = (uint32_t)(b0 + i) | ((uint32_t)j << 12) | ((uint32_t)cnt[i] << 22);
            lane_map.insert(lane_map.end(), row.begin(), row.end());
            n_phases++;
        }
    }
    if (!fused_ok) { fs.clear(); tab.clear(); lane_map.clear(); n_phases = 0; }
    DevProgram h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kProgramMagic;
    h.n_steps = (uint32_t)ds.size();
    h.n_leaves = (uint32_t)dl.size();
    h.n_leaf_entries = ldata.size() / 2;
    h.arena_elems = (uint64_t)p.arena_elems;
    const PTensor &F = p.tensors[p.final_tensor];
    h.final_off = (uint64_t)F.offset;
    h.n_inner = (uint32_t)p.n_inner;
    for (int i = 0; i < p.n_inner; i++)
        if (find_pos(F.modes, p.slices[i]) >= 0) h.final_present |= 1u << i;
    h.n_open = (uint32_t)p.open_qubits.size();
    for (size_t i = 0; i < p.open_qubits.size(); i++)
        if (find_pos(F.modes, m.n_vars + p.open_qubits[i]) >= 0) h.open_present |= 1u << i;
    h.zero_mask = m.zero_mask[0];
    h.zero_mask_hi = m.zero_mask[1];
    h.scalar_re = p.prog_scalar.real();
    h.scalar_im = p.prog_scalar.imag();
    h.n_outer = uint64_t(1) << ((int)p.slices.size() - p.n_inner);
    size_t off = align256(sizeof(DevProgram));
    h.steps_off = off;
    off = align256(off + ds.size() * sizeof(DevStep));
    h.leaves_off = off;
    off = align256(off + dl.size() * sizeof(DevLeaf));
    h.leaf_data_off = off;
    off = align256(off + ldata.size() * sizeof(float));
    if (!fs.empty()) {
        h.fused_steps_off = off;
        off = align256(off + fs.size() * sizeof(FusedStep));
        h.fused_tab_off = off;
        h.n_tab_entries = tab.size();
        h.fused_lane_map_off = h.fused_tab_off + tab.size() * sizeof(uint32_t);   // right after the tables
        h.n_fused_phases = (uint32_t)n_phases;
        h.fused_lanes = (uint32_t)lanes;
        off = align256(off + (tab.size() + lane_map.size()) * sizeof(uint32_t));
    }
    if (!rts.empty()) {
        h.regtile_off = off;
        off = align256(off + rts.size() * sizeof(RegTileStep));
    }
    if (!gms.empty()) {
        h.gemm_off = off;
        off = align256(off + gms.size() * sizeof(GemmStep));
    }
    // level phases (first step of each phase, then the step count)
    std::vector<uint32_t> level_first;
    for (const auto &ph : p.phases) level_first.push_back((uint32_t)ph.first);
    level_first.push_back((uint32_t)p.steps.size());
    h.level_phases_off = off;
    h.n_level_phases = (uint32_t)p.phases.size();
    off = align256(off + level_first.size() * sizeof(uint32_t));
    // gradient program
    std::vector<uint32_t> csr;
    std::vector<double> thetas;
    std::vector<GradEntry> gent;
    std::vector<uint32_t> gktab, gphase;
    if (p.opts.gradient) {
        // checkpointing: while one work item's gradient arena exceeds the memory budget, forward
        // values are recomputed in the backward pass instead of kept, largest first; a value
        // stays dropped only if that lowers the arena (at most 48 trial programs)
        std::vector<char> keep(p.tensors.size(), 1);
        if (!build_grad_program(p, dev_leaf, keep, err)) return false;
        if (p.grad_arena_elems * 8 > p.opts.mem_budget_bytes) {
            std::vector<int> cand;
            for (const PStep &st : p.steps)
                for (int t : {st.a, st.b})
                    if (t >= 0 && t != p.final_tensor && p.tensors[t].leaf < 0) cand.push_back(t);
            std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) {
                return p.tensors[x].modes.size() > p.tensors[y].modes.size();
            });
            int64_t best = p.grad_arena_elems;
            int trials = 0;
            for (int t : cand) {
                if (best * 8 <= p.opts.mem_budget_bytes || trials >= 48) break;
                keep[t] = 0;
                trials++;
                if (!build_grad_program(p, dev_leaf, keep, err)) return false;
                if (p.grad_arena_elems < best) best = p.grad_arena_elems;
                else keep[t] = 1;
            }
            if (!build_grad_program(p, dev_leaf, keep, err)) return false;
        }
        // parametrised leaves in the order of the derivative slots
        std::vector<ParamLeaf> ordered;
        for (int l : p.grad_param_leaves) ordered.push_back(pls[pleaf_of_leaf[l]]);
        pls = ordered;
        thetas.assign(p.n_params, 0.0);
        std::vector<char> seen(p.n_params, 0);
        for (int l : p.grad_param_leaves) {
            const HostTensor &hl = p.leaves[l];
            if (hl.param < p.n_params && !seen[hl.param]) { thetas[hl.param] = hl.theta; seen[hl.param] = 1; }
        }
        // CSR: parameter -> derivative slots
        csr.assign(p.n_params + 1, 0);
        for (const ParamLeaf &q : pls) csr[q.param + 1]++;
        for (int i = 0; i < p.n_params; i++) csr[i + 1] += csr[i];
        std::vector<uint32_t> fill(csr.begin(), csr.end() - 1), list(pls.size());
        for (size_t i = 0; i < pls.size(); i++) list[fill[pls[i].param]++] = (uint32_t)i;
        csr.insert(csr.end(), list.begin(), list.end());
        h.n_grad_steps = (uint32_t)p.grad_steps.size();
        h.n_param_leaves = (uint32_t)pls.size();
        h.n_params = (uint32_t)p.n_params;
        h.grad_arena_elems = (uint64_t)p.grad_arena_elems;
        h.final_fwd_off = (uint64_t)p.grad_final_off;
        h.gslot_off = (uint64_t)p.grad_gslot_off;
        h.grad_steps_off = off;
        off = align256(off + p.grad_steps.size() * sizeof(GenStep));
        h.params_off = off;
        off = align256(off + pls.size() * sizeof(ParamLeaf));
        h.codes_off = off;
        off = align256(off + codes.size());
        h.deriv_data_off = off;
        off = align256(off + ldata.size() * sizeof(float));
        h.thetas_off = off;
        off = align256(off + thetas.size() * sizeof(double));
        h.param_csr_off = off;
        off = align256(off + csr.size() * sizeof(uint32_t));
        h.grad_phases_off = off;
        h.n_grad_phases = (uint32_t)p.grad_phase_first.size() - 1;
        off = align256(off + p.grad_phase_first.size() * sizeof(uint32_t));
        h.grad_elem_off_off = off;
        off = align256(off + p.grad_elem_off.size() * sizeof(uint32_t));
        if (build_grad_tables(p, &gent, &gktab, &gphase)) {
            h.gentry_off = off;
            off = align256(off + gent.size() * sizeof(GradEntry));
            h.gktab_off = off;
            off = align256(off + std::max<size_t>(gktab.size(), 1) * sizeof(uint32_t));
            h.gphase_entry_off = off;
            off = align256(off + gphase.size() * sizeof(uint32_t));
        }
    }
    h.image_bytes = off;
    p.image.assign(off, 0);
    std::memcpy(p.image.data() + h.level_phases_off, level_first.data(), level_first.size() * sizeof(uint32_t));
    if (!rts.empty()) std::memcpy(p.image.data() + h.regtile_off, rts.data(), rts.size() * sizeof(RegTileStep));
    p.regtile = rts;
    if (!gms.empty()) std::memcpy(p.image.data() + h.gemm_off, gms.data(), gms.size() * sizeof(GemmStep));
    p.gemm = gms;
    if (p.opts.gradient) {
        unsigned char *img = p.image.data();
        if (!p.grad_steps.empty()) std::memcpy(img + h.grad_steps_off, p.grad_steps.data(), p.grad_steps.size() * sizeof(GenStep));
        if (!pls.empty()) std::memcpy(img + h.params_off, pls.data(), pls.size() * sizeof(ParamLeaf));
        if (!codes.empty()) std::memcpy(img + h.codes_off, codes.data(), codes.size());
        if (!thetas.empty()) std::memcpy(img + h.thetas_off, thetas.data(), thetas.size() * sizeof(double));
        if (!csr.empty()) std::memcpy(img + h.param_csr_off, csr.data(), csr.size() * sizeof(uint32_t));
        std::memcpy(img + h.grad_phases_off, p.grad_phase_first.data(), p.grad_phase_first.size() * sizeof(uint32_t));
        if (!p.grad_elem_off.empty())
            std::memcpy(img + h.grad_elem_off_off, p.grad_elem_off.data(), p.grad_elem_off.size() * sizeof(uint32_t));
        if (h.gentry_off) {
            std::memcpy(img + h.gentry_off, gent.data(), gent.size() * sizeof(GradEntry));
            if (!gktab.empty()) std::memcpy(img + h.gktab_off, gktab.data(), gktab.size() * sizeof(uint32_t));
            std::memcpy(img + h.gphase_entry_off, gphase.data(), gphase.size() * sizeof(uint32_t));
        }
    }
    std::memcpy(p.image.data(), &h, sizeof(h));
    if (!ds.empty()) std::memcpy(p.image.data() + h.steps_off, ds.data(), ds.size() * sizeof(DevStep));
    if (!dl.empty()) std::memcpy(p.image.data() + h.leaves_off, dl.data(), dl.size() * sizeof(DevLeaf));
    if (!ldata.empty()) std::memcpy(p.image.data() + h.leaf_data_off, ldata.data(), ldata.size() * sizeof(float));
    if (!fs.empty()) {
        std::memcpy(p.image.data() + h.fused_steps_off, fs.data(), fs.size() * sizeof(FusedStep));
        if (!tab.empty()) std::memcpy(p.image.data() + h.fused_tab_off, tab.data(), tab.size() * sizeof(uint32_t));
        if (!lane_map.empty())
            std::memcpy(p.image.data() + h.fused_lane_map_off, lane_map.data(), lane_map.size() * sizeof(uint32_t));
    }
    return true;
}

// Builds program, layouts, arena and stats for the current order/slices/n_inner.
bool build_program(Plan &p, std::string *err) {
    p.leaves.clear();
    p.tensors.clear();
    p.steps.clear();
    p.final_tensor = -1;
    ProgramBuilder b(p, p.model);
    if (!b.run()) { *err = b.err; return false; }
    p.prog_scalar = p.model.scalar * b.factor;
    schedule_levels(p);
    assign_layouts(p);
    p.arena_elems = allocate_arena(p);
    program_stats(p);
    return true;
}

}  // namespace

// Time estimate of a plan's contractions, in HBM byte-equivalents, summed over the work
// items of one bitstring; it ranks planning trials (Section 3.B ranks orders by flops alone,
// which leaves out that most steps are bandwidth bound). Fused engine (every tensor in
// shared memory): per step max(algorithmic bytes, flops / 12), about the FP32 FMA rate over
// the HBM bandwidth. Global-arena engines: the rates the step kernels reach on a GB300 in
// the 64-qubit benchmark, relative to the register-tiled SIMT kernel's streaming rate (about
// 5.5 TB/s): a SIMT step costs max(bytes, flops / 3.3) (its compute-bound steps run near 18
// TFLOP/s), a step the tensor cores take max(1.6 bytes, flops / 32) (about 3.5 TB/s and 175
// algorithmic TFLOP/s; flops / 16 with 8 summed entries, whose chunk is half padding).
double plan_estimate(const Plan &p) {
    double t = 0;
    const bool fused = p.engine == QVX_ENGINE_FUSED;
    for (size_t s = 0; s < p.steps.size(); s++) {
        double fl, by;
        step_work(p, p.steps[s], &fl, &by);
        if (fused) t += std::max(by, fl / 12.0);
        else if (!p.gemm.empty() && p.gemm[s].nk > 0) t += std::max(1.6 * by, fl / (p.gemm[s].nk == 3 ? 16.0 : 32.0));
        else t += std::max(by, fl / 3.3);
    }
    return t * std::ldexp(1.0, (int)p.slices.size() - p.n_inner);
}

void step_cost(const Plan &p, size_t s, double *flops, double *bytes) { step_work(p, p.steps[s], flops, bytes); }

namespace {

qvx_status plan_once(const qvx_circuit *c, const int32_t *order, int32_t n_order,
                     const int32_t *slices, int32_t n_slices, const qvx_plan_opts &opts,
                     Plan *p, std::string *err);

}  // namespace

// ---------------------------------------------------------------- entry point
// Section 3.B picks one ordering (QuickBB) and then the sliced variables; here every trial
// re-runs the randomised ordering, the slice choice and the re-ordering from its own seed,
// and the trial with the smallest estimate (plan_estimate) is kept. Trial 0 uses the given
// seed, so plan_trials = 1 is the single-trial planner.
qvx_status make_plan(const qvx_circuit *c, const int32_t *order, int32_t n_order,
                     const int32_t *slices, int32_t n_slices, const qvx_plan_opts &opts,
                     Plan *p, std::string *err) {
    const bool fixed = n_order > 0 && n_slices >= 0;
    const int trials = fixed ? 1 : std::max(1, opts.plan_trials);
    if (trials == 1) return plan_once(c, order, n_order, slices, n_slices, opts, p, err);
    // trials are independent: run them on host threads. Each thread keeps only its best
    // plan so far (at most one plan per thread besides the one being built); the best
    // overall is the lowest estimate, ties to the lowest trial index, so the result does not
    // depend on the thread count. Ranking fused-engine plans by their level count first was
    // measured on 6x6x25 (12 sliced, 5 open, 8 warps per item): 12 levels with twice the
    // bytes took 21.6 us per amplitude against 18.6 us for 15 levels, so the estimate alone
    // ranks.
    struct Best {
        int t = -1;
        double est = 0;
        Plan plan;
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int n_threads = (int)std::min<unsigned>(std::min<unsigned>(hw, 16u), (unsigned)trials);
    std::vector<Best> best(n_threads);
    std::vector<std::string> errs(trials);
    std::vector<qvx_status> st(trials, QVX_EUNSUPPORTED);
    std::vector<char> oom(trials, 0);
    std::atomic<int> next{0};
    auto work = [&](int w) {
        for (int t = next++; t < trials; t = next++) {
            qvx_plan_opts o = opts;
            // trial t's seed: an odd 64-bit multiplier keeps the trials' seeds distinct
            o.order_seed = opts.order_seed + uint64_t(t) * 0xD1B54A32D192ED03ull;
            try {
                Plan cand;
                st[t] = plan_once(c, order, n_order, slices, n_slices, o, &cand, &errs[t]);
                if (st[t] != QVX_OK) continue;
                const double est = plan_estimate(cand);
                Best &b = best[w];
                if (b.t < 0 || est < b.est || (est == b.est && t < b.t)) {
                    b.t = t;
                    b.est = est;
                    b.plan = std::move(cand);
                }
            } catch (const std::bad_alloc &) {
                oom[t] = 1;
            } catch (const std::exception &e) {
                st[t] = QVX_EUNSUPPORTED;
                errs[t] = e.what();
            }
        }
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < n_threads; i++) {
        try {
            pool.emplace_back(work, i);
        } catch (const std::system_error &) {
            break;   // fewer threads: the calling thread takes the remaining trials
        }
    }
    work(0);
    for (auto &th : pool) th.join();
    for (int t = 0; t < trials; t++) {
        if (oom[t]) throw std::bad_alloc();
        if (st[t] != QVX_OK && st[t] != QVX_EUNSUPPORTED) { *err = errs[t]; return st[t]; }  // bad input
    }
    int bw = -1;
    for (int w = 0; w < n_threads; w++) {
        const Best &b = best[w];
        if (b.t < 0) continue;
        if (bw < 0 || b.est < best[bw].est || (b.est == best[bw].est && b.t < best[bw].t)) bw = w;
    }
    if (bw < 0) { *err = errs[0]; return QVX_EUNSUPPORTED; }
    *p = std::move(best[bw].plan);
    return QVX_OK;
}

namespace {

qvx_status plan_once(const qvx_circuit *c, const int32_t *order, int32_t n_order,
                     const int32_t *slices, int32_t n_slices, const qvx_plan_opts &opts,
                     Plan *p, std::string *err) {
    p->opts = opts;
    if (!build_model(c, &p->model, err, opts.gradient != 0)) return QVX_EINVAL;
    if (opts.n_open_qubits < 0 || opts.n_open_qubits > 16) { *err = "opts: n_open_qubits must be in [0, 16]"; return QVX_EINVAL; }
    if (opts.n_open_qubits > 0 && opts.gradient) { *err = "open qubits are not supported with gradients"; return QVX_EUNSUPPORTED; }
    p->open_qubits.clear();
    for (int i = 0; i < opts.n_open_qubits; i++) {
        const int qb = opts.open_qubits[i];
        if (qb < 0 || qb >= c->n_qubits || find_pos(p->open_qubits, qb) >= 0) { *err = "open_qubits: bad or repeated qubit"; return QVX_EINVAL; }
        if ((p->model.zero_mask[qb >> 6] >> (qb & 63)) & 1ull) { *err = "open_qubits: a qubit without a non-diagonal gate has no output variable"; return QVX_EINVAL; }
        p->open_qubits.push_back(qb);
    }
    if (opts.gradient)
        for (int64_t i = 0; i < c->n_gates; i++)
            if (c->gates[i].kind == QVX_GATE_RXY && c->gates[i].param_index >= 0)
                p->n_params = std::max(p->n_params, c->gates[i].param_index + 1);
    const Model &m = p->model;
    const int nv = m.n_vars;
    Graph g;
    g.init(nv, m.edges);
    std::vector<char> none(nv, 0);
    int w0 = 0;
    std::vector<int> first;
    double c0 = best_order(g, none, opts, 1, &first, &w0);
    p->log2_cost_unsliced = c0 > 0 ? std::log2(c0) : 0;
    // slices: given, or greedy on the cost under the first order (Section 3.B.2-3)
    std::vector<char> removed(nv, 0);
    std::vector<int> sl;
    if (n_slices >= 0) {
        if (n_slices > 0 && !slices) { *err = "slices: null list"; return QVX_EINVAL; }
        for (int i = 0; i < n_slices; i++) {
            int v = slices[i];
            if (v < 0 || v >= nv || removed[v]) { *err = "slices: bad or repeated variable id"; return QVX_EINVAL; }
            removed[v] = 1;
            sl.push_back(v);
        }
    } else {
        int want = opts.n_slices;
        const double budget = (double)opts.mem_budget_bytes;
        std::vector<int> cur = first;    // the ordering the candidates are scored under
        uint64_t reseed = opts.order_seed ^ 0x5851F42D4C957F2Dull;
        bool any_cz = false;
        for (int v = 0; v < nv; v++) any_cz = any_cz || m.cz_count[v] >= 2;
        for (int it = 0; it < nv; it++) {
            int wd = 0;
            order_cost(g, cur, removed, &wd);
            bool fits = std::ldexp(8.0, wd) <= budget;
            if (want >= 0 ? (int)sl.size() >= want : fits) break;
            double best = -1;
            int bv = -1;
            for (int v = 0; v < nv; v++) {
                if (removed[v]) continue;
                if (opts.slice_rule == 2 && any_cz && m.cz_count[v] < 2) continue;
                removed[v] = 1;
                double cv = order_cost(g, cur, removed, nullptr);
                removed[v] = 0;
                if (best < 0 || cv < best) { best = cv; bv = v; }
            }
            if (bv < 0) break;
            removed[bv] = 1;
            sl.push_back(bv);
            if (opts.slice_rule == 1) {   // re-order the reduced graph before the next pick
                int w2 = 0;
                best_order(g, removed, opts, 3 + splitmix64(reseed) % 1000003, &cur, &w2);
            }
        }
    }
    if (sl.size() > 40) { *err = "more than 40 sliced variables"; return QVX_EUNSUPPORTED; }
    // the order: given, or re-ordered after removing the sliced vertices (Section 3.B.3)
    if (n_order > 0) {
        if (!order) { *err = "order: null list"; return QVX_EINVAL; }
        std::vector<char> seen(nv, 0);
        for (int i = 0; i < n_order; i++) {
            int v = order[i];
            if (v < 0 || v >= nv || seen[v] || removed[v]) { *err = "order: bad, repeated or sliced variable id"; return QVX_EINVAL; }
            seen[v] = 1;
            p->order.push_back(v);
        }
        if ((int)p->order.size() + (int)sl.size() != nv) { *err = "order: must hold every variable that is not sliced"; return QVX_EINVAL; }
        p->log2_cost = std::log2(std::max(1.0, order_cost(g, p->order, removed, &p->width)));
    } else {
        double cst = best_order(g, removed, opts, 2, &p->order, &p->width);
        p->log2_cost = cst > 0 ? std::log2(cst) : 0;
    }
    // inner slices: kept open inside one work item. Pick them greedily by the program's
    // flops, as many as requested or as fit the fused engine's per-warp memory.
    const int k = (int)sl.size();
    int inner_want = opts.inner_slices;
    p->slices = sl;
    p->n_inner = 0;
    if (!build_program(*p, err)) return QVX_EUNSUPPORTED;
    const int64_t fused_limit = int64_t(12) * 1024 / 8;   // complex64 entries per warp
    std::vector<int> inner, outer = sl;
    int target = inner_want >= 0 ? std::min(inner_want, k) : k;
    while ((int)inner.size() < target) {
        double best = -1;
        int bi = -1;
        int64_t best_arena = 0;
        for (size_t i = 0; i < outer.size(); i++) {
            std::vector<int> trial = inner;
            trial.push_back(outer[i]);
            for (size_t j = 0; j < outer.size(); j++)
                if (j != i) trial.push_back(outer[j]);
            p->slices = trial;
            p->n_inner = (int)inner.size() + 1;
            if (!build_program(*p, err)) return QVX_EUNSUPPORTED;
            double per_slice = p->flops_per_item / std::ldexp(1.0, p->n_inner);
            if (best < 0 || per_slice < best) { best = per_slice; bi = (int)i; best_arena = p->arena_elems; }
        }
        if (inner_want < 0 && (best_arena > fused_limit || (int)inner.size() >= 8 ||
                               k - (int)inner.size() - 1 < 8))
            break;   // auto: stay within shared memory and keep >= 256 work items
        inner.push_back(outer[bi]);
        outer.erase(outer.begin() + bi);
    }
    p->slices = inner;
    p->slices.insert(p->slices.end(), outer.begin(), outer.end());
    p->n_inner = (int)inner.size();
    if (!build_program(*p, err)) return QVX_EUNSUPPORTED;
    if (p->max_rank > std::min(30, opts.max_rank)) {
        *err = "a tensor of rank " + std::to_string(p->max_rank) + " exceeds max_rank";
        return QVX_EUNSUPPORTED;
    }
    // engine
    const int64_t arena_bytes = p->arena_elems * 8;
    p->warps_per_item = std::max(1, std::min(16, opts.warps_per_item));
    if (opts.engine == QVX_ENGINE_AUTO)
        p->engine = arena_bytes <= 48 * 1024 ? QVX_ENGINE_FUSED : QVX_ENGINE_PERSISTENT;
    else p->engine = opts.engine;
    if (p->engine == QVX_ENGINE_FUSED && arena_bytes > 200 * 1024) {
        *err = "fused engine: arena of " + std::to_string(arena_bytes) + " bytes exceeds shared memory";
        return QVX_EUNSUPPORTED;
    }
    if (p->engine == QVX_ENGINE_PERSISTENT) p->arena_elems = allocate_arena_unique(*p);
    if (!serialize(*p, err)) return QVX_EUNSUPPORTED;
    if (p->engine == QVX_ENGINE_FUSED &&
        reinterpret_cast<const DevProgram *>(p->image.data())->fused_steps_off == 0 && !p->steps.empty()) {
        if (opts.engine == QVX_ENGINE_FUSED) { *err = "fused engine: offsets exceed 16 bits"; return QVX_EUNSUPPORTED; }
        p->engine = QVX_ENGINE_PERSISTENT;
        p->arena_elems = allocate_arena_unique(*p);
        if (!serialize(*p, err)) return QVX_EUNSUPPORTED;
    }
    return QVX_OK;
}

}  // namespace

}  // namespace qvx
