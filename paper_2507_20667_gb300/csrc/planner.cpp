// Host planner: Greedy trees, the cost model, the fan-in tree and the simulated-annealing
// refinement of the partitioning (Sections 2.3-4.4 of arXiv 2507.20667).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <queue>
#include <thread>

#include "tn_internal.hpp"

namespace tn {

static const u128 kSizeCap = ((u128)1) << 120;

u128 legs_size(const Legs &l, const std::vector<int64_t> &edim, bool &ovf) {
    u128 p = 1;
    for (int32_t e : l) {
        p *= (u128)edim[e];
        if (p > kSizeCap) { ovf = true; p = kSizeCap; }
    }
    return p;
}

// Product of n(e) over legs(a) U legs(b): 2^vc of Eq. 3.3 as an integer product.
u128 union_size(const Legs &a, const Legs &b, const std::vector<int64_t> &edim, bool &ovf) {
    u128 p = 1;
    size_t i = 0, j = 0;
    while (i < a.size() || j < b.size()) {
        int32_t e;
        if (j == b.size() || (i < a.size() && a[i] < b[j])) e = a[i++];
        else if (i == a.size() || b[j] < a[i]) e = b[j++];
        else { e = a[i]; ++i; ++j; }
        p *= (u128)edim[e];
        if (p > kSizeCap) { ovf = true; p = kSizeCap; }
    }
    return p;
}

// Eq. 2.6: the legs of a contracted pair are the symmetric difference of the children's legs.
void legs_symdiff(const Legs &a, const Legs &b, Legs &out) {
    out.clear();
    size_t i = 0, j = 0;
    while (i < a.size() || j < b.size()) {
        if (j == b.size() || (i < a.size() && a[i] < b[j])) out.push_back(a[i++]);
        else if (i == a.size() || b[j] < a[i]) out.push_back(b[j++]);
        else { ++i; ++j; }
    }
}

bool legs_intersect(const Legs &a, const Legs &b) {
    size_t i = 0, j = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] == b[j]) return true;
        if (a[i] < b[j]) ++i; else ++j;
    }
    return false;
}

// ------------------------------------------------------------------------------------ Greedy
// The Greedy rule (Section 2.3 with the memory-reduction objective of Eq. 4.5): repeatedly
// contract the pair sharing a leg with the largest |A| + |B| - |A*B|; ties go to the
// lexicographically smallest (i, j) in local ids; new nodes take the next id; a set with no
// connected pair joins its two smallest tensors (by size, then id) by an outer product.
namespace {
struct Cand {
    i128 obj;
    int32_t i, j;
};
struct CandLess {  // priority_queue pops the "largest": higher obj, then smaller i, smaller j
    bool operator()(const Cand &x, const Cand &y) const {
        if (x.obj != y.obj) return x.obj < y.obj;
        if (x.i != y.i) return x.i > y.i;
        return x.j > y.j;
    }
};
}  // namespace

GreedyTree greedy_tree(const std::vector<const Legs *> &init, const std::vector<int64_t> &edim,
                       bool &ovf) {
    GreedyTree out;
    const int32_t s = (int32_t)init.size();
    if (s == 0) return out;
    std::vector<Legs> legs(2 * s - 1);
    std::vector<u128> size(2 * s - 1, 0);
    std::vector<char> alive(2 * s - 1, 0);
    for (int32_t i = 0; i < s; ++i) {
        legs[i] = *init[i];
        size[i] = legs_size(legs[i], edim, ovf);
        alive[i] = 1;
    }
    if (s == 1) {
        out.root_legs = legs[0];
        out.root_size = size[0];
        return out;
    }
    // holders: which (at most two) live nodes carry each edge
    std::vector<int32_t> touched;
    std::vector<std::array<int32_t, 2>> hold;
    std::vector<int32_t> slot(edim.size(), -1);
    auto add_holder = [&](int32_t e, int32_t v) {
        if (slot[e] < 0) {
            slot[e] = (int32_t)hold.size();
            hold.push_back({-1, -1});
            touched.push_back(e);
        }
        auto &h = hold[slot[e]];
        if (h[0] < 0) h[0] = v; else h[1] = v;
    };
    auto drop_holder = [&](int32_t e, int32_t v) {
        auto &h = hold[slot[e]];
        if (h[0] == v) { h[0] = h[1]; h[1] = -1; }
        else if (h[1] == v) h[1] = -1;
    };
    for (int32_t i = 0; i < s; ++i)
        for (int32_t e : legs[i]) add_holder(e, i);

    std::priority_queue<Cand, std::vector<Cand>, CandLess> pq;
    auto objective = [&](int32_t i, int32_t j) -> i128 {
        Legs r;
        legs_symdiff(legs[i], legs[j], r);
        return (i128)size[i] + (i128)size[j] - (i128)legs_size(r, edim, ovf);
    };
    auto push_pair = [&](int32_t a, int32_t b) {
        int32_t i = std::min(a, b), j = std::max(a, b);
        pq.push(Cand{objective(i, j), i, j});
    };
    for (int32_t e : touched) {
        auto &h = hold[slot[e]];
        if (h[0] >= 0 && h[1] >= 0) push_pair(h[0], h[1]);   // duplicates are harmless
    }
    int32_t next = s, n_alive = s;
    while (n_alive > 1) {
        int32_t i = -1, j = -1;
        while (!pq.empty()) {
            Cand c = pq.top();
            pq.pop();
            if (alive[c.i] && alive[c.j]) { i = c.i; j = c.j; break; }
        }
        if (i < 0) {  // no connected pair: outer product of the two smallest by (size, id)
            int32_t a = -1, b = -1;
            for (int32_t v = 0; v < next; ++v) {
                if (!alive[v]) continue;
                if (a < 0 || size[v] < size[a]) { b = a; a = v; }
                else if (b < 0 || size[v] < size[b]) b = v;
            }
            i = std::min(a, b);
            j = std::max(a, b);
        }
        const int32_t o = next++;
        legs_symdiff(legs[i], legs[j], legs[o]);
        size[o] = legs_size(legs[o], edim, ovf);
        u128 c = union_size(legs[i], legs[j], edim, ovf);
        out.con += c;
        if (out.con > kSizeCap) { ovf = true; out.con = kSizeCap; }
        u128 m = size[o] + size[i] + size[j];
        if (m > out.mem) out.mem = m;
        out.steps.emplace_back(i, j);
        alive[i] = alive[j] = 0;
        alive[o] = 1;
        --n_alive;
        for (int32_t e : legs[i]) drop_holder(e, i);
        for (int32_t e : legs[j]) drop_holder(e, j);
        for (int32_t e : legs[o]) add_holder(e, o);
        for (int32_t e : legs[o]) {
            auto &h = hold[slot[e]];
            int32_t other = (h[0] == o) ? h[1] : h[0];
            if (other >= 0 && other != o) push_pair(o, other);
        }
    }
    out.root_legs = legs[next - 1];
    out.root_size = size[next - 1];
    return out;
}

// ------------------------------------------------------------------------------------ fan-in
namespace {
struct Rng {  // xoshiro256** seeded through splitmix64
    uint64_t s[4];
    explicit Rng(uint64_t seed) {
        for (int i = 0; i < 4; ++i) {
            seed += 0x9E3779B97F4A7C15ull;
            uint64_t z = seed;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            s[i] = z ^ (z >> 31);
        }
    }
    static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
    uint64_t next() {
        uint64_t r = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
        s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]; s[2] ^= t; s[3] = rotl(s[3], 45);
        return r;
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    uint32_t below(uint32_t n) { return (uint32_t)(((next() >> 32) * (uint64_t)n) >> 32); }
};

uint64_t mix64(uint64_t h, uint64_t v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h * 0xff51afd7ed558ccdull;
}

}  // namespace

// The fan-in problem in the shared bitset form: compact edge ids are the union of the roots'
// legs in increasing edge order.
void fanin_input(const std::vector<Legs> &roots, const std::vector<u128> &part_con,
                 const std::vector<int64_t> &edim, uint64_t seed, FaninInput &in) {
    in.k = (int32_t)roots.size();
    in.seed = seed;
    in.part_con = part_con;
    std::vector<int32_t> ids;
    for (const Legs &r : roots) ids.insert(ids.end(), r.begin(), r.end());
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    in.W = std::max<int32_t>(1, (int32_t)((ids.size() + 63) / 64));
    in.unit = true;
    for (int32_t e : ids) in.unit = in.unit && edim[e] == 2;
    in.roots.assign((size_t)in.k * in.W, 0);
    for (int32_t i = 0; i < in.k; ++i)
        for (int32_t e : roots[i]) {
            const size_t x = (size_t)(std::lower_bound(ids.begin(), ids.end(), e) - ids.begin());
            in.roots[(size_t)i * in.W + x / 64] |= 1ull << (x % 64);
        }
    in.dims.clear();
    if (!in.unit) {
        in.dims.assign((size_t)64 * in.W, 1);
        for (size_t x = 0; x < ids.size(); ++x) in.dims[x] = edim[ids[x]];
    }
}

namespace {
// One Greedy pass (a RandomGreedy sample; noiseless when !noisy) over the k roots in legs[0..k):
// repeatedly merge the connected pair of live nodes that comes first in fanin::pair_before order
// (scores are fixed per pair, so a heap with lazy deletion holds them); a set with no connected
// pair merges its two smallest nodes (size, then id).  steps[2 s], steps[2 s + 1] = merge s.
void greedy_pass(int k, const fanin::Dims &d, bool noisy, uint64_t seed, uint64_t *legs, u128 *size,
                 uint8_t *alive, int16_t *steps, bool &sat) {
    const int W = d.W;
    struct Cand {
        i128 score;
        int32_t i, j;
    };
    auto later = [](const Cand &a, const Cand &b) { return fanin::pair_before(b.score, b.i, b.j, a.score, a.i, a.j); };
    std::priority_queue<Cand, std::vector<Cand>, decltype(later)> heap(later);
    auto push = [&](int i, int j) {
        const uint64_t *li = legs + (size_t)i * W, *lj = legs + (size_t)j * W;
        if (!fanin::intersects(li, lj, W)) return;
        const i128 obj = (i128)size[i] + (i128)size[j] - (i128)fanin::set_size(li, lj, 1, d, sat);
        heap.push(Cand{fanin::pair_score(obj, noisy, seed, (uint32_t)i, (uint32_t)j), i, j});
    };
    for (int i = 0; i < k; ++i) {
        size[i] = fanin::set_size(legs + (size_t)i * W, legs + (size_t)i * W, 0, d, sat);
        alive[i] = 1;
    }
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j) push(i, j);
    for (int it = 0; it < k - 1; ++it) {
        const int next = k + it;
        int bi = -1, bj = -1;
        while (!heap.empty()) {
            const Cand c = heap.top();
            heap.pop();
            if (alive[c.i] && alive[c.j]) {
                bi = c.i;
                bj = c.j;
                break;
            }
        }
        if (bi < 0) {   // no connected pair: the two smallest (size, then id)
            int a = -1, b = -1;
            for (int v = 0; v < next; ++v) {
                if (!alive[v]) continue;
                if (a < 0 || size[v] < size[a]) {
                    b = a;
                    a = v;
                } else if (b < 0 || size[v] < size[b]) {
                    b = v;
                }
            }
            bi = std::min(a, b);
            bj = std::max(a, b);
        }
        uint64_t *ln = legs + (size_t)next * W;
        for (int w = 0; w < W; ++w) ln[w] = legs[(size_t)bi * W + w] ^ legs[(size_t)bj * W + w];
        size[next] = fanin::set_size(ln, ln, 0, d, sat);
        alive[bi] = alive[bj] = 0;
        alive[next] = 1;
        steps[2 * it] = (int16_t)bi;
        steps[2 * it + 1] = (int16_t)bj;
        for (int x = 0; x < next; ++x)
            if (alive[x]) push(x, next);
    }
}

// Every merge order of k <= 4 roots (recursively: each pair of the live nodes, then the rest).
void enumerate_orders(std::vector<int32_t> &live, int32_t next, std::vector<int16_t> &cur,
                      const std::function<void(const std::vector<int16_t> &)> &visit) {
    if (live.size() == 1) {
        visit(cur);
        return;
    }
    for (size_t x = 0; x < live.size(); ++x)
        for (size_t y = x + 1; y < live.size(); ++y) {
            const int32_t a = live[x], b = live[y];
            std::vector<int32_t> rest;
            for (int32_t v : live) if (v != a && v != b) rest.push_back(v);
            rest.push_back(next);
            cur.push_back((int16_t)std::min(a, b));
            cur.push_back((int16_t)std::max(a, b));
            enumerate_orders(rest, next + 1, cur, visit);
            cur.resize(cur.size() - 2);
        }
}
}  // namespace

// The fan-in (reduction) tree of Section 4.4: for k <= 4 every merge order is tried; above that
// RandomGreedy keeps the best of `samples` Greedy passes (sample 0 noiseless, the others with the
// integer perturbation of fanin::pair_score).  Best = smallest con_dist, then smallest fan-in con,
// then first.  The batched GPU evaluator (fanin_eval.cu) makes the same choices.
FanIn fanin_host(const FaninInput &in, int samples, int sample, bool &ovf) {
    const int32_t k = in.k;
    FanIn out;
    if (k == 1) {
        out.con_dist = in.part_con[0];
        return out;
    }
    const fanin::Dims d{in.W, in.unit ? 1 : 0, in.dims.empty() ? nullptr : in.dims.data()};
    const size_t nn = 2 * (size_t)k - 1;
    std::vector<uint64_t> legs(nn * in.W, 0);
    std::copy(in.roots.begin(), in.roots.end(), legs.begin());
    std::vector<u128> size(nn), cost(nn);
    std::vector<int16_t> parent(nn), steps(2 * (size_t)(k - 1));
    std::vector<uint8_t> alive(nn);
    fanin::Counts best{0, 0, 0, false};
    std::vector<int16_t> best_steps;
    bool have = false, sat = false;
    auto consider = [&](const std::vector<int16_t> &st) {
        const fanin::Counts c = fanin::eval_steps(k, in.part_con.data(), st.data(), d, legs.data(), size.data(),
                                                  parent.data(), cost.data());
        sat = sat || c.sat;
        if (!have || fanin::better(c, best)) {
            best = c;
            best_steps = st;
            have = true;
        }
    };
    if (k <= 4) {
        std::vector<int32_t> live(k);
        for (int32_t i = 0; i < k; ++i) live[i] = i;
        std::vector<int16_t> cur;
        enumerate_orders(live, k, cur, consider);
    } else {
        const int s0 = sample >= 0 ? sample : 0, s1 = sample >= 0 ? sample + 1 : std::max(samples, 1);
        for (int smp = s0; smp < s1; ++smp) {
            greedy_pass(k, d, smp > 0, smp > 0 ? fanin::sample_seed(in.seed, smp) : 0, legs.data(), size.data(),
                        alive.data(), steps.data(), sat);
            consider(steps);
        }
    }
    if (sat) ovf = true;
    out.con_dist = best.con_dist;
    out.con = best.con;
    out.mem = best.mem;
    for (int32_t t = 0; t + 1 < k; ++t) out.steps.emplace_back(best_steps[2 * t], best_steps[2 * t + 1]);
    return out;
}

FanIn fanin_tree(const std::vector<Legs> &roots, const std::vector<u128> &part_con,
                 const std::vector<int64_t> &edim, int samples, uint64_t seed, bool &ovf) {
    FaninInput in;
    fanin_input(roots, part_con, edim, seed, in);
    return fanin_host(in, samples, -1, ovf);
}

// ------------------------------------------------------------------------------------ counts
tn_status plan_finalize(const Net &net, Plan &p) {
    const int32_t n = net.n;
    if ((int32_t)p.steps.size() != n - 1) return fail(TN_EINVAL, "a plan needs n_tensors - 1 steps");
    const int32_t nn = 2 * n - 1;
    std::vector<Legs> legs(nn);
    std::vector<u128> cost(nn, 0), sub(nn, 0), acc(nn, 0), size(nn, 0);
    std::vector<int32_t> parent(nn, -1), label(nn, -1), count(nn, 0);
    std::vector<int32_t> part_size(p.k, 0);
    bool ovf = false;
    for (int32_t t = 0; t < n; ++t) {
        legs[t] = net.legs[t];
        size[t] = legs_size(legs[t], net.edim, ovf);
        label[t] = p.part[t];
        count[t] = 1;
        if (p.part[t] < 0 || p.part[t] >= p.k) return fail(TN_EINVAL, "partition index out of range");
        part_size[p.part[t]]++;
    }
    for (int32_t k = 0; k < p.k; ++k)
        if (part_size[k] == 0) return fail(TN_EINVAL, "empty partition");
    u128 con = 0, mem = 0;
    for (int32_t s = 0; s < n - 1; ++s) {
        int32_t l = p.steps[s][0], r = p.steps[s][1], o = n + s;
        if (l < 0 || r < 0 || l >= o || r >= o || l == r || parent[l] >= 0 || parent[r] >= 0)
            return fail(TN_EINVAL, "steps do not form a binary contraction tree");
        p.steps[s][2] = o;
        parent[l] = parent[r] = o;
        legs_symdiff(legs[l], legs[r], legs[o]);
        size[o] = legs_size(legs[o], net.edim, ovf);
        cost[o] = union_size(legs[l], legs[r], net.edim, ovf);
        sub[o] = cost[o] + sub[l] + sub[r];
        con += cost[o];
        u128 m = size[o] + size[l] + size[r];
        if (m > mem) mem = m;
        count[o] = count[l] + count[r];
        label[o] = (label[l] >= 0 && label[l] == label[r]) ? label[l] : -1;
    }
    if (ovf) return fail(TN_EINVAL, "operation count exceeds 2^120");
    // acc(v): sum of 2^vc over the ancestors of v (v excluded), top-down.
    for (int32_t v = nn - 1; v >= 0; --v)
        acc[v] = parent[v] >= 0 ? acc[parent[v]] + cost[parent[v]] : 0;
    u128 cpar = 0;
    for (int32_t t = 0; t < n; ++t) cpar = std::max(cpar, acc[t]);     // Eq. 3.4
    // Eq. 2.7: each partition must be the leaf set of a subtree (a pure node covering it).
    p.part_root.assign(p.k, -1);
    for (int32_t v = 0; v < nn; ++v)
        if (label[v] >= 0 && count[v] == part_size[label[v]]) p.part_root[label[v]] = v;
    u128 cdist = 0;
    for (int32_t k = 0; k < p.k; ++k) {
        if (p.part_root[k] < 0) return fail(TN_EINVAL, "the tree does not accept the partitioning");
        int32_t r = p.part_root[k];
        cdist = std::max(cdist, sub[r] + acc[r]);                        // Eq. 3.5, comm = 0
    }
    p.step_part.assign(n - 1, -1);
    for (int32_t s = 0; s < n - 1; ++s) p.step_part[s] = label[n + s];
    p.con_serial = con;
    p.con_par = cpar;
    p.con_dist = cdist;
    p.mem = mem;
    return TN_OK;
}

// ------------------------------------------------------------------------------------ SA
namespace {
struct PartState {
    std::vector<int32_t> members;   // global tensor ids, increasing
    GreedyTree tree;
};

struct State {
    std::vector<int32_t> part;
    std::vector<PartState> parts;
    FanIn fan;                      // its steps are left empty when a device evaluated the state
    int32_t fan_sample = -1;        // then: the winning RandomGreedy sample
    u128 cost = 0;                  // con_dist
};

struct Ctx {
    const Net &net;
    int32_t k;
    int32_t samples;
    bool ovf = false;
    int32_t device = -1;            // >= 0: fan-in trees of k > 4 evaluated in batches on this GPU
    FaninWorkspace *ws = nullptr;
};

void rebuild_part(const Ctx &c, PartState &ps, bool &ovf) {
    std::vector<const Legs *> init;
    init.reserve(ps.members.size());
    for (int32_t t : ps.members) init.push_back(&c.net.legs[t]);
    ps.tree = greedy_tree(init, c.net.edim, ovf);
}

// EvaluateState (Section 4.4): Greedy trees are kept per partition; the fan-in tree and con_dist
// follow from the partition results.  The fan-in sampling seed is a hash of the partition roots,
// so the cost is a function of the state alone.
void state_fanin(const Ctx &c, const State &s, FaninInput &in) {
    std::vector<Legs> roots(c.k);
    std::vector<u128> pc(c.k);
    uint64_t h = 0x1234567ull;
    for (int32_t k = 0; k < c.k; ++k) {
        roots[k] = s.parts[k].tree.root_legs;
        pc[k] = s.parts[k].tree.con;
        for (int32_t e : roots[k]) h = mix64(h, (uint64_t)e * 131 + (uint64_t)k);
        h = mix64(h, (uint64_t)pc[k] ^ (uint64_t)(pc[k] >> 64));
    }
    fanin_input(roots, pc, c.net.edim, h, in);
}

void evaluate(const Ctx &c, State &s, bool &ovf) {
    FaninInput in;
    state_fanin(c, s, in);
    s.fan = fanin_host(in, c.samples, -1, ovf);
    s.fan_sample = -1;
    s.cost = s.fan.con_dist;
}

// Evaluate many states' fan-in trees on the context's device in one launch (k > 4).
tn_status evaluate_batch(const Ctx &c, std::vector<State *> &states, std::vector<char> *sat = nullptr) {
    std::vector<FaninInput> ins(states.size());
    for (size_t q = 0; q < states.size(); ++q) state_fanin(c, *states[q], ins[q]);
    std::vector<FaninBest> best;
    tn_status st = fanin_eval_device(c.device, ins, c.samples, best, *c.ws);
    if (st != TN_OK) return st;
    for (size_t q = 0; q < states.size(); ++q) {
        State &s = *states[q];
        s.fan = FanIn();
        s.fan.con_dist = best[q].counts.con_dist;
        s.fan.con = best[q].counts.con;
        s.fan.mem = best[q].counts.mem;
        s.fan_sample = best[q].sample;
        s.cost = s.fan.con_dist;
        if (sat) (*sat)[q] = best[q].counts.sat ? 1 : 0;
    }
    return TN_OK;
}

// The merge steps of a state evaluated on a device (the winning sample, replayed on the host).
void fill_fanin_steps(const Ctx &c, State &s, bool &ovf) {
    if (s.fan_sample < 0 || c.k <= 1) return;
    FaninInput in;
    state_fanin(c, s, in);
    s.fan = fanin_host(in, c.samples, s.fan_sample, ovf);
    s.fan_sample = -1;
}

// Rebalance (Algorithm 2): pick a source partition with at least two tensors, a node v of its tree
// other than the root (so the source never empties), the tensors under v, and a target partition
// (uniform for NAIVE; for DIRECTED the argmax of Eq. 4.5 between legs(v) and the target's root,
// ties to the lowest index); move the tensors and rebuild both Greedy trees and the fan-in tree.
bool propose(const Ctx &c, const State &cur, State &nxt, int32_t mode, Rng &rng, bool &ovf) {
    std::vector<int32_t> cand;
    for (int32_t k = 0; k < c.k; ++k)
        if (cur.parts[k].members.size() >= 2) cand.push_back(k);
    if (cand.empty()) return false;
    const int32_t src = cand[rng.below((uint32_t)cand.size())];
    const PartState &ps = cur.parts[src];
    const int32_t s = (int32_t)ps.members.size();
    const int32_t v = (int32_t)rng.below((uint32_t)(2 * s - 2));   // any node but the root
    // leaves under v
    std::vector<std::pair<int32_t, int32_t>> ch(2 * s - 1, {-1, -1});
    for (size_t t = 0; t < ps.tree.steps.size(); ++t) ch[s + t] = ps.tree.steps[t];
    std::vector<int32_t> moved, stack{v};
    while (!stack.empty()) {
        int32_t x = stack.back();
        stack.pop_back();
        if (x < s) moved.push_back(ps.members[x]);
        else { stack.push_back(ch[x].first); stack.push_back(ch[x].second); }
    }
    int32_t dst;
    if (mode == TN_SA_NAIVE) {
        dst = (int32_t)rng.below((uint32_t)(c.k - 1));
        if (dst >= src) ++dst;
    } else {
        // legs(v) = edges with exactly one end among the moved tensors (Eq. 2.6 applied up the
        // subtree), open legs included.
        Legs lv;
        {
            std::vector<int32_t> all;
            for (int32_t t : moved) all.insert(all.end(), c.net.legs[t].begin(), c.net.legs[t].end());
            std::sort(all.begin(), all.end());
            for (size_t i = 0; i < all.size();) {
                size_t j = i;
                while (j < all.size() && all[j] == all[i]) ++j;
                if ((j - i) % 2 == 1) lv.push_back(all[i]);
                i = j;
            }
        }
        u128 sv = legs_size(lv, c.net.edim, ovf);
        dst = -1;
        i128 best = 0;
        for (int32_t k = 0; k < c.k; ++k) {
            if (k == src) continue;
            const Legs &rl = cur.parts[k].tree.root_legs;
            Legs r;
            legs_symdiff(lv, rl, r);
            i128 obj = (i128)sv + (i128)cur.parts[k].tree.root_size - (i128)legs_size(r, c.net.edim, ovf);
            if (dst < 0 || obj > best) { best = obj; dst = k; }
        }
    }
    nxt = cur;
    std::sort(moved.begin(), moved.end());
    for (int32_t t : moved) nxt.part[t] = dst;
    auto &sm = nxt.parts[src].members;
    std::vector<int32_t> keep;
    std::set_difference(sm.begin(), sm.end(), moved.begin(), moved.end(), std::back_inserter(keep));
    sm.swap(keep);
    auto &dm = nxt.parts[dst].members;
    std::vector<int32_t> merged;
    std::merge(dm.begin(), dm.end(), moved.begin(), moved.end(), std::back_inserter(merged));
    dm.swap(merged);
    rebuild_part(c, nxt.parts[src], ovf);
    rebuild_part(c, nxt.parts[dst], ovf);
    return true;
}

// A move and the evaluation of the state it leads to.
bool rebalance(const Ctx &c, const State &cur, State &nxt, int32_t mode, Rng &rng, bool &ovf) {
    if (!propose(c, cur, nxt, mode, rng, ovf)) return false;
    evaluate(c, nxt, ovf);
    return true;
}

// Natural log of c_new / c_old on exact integer costs; a zero old cost makes any positive new
// cost infinitely worse.
double log_ratio(u128 cn, u128 cc) {
    if (cc == 0) return cn == 0 ? 0.0 : INFINITY;
    return std::log((double)cn) - std::log((double)cc);
}

// Metropolis rule of Eq. 4.2 on log-costs: a cheaper state is always taken (the probability
// exceeds one); a dearer one with probability exp(-log(c_new / c_old) / T).
bool metropolis_accept(u128 c_new, u128 c_old, double T, Rng &rng) {
    return std::exp(-log_ratio(c_new, c_old) / T) >= rng.uniform();
}

// Geometric cooling of Eq. 4.3-4.4: T(x) = T0 (Tf / T0)^x for search progress x in [0, 1].
struct Cooling {
    double T0, ratio;
    Cooling(double t0, double tf) : T0(t0), ratio(tf / t0) {}
    double at(double x) const { return T0 * std::pow(ratio, x); }
};

// How far the search has come: wall-clock time against a limit, or rounds against a fixed count
// (the deterministic mode).
struct SearchBudget {
    bool timed;
    double limit_s;
    int64_t rounds;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double seconds() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    // Progress x of round r, or a negative number when the budget is spent.
    double progress(int64_t r) const {
        if (timed) {
            const double e = seconds();
            return e >= limit_s ? -1.0 : e / limit_s;
        }
        return r >= rounds ? -1.0 : (double)r / (double)rounds;
    }
};

// One Markov chain: `moves` rebalancing moves from `start` at fixed temperature T.
struct Chain {
    State s;
    int32_t accepted = 0;
    bool ovf = false;
};
void run_chain(const Ctx &c, const State &start, int32_t moves, double T, int32_t mode, uint64_t seed,
               Chain &out) {
    Rng rng(seed);
    out.s = start;
    State cand;
    for (int32_t m = 0; m < moves; ++m) {
        if (!rebalance(c, out.s, cand, mode, rng, out.ovf)) break;
        if (metropolis_accept(cand.cost, out.s.cost, T, rng)) {
            out.s = std::move(cand);
            out.accepted++;
        }
    }
}

// One round of the division scheme (Algorithm 1, Section 4.3): p chains start from the same
// state, each runs ceil(N / p) moves with a seed drawn from (seed, round, chain), and the cheapest
// end state is kept (lowest chain index on ties, so the result does not depend on scheduling).
// The same round with the fan-in trees evaluated on a device: the chains advance in lockstep, every
// chain proposing its next move, then one batched launch evaluates all proposals, then every
// chain applies the Metropolis rule.  Each chain draws the same random numbers in the same order
// as in anneal_round and the device evaluation equals the host's, so the result is the same.
tn_status anneal_round_device(const Ctx &c, const State &from, int32_t chains, int32_t moves, double T,
                              int32_t mode, uint64_t seed, int64_t round, int32_t &accepted, State &out) {
    std::vector<Chain> res(chains);
    std::vector<Rng> rngs;
    std::vector<char> live(chains, 1);
    for (int32_t q = 0; q < chains; ++q) {
        res[q].s = from;
        rngs.emplace_back(mix64(mix64(seed, (uint64_t)round), (uint64_t)q + 1));
    }
    std::vector<State> cand(chains);
    for (int32_t m = 0; m < moves; ++m) {
        std::vector<State *> batch;
        std::vector<int32_t> who;
        for (int32_t q = 0; q < chains; ++q) {
            if (!live[q]) continue;
            if (!propose(c, res[q].s, cand[q], mode, rngs[q], res[q].ovf)) {
                live[q] = 0;
                continue;
            }
            batch.push_back(&cand[q]);
            who.push_back(q);
        }
        if (batch.empty()) break;
        tn_status st = evaluate_batch(c, batch);
        if (st != TN_OK) return st;
        for (int32_t q : who)
            if (metropolis_accept(cand[q].cost, res[q].s.cost, T, rngs[q])) {
                res[q].s = std::move(cand[q]);
                res[q].accepted++;
            }
    }
    int32_t win = 0;
    for (int32_t q = 0; q < chains; ++q) {
        accepted += res[q].accepted;
        if (res[q].s.cost < res[win].s.cost) win = q;
    }
    out = std::move(res[win].s);
    return TN_OK;
}

State anneal_round(const Ctx &c, const State &from, int32_t chains, int32_t moves, double T, int32_t mode,
                   uint64_t seed, int64_t round, int32_t &accepted) {
    std::vector<Chain> res(chains);
    auto go = [&](int32_t q) {
        run_chain(c, from, moves, T, mode, mix64(mix64(seed, (uint64_t)round), (uint64_t)q + 1), res[q]);
    };
    if (chains == 1) {
        go(0);
    } else {
        std::vector<std::thread> ts;
        for (int32_t q = 0; q < chains; ++q) ts.emplace_back(go, q);
        for (auto &t : ts) t.join();
    }
    int32_t win = 0;
    for (int32_t q = 0; q < chains; ++q) {
        accepted += res[q].accepted;
        if (res[q].s.cost < res[win].s.cost) win = q;
    }
    return std::move(res[win].s);
}

// Restart policy (Algorithm 1): remember the cheapest state seen; when `patience` rounds pass
// without a strictly cheaper state, continue from the remembered one.
struct BestTracker {
    State best;
    int64_t last_gain = -1;
    int32_t restarts = 0;
    void observe(State &cur, int64_t round, int32_t patience) {
        if (cur.cost < best.cost) {
            best = cur;
            last_gain = round;
        } else if (round - last_gain >= patience) {
            cur = best;
            last_gain = round;
            ++restarts;
        }
    }
};
}  // namespace

tn_status eval_states(const Net &net, int32_t k, int32_t samples, int32_t device, int32_t n_states,
                      const int32_t *parts, std::vector<StateCounts> &out) {
    if (k < 1 || k > net.n) return fail(TN_EINVAL, "k must satisfy 1 <= k <= n_tensors");
    if (n_states < 0 || (n_states > 0 && !parts)) return fail(TN_EINVAL, "NULL parts");
    Ctx c{net, k, samples};
    FaninWorkspace ws;
    struct WsGuard {
        FaninWorkspace &w;
        ~WsGuard() { fanin_workspace_free(w); }
    } ws_guard{ws};
    if (device >= 0 && k > 4) {
        c.device = device;
        c.ws = &ws;
    }
    std::vector<State> st(n_states);
    std::vector<char> ovfs(n_states, 0);
    // partition trees on the host, in parallel over states
    auto build = [&](int32_t lo, int32_t hi, bool *bad) {
        for (int32_t q = lo; q < hi; ++q) {
            State &s = st[q];
            s.part.assign(parts + (size_t)q * net.n, parts + (size_t)(q + 1) * net.n);
            s.parts.assign(k, PartState());
            for (int32_t t = 0; t < net.n; ++t) {
                if (s.part[t] < 0 || s.part[t] >= k) { *bad = true; return; }
                s.parts[s.part[t]].members.push_back(t);
            }
            for (int32_t p = 0; p < k; ++p) {
                if (s.parts[p].members.empty()) { *bad = true; return; }
                bool ov = false;
                rebuild_part(c, s.parts[p], ov);
                if (ov) ovfs[q] = 1;
            }
        }
    };
    const int32_t nt = std::max<int32_t>(1, std::min<int32_t>((int32_t)std::thread::hardware_concurrency(), 16));
    std::vector<std::thread> ts;
    std::vector<char> bad(nt, 0);
    for (int32_t w = 0; w < nt; ++w) {
        const int32_t lo = (int32_t)((int64_t)n_states * w / nt), hi = (int32_t)((int64_t)n_states * (w + 1) / nt);
        ts.emplace_back([&, lo, hi, w] {
            bool b = false;
            build(lo, hi, &b);
            bad[w] = b;
        });
    }
    for (auto &t : ts) t.join();
    for (char b : bad)
        if (b) return fail(TN_EINVAL, "a state has a partition index outside [0, k) or an empty partition");
    if (c.device >= 0) {
        std::vector<State *> ptr;
        for (State &s : st) ptr.push_back(&s);
        std::vector<char> fsat(n_states, 0);
        tn_status r = evaluate_batch(c, ptr, &fsat);
        if (r != TN_OK) return r;
        for (int32_t q = 0; q < n_states; ++q) ovfs[q] = ovfs[q] || fsat[q];
    } else {
        std::vector<std::thread> ev;
        for (int32_t w = 0; w < nt; ++w) {
            const int32_t lo = (int32_t)((int64_t)n_states * w / nt), hi = (int32_t)((int64_t)n_states * (w + 1) / nt);
            ev.emplace_back([&, lo, hi] {
                for (int32_t q = lo; q < hi; ++q) {
                    bool ov = false;
                    evaluate(c, st[q], ov);
                    if (ov) ovfs[q] = 1;
                }
            });
        }
        for (auto &t : ev) t.join();
    }
    out.assign(n_states, StateCounts());
    for (int32_t q = 0; q < n_states; ++q) {
        StateCounts &r = out[q];
        u128 con = st[q].fan.con, mem = st[q].fan.mem;
        for (const PartState &ps : st[q].parts) {
            con += ps.tree.con;
            mem = std::max(mem, ps.tree.mem);
        }
        r.con_serial = con;
        r.con_dist = st[q].cost;
        r.mem = mem;
        r.saturated = ovfs[q] || con >= kSizeCap || st[q].cost >= kSizeCap || mem >= kSizeCap;
    }
    return TN_OK;
}

tn_status plan_run(const Net &net, const tn_plan_opts &o, Plan &out) {
    auto t_start = std::chrono::steady_clock::now();
    const int32_t n = net.n;
    if (o.k < 1 || o.k > n) return fail(TN_EINVAL, "k must satisfy 1 <= k <= n_tensors");
    if (o.threads < 1 || o.steps_per_temp < 1 || o.restart_threshold < 1)
        return fail(TN_EINVAL, "threads, steps_per_temp and restart_threshold must be >= 1");
    if (!(o.T0 > 0) || !(o.Tf > 0)) return fail(TN_EINVAL, "temperatures must be positive");
    if (o.time_limit_s <= 0 && o.iterations < 0) return fail(TN_EINVAL, "iterations must be >= 0");
    if (o.mode != TN_SA_NAIVE && o.mode != TN_SA_DIRECTED) return fail(TN_EINVAL, "unknown SA mode");
    Ctx c{net, o.k, o.fanin_samples};
    bool ovf = false;
    FaninWorkspace ws;
    struct WsGuard {
        FaninWorkspace &w;
        ~WsGuard() { fanin_workspace_free(w); }
    } ws_guard{ws};
    if (o.fanin_device >= 0 && o.k > 4) {
        c.device = o.fanin_device;
        c.ws = &ws;
    }

    // initial partitioning
    State init;
    init.part.assign(n, 0);
    if (o.k > 1) {
        if (o.initial == TN_INIT_GIVEN) {
            if (!o.initial_part) return fail(TN_EINVAL, "TN_INIT_GIVEN needs initial_part");
            for (int32_t t = 0; t < n; ++t) {
                if (o.initial_part[t] < 0 || o.initial_part[t] >= o.k)
                    return fail(TN_EINVAL, "initial_part entry out of range");
                init.part[t] = o.initial_part[t];
            }
        } else if (o.initial == TN_INIT_QUBIT_BLOCK) {
            if (!o.position) return fail(TN_EINVAL, "TN_INIT_QUBIT_BLOCK needs a position hint");
            int64_t span = 0;
            for (int32_t t = 0; t < n; ++t) {
                if (o.position[t] < 0) return fail(TN_EINVAL, "negative position hint");
                span = std::max(span, (int64_t)o.position[t] + 1);
            }
            for (int32_t t = 0; t < n; ++t) init.part[t] = (int32_t)((int64_t)o.position[t] * o.k / span);
        } else if (o.initial == TN_INIT_BFS) {
            // balanced breadth-first split: BFS order from tensor 0 (restarting in unvisited
            // components), cut into k contiguous chunks of near-equal size
            std::vector<std::vector<int32_t>> nb(n);
            for (const tn_edge &e : net.edges)
                if (e.v >= 0) { nb[e.u].push_back(e.v); nb[e.v].push_back(e.u); }
            std::vector<int32_t> order, seen(n, 0);
            for (int32_t r = 0; r < n; ++r) {
                if (seen[r]) continue;
                seen[r] = 1;
                size_t head = order.size();
                order.push_back(r);
                while (head < order.size()) {
                    int32_t x = order[head++];
                    for (int32_t y : nb[x]) if (!seen[y]) { seen[y] = 1; order.push_back(y); }
                }
            }
            for (int32_t i = 0; i < n; ++i) init.part[order[i]] = (int32_t)((int64_t)i * o.k / n);
        } else {
            return fail(TN_EINVAL, "unknown initial partition mode");
        }
    }
    init.parts.resize(o.k);
    for (int32_t t = 0; t < n; ++t) init.parts[init.part[t]].members.push_back(t);
    for (int32_t k = 0; k < o.k; ++k)
        if (init.parts[k].members.empty()) return fail(TN_EINVAL, "initial partition has an empty part");
    // Sizes and costs saturate at 2^120 during the search: a saturated state is merely very
    // expensive, so the annealing can still move away from it.  Only the final plan must fit.
    for (int32_t k = 0; k < o.k; ++k) rebuild_part(c, init.parts[k], ovf);
    if (c.device >= 0) {
        std::vector<State *> one{&init};
        tn_status st = evaluate_batch(c, one);
        if (st != TN_OK) return st;
    } else {
        evaluate(c, init, ovf);
    }

    // Simulated annealing (Section 4.3, Algorithm 1): rounds of parallel chains at a falling
    // temperature, with restarts from the best state.
    BestTracker track;
    track.best = init;
    int32_t accepted = 0, iters = 0;
    if (o.k > 1) {
        const Cooling cool(o.T0, o.Tf);
        const SearchBudget budget{o.time_limit_s > 0, o.time_limit_s, (int64_t)o.iterations};
        const int32_t moves = (o.steps_per_temp + o.threads - 1) / o.threads;
        State cur = init;
        for (int64_t round = 0;; ++round) {
            const double x = budget.progress(round);
            if (x < 0) break;
            if (c.device >= 0) {
                State nxt;
                tn_status st = anneal_round_device(c, cur, o.threads, moves, cool.at(x), o.mode, o.seed, round,
                                                   accepted, nxt);
                if (st != TN_OK) return st;
                cur = std::move(nxt);
            } else {
                cur = anneal_round(c, cur, o.threads, moves, cool.at(x), o.mode, o.seed, round, accepted);
            }
            ++iters;
            track.observe(cur, round, o.restart_threshold);
        }
    }
    State &best = track.best;
    fill_fanin_steps(c, best, ovf);
    const int32_t restarts = track.restarts;
    // assemble the plan from the best state
    out = Plan();
    out.n = n;
    out.k = o.k;
    out.part = best.part;
    std::vector<int32_t> root_id(o.k);
    for (int32_t k = 0; k < o.k; ++k) {
        const PartState &ps = best.parts[k];
        std::vector<int32_t> gid(ps.members.begin(), ps.members.end());
        for (auto &st : ps.tree.steps) {
            int32_t a = gid[st.first], b = gid[st.second];
            int32_t oid = n + (int32_t)out.steps.size();
            out.steps.push_back({std::min(a, b), std::max(a, b), oid});
            gid.push_back(oid);
        }
        root_id[k] = gid.back();
    }
    {
        std::vector<int32_t> gid(root_id);
        for (auto &st : best.fan.steps) {
            int32_t a = gid[st.first], b = gid[st.second];
            int32_t oid = n + (int32_t)out.steps.size();
            out.steps.push_back({std::min(a, b), std::max(a, b), oid});
            gid.push_back(oid);
        }
    }
    tn_status s = plan_finalize(net, out);
    if (s != TN_OK) return s;
    out.init_con_dist = init.cost;
    out.sa_iterations = iters;
    out.sa_accepted = accepted;
    out.sa_restarts = restarts;
    out.plan_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    return TN_OK;
}

}  // namespace tn
