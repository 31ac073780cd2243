// Program compiler and runtime.
//
// compile(): turns (network structure, plan, precision) into a device step list -- per-step
// layouts and fused index maps, kernel class, work tiles, dependencies, a static memory plan for
// every intermediate (offsets into one arena).  Nets with the same structure that use the same
// plan share one compiled list and differ only in their leaves.
//
// A batch is a set of jobs (independent contractions).  It is executed either by the subtree-
// program kernels plus the persistent dataflow kernel -- one launch of each for all jobs, and for
// every dependency phase of dense tensor-core steps a pack launch, a grouped GEMM launch and one
// more dataflow launch (the default) -- or, as a reference mode, by one launch per step and job
// recorded into a CUDA graph.  A program is a batch of one job.
#include <algorithm>
#include <array>
#include <atomic>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "local_ops.cuh"
#include "tn_internal.hpp"

using namespace tn;

#include "compile.cuh"

struct tn_ctx {
    int32_t device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    int32_t mode = 0;                 // tn_exec_mode
    tn_exec_config cfg{-1, 0, 1, 64, 32, 16, 1, 4000000, 1, 1, 0};   // programs, TC, waits, graphs, order, TC tile
    tn_batch *cached = nullptr;       // batch of one reused by tn_contract, keyed by the unique
    uint64_t cached_net = 0, cached_plan = 0;   // ids of the net and plan (never by address)
    tn_precision cached_prec = TN_C64;
    // Batches, programs and servers made from the context hold a reference; tn_ctx_free only marks
    // the context, which is deleted when its last dependent is freed (garbage collectors may free
    // a context before the batches that use it).
    std::atomic<int32_t> refs{0};
    bool freed = false;
};

namespace tn {
void ctx_retain(tn_ctx *c) { c->refs.fetch_add(1); }
void ctx_destroy_now(tn_ctx *c) {
    cudaSetDevice(c->device);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}
void ctx_release(tn_ctx *c) {
    if (c && c->refs.fetch_sub(1) == 1 && c->freed) ctx_destroy_now(c);
}
}  // namespace tn

struct tn_batch {
    tn_ctx *ctx = nullptr;
    tn_precision prec = TN_C64;
    bool c128 = false;
    int32_t elem = 8;
    int32_t mode = 0;
    int32_t n_jobs = 0;
    std::vector<const tn_net *> nets;
    std::vector<uint64_t> uploaded;
    std::vector<Compiled> comp;
    std::vector<int32_t> job_comp;
    std::vector<JobPtrs> jobs;
    std::vector<int64_t> leaf64_off;  // per job, element offset into d_leaf64
    int64_t leaf_elems_total = 0;
    int32_t max_leaves = 0;
    int64_t max_leaf_elems = 0;      // the largest leaf of any job
    // device memory: one allocation, carved
    void *d_block = nullptr;
    double2 *d_leaf64 = nullptr;
    JobPtrs *d_jobs = nullptr;
    WorkItem *d_work = nullptr;
    int64_t n_work = 0;
    // dependency phases (step_phases): per phase the range of its dataflow items in d_work and of
    // its tensor-core pack units and GEMM tiles in d_pack / d_gemm (persistent mode)
    struct Phase {
        int64_t work0 = 0, n_work = 0;
        int32_t pack0 = 0, n_pack = 0, gemm0 = 0, n_gemm = 0;
    };
    std::vector<Phase> phases;
    WorkItem *d_pack = nullptr, *d_gemm = nullptr;
    std::vector<TcRange> tc_ranges;   // every tensor-core step's units and tiles (both modes)
    std::vector<int32_t> h_work_phase;
    std::vector<WorkItem> h_work;     // the full work list (tn_batch_debug_hold uploads subsets)
    std::vector<std::pair<int32_t, int32_t>> held;   // (job, step) left out by tn_batch_debug_hold
    long long wait_ns = 4000000000LL; // a dependency wait of the persistent kernel gives up after this
    WorkItem *d_local = nullptr;      // (job, pseudo-step) of every subtree program
    int32_t n_warp_items = 0;         // warp programs (first in d_local), then block programs
    int32_t n_block_items = 0;
    int32_t n_big_items = 0;          // large programs (last in d_local)
    int32_t dyn_big = 0;              // dynamic shared memory of the large-program launch
    uint32_t *d_counter = nullptr;
    DeviceResult *d_res = nullptr;
    char *d_reset = nullptr;          // results, maxbits, done, counter: zeroed before every run
    size_t reset_bytes = 0;
    size_t footprint = 0, arena_total = 0;
    int32_t grid = 0;
    int32_t dyn_smem = 0;             // dynamic shared memory of the subtree-program kernel
    long long *d_prof = nullptr;      // optional per-kind cycle counters (tn_batch_set_profiling)
    // host
    double *h_pinned = nullptr;
    DeviceResult *h_res = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // ring of per-run event lists (persistent mode): one event at the start of the contraction
    // kernels and one after every launch slot -- warp programs, block and large programs, then per
    // phase the pack, GEMM and dataflow launches (a slot whose launch is empty records no time)
    static constexpr int kRing = 256;
    std::vector<cudaEvent_t> kev[kRing];
    // persistent runs replayed from a CUDA graph (tn_exec_config.graph_capture): the graph holds
    // the reset, the leaf conversion and every launch of a run, with its own per-slot events
    // (gev, the last replay's); the ring then holds only a start and an end event per run
    cudaGraphExec_t pgexec = nullptr;
    std::vector<cudaEvent_t> gev;
    bool replay = false;
    int64_t runs = 0;
    // pending tensor updates (tn_batch_set_tensors): headers {dst element offset, count, src
    // element offset} and complex128 values, staged in pinned memory, applied on the device
    // staged tensor updates, written by tn_batch_set_tensors straight into pinned host memory: two
    // staging sets used in turn, so a set is refilled only once the copy of the run before last
    // out of it has completed (its event), and the filling overlaps the run in flight
    struct Pinned {
        char *p = nullptr;
        size_t size = 0, cap = 0;
    };
    struct Stage {
        Pinned hdr, val;              // {dst offset, count, src offset} per update; the values
        cudaEvent_t ev = nullptr;     // recorded after the copies out of this set
        bool copying = false;
    };
    Stage stage[2];
    int32_t cur_stage = 0;
    char *d_upd = nullptr;
    size_t d_upd_cap = 0;
    size_t last_h2d = 0;
    tn_run_info info{};
    bool ran = false;
};

struct tn_program {
    tn_batch *b = nullptr;
};

namespace {

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess)                                                             \
            return fail(TN_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));     \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

int32_t ilog2(int64_t x) {
    int32_t r = 0;
    while ((((int64_t)1) << r) < x) ++r;
    return r;
}

uint64_t shape_hash(const Net &net) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix((uint64_t)net.n);
    for (int32_t d : net.degree) mix((uint64_t)d);
    for (int64_t d : net.dims) mix((uint64_t)d);
    for (const tn_edge &e : net.edges) {
        mix((uint64_t)(uint32_t)e.u); mix((uint64_t)(uint32_t)e.a);
        mix((uint64_t)(uint32_t)e.v); mix((uint64_t)(uint32_t)e.b);
    }
    return h;
}

// Build a fused group list from legs listed outermost -> innermost with their strides.
bool make_groups(const std::vector<int64_t> &dim, const std::vector<int64_t> &sa,
                 const std::vector<int64_t> &sb, bool two, Groups &g) {
    std::memset(&g, 0, sizeof(g));
    int32_t n = 0;
    for (int32_t i = (int32_t)dim.size() - 1; i >= 0; --i) {   // innermost first
        if (dim[i] == 1) continue;
        if (n > 0 && sa[i] == g.sa[n - 1] * g.dim[n - 1] &&
            (!two || sb[i] == g.sb[n - 1] * g.dim[n - 1])) {
            g.dim[n - 1] *= dim[i];
            continue;
        }
        if (n == kMaxGroups) return false;
        g.dim[n] = dim[i];
        g.sa[n] = sa[i];
        g.sb[n] = two ? sb[i] : 0;
        ++n;
    }
    g.n = n;
    g.pow2 = 1;
    int32_t bit = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (!is_pow2(g.dim[i])) g.pow2 = 0;
        g.lsb[i] = bit;
        g.mask[i] = g.dim[i] - 1;
        bit += ilog2(g.dim[i]);
    }
    return true;
}

// Free blocks of the arena (offset -> size), coalescing neighbours.
struct Pool {
    std::map<size_t, size_t> blocks;
    void release(size_t off, size_t sz) {
        auto it = blocks.emplace(off, sz).first;
        auto nx = std::next(it);
        if (nx != blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            blocks.erase(nx);
        }
        if (it != blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                blocks.erase(it);
            }
        }
    }
    bool take(size_t sz, size_t &off) {   // best fit
        auto best = blocks.end();
        for (auto it = blocks.begin(); it != blocks.end(); ++it)
            if (it->second >= sz && (best == blocks.end() || it->second < best->second)) best = it;
        if (best == blocks.end()) return false;
        off = best->first;
        const size_t rest = best->second - sz;
        blocks.erase(best);
        if (rest) blocks[off + sz] = rest;
        return true;
    }
    void absorb(Pool &o) {
        if (o.blocks.size() > blocks.size()) std::swap(blocks, o.blocks);
        for (auto &b : o.blocks) release(b.first, b.second);
        o.blocks.clear();
    }
};

// Static memory plan that is valid for ANY execution order consistent with the tree's
// dependencies: a buffer freed inside a subtree (its last reader is in that subtree) may be
// reused only by that subtree's ancestors, which run after every step of the subtree; sibling
// subtrees may run concurrently and so draw fresh memory from the top of the arena.  A step's
// output never overlaps its own operands.  Returns the arena size.
size_t plan_memory(const Plan &plan, int32_t n, const std::vector<size_t> &bytes,
                   std::vector<size_t> &off) {
    const int32_t nn = 2 * n - 1;
    std::vector<Pool> pool(nn);
    size_t top = 0;
    off.assign(nn, 0);
    for (int32_t s = 0; s < n - 1; ++s) {
        const int32_t l = plan.steps[s][0], r = plan.steps[s][1], o = n + s;
        Pool p;
        p.absorb(pool[l]);
        p.absorb(pool[r]);
        if (s != n - 2 && bytes[o] > 0) {   // the root's value goes to the result record
            size_t at;
            if (!p.take(bytes[o], at)) {
                at = top;
                top += bytes[o];
            }
            off[o] = at;
        }
        for (int32_t x : {l, r})
            if (x >= n && bytes[x] > 0) p.release(off[x], bytes[x]);
        pool[o].blocks.swap(p.blocks);
    }
    return top;
}

// Rows per work tile of a global ROWS step: large enough to amortise the tile's fixed cost
// (descriptor, scales, B staging, completion fence), 16 rows per thread at most.
int32_t rows_per_tile(int64_t M) {
    if (M <= 4096) return (int32_t)std::max<int64_t>(M, 1);
    return 4096;
}

// Geometry of one pairwise step: which child plays A (the larger), the free / shared legs with
// their strides (outermost first), and M, N, K.
struct Geom {
    int32_t a = -1, b = -1;
    int64_t M = 1, N = 1, K = 1;
    std::vector<int64_t> md, ms, nd, ns, kd, ksa, ksb;
};

// Local (shared-memory) form of a leg-group list; false if it needs more than kLG groups.
bool make_lgroups(const std::vector<int64_t> &dim, const std::vector<int64_t> &sa,
                  const std::vector<int64_t> &sb, bool two, int32_t *o_dim, int32_t *o_sa, int32_t *o_sb,
                  uint8_t *o_lsb, uint8_t &count, bool &pow2) {
    Groups g;
    if (!make_groups(dim, sa, sb, two, g) || g.n > kLG) return false;
    count = (uint8_t)g.n;
    for (int32_t i = 0; i < g.n; ++i) {
        if (g.dim[i] > (1 << 30) || g.sa[i] > (1 << 30) || g.sb[i] > (1 << 30)) return false;
        o_dim[i] = (int32_t)g.dim[i];
        o_sa[i] = (int32_t)g.sa[i];
        if (o_sb) o_sb[i] = (int32_t)g.sb[i];
        o_lsb[i] = (uint8_t)g.lsb[i];
    }
    if (!g.pow2) pow2 = false;
    return true;
}

// Tabulate the index maps of a small step with at most kTabOut outputs and kTabK shared indices
// (LFLAG_TAB): the warp then reads each offset instead of decoding the index over the leg groups.
// The decode is the one the kernels perform (digits by shift and mask, or by division).
void tabulate_small(LocalStep &ls) {
    if (!(ls.flags & LFLAG_SMALL) || (int64_t)ls.M * ls.N > kTabOut || ls.K > kTabK) return;
    auto dec = [&](int32_t n, const int32_t *dim, const int32_t *str, const uint8_t *lsb, int32_t idx) {
        int64_t off = 0;
        for (int32_t i = 0; i < n; ++i) {
            int64_t d;
            if (ls.pow2) {
                d = (idx >> lsb[i]) & (dim[i] - 1);
            } else {
                d = idx % dim[i];
                idx /= dim[i];
            }
            off += d * str[i];
        }
        return off;
    };
    uint32_t t[kTabOut + kTabK] = {};
    for (int32_t o = 0; o < ls.M * ls.N; ++o) {
        const int64_t a = dec(ls.nm, ls.m_dim, ls.m_str, ls.m_lsb, o / ls.N);
        const int64_t b = dec(ls.nn, ls.n_dim, ls.n_str, ls.n_lsb, o % ls.N);
        if (a > 0xffff || b > 0xffff) return;
        t[o] = (uint32_t)a | ((uint32_t)b << 16);
    }
    for (int32_t k = 0; k < ls.K; ++k) {
        const int64_t a = dec(ls.nk, ls.k_dim, ls.k_sa, ls.k_lsb, k);
        const int64_t b = dec(ls.nk, ls.k_dim, ls.k_sb, ls.k_lsb, k);
        if (a > 0xffff || b > 0xffff) return;
        t[kTabOut + k] = (uint32_t)a | ((uint32_t)b << 16);
    }
    std::memcpy(reinterpret_cast<char *>(&ls) + offsetof(LocalStep, m_dim), t, sizeof(t));
    ls.flags |= LFLAG_TAB;
}

struct LocalPlan {
    std::vector<int32_t> nodes;      // internal nodes in execution order (wave by wave)
    std::vector<char> small;         // per entry of `nodes`: one warp runs it
    std::vector<LocalWave> waves;
    std::vector<int32_t> leaves;     // leaves, increasing
    std::vector<int64_t> loc;        // per node of the subtree: shared-memory element offset
    std::unordered_map<int32_t, int32_t> idx;   // node -> position in loc / slot
    std::vector<std::vector<int32_t>> wave_inputs;  // lazy programs: inputs staged before each wave
    int64_t leaf_elems = 0, arena_elems = 0;
    int32_t smem_bytes = 0;
};

// A step one warp runs on its own (no block barrier): few outputs and a short shared index.
bool small_step(const Geom &g, bool job_root) {
    return !job_root && g.M * g.N <= 256 && g.K <= 256 && g.M * g.N * g.K <= 4096;
}

// Can the subtree rooted at v run in one block within `budget` bytes of dynamic shared memory?
// Steps are grouped into waves of mutually independent steps (wave = 1 + the latest wave among
// the step's children inside the subtree); a wave runs its small steps one per warp and its big
// steps with the whole block.  The memory plan is simulated in that order: all outputs of a wave
// are placed (best fit) before the inputs it consumed are released.
// lazy: each input is staged into the pool right before the wave that consumes it and released
// after it (large programs), instead of all inputs up front below the pool.
bool local_fit(int32_t v, int32_t n, const Plan &plan, const std::vector<Geom> &geo,
               const std::vector<int64_t> &size, int32_t elem, int32_t budget,
               const std::vector<int32_t> &input_prog, bool lazy, LocalPlan &lp) {
    lp = LocalPlan();
    std::vector<int32_t> nodes, stack{v};
    while (!stack.empty()) {
        int32_t x = stack.back();
        stack.pop_back();
        // inputs: network leaves and the results of earlier programs (already in device memory)
        if (x < n || (x != v && input_prog[x] >= 0)) { lp.leaves.push_back(x); continue; }
        nodes.push_back(x);
        stack.push_back(plan.steps[x - n][0]);
        stack.push_back(plan.steps[x - n][1]);
    }
    std::unordered_set<int32_t> inner(nodes.begin(), nodes.end());
    std::sort(nodes.begin(), nodes.end());
    std::sort(lp.leaves.begin(), lp.leaves.end());
    const int64_t slots = (int64_t)nodes.size() + (int64_t)lp.leaves.size();
    if (slots > 32000) return false;
    // element offsets inside one operand are packed in 16 bits by the small-step path
    for (int32_t x : nodes)
        if (size[x] > 0xffff) return false;
    for (int32_t t : lp.leaves)
        if (size[t] > 0xffff) return false;
    // waves and execution order
    std::unordered_map<int32_t, int32_t> wave;
    int32_t n_waves = 0;
    for (int32_t x : nodes) {
        int32_t w = 0;
        for (int32_t c : {plan.steps[x - n][0], plan.steps[x - n][1]})
            if (inner.count(c)) w = std::max(w, wave[c]);
        wave[x] = w + 1;
        n_waves = std::max(n_waves, w + 1);
    }
    const int32_t root_id = 2 * n - 2;
    std::vector<std::vector<int32_t>> by_wave(n_waves + 1);
    for (int32_t x : nodes) by_wave[wave[x]].push_back(x);
    for (int32_t w = 1; w <= n_waves; ++w) {
        LocalWave W{(int32_t)lp.nodes.size(), 0, 0, 0, 0, {0, 0, 0}};
        for (int pass = 0; pass < 2; ++pass)
            for (int32_t x : by_wave[w]) {
                const bool sm = small_step(geo[x - n], x == root_id);
                if (sm != (pass == 0)) continue;
                lp.nodes.push_back(x);
                lp.small.push_back(sm ? 1 : 0);
                if (sm) W.n_small++; else W.n_big++;
            }
        lp.waves.push_back(W);
    }
    const int64_t fixed = (int64_t)local_fixed_bytes((int32_t)lp.nodes.size(), (int32_t)lp.waves.size(), (int32_t)slots);
    int64_t pos = 0;
    for (int32_t t : lp.leaves) {
        lp.idx[t] = (int32_t)lp.loc.size();
        lp.loc.push_back(pos);   // lazy: set when the input is staged
        if (!lazy) pos += size[t];
    }
    lp.leaf_elems = (pos + 1) / 2 * 2;   // keep the arena 16-byte aligned
    if (fixed + lp.leaf_elems * elem > budget) return false;
    Pool pool;
    int64_t top = 0;
    std::unordered_map<int32_t, int64_t> asz;
    // lazy: the inputs of wave w are copied while wave w - 1 runs, so they are placed when wave
    // w - 1's results are, clear of everything wave w - 1 touches (each input has one consumer)
    auto place_inputs = [&](size_t wi) {
        const LocalWave &W = lp.waves[wi];
        const int32_t end = W.first + W.n_small + W.n_big;
        for (int32_t i = W.first; i < end; ++i) {
            const int32_t x = lp.nodes[i];
            for (int32_t c : {plan.steps[x - n][0], plan.steps[x - n][1]}) {
                if (inner.count(c)) continue;
                const int64_t sz = (size[c] + 1) / 2 * 2;
                size_t at;
                if (!pool.take((size_t)sz, at)) {
                    at = (size_t)top;
                    top += sz;
                }
                lp.loc[lp.idx[c]] = (int64_t)at;
                asz[c] = sz;
                lp.wave_inputs[wi].push_back(c);
            }
        }
    };
    if (lazy) {
        lp.wave_inputs.assign(lp.waves.size(), {});
        if (!lp.waves.empty()) place_inputs(0);
    }
    for (size_t wi = 0; wi < lp.waves.size(); ++wi) {
        const LocalWave &W = lp.waves[wi];
        const int32_t end = W.first + W.n_small + W.n_big;
        for (int32_t i = W.first; i < end; ++i) {
            const int32_t x = lp.nodes[i];
            const int64_t sz = (size[x] + 1) / 2 * 2;
            size_t at;
            if (!pool.take((size_t)sz, at)) {
                at = (size_t)top;
                top += sz;
            }
            lp.idx[x] = (int32_t)lp.loc.size();
            lp.loc.push_back(lp.leaf_elems + (int64_t)at);
            asz[x] = sz;
        }
        if (lazy && wi + 1 < lp.waves.size()) place_inputs(wi + 1);
        if (fixed + (lp.leaf_elems + top) * elem > budget) return false;
        for (int32_t i = W.first; i < end; ++i) {
            const int32_t x = lp.nodes[i];
            for (int32_t c : {plan.steps[x - n][0], plan.steps[x - n][1]})
                if (inner.count(c) || lazy) pool.release((size_t)(lp.loc[lp.idx[c]] - lp.leaf_elems), (size_t)asz[c]);
        }
    }
    lp.arena_elems = top;
    lp.smem_bytes = (int32_t)(fixed + (lp.leaf_elems + top) * elem);
    if (lp.leaf_elems + top > (1LL << 30)) return false;
    // every step must fit the compact descriptor
    for (int32_t x : lp.nodes) {
        const Geom &g = geo[x - n];
        LocalStep ls;
        bool p2 = true;
        if (!make_lgroups(g.md, g.ms, g.ms, false, ls.m_dim, ls.m_str, nullptr, ls.m_lsb, ls.nm, p2) ||
            !make_lgroups(g.nd, g.ns, g.ns, false, ls.n_dim, ls.n_str, nullptr, ls.n_lsb, ls.nn, p2) ||
            !make_lgroups(g.kd, g.ksa, g.ksb, true, ls.k_dim, ls.k_sa, ls.k_sb, ls.k_lsb, ls.nk, p2))
            return false;
    }
    return true;
}

// A warp program: a subtree whose steps are all small, run by one warp in plan order with its
// intermediates in a kWarpSlice-byte shared-memory slice; leaves are read from device memory and
// the root's value is written there.
struct WarpPlan {
    std::vector<int32_t> nodes;                 // internal nodes, plan order
    std::vector<int32_t> leaves;                // leaves, increasing
    std::unordered_map<int32_t, int32_t> slot;  // node (leaf or internal) -> scale slot
    std::unordered_map<int32_t, int64_t> loc;   // node (not the root) -> element offset in the slice
    int32_t smem_bytes = 0;
};

bool warp_fit(int32_t v, int32_t n, const Plan &plan, const std::vector<Geom> &geo,
              const std::vector<int64_t> &size, int32_t elem, WarpPlan &wp) {
    wp = WarpPlan();
    const int32_t root_id = 2 * n - 2;
    std::vector<int32_t> stack{v};
    while (!stack.empty()) {
        const int32_t x = stack.back();
        stack.pop_back();
        if (x < n) {
            if (size[x] > 0xffff) return false;
            wp.leaves.push_back(x);
            continue;
        }
        if (!small_step(geo[x - n], x == root_id) || size[x] > 0xffff) return false;
        wp.nodes.push_back(x);
        if (wp.nodes.size() > 4096) return false;
        stack.push_back(plan.steps[x - n][0]);
        stack.push_back(plan.steps[x - n][1]);
    }
    std::sort(wp.nodes.begin(), wp.nodes.end());
    std::sort(wp.leaves.begin(), wp.leaves.end());
    int32_t ns = 0;
    for (int32_t t : wp.leaves) wp.slot[t] = ns++;
    for (int32_t x : wp.nodes) wp.slot[x] = ns++;
    const int64_t fixed = (int64_t)warp_fixed_bytes(ns);
    // leaves at the bottom of the slice (staged once), intermediates above them
    int64_t lpos = 0;
    for (int32_t t : wp.leaves) {
        wp.loc[t] = lpos;
        lpos += (size[t] + 1) / 2 * 2;   // 16-byte granules
    }
    if (fixed + lpos * elem > kWarpSlice) return false;
    Pool pool;
    int64_t top = 0;
    std::unordered_map<int32_t, int64_t> asz;
    for (int32_t x : wp.nodes) {
        if (x != v) {
            const int64_t sz = (size[x] + 1) / 2 * 2;
            size_t at;
            if (!pool.take((size_t)sz, at)) {
                at = (size_t)top;
                top += sz;
            }
            wp.loc[x] = lpos + (int64_t)at;
            asz[x] = sz;
            if (fixed + (lpos + top) * elem > kWarpSlice) return false;
        }
        for (int32_t c : {plan.steps[x - n][0], plan.steps[x - n][1]})
            if (c >= n) pool.release((size_t)(wp.loc[c] - lpos), (size_t)asz[c]);
    }
    wp.smem_bytes = (int32_t)(fixed + (lpos + top) * elem);
    for (int32_t x : wp.nodes) {
        const Geom &g = geo[x - n];
        LocalStep ls;
        bool p2 = true;
        if (!make_lgroups(g.md, g.ms, g.ms, false, ls.m_dim, ls.m_str, nullptr, ls.m_lsb, ls.nm, p2) ||
            !make_lgroups(g.nd, g.ns, g.ns, false, ls.n_dim, ls.n_str, nullptr, ls.n_lsb, ls.nn, p2) ||
            !make_lgroups(g.kd, g.ksa, g.ksb, true, ls.k_dim, ls.k_sa, ls.k_sb, ls.k_lsb, ls.nk, p2))
            return false;
    }
    return true;
}

// Staging records of one program input (a leaf, or a warp program's result): pieces of at most
// kStagePiece elements, so that each thread of the staging loop copies one piece with one burst of
// loads; the first piece carries the input's scale slot and node.
constexpr int32_t kStagePiece = 16;
tn_status push_input(std::vector<LeafRef> &out, int64_t goff, int64_t count, int64_t smem_off, int32_t slot,
                     int32_t node, int32_t src) {
    for (int64_t p = 0; p < std::max<int64_t>(count, 1); p += kStagePiece) {
        LeafRef r;
        r.global_off = goff + p;
        r.pad = 0;
        r.count = (int32_t)std::min<int64_t>(kStagePiece, count - p);
        r.smem_off = (int32_t)(smem_off + p);
        r.slot = p == 0 ? slot : -1;
        r.node = node;
        r.src = src;
        out.push_back(r);
    }
    return TN_OK;
}

}  // namespace

int32_t tn::tc_mode_of(int32_t prec) { return prec == TN_BF16_SPLIT ? 1 : prec == TN_TF32_SPLIT ? 2 : 0; }

tn::CompileOpts tn::compile_opts(const tn_exec_config &cfg, int32_t prec, bool c128) {
    CompileOpts o;
    o.elem = c128 ? 16 : 8;
    o.local_budget = cfg.local_budget >= 0 ? cfg.local_budget : local_smem_budget(c128, 2);
    o.big_budget = (o.local_budget > 0 && cfg.big_programs) ? local_smem_budget(c128, 1) : 0;
    o.warp_programs = cfg.warp_programs != 0;
    o.tc_mode = tc_mode_of(prec);
    o.tc_min_m = cfg.tc_min_m;
    o.tc_min_n = cfg.tc_min_n;
    o.tc_min_k = cfg.tc_min_k;
    o.rows_chains = cfg.rows_chains != 0;
    o.tc_tile_n = cfg.tc_tile_n;
    return o;
}

namespace {
// Options of the device-free compile statistics: the given block budget, and for large programs
// twice that (a device gives one block per SM about twice what two blocks per SM get), at most
// 200 KB.
CompileOpts stats_opts(int32_t prec, int32_t local_budget) {
    CompileOpts o;
    o.elem = prec == TN_C128 ? 16 : 8;
    o.local_budget = local_budget;
    o.big_budget = local_budget > 0 ? std::min(2 * local_budget, 200 * 1024) : 0;
    o.tc_mode = tc_mode_of(prec);
    return o;
}
}  // namespace

tn_status tn::compile(Compiled &c, const Net &net, const Plan &plan, const CompileOpts &opt) {
    const int32_t elem = opt.elem, local_budget = opt.local_budget, big_budget = opt.big_budget,
                  tc_mode = opt.tc_mode;
    const bool use_tc = tc_mode != 0;
    const int32_t n = net.n, nn = 2 * n - 1;
    c.n = n;
    c.n_nodes = nn;
    std::vector<std::vector<int32_t>> layout(nn);
    std::vector<int64_t> size(nn, 1);
    for (int32_t t = 0; t < n; ++t) {
        layout[t] = net.axis_edge[t];
        size[t] = net.data_off[t + 1] - net.data_off[t];
    }
    c.leaf_off.assign(net.data_off.begin(), net.data_off.end());
    const size_t esz = (size_t)elem;
    // pass 1: layouts and geometry of every step
    std::vector<Geom> geo(std::max(n - 1, 0));
    for (int32_t s = 0; s < n - 1; ++s) {
        const int32_t l = plan.steps[s][0], r = plan.steps[s][1], o = n + s;
        Geom &g = geo[s];
        g.a = size[l] >= size[r] ? l : r;
        g.b = (g.a == l) ? r : l;
        const auto &LA = layout[g.a], &LB = layout[g.b];
        std::vector<int64_t> strA(LA.size()), strB(LB.size());
        int64_t acc = 1;
        for (int32_t i = (int32_t)LA.size() - 1; i >= 0; --i) { strA[i] = acc; acc *= net.edim[LA[i]]; }
        acc = 1;
        for (int32_t i = (int32_t)LB.size() - 1; i >= 0; --i) { strB[i] = acc; acc *= net.edim[LB[i]]; }
        std::vector<int32_t> out;
        for (size_t i = 0; i < LA.size(); ++i) {
            const int32_t e = LA[i];
            auto jt = std::find(LB.begin(), LB.end(), e);
            if (jt == LB.end()) {
                g.md.push_back(net.edim[e]); g.ms.push_back(strA[i]); out.push_back(e); g.M *= net.edim[e];
            } else {
                g.kd.push_back(net.edim[e]); g.ksa.push_back(strA[i]); g.ksb.push_back(strB[jt - LB.begin()]);
                g.K *= net.edim[e];
            }
        }
        for (size_t i = 0; i < LB.size(); ++i) {
            const int32_t e = LB[i];
            if (std::find(LA.begin(), LA.end(), e) == LA.end()) {
                g.nd.push_back(net.edim[e]); g.ns.push_back(strB[i]); out.push_back(e); g.N *= net.edim[e];
            }
        }
        layout[o] = out;
        size[o] = g.M * g.N;
        if (s == n - 2 && g.M * g.N != 1)
            return fail(TN_EUNSUPPORTED, "open networks are not supported by tn_contract");
        c.flops += 8.0 * (double)g.M * (double)g.N * (double)g.K;
        c.bytes += (double)(size[g.a] + size[g.b] + size[o]) * (double)esz;
    }
    // pass 2: CTA-resident subtree programs -- the maximal subtrees that fit the budget
    // Warp programs first (maximal subtrees of small steps), then block programs (maximal subtrees
    // that fit the budget, whose inputs are leaves and warp-program results).
    std::vector<int32_t> prog_of(nn, -1);     // program index for every internal node inside one
    std::vector<int32_t> wprog_of(nn, -1);    // the same, warp programs only
    std::vector<LocalPlan> lplans;
    std::vector<WarpPlan> wplans;
    std::vector<int32_t> proot, wroot;
    std::vector<int32_t> pkind;                // ProgKind of each entry of proot
    if (local_budget > 0 && n > 1) {
        std::vector<int32_t> stack{nn - 1};
        while (!stack.empty()) {
            const int32_t v = stack.back();
            stack.pop_back();
            if (v < n) continue;
            WarpPlan wp;
            if (opt.warp_programs && warp_fit(v, n, plan, geo, size, elem, wp)) {
                for (int32_t x : wp.nodes) wprog_of[x] = (int32_t)wroot.size();
                wroot.push_back(v);
                wplans.push_back(std::move(wp));
            } else {
                stack.push_back(plan.steps[v - n][0]);
                stack.push_back(plan.steps[v - n][1]);
            }
        }
        stack.assign(1, nn - 1);
        while (!stack.empty()) {
            const int32_t v = stack.back();
            stack.pop_back();
            if (v < n || wprog_of[v] >= 0) continue;
            LocalPlan lp;
            if (local_fit(v, n, plan, geo, size, elem, local_budget, wprog_of, false, lp)) {
                for (int32_t x : lp.nodes) prog_of[x] = (int32_t)proot.size();
                proot.push_back(v);
                pkind.push_back(PROG_BLOCK);
                lplans.push_back(std::move(lp));
            } else {
                stack.push_back(plan.steps[v - n][0]);
                stack.push_back(plan.steps[v - n][1]);
            }
        }
        // large programs: maximal subtrees within the one-block-per-SM budget whose inputs are
        // leaves and the results of the programs above, each input staged when it is consumed
        if (big_budget > local_budget) {
            std::vector<int32_t> covered(nn, -1);
            for (int32_t v = n; v < nn; ++v)
                if (wprog_of[v] >= 0 || prog_of[v] >= 0) covered[v] = 1;
            stack.assign(1, nn - 1);
            while (!stack.empty()) {
                const int32_t v = stack.back();
                stack.pop_back();
                if (v < n || covered[v] >= 0) continue;
                LocalPlan lp;
                if (local_fit(v, n, plan, geo, size, elem, big_budget, covered, true, lp) && lp.nodes.size() > 1) {
                    for (int32_t x : lp.nodes) prog_of[x] = (int32_t)proot.size();
                    proot.push_back(v);
                    pkind.push_back(PROG_BIG);
                    lplans.push_back(std::move(lp));
                } else {
                    stack.push_back(plan.steps[v - n][0]);
                    stack.push_back(plan.steps[v - n][1]);
                }
            }
        }
        // warp programs are numbered after the block and large programs
        for (int32_t v = n; v < nn; ++v)
            if (wprog_of[v] >= 0) prog_of[v] = (int32_t)proot.size() + wprog_of[v];
    }
    std::vector<char> is_proot(nn, 0);
    for (int32_t v : proot) is_proot[v] = 1;
    for (int32_t v : wroot) is_proot[v] = 1;
    // global memory: outputs of global steps and of programs (not the intermediates of programs)
    std::vector<size_t> bytes(nn, 0), arena_off;
    for (int32_t v = n; v < nn; ++v)
        if (prog_of[v] < 0 || is_proot[v]) bytes[v] = align_up((size_t)size[v] * esz, 256);
    c.arena_bytes = std::max(plan_memory(plan, n, bytes, arena_off), (size_t)256);
    // pass 3: the global step list (plan order), programs as single pseudo-steps
    std::vector<int32_t> producer(nn, -1), level(nn, 0);
    c.steps.clear();
    for (int32_t s = 0; s < n - 1; ++s) {
        const int32_t o = n + s;
        if (prog_of[o] >= 0 && !is_proot[o]) continue;
        const Geom &g = geo[s];
        const bool root = (s == n - 2);
        StepDesc d;
        std::memset(&d, 0, sizeof(d));
        d.ktab_off = -1;
        d.chain_next = -1;
        d.M = g.M; d.N = g.N; d.K = g.K;
        d.node_a = g.a; d.node_b = g.b; d.node_c = o;
        d.c_off = (int64_t)(arena_off[o] / esz);
        if (is_proot[o]) {
            d.kind = STEP_LOCAL;
            d.ntiles = 1;
            d.tile_rows = prog_of[o];
            d.dep0 = d.dep1 = -1;
            d.level = 1;
            if (root) d.flags |= FLAG_ROOT | FLAG_NO_C;
            c.steps.push_back(d);
            c.counts[STEP_LOCAL]++;
            producer[o] = (int32_t)c.steps.size() - 1;
            level[o] = 1;
            continue;
        }
        if (!make_groups(g.md, g.ms, g.ms, false, d.m) || !make_groups(g.nd, g.ns, g.ns, false, d.n) ||
            !make_groups(g.kd, g.ksa, g.ksb, true, d.k))
            return fail(TN_EUNSUPPORTED, "step " + std::to_string(s) + " has more than 32 leg groups");
        auto where = [&](int32_t v, int64_t &off) -> bool {
            if (v < n) { off = c.leaf_off[v]; return true; }
            off = (int64_t)(arena_off[v] / esz);
            return false;
        };
        if (where(g.a, d.a_off)) d.flags |= FLAG_A_LEAF;
        if (where(g.b, d.b_off)) d.flags |= FLAG_B_LEAF;
        d.dep0 = producer[g.a];
        d.dep1 = producer[g.b];
        d.level = 1 + std::max(level[g.a], level[g.b]);
        const int64_t M = g.M, N = g.N, K = g.K;
        const bool dot = root || (M * N <= kDotMaxOut && K > kRowsMaxK);
        if (dot) {
            StepDesc p = d;
            p.kind = STEP_DOTP;
            p.flags |= FLAG_NO_C;
            p.tile_rows = kDotChunk;
            p.ntiles = (int32_t)((K + kDotChunk - 1) / kDotChunk);
            p.part_off = (int32_t)c.n_partials;
            c.n_partials += (int64_t)p.ntiles * kDotMaxOut;
            // tabulate the shared-index offsets (the tile then reads one int2 per index instead of
            // decomposing the index over its leg groups) when the table stays small
            if (K <= (1 << 20)) {
                bool fits = true;
                const size_t t0 = c.ktab.size();
                c.ktab.resize(t0 + (size_t)K);
                for (int64_t k = 0; k < K && fits; ++k) {
                    int64_t idx = k, oa = 0, ob = 0;
                    for (int32_t i = 0; i < p.k.n; ++i) {
                        const int64_t dg = idx % p.k.dim[i];
                        idx /= p.k.dim[i];
                        oa += dg * p.k.sa[i];
                        ob += dg * p.k.sb[i];
                    }
                    if (oa > 0x7fffffffLL || ob > 0x7fffffffLL) fits = false;
                    c.ktab[t0 + (size_t)k] = make_int2((int32_t)oa, (int32_t)ob);
                }
                if (fits && t0 <= 0x7fffffffULL) p.ktab_off = (int32_t)t0;
                else c.ktab.resize(t0);
                // one complex64 tile over a vector operand read in a permuted order: stage the more
                // permuted one (counted in breaks of unit stride along k) in shared memory
                if (p.ktab_off >= 0 && elem == 8 && p.ntiles == 1 && K <= kRowsSmemElems) {
                    int64_t brk_a = 0, brk_b = 0;
                    for (int64_t k = 1; k < K; ++k) {
                        const int2 u = c.ktab[t0 + (size_t)k - 1], v = c.ktab[t0 + (size_t)k];
                        brk_a += v.x != u.x + 1;
                        brk_b += v.y != u.y + 1;
                    }
                    const bool a_ok = M == 1 && !(p.flags & FLAG_A_LEAF), b_ok = N == 1 && !(p.flags & FLAG_B_LEAF);
                    if (b_ok && brk_b > 0 && (brk_b >= brk_a || !a_ok)) p.flags |= FLAG_DOT_SMEM_B;
                    else if (a_ok && brk_a > 0) p.flags |= FLAG_DOT_SMEM_A;
                }
            }
            c.steps.push_back(p);
            StepDesc f = d;
            f.kind = STEP_DOTF;
            f.ntiles = 1;
            f.tile_rows = p.ntiles;
            f.part_off = p.part_off;
            f.dep0 = (int32_t)c.steps.size() - 1;
            f.dep1 = -1;
            f.level = d.level + 1;
            if (root) f.flags |= FLAG_ROOT | FLAG_NO_C;
            c.steps.push_back(f);
            c.counts[STEP_DOTP]++;
        } else if (N <= kRowsMaxN && K <= kRowsMaxK && K * N <= kRowsMaxKN) {
            d.kind = STEP_ROWS;
            d.tile_rows = rows_per_tile(M);
            d.ntiles = (int32_t)((M + d.tile_rows - 1) / d.tile_rows);
            // complex64 steps whose A fits shared memory are staged through it (one tile, every
            // thread owning 32 / NT rows in one pass)
            const int64_t nt = N <= 4 ? 4 : (N <= 8 ? 8 : 16);
            if (elem == 8 && K <= 16 && !(d.flags & FLAG_A_LEAF) && M * K <= kRowsSmemElems &&
                M * (N + 1) <= kRowsSmemElems && M <= (int64_t)kThreads * (32 / nt)) {
                d.flags |= FLAG_A_SMEM;
                d.tile_rows = (int32_t)M;
                d.ntiles = 1;
            }
            c.steps.push_back(d);
            c.counts[STEP_ROWS]++;
        } else if (use_tc && M >= opt.tc_min_m && N >= opt.tc_min_n && K >= opt.tc_min_k) {
            // dense step on the tensor cores: operands packed into split images, then 128 x 128
            // complex output tiles, BF16 or TF32 split
            d.kind = STEP_TC;
            if (tc_mode == 2) d.flags |= FLAG_TF32;
            if (d.m.n > 0 && d.m.sa[0] == 1 && !(d.k.n > 0 && d.k.sa[0] == 1)) d.flags |= FLAG_A_MCONT;
            if (d.n.n > 0 && d.n.sa[0] == 1) d.flags |= FLAG_B_NCONT;
            // output tile width: 64 complex columns when the step is that narrow (or forced)
            const int nc = opt.tc_tile_n == 64 || (opt.tc_tile_n == 0 && N <= 64) ? 64 : kTcColsMax;
            d.tile_rows = nc;
            const int64_t tiles = ((M + kTcRows - 1) / kTcRows) * ((N + nc - 1) / nc);
            if (tiles > 0x7fffffffLL || tc_pack_units(M, N, K, tc_mode == 2, nc) > 0x7fffffffLL)
                return fail(TN_EUNSUPPORTED, "step too large");
            d.ntiles = (int32_t)tiles;
            c.steps.push_back(d);
            c.counts[STEP_TC]++;
        } else {
            d.kind = STEP_TILE;
            // narrow complex64 outputs (N <= 32) use 128 x 32 tiles so no thread computes padding
            const bool narrow = N <= kTileN / 2 && elem == 8;
            d.tile_rows = narrow ? kTileNarrow : 0;
            const int64_t tm = narrow ? 2 * kTileM : kTileM, tn = narrow ? kTileN / 2 : kTileN;
            const int64_t tiles = ((M + tm - 1) / tm) * ((N + tn - 1) / tn);
            if (tiles > 0x7fffffffLL) return fail(TN_EUNSUPPORTED, "step too large");
            d.ntiles = (int32_t)tiles;
            c.steps.push_back(d);
            c.counts[STEP_TILE]++;
        }
        producer[o] = (int32_t)c.steps.size() - 1;
        level[o] = c.steps.back().level;
    }
    // ROWS chains: step t continues step s in the same persistent block, with s's C kept in
    // shared memory as t's A, when both stage A through shared memory, A of t is C of s (its only
    // consumer: the plan is a tree), N of s is a power of two (C's rotated layout) and B of t is a
    // leaf or a program output (complete before the dataflow launch, so the chain never waits
    // inside).  Steps are in plan order, so s precedes t.
    if (opt.rows_chains) {
        std::vector<int32_t> chain_len(c.steps.size(), 1);
        for (size_t ti = 0; ti < c.steps.size(); ++ti) {
            StepDesc &t = c.steps[ti];
            if (t.kind != STEP_ROWS || !(t.flags & FLAG_A_SMEM) || t.dep0 < 0) continue;
            StepDesc &s = c.steps[t.dep0];
            if (s.kind != STEP_ROWS || !(s.flags & FLAG_A_SMEM) || s.chain_next >= 0 || s.node_c != t.node_a)
                continue;
            if ((s.N & (s.N - 1)) != 0 || s.M * s.N != t.M * t.K) continue;
            if (t.dep1 >= 0 && c.steps[t.dep1].kind != STEP_LOCAL) continue;
            if (chain_len[t.dep0] >= kMaxChain) continue;
            s.chain_next = (int32_t)ti;
            t.flags |= FLAG_CHAIN_CONT;
            int32_t lg = 0;
            while ((1LL << lg) < s.N) ++lg;
            t.a_lgn = lg;
            chain_len[ti] = chain_len[t.dep0] + 1;
        }
    }
    // algorithmic bytes by executing kernel class
    for (int32_t st = 0; st < n - 1; ++st) {
        const int32_t o = n + st;
        const Geom &g = geo[st];
        const double bb = (double)(size[g.a] + size[g.b] + size[o]) * (double)esz;
        int cls = 3;
        if (wprog_of[o] >= 0) cls = 0;
        else if (prog_of[o] >= 0) cls = 1;
        else if (producer[o] >= 0 && c.steps[producer[o]].kind == STEP_TC) cls = 2;
        c.bytes_cls[cls] += bb;
    }
    // packed operand images of the tensor-core steps: after the intermediates, never reused
    {
        size_t img = align_up(c.arena_bytes, 1024);
        for (StepDesc &d : c.steps) {
            if (d.kind != STEP_TC) continue;
            size_t a_bytes = 0;
            const size_t all = tc_image_bytes(d.M, d.N, d.K, (d.flags & FLAG_TF32) != 0, d.tile_rows, &a_bytes);
            d.img_a = (int64_t)img;
            d.img_b = (int64_t)(img + a_bytes);
            img = align_up(img + all, 1024);
        }
        c.arena_bytes = img;
    }
    // pass 4: the programs' compact step lists
    c.progs.clear();
    c.lsteps.clear();
    c.leafrefs.clear();
    c.lwaves.clear();
    c.dyn_smem = 0;
    for (size_t pi = 0; pi < proot.size(); ++pi) {
        const LocalPlan &lp = lplans[pi];
        const int32_t v = proot[pi];
        LocalProg P;
        std::memset(&P, 0, sizeof(P));
        P.first_step = (int32_t)c.lsteps.size();
        P.n_steps = (int32_t)lp.nodes.size();
        P.first_leaf = (int32_t)c.leafrefs.size();
        P.n_leaves = (int32_t)lp.leaves.size();
        P.n_slots = (int32_t)lp.loc.size();
        P.smem_bytes = lp.smem_bytes;
        P.root_node = v;
        P.root_slot = lp.idx.at(v);
        P.root_smem_off = (int32_t)lp.loc[lp.idx.at(v)];
        P.root_size = (int32_t)size[v];
        P.root_c_off = (int64_t)(arena_off[v] / esz);
        P.flags = (v == nn - 1) ? LFLAG_JOB_ROOT : 0;
        P.first_wave = (int32_t)c.lwaves.size();
        P.n_waves = (int32_t)lp.waves.size();
        P.kind = pkind[pi];
        auto stage = [&](int32_t t) -> tn_status {
            const int64_t goff = t < n ? c.leaf_off[t] : (int64_t)(arena_off[t] / esz);
            return push_input(c.leafrefs, goff, size[t], lp.loc[lp.idx.at(t)], lp.idx.at(t), t, t < n ? 0 : 1);
        };
        // wave step indices are relative to the program (its descriptors are staged per program)
        for (size_t wi = 0; wi < lp.waves.size(); ++wi) {
            LocalWave W = lp.waves[wi];
            if (P.kind == PROG_BIG) {
                W.first_in = (int32_t)c.leafrefs.size();
                for (int32_t t : lp.wave_inputs[wi]) {
                    tn_status st = stage(t);
                    if (st != TN_OK) return st;
                }
                W.n_in = (int32_t)c.leafrefs.size() - W.first_in;
            }
            c.lwaves.push_back(W);
        }
        P.first_leaf = (int32_t)c.leafrefs.size();
        if (P.kind != PROG_BIG)
            for (int32_t t : lp.leaves) {
                tn_status st = stage(t);
                if (st != TN_OK) return st;
            }
        P.n_leaves = (int32_t)c.leafrefs.size() - P.first_leaf;
        for (size_t si = 0; si < lp.nodes.size(); ++si) {
            const int32_t x = lp.nodes[si];
            const Geom &g = geo[x - n];
            LocalStep ls;
            std::memset(&ls, 0, sizeof(ls));
            ls.M = (int32_t)g.M; ls.N = (int32_t)g.N; ls.K = (int32_t)g.K;
            ls.a_off = (int32_t)lp.loc[lp.idx.at(g.a)];
            ls.b_off = (int32_t)lp.loc[lp.idx.at(g.b)];
            ls.c_off = (int32_t)lp.loc[lp.idx.at(x)];
            ls.sa = (int16_t)lp.idx.at(g.a);
            ls.sb = (int16_t)lp.idx.at(g.b);
            ls.sc = (int16_t)lp.idx.at(x);
            bool p2 = true;
            make_lgroups(g.md, g.ms, g.ms, false, ls.m_dim, ls.m_str, nullptr, ls.m_lsb, ls.nm, p2);
            make_lgroups(g.nd, g.ns, g.ns, false, ls.n_dim, ls.n_str, nullptr, ls.n_lsb, ls.nn, p2);
            make_lgroups(g.kd, g.ksa, g.ksb, true, ls.k_dim, ls.k_sa, ls.k_sb, ls.k_lsb, ls.nk, p2);
            ls.pow2 = p2 ? 1 : 0;
            if (x == nn - 1) {
                ls.mode = LMODE_REDUCE;
                ls.flags = LFLAG_JOB_ROOT;
            } else if (g.N <= kRowsMaxN && g.K <= kRowsMaxK) {
                ls.mode = LMODE_ROWS;
            } else if (g.M >= 32 && g.N >= 32) {
                ls.mode = LMODE_GEMM;
            } else {
                ls.mode = LMODE_REDUCE;
            }
            if (lp.small[si]) ls.flags |= LFLAG_SMALL;
            tabulate_small(ls);
            c.lsteps.push_back(ls);
        }
        if (P.kind == PROG_BIG) {
            c.dyn_big = std::max(c.dyn_big, P.smem_bytes);
            c.counts[9]++;
        } else {
            c.dyn_smem = std::max(c.dyn_smem, P.smem_bytes);
        }
        c.progs.push_back(P);
    }
    c.counts[6] = (int32_t)c.lsteps.size();
    // warp programs
    for (size_t wi = 0; wi < wroot.size(); ++wi) {
        const WarpPlan &wp = wplans[wi];
        const int32_t v = wroot[wi];
        LocalProg P;
        std::memset(&P, 0, sizeof(P));
        P.first_step = (int32_t)c.lsteps.size();
        P.n_steps = (int32_t)wp.nodes.size();
        P.n_slots = (int32_t)(wp.leaves.size() + wp.nodes.size());
        P.first_leaf = (int32_t)c.leafrefs.size();
        for (int32_t t : wp.leaves) {
            tn_status st = push_input(c.leafrefs, c.leaf_off[t], size[t], wp.loc.at(t), wp.slot.at(t), t, 0);
            if (st != TN_OK) return st;
        }
        P.n_leaves = (int32_t)c.leafrefs.size() - P.first_leaf;
        P.smem_bytes = wp.smem_bytes;
        P.root_node = v;
        P.root_slot = wp.slot.at(v);
        P.root_size = (int32_t)size[v];
        P.root_c_off = (int64_t)(arena_off[v] / esz);
        P.kind = PROG_WARP;
        for (int32_t x : wp.nodes) {
            const Geom &g = geo[x - n];
            LocalStep ls;
            std::memset(&ls, 0, sizeof(ls));
            ls.M = (int32_t)g.M; ls.N = (int32_t)g.N; ls.K = (int32_t)g.K;
            ls.flags = LFLAG_SMALL;
            ls.a_off = (int32_t)wp.loc.at(g.a);
            ls.sa = (int16_t)wp.slot.at(g.a);
            ls.b_off = (int32_t)wp.loc.at(g.b);
            ls.sb = (int16_t)wp.slot.at(g.b);
            if (x == v) ls.flags |= LFLAG_C_OUT;
            else ls.c_off = (int32_t)wp.loc.at(x);
            ls.sc = (int16_t)wp.slot.at(x);
            bool p2 = true;
            make_lgroups(g.md, g.ms, g.ms, false, ls.m_dim, ls.m_str, nullptr, ls.m_lsb, ls.nm, p2);
            make_lgroups(g.nd, g.ns, g.ns, false, ls.n_dim, ls.n_str, nullptr, ls.n_lsb, ls.nn, p2);
            make_lgroups(g.kd, g.ksa, g.ksb, true, ls.k_dim, ls.k_sa, ls.k_sb, ls.k_lsb, ls.nk, p2);
            ls.pow2 = p2 ? 1 : 0;
            ls.mode = LMODE_ROWS;
            tabulate_small(ls);
            c.lsteps.push_back(ls);
        }
        c.dyn_smem = std::max(c.dyn_smem, (int32_t)kWarpSlice);
        c.progs.push_back(P);
        c.counts[7]++;
        c.counts[8] += P.n_steps;
    }
    c.total_tiles = 0;
    for (const StepDesc &d : c.steps) c.total_tiles += d.ntiles;
    return TN_OK;
}

WorkItem tn::dataflow_item(const Compiled &c, uint32_t job, int32_t step, int32_t tile) {
    const StepDesc &d = c.steps[step];
    WorkItem w;
    w.job = job;
    w.step = (uint32_t)step;
    w.tile = (uint32_t)tile;
    w.dep0 = d.dep0;
    w.dep1 = d.dep1;
    w.need0 = d.dep0 >= 0 ? (uint32_t)c.steps[d.dep0].ntiles : 0u;
    w.need1 = d.dep1 >= 0 ? (uint32_t)c.steps[d.dep1].ntiles : 0u;
    return w;
}

void tn::path_weights(const Compiled &c, std::vector<double> &path) {
    const size_t ns = c.steps.size();
    std::vector<int32_t> consumer(ns, -1);
    for (size_t s = 0; s < ns; ++s) {
        if (c.steps[s].dep0 >= 0) consumer[c.steps[s].dep0] = (int32_t)s;
        if (c.steps[s].dep1 >= 0) consumer[c.steps[s].dep1] = (int32_t)s;
    }
    path.assign(ns, 0.0);
    for (size_t s = ns; s-- > 0;) {   // consumers follow their producers
        const StepDesc &d = c.steps[s];
        const double w = d.kind == STEP_LOCAL ? 0.0 : (double)d.M * (double)d.N * (double)d.K;
        path[s] = w + (consumer[s] >= 0 ? path[consumer[s]] : 0.0);
    }
}

int32_t tn::step_phases(const Compiled &c, std::vector<int32_t> &phase) {
    phase.assign(c.steps.size(), 0);
    int32_t top = 0;
    for (size_t s = 0; s < c.steps.size(); ++s) {   // producers precede their consumers
        const StepDesc &d = c.steps[s];
        int32_t p = 0;
        if (d.dep0 >= 0) p = std::max(p, phase[d.dep0]);
        if (d.dep1 >= 0) p = std::max(p, phase[d.dep1]);
        if (d.kind == STEP_TC) ++p;
        phase[s] = p;
        top = std::max(top, p);
    }
    return top + 1;
}

void tn::phase_templates(const Compiled &c, std::vector<PhaseTemplate> &out) {
    std::vector<int32_t> phase;
    const int32_t np = step_phases(c, phase);
    out.assign(np, PhaseTemplate());
    std::vector<std::array<int32_t, 3>> order;   // phase, level, step
    for (size_t s = 0; s < c.steps.size(); ++s)
        if (c.steps[s].kind != STEP_LOCAL && !(c.steps[s].flags & FLAG_CHAIN_CONT))
            order.push_back({phase[s], c.steps[s].level, (int32_t)s});
    std::sort(order.begin(), order.end());
    for (auto &o : order) {
        const StepDesc &d = c.steps[o[2]];
        PhaseTemplate &pt = out[o[0]];
        if (d.kind == STEP_TC) {
            const int64_t units = tc_pack_units(d.M, d.N, d.K, (d.flags & FLAG_TF32) != 0, d.tile_rows);
            for (int64_t u = 0; u < units; ++u) pt.pack.push_back({0u, (uint32_t)o[2], (uint32_t)u});
            for (int32_t t = 0; t < d.ntiles; ++t) pt.gemm.push_back({0u, (uint32_t)o[2], (uint32_t)t});
            continue;
        }
        for (int32_t t = 0; t < d.ntiles; ++t) {
            pt.work.push_back(dataflow_item(c, 0u, o[2], t));
            pt.level.push_back(o[1]);
        }
    }
}

namespace {

tn_status upload_leaves(tn_batch *b, int32_t job) {
    const Net &net = b->nets[job]->impl;
    const size_t bytes = sizeof(double) * net.data.size();
    double *stage = b->h_pinned + 2 * b->leaf64_off[job];
    if (bytes) {
        std::memcpy(stage, net.data.data(), bytes);
        CK(cudaMemcpyAsync(b->d_leaf64 + b->leaf64_off[job], stage, bytes, cudaMemcpyHostToDevice,
                           b->ctx->stream));
    }
    b->uploaded[job] = net.version;
    return TN_OK;
}

// Ranges of the phases' dataflow items in a work list built phase by phase (item i in phase ph[i]).
void set_phase_ranges(tn_batch *b, const std::vector<int32_t> &ph) {
    for (tn_batch::Phase &p : b->phases) p.work0 = p.n_work = 0;
    for (size_t i = 0; i < ph.size(); ++i) {
        tn_batch::Phase &p = b->phases[ph[i]];
        if (p.n_work == 0) p.work0 = (int64_t)i;
        p.n_work++;
    }
}

// The stage of the last enqueue_run that failed (for the error message).
thread_local const char *t_enqueue_stage = "";

// Enough events in `ev` for one persistent run: a start event and one after every launch slot.
cudaError_t ensure_events(std::vector<cudaEvent_t> &ev, size_t n) {
    while (ev.size() < n) {
        cudaEvent_t x = nullptr;
        const cudaError_t e = cudaEventCreate(&x);
        if (e != cudaSuccess) return e;
        ev.push_back(x);
    }
    return cudaSuccess;
}

// The contraction kernels of one persistent run, ev[0] recorded first and one event after every
// launch slot: warp programs, block and large programs, then per phase the pack, GEMM and
// dataflow launches.
cudaError_t enqueue_persistent(tn_batch *b, cudaStream_t st, std::vector<cudaEvent_t> &ev, bool capturing) {
    // inside a stream capture an event becomes a graph event-record node only when recorded as
    // an external event
    const unsigned rec_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaError_t e = cudaSuccess;
    e = ensure_events(ev, 3 + 3 * b->phases.size());
    if (e != cudaSuccess) return e;
    size_t k = 0;
    e = cudaEventRecordWithFlags(ev[k++], st, rec_flags);
    if (e == cudaSuccess) {
        t_enqueue_stage = "warp programs";
        e = launch_local(b->c128, b->d_jobs, b->d_local, b->n_warp_items, 0, 0, b->dyn_smem, b->dyn_big,
                         b->d_prof, st);
    }
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[k++], st, rec_flags);
    if (e == cudaSuccess) {
        t_enqueue_stage = "subtree programs";
        e = launch_local(b->c128, b->d_jobs, b->d_local + b->n_warp_items, 0, b->n_block_items, b->n_big_items,
                         b->dyn_smem, b->dyn_big, b->d_prof, st);
    }
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[k++], st, rec_flags);
    const bool tf32 = b->prec == TN_TF32_SPLIT;
    for (size_t p = 0; e == cudaSuccess && p < b->phases.size(); ++p) {
        const tn_batch::Phase &ph = b->phases[p];
        uint32_t *cnt = b->d_counter + 3 * p;
        if (ph.n_pack > 0) {
            t_enqueue_stage = "tensor-core operand packing";
            e = launch_tc_pack(tf32, b->d_jobs, b->d_pack + ph.pack0, ph.n_pack, st);
        }
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[k++], st, rec_flags);
        if (e == cudaSuccess && ph.n_gemm > 0) {
            t_enqueue_stage = "tensor-core GEMM";
            e = launch_tc_gemm(tf32, b->d_jobs, b->d_gemm + ph.gemm0, ph.n_gemm, reinterpret_cast<int32_t *>(cnt + 2),
                               b->wait_ns, st);
        }
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[k++], st, rec_flags);
        if (e == cudaSuccess && ph.n_work > 0) {
            t_enqueue_stage = "dataflow kernel";
            e = launch_persistent(b->c128, b->d_jobs, b->d_work + ph.work0, ph.n_work, cnt, b->grid, b->wait_ns,
                                  b->d_prof, st);
        }
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[k++], st, rec_flags);
    }
    return e;
}

cudaError_t enqueue_run(tn_batch *b, cudaStream_t st) {
    // a non-sticky error left by an earlier runtime call of this thread (another library's, say)
    // would otherwise be reported by the launch checks below
    (void)cudaGetLastError();
    t_enqueue_stage = "reset";
    cudaError_t e = cudaMemsetAsync(b->d_reset, 0, b->reset_bytes, st);
    if (e == cudaSuccess) {
        t_enqueue_stage = "leaf conversion";
        e = launch_leaf_convert(b->c128, b->d_jobs, b->n_jobs, b->max_leaves, b->max_leaf_elems, st);
    }
    if (e != cudaSuccess) return e;
    if (b->mode == TN_EXEC_PERSISTENT) {
        e = enqueue_persistent(b, st, b->kev[b->runs % tn_batch::kRing], false);
        b->runs++;
    } else {
        const bool tf32 = b->prec == TN_TF32_SPLIT;
        size_t r = 0;   // tensor-core ranges, in (job, step) order
        for (int32_t jb = 0; e == cudaSuccess && jb < b->n_jobs; ++jb) {
            const Compiled &c = b->comp[b->job_comp[jb]];
            for (size_t s = 0; e == cudaSuccess && s < c.steps.size(); ++s) {
                if (c.steps[s].kind == STEP_TC) {
                    const TcRange &tr = b->tc_ranges[r++];
                    e = launch_tc_pack(tf32, b->d_jobs, b->d_pack + tr.pack0, tr.n_pack, st);
                    if (e == cudaSuccess)
                        e = launch_tc_gemm(tf32, b->d_jobs, b->d_gemm + tr.gemm0, tr.n_gemm,
                                           reinterpret_cast<int32_t *>(b->d_counter + 2), b->wait_ns, st);
                    continue;
                }
                e = launch_step(b->c128, c.steps[s], (int32_t)s, b->jobs[jb], std::max(b->dyn_smem, b->dyn_big), st);
            }
        }
    }
    for (int32_t jb = 0; e == cudaSuccess && jb < b->n_jobs; ++jb)
        if (b->comp[b->job_comp[jb]].n == 1) e = launch_finish_leaf(b->c128, b->jobs[jb], st);
    return e;
}

// Capture one persistent run -- reset, leaf conversion, all launches with the graph's own events
// -- into b->pgexec (replaced if present).
tn_status record_persistent_graph(tn_batch *b) {
    cudaStream_t st = b->ctx->stream;
    if (b->pgexec) {
        CK(cudaStreamSynchronize(st));
        cudaGraphExecDestroy(b->pgexec);
        b->pgexec = nullptr;
    }
    cudaError_t err = ensure_events(b->gev, 3 + 3 * b->phases.size());
    if (err != cudaSuccess) return fail(TN_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(err));
    (void)cudaGetLastError();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    err = cudaMemsetAsync(b->d_reset, 0, b->reset_bytes, st);
    if (err == cudaSuccess) err = launch_leaf_convert(b->c128, b->d_jobs, b->n_jobs, b->max_leaves, b->max_leaf_elems, st);
    if (err == cudaSuccess) err = enqueue_persistent(b, st, b->gev, true);
    for (int32_t jb = 0; err == cudaSuccess && jb < b->n_jobs; ++jb)
        if (b->comp[b->job_comp[jb]].n == 1) err = launch_finish_leaf(b->c128, b->jobs[jb], st);
    cudaGraph_t g = nullptr;
    cudaError_t err2 = cudaStreamEndCapture(st, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(TN_ECUDA, std::string("recording the run: ") + cudaGetErrorString(err));
    }
    if (err2 != cudaSuccess) return fail(TN_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(err2));
    err = cudaGraphInstantiate(&b->pgexec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return fail(TN_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(err));
    return TN_OK;
}

tn_status record_graph(tn_batch *b) {
    cudaStream_t st = b->ctx->stream;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = enqueue_run(b, st);
    cudaGraph_t g = nullptr;
    cudaError_t err2 = cudaStreamEndCapture(st, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(TN_ECUDA, std::string("recording the program: ") + cudaGetErrorString(err));
    }
    if (err2 != cudaSuccess) return fail(TN_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(err2));
    err = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return fail(TN_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(err));
    return TN_OK;
}

void batch_destroy(tn_batch *b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->pgexec) cudaGraphExecDestroy(b->pgexec);
    for (cudaEvent_t e : b->gev)
        if (e) cudaEventDestroy(e);
    for (auto &list : b->kev)
        for (cudaEvent_t e : list)
            if (e) cudaEventDestroy(e);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->d_block) cudaFree(b->d_block);
    if (b->h_pinned) cudaFreeHost(b->h_pinned);
    if (b->h_res) cudaFreeHost(b->h_res);
    for (tn_batch::Stage &sg : b->stage) {
        if (sg.hdr.p) cudaFreeHost(sg.hdr.p);
        if (sg.val.p) cudaFreeHost(sg.val.p);
        if (sg.ev) cudaEventDestroy(sg.ev);
    }
    if (b->d_upd) cudaFree(b->d_upd);
    if (b->d_prof) cudaFree(b->d_prof);
    tn_ctx *ctx = b->ctx;
    delete b;
    ctx_release(ctx);
}

tn_status batch_create(tn_ctx *ctx, int32_t n, const tn_net *const *nets, const tn_plan *const *plans,
                       tn_precision prec, tn_batch **out) {
    if (!ctx || !out || n < 1 || !nets || !plans) return fail(TN_EINVAL, "NULL argument or empty batch");
    if (prec < TN_C128 || prec > TN_BF16_SPLIT) return fail(TN_EINVAL, "unknown precision");
    for (int32_t i = 0; i < n; ++i) {
        if (!nets[i] || !plans[i]) return fail(TN_EINVAL, "NULL net or plan in the batch");
        if (plans[i]->impl.n != nets[i]->impl.n) return fail(TN_EINVAL, "plan and network do not match");
        if (!nets[i]->impl.closed) return fail(TN_EUNSUPPORTED, "open networks are not supported by tn_contract");
    }
    CK(cudaSetDevice(ctx->device));
    // admission: mem(B) of Eq. 3.1 (elements of the largest step's operands and result) is a lower
    // bound of a job's device footprint; refuse before compiling if it cannot fit
    {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        const double elem = prec == TN_C128 ? 16.0 : 8.0;
        double need = 0;
        for (int32_t i = 0; i < n; ++i) need += (double)plans[i]->impl.mem * elem;
        if (ctx->budget && need > (double)ctx->budget)
            return fail(TN_EBUDGET, "the plans need at least " + std::to_string(need) +
                                        " bytes (Eq. 3.1), above the context's budget");
        if (need > (double)free_b)
            return fail(TN_EBUDGET, "the plans need at least " + std::to_string(need) +
                                        " bytes (Eq. 3.1), above the free device memory");
    }
    tn_batch *b = new (std::nothrow) tn_batch;
    if (!b) return fail(TN_ENOMEM, "allocating the batch");
    b->ctx = ctx;
    ctx_retain(ctx);
    b->prec = prec;
    b->c128 = (prec == TN_C128);
    b->elem = b->c128 ? 16 : 8;
    b->mode = ctx->mode;
    b->n_jobs = n;
    b->nets.assign(nets, nets + n);
    b->uploaded.assign(n, ~0ull);
    b->job_comp.assign(n, -1);
    // compile every distinct (structure, plan) once
    CompileOpts copt = compile_opts(ctx->cfg, prec, b->c128);
    std::unordered_map<std::string, int32_t> seen;
    for (int32_t i = 0; i < n; ++i) {
        const Net &net = nets[i]->impl;
        const uint64_t h = shape_hash(net);
        const std::string key = std::to_string(plans[i]->impl.uid) + ":" + std::to_string(h);
        auto it = seen.find(key);
        if (it != seen.end()) { b->job_comp[i] = it->second; continue; }
        Compiled c;
        tn_status s = compile(c, net, plans[i]->impl, copt);
        if (s != TN_OK) { batch_destroy(b); return s; }
        c.plan_uid = plans[i]->impl.uid;
        c.shape_hash = h;
        b->job_comp[i] = (int32_t)b->comp.size();
        seen[key] = b->job_comp[i];
        b->comp.push_back(std::move(c));
    }
    // device layout
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max(bytes, (size_t)16), 256); return o; };
    std::vector<size_t> o_steps(b->comp.size()), o_loff(b->comp.size());
    std::vector<size_t> o_progs(b->comp.size()), o_lsteps(b->comp.size()), o_lrefs(b->comp.size()),
        o_lwaves(b->comp.size()), o_ktab(b->comp.size());
    for (size_t ci = 0; ci < b->comp.size(); ++ci) {
        o_steps[ci] = carve(sizeof(StepDesc) * b->comp[ci].steps.size());
        o_loff[ci] = carve(sizeof(int64_t) * b->comp[ci].leaf_off.size());
        o_progs[ci] = carve(sizeof(LocalProg) * b->comp[ci].progs.size());
        o_lsteps[ci] = carve(sizeof(LocalStep) * b->comp[ci].lsteps.size());
        o_lrefs[ci] = carve(sizeof(LeafRef) * b->comp[ci].leafrefs.size());
        o_lwaves[ci] = carve(sizeof(LocalWave) * b->comp[ci].lwaves.size());
        o_ktab[ci] = carve(sizeof(int2) * b->comp[ci].ktab.size());
        b->dyn_smem = std::max(b->dyn_smem, b->comp[ci].dyn_smem);
        b->dyn_big = std::max(b->dyn_big, b->comp[ci].dyn_big);
    }
    b->leaf64_off.assign(n, 0);
    int64_t leaf_total = 0;
    for (int32_t i = 0; i < n; ++i) {
        b->leaf64_off[i] = leaf_total;
        leaf_total += b->comp[b->job_comp[i]].leaf_off.back();
        b->max_leaves = std::max(b->max_leaves, b->comp[b->job_comp[i]].n);
        {
            const std::vector<int64_t> &lo = b->comp[b->job_comp[i]].leaf_off;
            for (size_t t = 0; t + 1 < lo.size(); ++t) b->max_leaf_elems = std::max(b->max_leaf_elems, lo[t + 1] - lo[t]);
        }
    }
    b->leaf_elems_total = leaf_total;
    const size_t o_leaf64 = carve(sizeof(double2) * (size_t)leaf_total);
    const size_t o_leaf = carve((size_t)b->elem * (size_t)leaf_total);
    std::vector<size_t> o_arena(n), o_part(n), o_exp(n);
    for (int32_t i = 0; i < n; ++i) {
        const Compiled &c = b->comp[b->job_comp[i]];
        o_arena[i] = carve(c.arena_bytes);
        o_part[i] = carve(sizeof(double2) * (size_t)c.n_partials);
        o_exp[i] = carve(sizeof(int32_t) * (size_t)c.n_nodes);
        b->arena_total += c.arena_bytes;
    }
    const size_t o_jobs = carve(sizeof(JobPtrs) * (size_t)n);
    // work lists per dependency phase (step_phases): dataflow items in (level, job, step, tile)
    // order, and the pack units and GEMM tiles of the tensor-core steps in (job, step) order
    std::vector<WorkItem> work, packs, gemms, local_items, warp_items, big_items;
    std::vector<int32_t> work_phase;
    {
        std::vector<std::vector<int32_t>> phase_of(b->comp.size());
        int32_t np = 1;
        for (size_t ci = 0; ci < b->comp.size(); ++ci) np = std::max(np, step_phases(b->comp[ci], phase_of[ci]));
        int64_t total = 0;
        for (int32_t i = 0; i < n; ++i) total += b->comp[b->job_comp[i]].total_tiles;
        if (total >= 0xffffffffLL) { batch_destroy(b); return fail(TN_EUNSUPPORTED, "too many work tiles"); }
        for (int32_t i = 0; i < n; ++i) {
            const Compiled &c = b->comp[b->job_comp[i]];
            for (size_t st = 0; st < c.steps.size(); ++st) {
                const StepDesc &d = c.steps[st];
                if (d.kind != STEP_LOCAL) continue;
                const LocalProg &P = c.progs[d.tile_rows];
                (P.kind == PROG_WARP ? warp_items : P.kind == PROG_BIG ? big_items : local_items)
                    .push_back({(uint32_t)i, (uint32_t)st, 0u});
            }
        }
        auto add_tc = [&](int32_t job, int32_t st) {
            const StepDesc &d = b->comp[b->job_comp[job]].steps[st];
            const int64_t units = tc_pack_units(d.M, d.N, d.K, (d.flags & FLAG_TF32) != 0, d.tile_rows);
            TcRange r{job, st, (int32_t)packs.size(), (int32_t)units, (int32_t)gemms.size(), d.ntiles};
            for (int64_t u = 0; u < units; ++u) packs.push_back({(uint32_t)job, (uint32_t)st, (uint32_t)u});
            for (int32_t t = 0; t < d.ntiles; ++t) gemms.push_back({(uint32_t)job, (uint32_t)st, (uint32_t)t});
            b->tc_ranges.push_back(r);
        };
        if (b->mode == TN_EXEC_PERSISTENT) {
            work.reserve((size_t)total);
            b->phases.assign(np, tn_batch::Phase());
            // order key of every step: its dependency level, or (critical path first) minus the
            // weight of its path to the root
            std::vector<std::vector<double>> key(b->comp.size());
            for (size_t ci = 0; ci < b->comp.size(); ++ci) {
                const Compiled &c = b->comp[ci];
                key[ci].assign(c.steps.size(), 0.0);
                if (ctx->cfg.schedule == 1) {
                    std::vector<double> path;
                    path_weights(c, path);
                    for (size_t st = 0; st < c.steps.size(); ++st) key[ci][st] = -path[st];
                } else {
                    for (size_t st = 0; st < c.steps.size(); ++st) key[ci][st] = c.steps[st].level;
                }
            }
            for (int32_t p = 0; p < np; ++p) {
                tn_batch::Phase &ph = b->phases[p];
                std::vector<std::tuple<double, int32_t, int32_t>> order;   // key, job, step
                for (int32_t i = 0; i < n; ++i) {
                    const Compiled &c = b->comp[b->job_comp[i]];
                    const std::vector<int32_t> &phs = phase_of[b->job_comp[i]];
                    for (size_t st = 0; st < c.steps.size(); ++st)
                        if (phs[st] == p && c.steps[st].kind != STEP_LOCAL && !(c.steps[st].flags & FLAG_CHAIN_CONT))
                            order.emplace_back(key[b->job_comp[i]][st], i, (int32_t)st);
                }
                std::sort(order.begin(), order.end());
                ph.pack0 = (int32_t)packs.size();
                ph.gemm0 = (int32_t)gemms.size();
                for (auto &o : order)
                    if (b->comp[b->job_comp[std::get<1>(o)]].steps[std::get<2>(o)].kind == STEP_TC)
                        add_tc(std::get<1>(o), std::get<2>(o));
                ph.n_pack = (int32_t)packs.size() - ph.pack0;
                ph.n_gemm = (int32_t)gemms.size() - ph.gemm0;
                for (auto &o : order) {
                    const int32_t job = std::get<1>(o), st = std::get<2>(o);
                    const Compiled &cj = b->comp[b->job_comp[job]];
                    const StepDesc &d = cj.steps[st];
                    if (d.kind == STEP_TC) continue;
                    for (int32_t t = 0; t < d.ntiles; ++t) {
                        work.push_back(dataflow_item(cj, (uint32_t)job, st, t));
                        work_phase.push_back(p);
                    }
                }
            }
        } else {
            for (int32_t i = 0; i < n; ++i) {
                const Compiled &c = b->comp[b->job_comp[i]];
                for (size_t st = 0; st < c.steps.size(); ++st)
                    if (c.steps[st].kind == STEP_TC) add_tc(i, (int32_t)st);
            }
        }
    }
    b->n_work = (int64_t)work.size();
    set_phase_ranges(b, work_phase);
    b->wait_ns = (long long)ctx->cfg.wait_limit_us * 1000;
    // warp programs first, longest first (a block of four warps lasts as long as its longest
    // program), then the block programs
    std::stable_sort(warp_items.begin(), warp_items.end(), [&](const WorkItem &x, const WorkItem &y) {
        const Compiled &cx = b->comp[b->job_comp[x.job]], &cy = b->comp[b->job_comp[y.job]];
        return cx.progs[cx.steps[x.step].tile_rows].n_steps > cy.progs[cy.steps[y.step].tile_rows].n_steps;
    });
    b->n_warp_items = (int32_t)warp_items.size();
    b->n_block_items = (int32_t)local_items.size();
    b->n_big_items = (int32_t)big_items.size();
    local_items.insert(local_items.begin(), warp_items.begin(), warp_items.end());
    local_items.insert(local_items.end(), big_items.begin(), big_items.end());
    const size_t o_work = carve(sizeof(WorkItem) * work.size());
    const size_t o_litems = carve(sizeof(WorkItem) * local_items.size());
    const size_t o_pack = carve(sizeof(WorkItem) * packs.size());
    const size_t o_gemm = carve(sizeof(WorkItem) * gemms.size());
    // reset region: results, maxbits, done, counter
    const size_t o_reset = off;
    const size_t o_res = carve(sizeof(DeviceResult) * (size_t)n);
    std::vector<size_t> o_max(n), o_done(n);
    for (int32_t i = 0; i < n; ++i) {
        const Compiled &c = b->comp[b->job_comp[i]];
        o_max[i] = carve(sizeof(uint32_t) * (size_t)c.n_nodes);
        o_done[i] = carve(sizeof(int32_t) * c.steps.size());
    }
    // per phase: the dataflow launch's claim counter and abort flag, the GEMM launch's abort flag
    const size_t o_counter = carve(3 * sizeof(uint32_t) * std::max<size_t>(b->phases.size(), 1));
    b->reset_bytes = off - o_reset;
    b->footprint = off;
    if (ctx->budget && b->footprint > ctx->budget) {
        batch_destroy(b);
        return fail(TN_EBUDGET, "the batch needs " + std::to_string(off) + " bytes of device memory");
    }
    cudaError_t e = cudaMalloc(&b->d_block, off);
    if (e != cudaSuccess) {
        batch_destroy(b);
        return fail(e == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA, cudaGetErrorString(e));
    }
    char *base = static_cast<char *>(b->d_block);
    for (size_t ci = 0; ci < b->comp.size(); ++ci) {
        b->comp[ci].d_steps = reinterpret_cast<StepDesc *>(base + o_steps[ci]);
        b->comp[ci].d_leaf_off = reinterpret_cast<int64_t *>(base + o_loff[ci]);
        b->comp[ci].d_progs = reinterpret_cast<LocalProg *>(base + o_progs[ci]);
        b->comp[ci].d_lsteps = reinterpret_cast<LocalStep *>(base + o_lsteps[ci]);
        b->comp[ci].d_leafrefs = reinterpret_cast<LeafRef *>(base + o_lrefs[ci]);
        b->comp[ci].d_lwaves = reinterpret_cast<LocalWave *>(base + o_lwaves[ci]);
        b->comp[ci].d_ktab = reinterpret_cast<int2 *>(base + o_ktab[ci]);
    }
    b->d_leaf64 = reinterpret_cast<double2 *>(base + o_leaf64);
    char *d_leaf = base + o_leaf;
    b->d_jobs = reinterpret_cast<JobPtrs *>(base + o_jobs);
    b->d_work = reinterpret_cast<WorkItem *>(base + o_work);
    b->d_local = reinterpret_cast<WorkItem *>(base + o_litems);
    b->d_pack = reinterpret_cast<WorkItem *>(base + o_pack);
    b->d_gemm = reinterpret_cast<WorkItem *>(base + o_gemm);
    b->d_reset = base + o_reset;
    b->d_res = reinterpret_cast<DeviceResult *>(base + o_res);
    b->d_counter = reinterpret_cast<uint32_t *>(base + o_counter);
    b->jobs.resize(n);
    for (int32_t i = 0; i < n; ++i) {
        const Compiled &c = b->comp[b->job_comp[i]];
        JobPtrs &j = b->jobs[i];
        j.leaf64 = b->d_leaf64 + b->leaf64_off[i];
        j.leaf_off = c.d_leaf_off;
        j.leaf = d_leaf + (size_t)b->elem * (size_t)b->leaf64_off[i];
        j.arena = base + o_arena[i];
        j.partials = reinterpret_cast<double2 *>(base + o_part[i]);
        j.exp2 = reinterpret_cast<int32_t *>(base + o_exp[i]);
        j.maxbits = reinterpret_cast<uint32_t *>(base + o_max[i]);
        j.done = reinterpret_cast<int32_t *>(base + o_done[i]);
        j.result = b->d_res + i;
        j.steps = c.d_steps;
        j.progs = c.d_progs;
        j.lsteps = c.d_lsteps;
        j.leafrefs = c.d_leafrefs;
        j.lwaves = c.d_lwaves;
        j.ktab = c.d_ktab;
        j.n_steps = (int32_t)c.steps.size();
        j.n_leaves = c.n;
    }
    if (cudaMallocHost(&b->h_pinned, std::max((size_t)16, sizeof(double2) * (size_t)leaf_total)) != cudaSuccess ||
        cudaMallocHost(&b->h_res, sizeof(DeviceResult) * (size_t)n) != cudaSuccess) {
        batch_destroy(b);
        return fail(TN_ENOMEM, "pinned host buffers");
    }
    cudaStream_t st = ctx->stream;
    for (size_t ci = 0; ci < b->comp.size() && e == cudaSuccess; ++ci) {
        const Compiled &c = b->comp[ci];
        if (!c.steps.empty())
            e = cudaMemcpyAsync(c.d_steps, c.steps.data(), sizeof(StepDesc) * c.steps.size(),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c.d_leaf_off, c.leaf_off.data(), sizeof(int64_t) * c.leaf_off.size(),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !c.progs.empty())
            e = cudaMemcpyAsync(c.d_progs, c.progs.data(), sizeof(LocalProg) * c.progs.size(),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !c.lsteps.empty())
            e = cudaMemcpyAsync(c.d_lsteps, c.lsteps.data(), sizeof(LocalStep) * c.lsteps.size(),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !c.leafrefs.empty())
            e = cudaMemcpyAsync(c.d_leafrefs, c.leafrefs.data(), sizeof(LeafRef) * c.leafrefs.size(),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !c.lwaves.empty())
            e = cudaMemcpyAsync(c.d_lwaves, c.lwaves.data(), sizeof(LocalWave) * c.lwaves.size(),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !c.ktab.empty())
            e = cudaMemcpyAsync(c.d_ktab, c.ktab.data(), sizeof(int2) * c.ktab.size(), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_jobs, b->jobs.data(), sizeof(JobPtrs) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !work.empty())
        e = cudaMemcpyAsync(b->d_work, work.data(), sizeof(WorkItem) * work.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !local_items.empty())
        e = cudaMemcpyAsync(b->d_local, local_items.data(), sizeof(WorkItem) * local_items.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !packs.empty())
        e = cudaMemcpyAsync(b->d_pack, packs.data(), sizeof(WorkItem) * packs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !gemms.empty())
        e = cudaMemcpyAsync(b->d_gemm, gemms.data(), sizeof(WorkItem) * gemms.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e != cudaSuccess) { batch_destroy(b); return fail(TN_ECUDA, cudaGetErrorString(e)); }
    b->h_work = std::move(work);
    b->h_work_phase = std::move(work_phase);
    b->grid = persistent_grid(b->c128);
    if (b->grid <= 0) { batch_destroy(b); return fail(TN_ECUDA, "occupancy query failed"); }
    tn_status s = TN_OK;
    for (int32_t i = 0; i < n && s == TN_OK; ++i) s = upload_leaves(b, i);
    if (s == TN_OK && b->mode == TN_EXEC_GRAPH) s = record_graph(b);
    b->replay = b->mode == TN_EXEC_PERSISTENT && ctx->cfg.graph_capture != 0;
    if (s == TN_OK && b->replay) s = record_persistent_graph(b);
    if (s == TN_OK) {
        e = cudaStreamSynchronize(st);   // the uploads read host buffers that must stay alive
        if (e != cudaSuccess) s = fail(TN_ECUDA, cudaGetErrorString(e));
    }
    if (s != TN_OK) { batch_destroy(b); return s; }
    // run statistics
    b->info = tn_run_info{};
    for (int32_t i = 0; i < n; ++i) {
        const Compiled &c = b->comp[b->job_comp[i]];
        b->info.flops += c.flops;
        b->info.bytes += c.bytes;
        b->info.bytes_warp += c.bytes_cls[0];
        b->info.bytes_block += c.bytes_cls[1];
        b->info.bytes_tc += c.bytes_cls[2];
        b->info.bytes_flow += c.bytes_cls[3];
        b->info.n_gather += c.counts[STEP_ROWS];
        b->info.n_tile += c.counts[STEP_TILE];
        b->info.n_dot += c.counts[STEP_DOTP];
        b->info.n_tc += c.counts[STEP_TC];
        b->info.n_local += c.counts[STEP_LOCAL] - c.counts[7];
        b->info.n_local_steps += c.counts[6] + c.counts[8];
        b->info.n_warp_progs += c.counts[7];
    }
    b->info.dyn_smem = b->dyn_smem;
    b->info.arena_bytes = b->arena_total;
    if (b->mode == TN_EXEC_PERSISTENT) {
        // leaf conversion, warp programs, block programs, large programs; per phase the pack,
        // GEMM and dataflow launches
        b->info.launches = 1 + (b->n_warp_items > 0 ? 1 : 0) + (b->n_block_items > 0 ? 1 : 0) +
                           (b->n_big_items > 0 ? 1 : 0);
        for (const tn_batch::Phase &ph : b->phases)
            b->info.launches += (ph.n_pack > 0) + (ph.n_gemm > 0) + (ph.n_work > 0);
    } else {
        int32_t l = 1;
        for (int32_t i = 0; i < n; ++i) {
            const Compiled &c = b->comp[b->job_comp[i]];
            l += (int32_t)c.steps.size() + c.counts[STEP_TC];   // a tensor-core step: pack and GEMM
        }
        b->info.launches = l;
    }
    for (int32_t i = 0; i < n; ++i)
        if (b->comp[b->job_comp[i]].n == 1) b->info.launches++;
    *out = b;
    return TN_OK;
}

// Copy the pending tensor updates to the device in one transfer and scatter them into the
// resident complex128 leaves.
tn_status apply_updates(tn_batch *b, cudaStream_t st) {
    tn_batch::Stage &sg = b->stage[b->cur_stage];
    const size_t n_upd = sg.hdr.size / (3 * sizeof(int64_t));
    if (n_upd == 0) return TN_OK;
    const size_t hdr_bytes = align_up(sg.hdr.size, 16);
    const size_t bytes = hdr_bytes + sg.val.size;
    if (bytes > b->d_upd_cap) {
        if (b->d_upd) cudaFree(b->d_upd);
        b->d_upd = nullptr;
        b->d_upd_cap = 0;
        cudaError_t e = cudaMalloc(&b->d_upd, bytes);
        if (e != cudaSuccess) return fail(TN_ENOMEM, cudaGetErrorString(e));
        b->d_upd_cap = bytes;
    }
    if (!sg.ev) CK(cudaEventCreateWithFlags(&sg.ev, cudaEventDisableTiming));
    CK(cudaMemcpyAsync(b->d_upd, sg.hdr.p, sg.hdr.size, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->d_upd + hdr_bytes, sg.val.p, sg.val.size, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(sg.ev, st));
    sg.copying = true;
    CK(launch_scatter_updates(reinterpret_cast<const int64_t *>(b->d_upd),
                              reinterpret_cast<const double2 *>(b->d_upd + hdr_bytes), (int64_t)n_upd,
                              b->d_leaf64, st));
    b->last_h2d += bytes;
    sg.hdr.size = 0;
    sg.val.size = 0;
    b->cur_stage ^= 1;
    return TN_OK;
}

tn_status batch_run(tn_batch *b, void *d_results) {
    CK(cudaSetDevice(b->ctx->device));
    cudaStream_t st = b->ctx->stream;
    bool synced = false;
    b->last_h2d = 0;
    for (int32_t i = 0; i < b->n_jobs; ++i)
        if (b->uploaded[i] != b->nets[i]->impl.version) {
            if (!synced) { CK(cudaStreamSynchronize(st)); synced = true; }   // staging in flight
            tn_status s = upload_leaves(b, i);
            if (s != TN_OK) return s;
            b->last_h2d += sizeof(double) * b->nets[i]->impl.data.size();
        }
    {
        tn_status s = apply_updates(b, st);
        if (s != TN_OK) return s;
    }
    CK(cudaEventRecord(b->ev0, st));
    if (b->mode == TN_EXEC_GRAPH) {
        CK(cudaGraphLaunch(b->gexec, st));
    } else if (b->replay) {
        std::vector<cudaEvent_t> &ev = b->kev[b->runs % tn_batch::kRing];
        CK(ensure_events(ev, 2));
        CK(cudaEventRecord(ev[0], st));
        CK(cudaGraphLaunch(b->pgexec, st));
        CK(cudaEventRecord(ev[1], st));
        b->runs++;
    } else {
        const cudaError_t e = enqueue_run(b, st);
        if (e != cudaSuccess)
            return fail(TN_ECUDA, std::string("run (") + t_enqueue_stage + "): " + cudaGetErrorString(e));
    }
    CK(cudaEventRecord(b->ev1, st));
    if (d_results && d_results != (void *)b->d_res)
        CK(cudaMemcpyAsync(d_results, b->d_res, sizeof(DeviceResult) * (size_t)b->n_jobs,
                           cudaMemcpyDeviceToDevice, st));
    b->ran = true;
    return TN_OK;
}

tn_status batch_info(tn_batch *b, tn_run_info *info) {
    b->info.h2d_bytes = (double)b->last_h2d;
    if (b->ran) {
        CK(cudaSetDevice(b->ctx->device));
        CK(cudaEventSynchronize(b->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        b->info.device_ms = ms;
    }
    *info = b->info;
    return TN_OK;
}

// Copy the results to the host (blocking).
tn_status batch_results(tn_batch *b, double *amps, int32_t *exp2, int32_t *status) {
    CK(cudaSetDevice(b->ctx->device));
    cudaStream_t st = b->ctx->stream;
    CK(cudaMemcpyAsync(b->h_res, b->d_res, sizeof(DeviceResult) * (size_t)b->n_jobs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool timeout = false;
    for (int32_t i = 0; i < b->n_jobs; ++i) {
        const DeviceResult &r = b->h_res[i];
        if (amps) { amps[2 * i] = r.re; amps[2 * i + 1] = r.im; }
        if (exp2) exp2[i] = r.exp2;
        if (status) status[i] = r.status;
        if (r.status != 0) timeout = true;
    }
    if (timeout && !status) return fail(TN_ETIMEOUT, "a device-side wait gave up");
    return TN_OK;
}

}  // namespace

extern "C" {

tn_status tn_ctx_create(int32_t device, void *cuda_stream, size_t hbm_budget_bytes, tn_ctx **out) {
    if (!out) return fail(TN_EINVAL, "out is NULL");
    int count = 0;
    CK(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(TN_ECUDA, "no such CUDA device");
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(TN_ECUDA, "this library targets sm_103a (GB300); device is sm_" +
                                  std::to_string(prop.major) + std::to_string(prop.minor));
    CK(cudaSetDevice(device));
    tn_ctx *c = new (std::nothrow) tn_ctx;
    if (!c) return fail(TN_ENOMEM, "allocating the context");
    c->device = device;
    c->budget = hbm_budget_bytes;
    c->mode = TN_EXEC_PERSISTENT;
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return fail(TN_ECUDA, cudaGetErrorString(e)); }
        c->own_stream = true;
    }
    *out = c;
    return TN_OK;
}

tn_status tn_plan_compile_stats(const tn_net *net, const tn_plan *plan, tn_precision prec,
                                int32_t local_budget, tn_compile_stats *out) {
    if (!net || !plan || !out) return fail(TN_EINVAL, "NULL argument");
    if (prec < TN_C128 || prec > TN_BF16_SPLIT) return fail(TN_EINVAL, "unknown precision");
    if (plan->impl.n != net->impl.n) return fail(TN_EINVAL, "plan and network do not match");
    if (!net->impl.closed) return fail(TN_EUNSUPPORTED, "open networks are not supported by tn_contract");
    Compiled c;
    tn_status s = compile(c, net->impl, plan->impl, stats_opts(prec, local_budget));
    if (s != TN_OK) return s;
    tn_compile_stats st;
    std::memset(&st, 0, sizeof(st));
    st.global_steps = (int32_t)c.steps.size();
    st.n_rows = c.counts[STEP_ROWS];
    st.n_tile = c.counts[STEP_TILE];
    st.n_dot = c.counts[STEP_DOTP];
    st.n_local = c.counts[STEP_LOCAL] - c.counts[7];
    st.n_local_steps = c.counts[6];
    st.n_warp_progs = c.counts[7];
    st.n_warp_steps = c.counts[8];
    st.n_chained = 0;
    for (const StepDesc &d : c.steps) st.n_chained += (d.flags & FLAG_CHAIN_CONT) ? 1 : 0;
    st.max_local_smem = c.dyn_smem;
    st.total_tiles = c.total_tiles;
    st.arena_bytes = c.arena_bytes;
    st.flops = c.flops;
    st.bytes = c.bytes;
    int32_t lv = 0;
    for (const StepDesc &d : c.steps) lv = std::max(lv, d.level);
    st.levels = lv;
    *out = st;
    return TN_OK;
}

tn_status tn_plan_compile_steps(const tn_net *net, const tn_plan *plan, tn_precision prec,
                                int32_t local_budget, int64_t *out, int32_t cap, int32_t *n_out) {
    if (!net || !plan || !n_out) return fail(TN_EINVAL, "NULL argument");
    if (prec < TN_C128 || prec > TN_BF16_SPLIT) return fail(TN_EINVAL, "unknown precision");
    if (plan->impl.n != net->impl.n) return fail(TN_EINVAL, "plan and network do not match");
    if (!net->impl.closed) return fail(TN_EUNSUPPORTED, "open networks are not supported by tn_contract");
    Compiled c;
    tn_status s = compile(c, net->impl, plan->impl, stats_opts(prec, local_budget));
    if (s != TN_OK) return s;
    const int32_t n = (int32_t)c.steps.size();
    for (int32_t i = 0; i < n && i < cap && out; ++i) {
        const StepDesc &d = c.steps[i];
        int64_t *r = out + 8 * (int64_t)i;
        r[0] = d.kind; r[1] = d.M; r[2] = d.N; r[3] = d.K; r[4] = d.ntiles; r[5] = d.level;
        r[6] = d.kind == STEP_LOCAL ? c.progs[d.tile_rows].n_steps : (d.kind == STEP_ROWS ? d.chain_next : 0);
        r[7] = d.kind == STEP_LOCAL ? c.progs[d.tile_rows].smem_bytes : 0;
    }
    *n_out = n;
    return TN_OK;
}

namespace {
void drop_cached(tn_ctx *c) {
    if (c->cached) {
        cudaSetDevice(c->device);
        cudaStreamSynchronize(c->stream);
        batch_destroy(c->cached);
        c->cached = nullptr;
    }
}
}  // namespace

tn_status tn_ctx_set_local_budget(tn_ctx *c, int32_t bytes) {
    if (!c) return fail(TN_EINVAL, "NULL ctx");
    if (bytes < -1) return fail(TN_EINVAL, "bytes must be -1 (automatic), 0 (off) or positive");
    drop_cached(c);
    c->cfg.local_budget = bytes;
    return TN_OK;
}

tn_status tn_ctx_get_config(const tn_ctx *c, tn_exec_config *cfg) {
    if (!c || !cfg) return fail(TN_EINVAL, "NULL argument");
    *cfg = c->cfg;
    return TN_OK;
}

tn_status tn_ctx_set_config(tn_ctx *c, const tn_exec_config *cfg) {
    if (!c || !cfg) return fail(TN_EINVAL, "NULL argument");
    if (cfg->local_budget < -1 || cfg->tc_min_m < 1 || cfg->tc_min_n < 1 || cfg->tc_min_k < 1 ||
        cfg->wait_limit_us < 1)
        return fail(TN_EINVAL, "invalid configuration");
    drop_cached(c);
    c->cfg = *cfg;
    c->cfg.big_programs = cfg->big_programs ? 1 : 0;
    c->cfg.warp_programs = cfg->warp_programs ? 1 : 0;
    c->cfg.rows_chains = cfg->rows_chains ? 1 : 0;
    c->cfg.graph_capture = cfg->graph_capture ? 1 : 0;
    if (cfg->schedule < 0 || cfg->schedule > 1) return fail(TN_EINVAL, "schedule must be 0 or 1");
    if (cfg->tc_tile_n != 0 && cfg->tc_tile_n != 64 && cfg->tc_tile_n != 128)
        return fail(TN_EINVAL, "tc_tile_n must be 0, 64 or 128");
    return TN_OK;
}

tn_status tn_ctx_set_exec_mode(tn_ctx *c, int32_t mode) {
    if (!c) return fail(TN_EINVAL, "NULL ctx");
    if (mode != TN_EXEC_PERSISTENT && mode != TN_EXEC_GRAPH) return fail(TN_EINVAL, "unknown mode");
    if (c->mode != mode && c->cached) {
        cudaSetDevice(c->device);
        cudaStreamSynchronize(c->stream);
        batch_destroy(c->cached);
        c->cached = nullptr;
    }
    c->mode = mode;
    return TN_OK;
}

void tn_ctx_free(tn_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    tn_batch *cached = c->cached;
    c->cached = nullptr;
    c->freed = true;
    c->refs.fetch_add(1);      // keep the context alive while its cached batch is destroyed
    batch_destroy(cached);
    ctx_release(c);            // deletes it now unless other batches, programs or servers remain
}

tn_status tn_ctx_device(const tn_ctx *c, int32_t *device) {
    if (!c || !device) return fail(TN_EINVAL, "NULL argument");
    *device = c->device;
    return TN_OK;
}

tn_status tn_ctx_synchronize(tn_ctx *c) {
    if (!c) return fail(TN_EINVAL, "NULL ctx");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    return TN_OK;
}

tn_status tn_program_create(tn_ctx *ctx, const tn_net *net, const tn_plan *plan, tn_precision prec,
                            tn_program **out) {
    if (!ctx || !net || !plan || !out) return fail(TN_EINVAL, "NULL argument");
    tn_program *p = new (std::nothrow) tn_program;
    if (!p) return fail(TN_ENOMEM, "allocating the program");
    tn_status s = batch_create(ctx, 1, &net, &plan, prec, &p->b);
    if (s != TN_OK) { delete p; return s; }
    *out = p;
    return TN_OK;
}

tn_status tn_program_run(tn_program *p, void *d_result) {
    if (!p || !d_result) return fail(TN_EINVAL, "NULL argument");
    return batch_run(p->b, d_result);
}

tn_status tn_program_footprint(const tn_program *p, size_t *bytes) {
    if (!p || !bytes) return fail(TN_EINVAL, "NULL argument");
    *bytes = p->b->footprint;
    return TN_OK;
}

tn_status tn_program_last_info(const tn_program *p, tn_run_info *info) {
    if (!p || !info) return fail(TN_EINVAL, "NULL argument");
    return batch_info(p->b, info);
}

void tn_program_free(tn_program *p) {
    if (!p) return;
    cudaSetDevice(p->b->ctx->device);
    cudaStreamSynchronize(p->b->ctx->stream);
    batch_destroy(p->b);
    delete p;
}

tn_status tn_batch_create(tn_ctx *ctx, int32_t n, const tn_net *const *nets, const tn_plan *const *plans,
                          tn_precision prec, tn_batch **out) {
    return batch_create(ctx, n, nets, plans, prec, out);
}

tn_status tn_batch_run(tn_batch *b, void *d_results) {
    if (!b) return fail(TN_EINVAL, "NULL batch");
    return batch_run(b, d_results);
}

tn_status tn_batch_results(tn_batch *b, double *amps, int32_t *exp2, int32_t *status) {
    if (!b) return fail(TN_EINVAL, "NULL batch");
    return batch_results(b, amps, exp2, status);
}

tn_status tn_batch_set_profiling(tn_batch *b, int32_t on) {
    if (!b) return fail(TN_EINVAL, "NULL batch");
    CK(cudaSetDevice(b->ctx->device));
    CK(cudaStreamSynchronize(b->ctx->stream));
    if (on && !b->d_prof) {
        CK(cudaMalloc(&b->d_prof, sizeof(long long) * 2 * kProfSlots));
        CK(cudaMemset(b->d_prof, 0, sizeof(long long) * 2 * kProfSlots));
    } else if (!on && b->d_prof) {
        cudaFree(b->d_prof);
        b->d_prof = nullptr;
    }
    if (b->replay) return record_persistent_graph(b);   // the launches' profiling pointer changed
    return TN_OK;
}

tn_status tn_batch_profile(tn_batch *b, int64_t *cycles, int64_t *items) {
    if (!b || !cycles || !items) return fail(TN_EINVAL, "NULL argument");
    if (!b->d_prof) return fail(TN_EINVAL, "profiling is off (tn_batch_set_profiling)");
    CK(cudaSetDevice(b->ctx->device));
    CK(cudaStreamSynchronize(b->ctx->stream));
    long long h[2 * kProfSlots];
    CK(cudaMemcpy(h, b->d_prof, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < kProfSlots; ++i) { cycles[i] = h[i]; items[i] = h[kProfSlots + i]; }
    return TN_OK;
}

tn_status tn_batch_debug_hold(tn_batch *b, int32_t job, int32_t step) {
    if (!b) return fail(TN_EINVAL, "NULL batch");
    if (b->mode != TN_EXEC_PERSISTENT) return fail(TN_EINVAL, "only the persistent mode has a work list");
    if (job >= b->n_jobs) return fail(TN_EINVAL, "job index out of range");
    std::vector<std::pair<int32_t, int32_t>> held;
    if (job >= 0) {
        for (const auto &h : b->held)
            if (h.first != job) held.push_back(h);
        if (step >= 0) {
            bool found = false;
            for (const WorkItem &w : b->h_work) found = found || ((int32_t)w.job == job && (int32_t)w.step == step);
            if (!found) return fail(TN_EINVAL, "the step has no tile in the persistent work list");
            for (const auto &h : b->held)
                if (h.first == job) held.push_back(h);
            held.push_back({job, step});
        }
    }
    std::vector<WorkItem> kept;
    std::vector<int32_t> kept_phase;
    kept.reserve(b->h_work.size());
    for (size_t i = 0; i < b->h_work.size(); ++i) {
        const WorkItem &w = b->h_work[i];
        bool drop = false;
        for (const auto &h : held) drop = drop || ((int32_t)w.job == h.first && (int32_t)w.step == h.second);
        if (!drop) {
            kept.push_back(w);
            kept_phase.push_back(b->h_work_phase[i]);
        }
    }
    CK(cudaSetDevice(b->ctx->device));
    CK(cudaStreamSynchronize(b->ctx->stream));
    if (!kept.empty()) CK(cudaMemcpy(b->d_work, kept.data(), sizeof(WorkItem) * kept.size(), cudaMemcpyHostToDevice));
    b->n_work = (int64_t)kept.size();
    set_phase_ranges(b, kept_phase);
    b->held.swap(held);
    if (b->replay) return record_persistent_graph(b);   // the launches' work counts changed
    return TN_OK;
}

// Grow a pinned staging buffer to hold `need` bytes, keeping its contents.
static tn_status pinned_reserve(tn_batch::Pinned &buf, size_t need) {
    if (need <= buf.cap) return TN_OK;
    size_t cap = std::max<size_t>(need, 2 * buf.cap);
    char *p = nullptr;
    cudaError_t e = cudaMallocHost(&p, cap);
    if (e != cudaSuccess) return fail(TN_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    if (buf.size) std::memcpy(p, buf.p, buf.size);
    if (buf.p) cudaFreeHost(buf.p);
    buf.p = p;
    buf.cap = cap;
    return TN_OK;
}

tn_status tn_batch_set_tensors(tn_batch *b, int32_t count, const int32_t *job, const int32_t *tensor,
                               const double *data) {
    if (!b || (count > 0 && (!job || !tensor || !data))) return fail(TN_EINVAL, "NULL argument");
    if (count < 0) return fail(TN_EINVAL, "count must be >= 0");
    // validate everything first: a rejected call stages nothing
    size_t n_val = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (job[i] < 0 || job[i] >= b->n_jobs) return fail(TN_EINVAL, "job index out of range");
        const Compiled &c = b->comp[b->job_comp[job[i]]];
        if (tensor[i] < 0 || tensor[i] >= c.n) return fail(TN_EINVAL, "tensor index out of range");
        n_val += 2 * (size_t)(c.leaf_off[tensor[i] + 1] - c.leaf_off[tensor[i]]);
    }
    if (count == 0) return TN_OK;
    if (!entries_in_range(data, n_val))
        return fail(TN_EINVAL, "tensor entries must be finite and below 2^127 in magnitude");
    tn_batch::Stage &sg = b->stage[b->cur_stage];
    if (sg.copying) {   // the copy out of this set, two runs ago, must be done before it is refilled
        CK(cudaSetDevice(b->ctx->device));
        CK(cudaEventSynchronize(sg.ev));
        sg.copying = false;
    }
    tn_status s = pinned_reserve(sg.hdr, sg.hdr.size + 3 * sizeof(int64_t) * (size_t)count);
    if (s == TN_OK) s = pinned_reserve(sg.val, sg.val.size + sizeof(double) * n_val);
    if (s != TN_OK) return s;
    int64_t *hdr = reinterpret_cast<int64_t *>(sg.hdr.p + sg.hdr.size);
    double *val = reinterpret_cast<double *>(sg.val.p + sg.val.size);
    int64_t vpos = (int64_t)(sg.val.size / (2 * sizeof(double)));   // complex entries staged so far
    size_t src = 0;
    for (int32_t i = 0; i < count; ++i) {
        const Compiled &c = b->comp[b->job_comp[job[i]]];
        const int64_t off = c.leaf_off[tensor[i]], cnt = c.leaf_off[tensor[i] + 1] - off;
        hdr[3 * i] = b->leaf64_off[job[i]] + off;
        hdr[3 * i + 1] = cnt;
        hdr[3 * i + 2] = vpos;
        std::memcpy(val, data + src, sizeof(double) * 2 * (size_t)cnt);
        val += 2 * cnt;
        src += 2 * (size_t)cnt;
        vpos += cnt;
    }
    sg.hdr.size += 3 * sizeof(int64_t) * (size_t)count;
    sg.val.size += sizeof(double) * n_val;
    return TN_OK;
}

tn_status tn_batch_footprint(const tn_batch *b, size_t *bytes) {
    if (!b || !bytes) return fail(TN_EINVAL, "NULL argument");
    *bytes = b->footprint;
    return TN_OK;
}

tn_status tn_batch_last_info(const tn_batch *b, tn_run_info *info) {
    if (!b || !info) return fail(TN_EINVAL, "NULL argument");
    return batch_info(const_cast<tn_batch *>(b), info);
}

tn_status tn_batch_kernel_ms(const tn_batch *b, int32_t n_runs, double *mean_ms) {
    if (!b || !mean_ms) return fail(TN_EINVAL, "NULL argument");
    if (b->mode != TN_EXEC_PERSISTENT) return fail(TN_EUNSUPPORTED, "only the persistent mode is timed per run");
    if (n_runs < 1 || n_runs > tn_batch::kRing || n_runs > b->runs)
        return fail(TN_EINVAL, "n_runs must be in [1, min(256, runs so far)]");
    CK(cudaSetDevice(b->ctx->device));
    double total = 0;
    const size_t n_ev = b->replay ? 2 : 3 + 3 * b->phases.size();
    for (int64_t r = b->runs - n_runs; r < b->runs; ++r) {
        const std::vector<cudaEvent_t> &ev = b->kev[r % tn_batch::kRing];
        if (ev.size() < n_ev) return fail(TN_EINVAL, "no timing of that run");
        CK(cudaEventSynchronize(ev[n_ev - 1]));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ev[0], ev[n_ev - 1]));
        total += ms;
    }
    *mean_ms = total / n_runs;
    return TN_OK;
}

tn_status tn_batch_kernel_times(const tn_batch *b, int32_t n_runs, double *mean_ms) {
    if (!b || !mean_ms) return fail(TN_EINVAL, "NULL argument");
    if (b->mode != TN_EXEC_PERSISTENT) return fail(TN_EUNSUPPORTED, "only the persistent mode is timed per run");
    if (n_runs < 1 || n_runs > tn_batch::kRing || n_runs > b->runs)
        return fail(TN_EINVAL, "n_runs must be in [1, min(256, runs so far)]");
    CK(cudaSetDevice(b->ctx->device));
    double acc[5] = {0, 0, 0, 0, 0};
    const size_t n_ev = 3 + 3 * b->phases.size();
    if (b->replay) n_runs = 1;   // the graph's events time its last replay
    for (int64_t r = b->runs - n_runs; r < b->runs; ++r) {
        const std::vector<cudaEvent_t> &ev = b->replay ? b->gev : b->kev[r % tn_batch::kRing];
        if (ev.size() < n_ev) return fail(TN_EINVAL, "no timing of that run");
        CK(cudaEventSynchronize(ev[n_ev - 1]));
        for (size_t i = 0; i + 1 < n_ev; ++i) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            // slots: 0 warp programs, 1 block and large programs, then (pack, GEMM, dataflow) per phase
            const int cls = i < 2 ? (int)i : 2 + (int)((i - 2) % 3);
            acc[cls] += ms;
        }
    }
    for (int c = 0; c < 5; ++c) mean_ms[c] = acc[c] / n_runs;
    return TN_OK;
}

void tn_batch_free(tn_batch *b) {
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    if (b->ctx->cached == b) b->ctx->cached = nullptr;
    batch_destroy(b);
}

tn_status tn_contract(tn_ctx *ctx, const tn_net *net, const tn_plan *plan, tn_precision prec,
                      double out_amp[2], int32_t *out_exp2, tn_run_info *info) {
    if (!ctx || !net || !plan || !out_amp || !out_exp2) return fail(TN_EINVAL, "NULL argument");
    CK(cudaSetDevice(ctx->device));
    if (!(ctx->cached && ctx->cached_net == net->impl.uid && ctx->cached_plan == plan->impl.uid &&
          ctx->cached_prec == prec)) {
        if (ctx->cached) {
            cudaStreamSynchronize(ctx->stream);
            batch_destroy(ctx->cached);
            ctx->cached = nullptr;
        }
        tn_batch *b = nullptr;
        tn_status s = batch_create(ctx, 1, &net, &plan, prec, &b);
        if (s != TN_OK) return s;
        ctx->cached = b;
        ctx->cached_net = net->impl.uid;
        ctx->cached_plan = plan->impl.uid;
        ctx->cached_prec = prec;
    }
    tn_batch *b = ctx->cached;
    b->nets[0] = net;               // the same net (by id); refresh the address
    b->uploaded[0] = ~0ull;         // end to end: the leaves are copied from the host every call
    tn_status s = batch_run(b, nullptr);
    if (s != TN_OK) return s;
    double amp[2];
    int32_t e2 = 0;
    s = batch_results(b, amp, &e2, nullptr);
    if (s != TN_OK) return s;
    out_amp[0] = amp[0];
    out_amp[1] = amp[1];
    *out_exp2 = e2;
    if (info) return batch_info(b, info);
    return TN_OK;
}

tn_status tn_batch_contract(tn_ctx *ctx, int32_t n, const tn_net *const *nets, const tn_plan *const *plans,
                            tn_precision prec, double *out_amps, int32_t *out_exp2) {
    if (!out_amps || !out_exp2) return fail(TN_EINVAL, "NULL output");
    tn_batch *b = nullptr;
    tn_status s = batch_create(ctx, n, nets, plans, prec, &b);
    if (s != TN_OK) return s;
    s = batch_run(b, nullptr);
    if (s == TN_OK) s = batch_results(b, out_amps, out_exp2, nullptr);
    tn_batch_free(b);
    return s;
}

tn_status tn_permute(tn_ctx *ctx, const void *d_in, void *d_out, int32_t elem_bytes, int32_t rank,
                     const int64_t *dims, const int32_t *perm) {
    if (!ctx || (!d_in && rank > 0) || !d_out || (rank > 0 && (!dims || !perm)))
        return fail(TN_EINVAL, "NULL argument");
    if (rank < 0 || rank > 32) return fail(TN_EINVAL, "rank must be in [0, 32]");
    if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16)
        return fail(TN_EINVAL, "elem_bytes must be 1, 2, 4, 8 or 16");
    std::vector<int> seen(rank, 0);
    for (int32_t t = 0; t < rank; ++t) {
        if (perm[t] < 0 || perm[t] >= rank || seen[perm[t]]) return fail(TN_EINVAL, "perm is not a permutation");
        seen[perm[t]] = 1;
        if (dims[t] < 1) return fail(TN_EINVAL, "dims must be >= 1");
    }
    CK(cudaSetDevice(ctx->device));
    CK(launch_permute(d_in, d_out, elem_bytes, rank, dims, perm, ctx->stream));
    return TN_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------ autotuner

tn_status tn_ctx_autotune(tn_ctx *ctx, int32_t n, const tn_net *const *nets, const tn_plan *const *plans,
                          tn_precision prec, int32_t runs, tn_exec_config *out_best, double *out_ms,
                          double *cand_ms, int32_t cap, int32_t *n_cand) {
    if (!ctx || n < 1 || !nets || !plans || runs < 1 || cap < 0) return fail(TN_EINVAL, "invalid argument");
    if (prec < TN_C128 || prec > TN_BF16_SPLIT) return fail(TN_EINVAL, "unknown precision");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(TN_ECUDA, "cudaSetDevice");
    const bool c128 = prec == TN_C128;
    // candidates: program kinds on and off, block budgets for two and three blocks per SM, no
    // programs; in the split precisions the tensor-core thresholds too
    const int32_t b3 = local_smem_budget(c128, 3);
    std::vector<tn_exec_config> cands = {
        {-1, 1, 1, 64, 32, 16, 1}, {-1, 0, 1, 64, 32, 16, 1}, {-1, 0, 1, 64, 32, 16, 0},
        {-1, 1, 0, 64, 32, 16, 1}, {b3, 1, 1, 64, 32, 16, 1}, {b3, 0, 1, 64, 32, 16, 1},
        {0, 0, 0, 64, 32, 16, 1}};
    if (tc_mode_of(prec)) {
        const int32_t off = 1 << 30;
        cands.push_back({-1, 1, 1, off, off, off, 1});
        cands.push_back({-1, 0, 1, off, off, off, 1});
        cands.push_back({-1, 1, 1, 32, 32, 16, 1});
        cands.push_back({-1, 0, 1, 32, 32, 16, 1});
    }
    const tn_exec_config saved = ctx->cfg;
    drop_cached(ctx);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(TN_ECUDA, "cudaEventCreate");
    }
    double best_ms = -1;
    int32_t best = -1;
    tn_status first_err = TN_OK;
    std::string first_msg;
    for (tn_exec_config &c : cands) {
        c.wait_limit_us = saved.wait_limit_us;
        c.graph_capture = saved.graph_capture;
        c.schedule = 1;
        c.tc_tile_n = 0;
    }
    {   // the dependency-level order with the default program configuration
        tn_exec_config lv = cands[1];
        lv.schedule = 0;
        cands.push_back(lv);
    }
    if (tc_mode_of(prec)) {   // 128-column tiles for every dense step
        tn_exec_config wide = cands[1];
        wide.tc_tile_n = 128;
        cands.push_back(wide);
    }
    for (size_t i = 0; i < cands.size(); ++i) {
        ctx->cfg = cands[i];
        tn_batch *b = nullptr;
        double ms = -1;
        tn_status s = batch_create(ctx, n, nets, plans, prec, &b);
        if (s == TN_OK) {
            for (int w = 0; w < 2 && s == TN_OK; ++w) s = batch_run(b, nullptr);
            if (s == TN_OK && cudaEventRecord(e0, ctx->stream) == cudaSuccess) {
                for (int32_t r = 0; r < runs && s == TN_OK; ++r) s = batch_run(b, nullptr);
                float t = 0.f;
                if (s == TN_OK && cudaEventRecord(e1, ctx->stream) == cudaSuccess &&
                    cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
                    ms = (double)t / runs;
            }
            batch_destroy(b);
        }
        if (s != TN_OK && first_err == TN_OK) {
            first_err = s;
            first_msg = tn_last_error();
        }
        if (cand_ms && (int32_t)i < cap) cand_ms[i] = ms;
        if (ms > 0 && (best < 0 || ms < best_ms)) {
            best_ms = ms;
            best = (int32_t)i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_cand) *n_cand = (int32_t)cands.size();
    if (best < 0) {
        ctx->cfg = saved;
        return fail(first_err == TN_OK ? TN_ECUDA : first_err, "autotune: no candidate ran: " + first_msg);
    }
    ctx->cfg = cands[best];
    if (out_best) *out_best = cands[best];
    if (out_ms) *out_ms = best_ms;
    return TN_OK;
}
