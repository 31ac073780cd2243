// Internal host-side data structures shared by the planner, the program compiler and the C ABI.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "tnsa.h"
#include "fanin_core.cuh"

namespace tn {

using u128 = unsigned __int128;
using i128 = __int128;

// Thread-local error message (tn_last_error) and status plumbing.
tn_status fail(tn_status s, const std::string &msg);
void set_error(const std::string &msg);

inline tn_u128 to_abi(u128 x) { return tn_u128{(uint64_t)x, (uint64_t)(x >> 64)}; }

// Tensor entries the engine accepts: finite, with |Re| and |Im| below 2^127.  The per-step scaling
// tracks each tensor's max-abs in FP32, so larger leaf entries (possible only in complex128) would
// saturate it; intermediates of any size are fine (every step rescales its operands).
constexpr double kMaxEntry = 170141183460469231731687303715884105728.0;   // 2^127
inline bool entries_in_range(const double *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(p[i] < kMaxEntry && p[i] > -kMaxEntry)) return false;   // NaN fails both
    return true;
}

// Sorted set of edge ids (the legs of a tensor, Eq. 2.2 / Eq. 2.6).
using Legs = std::vector<int32_t>;

// A network as given to tn_build (Eq. 2.1).
struct Net {
    int32_t n = 0;                       // tensors
    int32_t n_edges = 0;
    std::vector<int32_t> degree;
    std::vector<int64_t> dim_off;        // [n+1] offsets into dims
    std::vector<int64_t> dims;           // concatenated dims
    std::vector<int64_t> data_off;       // [n+1] offsets (complex elements) into data
    std::vector<double> data;            // complex128 interleaved
    std::vector<tn_edge> edges;
    std::vector<int64_t> edim;           // dimension of each edge
    std::vector<std::vector<int32_t>> axis_edge;  // edge id of each axis of each tensor
    std::vector<Legs> legs;              // sorted legs of each tensor
    bool closed = true;
    uint64_t version = 0;                // bumped by tn_net_set_tensor
    uint64_t uid = 0;                    // unique per created net (addresses can be reused)
};

// Saturating products of edge dimensions; `ovf` is set on overflow of 2^120.
u128 legs_size(const Legs &l, const std::vector<int64_t> &edim, bool &ovf);
u128 union_size(const Legs &a, const Legs &b, const std::vector<int64_t> &edim, bool &ovf);
void legs_symdiff(const Legs &a, const Legs &b, Legs &out);
bool legs_intersect(const Legs &a, const Legs &b);

// Result of the Greedy rule over a set of tensors (local ids 0..s-1, new nodes s, s+1, ...).
struct GreedyTree {
    std::vector<std::pair<int32_t, int32_t>> steps;   // (smaller local id, larger local id)
    u128 con = 0;          // sum of 2^vc over its internal nodes (Eq. 3.2)
    u128 mem = 0;          // Eq. 3.1 restricted to this tree
    Legs root_legs;
    u128 root_size = 0;
};
GreedyTree greedy_tree(const std::vector<const Legs *> &init, const std::vector<int64_t> &edim,
                       bool &ovf);

// Fan-in tree over the k partition results (Section 4.4).
struct FanIn {
    std::vector<std::pair<int32_t, int32_t>> steps;   // over local ids 0..k-1, new nodes k, ...
    u128 con_dist = 0;     // Eq. 3.5 with con = con_serial, comm = 0
    u128 con = 0;          // sum of the fan-in nodes' 2^vc
    u128 mem = 0;
};
FanIn fanin_tree(const std::vector<Legs> &roots, const std::vector<u128> &part_con,
                 const std::vector<int64_t> &edim, int samples, uint64_t seed, bool &ovf);

// A fan-in problem in the shared bitset form (fanin_core.cuh): the k roots' legs over compact
// edge ids (the union of the roots' legs, in increasing edge order), their dimensions, the
// partition results' con and the sampling seed.
struct FaninInput {
    int32_t k = 0, W = 0;
    bool unit = true;                   // every compact edge has dimension 2
    std::vector<uint64_t> roots;        // [k][W]
    std::vector<int64_t> dims;          // [64 W] (empty when unit)
    std::vector<u128> part_con;         // [k]
    uint64_t seed = 0;
};
void fanin_input(const std::vector<Legs> &roots, const std::vector<u128> &part_con,
                 const std::vector<int64_t> &edim, uint64_t seed, FaninInput &in);
// The fan-in tree on the host: every merge order for k <= 4, else the best of `samples`
// RandomGreedy samples; `sample` >= 0 evaluates that single sample only (k > 4).
FanIn fanin_host(const FaninInput &in, int samples, int sample, bool &ovf);

// The best sample of a batched evaluation.
struct FaninBest {
    fanin::Counts counts{0, 0, 0, false};
    int32_t sample = 0;
};
// Device buffers and stream kept across batched evaluations.
struct FaninWorkspace {
    void *d_buf = nullptr, *h_buf = nullptr, *stream = nullptr;
    size_t cap = 0;
};
// Batched fan-in evaluation on a CUDA device (k > 4): bit-identical to fanin_host.
tn_status fanin_eval_device(int32_t device, const std::vector<FaninInput> &ins, int32_t samples,
                            std::vector<FaninBest> &result, FaninWorkspace &ws);
void fanin_workspace_free(FaninWorkspace &ws);

struct Plan {
    int32_t n = 0, k = 1;
    std::vector<int32_t> part;                       // partition of each tensor
    std::vector<std::array<int32_t, 3>> steps;       // (left, right, out) global node ids
    std::vector<int32_t> step_part;                  // partition of each step, -1 = fan-in
    std::vector<int32_t> part_root;                  // node id of root(B_k)
    u128 con_serial = 0, con_dist = 0, con_par = 0, mem = 0, init_con_dist = 0;
    int32_t sa_iterations = 0, sa_accepted = 0, sa_restarts = 0;
    double plan_seconds = 0;
    uint64_t uid = 0;                    // unique per created plan
};

uint64_t next_uid();

// Recompute all counts of a plan from its steps (Eq. 3.1-3.5); checks tree and acceptance.
tn_status plan_finalize(const Net &net, Plan &plan);

tn_status plan_run(const Net &net, const tn_plan_opts &opts, Plan &out);

// EvaluateState (Section 4.4) for many partitions at once: each state's Greedy partition trees
// (host threads) and fan-in tree (on `device` in one batched launch when k > 4 and device >= 0,
// else on the host); the counts of the plan the planner would assemble from it.
struct StateCounts {
    u128 con_serial = 0, con_dist = 0, mem = 0;
    bool saturated = false;     // some size or cost reached 2^120: the counts are lower bounds
};
tn_status eval_states(const Net &net, int32_t k, int32_t samples, int32_t device, int32_t n_states,
                      const int32_t *parts, std::vector<StateCounts> &out);

}  // namespace tn

struct tn_net { tn::Net impl; };
struct tn_plan { tn::Plan impl; };
