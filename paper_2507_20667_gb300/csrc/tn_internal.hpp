// Internal host-side data structures shared by the planner, the program compiler and the C ABI.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "tnsa.h"

namespace tn {

using u128 = unsigned __int128;
using i128 = __int128;

// Thread-local error message (tn_last_error) and status plumbing.
tn_status fail(tn_status s, const std::string &msg);
void set_error(const std::string &msg);

inline tn_u128 to_abi(u128 x) { return tn_u128{(uint64_t)x, (uint64_t)(x >> 64)}; }

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

}  // namespace tn

struct tn_net { tn::Net impl; };
struct tn_plan { tn::Plan impl; };
