// Program compilation shared by the batch executor and the serving loop.
#pragma once

#include <cstdint>
#include <vector>

#include "kernels.cuh"
#include "tn_internal.hpp"

namespace tn {

struct Compiled {
    std::vector<StepDesc> steps;
    std::vector<LocalProg> progs;
    std::vector<LocalStep> lsteps;
    std::vector<LeafRef> leafrefs;
    std::vector<LocalWave> lwaves;
    std::vector<int64_t> leaf_off;   // [n + 1] element offsets of the leaves
    int32_t n = 0, n_nodes = 0;
    size_t arena_bytes = 0;
    int64_t n_partials = 0;          // double2 entries
    int64_t total_tiles = 0;
    int32_t dyn_smem = 0;            // largest shared-memory need of a local program
    double flops = 0, bytes = 0;
    // by StepKind ([5] = block programs); [6] = steps inside block programs; [7] = warp programs,
    // [8] = steps inside warp programs
    int32_t counts[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t plan_uid = 0, shape_hash = 0;
    // device copies (inside the batch's allocation)
    StepDesc *d_steps = nullptr;
    int64_t *d_leaf_off = nullptr;
    LocalProg *d_progs = nullptr;
    LocalStep *d_lsteps = nullptr;
    LeafRef *d_leafrefs = nullptr;
    LocalWave *d_lwaves = nullptr;
};


// Compile (network structure, plan) for complex elements of `elem` bytes: the global dataflow
// step list, the CTA-resident subtree programs (maximal subtrees whose working set fits
// `local_budget` bytes of shared memory; 0 = none) and the arena plan of one contraction.
// use_tc: dense steps go to the tensor cores (BF16 split).
tn_status compile(Compiled &c, const Net &net, const Plan &plan, int32_t elem, int32_t local_budget,
                  bool use_tc);

// Sorted work items (level, step, tile) of one compiled structure, subtree programs excluded.
void work_template(const Compiled &c, std::vector<WorkItem> &items, std::vector<int32_t> &item_level);

}  // namespace tn
