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
    std::vector<int2> ktab;          // shared-index offset tables of DOTP steps
    std::vector<int64_t> leaf_off;   // [n + 1] element offsets of the leaves
    int32_t n = 0, n_nodes = 0;
    size_t arena_bytes = 0;
    int64_t n_partials = 0;          // double2 entries
    int64_t total_tiles = 0;
    int32_t dyn_smem = 0;            // largest shared-memory need of a block (or warp) program
    int32_t dyn_big = 0;             // largest shared-memory need of a large program
    double flops = 0, bytes = 0;
    // algorithmic bytes by the kernel class that executes the step: [0] warp programs, [1] block
    // and large programs, [2] tensor-core GEMM, [3] dataflow kernel
    double bytes_cls[4] = {0, 0, 0, 0};
    // by StepKind ([5] = all programs); [6] = steps inside block and large programs; [7] = warp
    // programs, [8] = steps inside warp programs; [9] = large programs
    int32_t counts[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t plan_uid = 0, shape_hash = 0;
    // device copies (inside the batch's allocation)
    StepDesc *d_steps = nullptr;
    int64_t *d_leaf_off = nullptr;
    LocalProg *d_progs = nullptr;
    LocalStep *d_lsteps = nullptr;
    LeafRef *d_leafrefs = nullptr;
    LocalWave *d_lwaves = nullptr;
    int2 *d_ktab = nullptr;
};


// What the compiler may use.  Programs: warp programs (maximal subtrees of small steps), block
// programs (maximal subtrees whose working set fits local_budget bytes of shared memory; 0 = no
// programs at all) and large programs (maximal subtrees within big_budget bytes, inputs staged
// when consumed; none if big_budget <= local_budget).  tc_mode: dense steps (M >= tc_min_m,
// N >= tc_min_n, K >= tc_min_k) go to the tensor cores, 1 = BF16 split, 2 = TF32 split.
// rows_chains: link chains of ROWS steps that the persistent kernel runs with the tensor kept in
// shared memory.
struct CompileOpts {
    int32_t elem = 8;                 // bytes per complex element (8: complex64, 16: complex128)
    int32_t local_budget = 0;
    int32_t big_budget = 0;
    bool warp_programs = true;
    int32_t tc_mode = 0;
    int32_t tc_min_m = 64, tc_min_n = 32, tc_min_k = 16;
    int32_t tc_tile_n = 0;            // dense-step tile width: 0 automatic (64 if N <= 64), 64, 128
    bool rows_chains = true;
};

// Compile (network structure, plan): the global dataflow step list, the subtree programs and the
// arena plan of one contraction.
tn_status compile(Compiled &c, const Net &net, const Plan &plan, const CompileOpts &o);

// Reference counting of contexts by the objects made from them (tn_ctx_free defers the delete).
void ctx_retain(tn_ctx *c);
void ctx_release(tn_ctx *c);

// Tensor-core mode of a precision (0: CUDA cores only).
int32_t tc_mode_of(int32_t prec);

// Compiler options of an execution configuration on the current device.
CompileOpts compile_opts(const tn_exec_config &cfg, int32_t prec, bool c128);

// The dataflow work item of tile `tile` of step `step` (with the step's dependencies).
WorkItem dataflow_item(const Compiled &c, uint32_t job, int32_t step, int32_t tile);

// Weight of the path from every global step to the root: the sum of M N K (2^vc of Eq. 3.3) over
// the step and its consumers up to the root -- the path sums whose maximum over the leaves is
// con_par (Eq. 3.4).  Programs count as zero.
void path_weights(const Compiled &c, std::vector<double> &path);

// Dependency phases.  A dense tensor-core step runs in its own pack and GEMM launches, so the
// persistent dataflow launches are cut at them: phase(TC step) = 1 + the largest phase of its
// producers, phase(other step) = the largest phase of its producers (programs: 0).  A run is, for
// p = 0, 1, ...: the pack and GEMM launches of the TC steps of phase p (none for p = 0), then the
// persistent launch of the other steps of phase p.  Returns the number of phases.
int32_t step_phases(const Compiled &c, std::vector<int32_t> &phase);

// Per phase of one compiled structure (job index 0): the dataflow work items sorted by (level,
// step, tile) with their levels, the pack units and the GEMM tiles of its tensor-core steps.
struct PhaseTemplate {
    std::vector<WorkItem> work;
    std::vector<int32_t> level;
    std::vector<WorkItem> pack, gemm;
};
void phase_templates(const Compiled &c, std::vector<PhaseTemplate> &out);

// The pack units and GEMM tiles of one tensor-core step of one job, as ranges of a run's lists.
struct TcRange {
    int32_t job, step, pack0, n_pack, gemm0, n_gemm;
};

}  // namespace tn
