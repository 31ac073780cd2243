/*
 * tnsa.h -- C ABI of the GB300 engine that contracts a quantum-circuit tensor network split into
 * k partitions (arXiv 2507.20667, "Optimizing tensor network partitioning using Simulated
 * Annealing").  Plain C types only: host or device pointers, sizes, status codes.
 *
 * Conventions used by every entry point
 *   - Status codes only; no exceptions cross the ABI.  On any status other than TN_OK the
 *     out-parameters are left untouched and tn_last_error() returns a message for this thread.
 *   - Handles (tn_net, tn_plan, tn_ctx, tn_program) are owned by the caller and released with the
 *     matching *_free.  Nets and plans are immutable after creation and may be shared between
 *     threads; a tn_ctx (and every tn_program made from it) is bound to one device and one CUDA
 *     stream and is not thread-safe.
 *   - Complex numbers are interleaved (re, im).  Tensors are row-major: axis 0 is the slowest.
 *   - Amplitudes are returned as a mantissa and a power of two: value = (re + i im) * 2^exp2.
 *   - Operation counts can exceed 2^64, so they are returned as unsigned 128-bit integers.
 *   - No entry point falls back to the CPU: compute entry points fail with TN_ECUDA when no
 *     usable sm_103a device is present.
 */
#ifndef TNSA_H
#define TNSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TN_OK = 0,
    TN_EINVAL = 1,        /* malformed network, plan, option or argument */
    TN_ENOMEM = 2,        /* host or device allocation failed */
    TN_EBUDGET = 3,       /* the plan's device footprint exceeds the context's budget */
    TN_ECUDA = 4,         /* a CUDA call failed or no usable device */
    TN_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    TN_EUNSUPPORTED = 6   /* valid request outside what this library supports */
} tn_status;

/* Arithmetic used for the pairwise contractions.
 *   TN_C128        complex128 everywhere (correctness variant, CUDA cores).
 *   TN_C64         complex64 storage and arithmetic (CUDA cores).
 *   TN_TF32_SPLIT  complex64 storage; dense steps on tensor cores with a 3-term TF32 hi/lo split.
 *   TN_BF16_SPLIT  complex64 storage; dense steps on tensor cores with a 3-term BF16 hi/lo split,
 *                  FP32 accumulation.
 * In every mode the last, scalar-producing contraction accumulates in FP64. */
typedef enum { TN_C128 = 0, TN_C64 = 1, TN_TF32_SPLIT = 2, TN_BF16_SPLIT = 3 } tn_precision;

/* Target selection of the simulated-annealing move (Algorithm 2). */
typedef enum { TN_SA_NAIVE = 0, TN_SA_DIRECTED = 1 } tn_sa_mode;

/* One edge ((u, a), (v, b)) of Eq. 2.1, 0-based axes.  v = -1 is the dummy vertex (an open leg);
 * b is then ignored. */
typedef struct { int32_t u, a, v, b; } tn_edge;

typedef struct { uint64_t lo, hi; } tn_u128;

typedef struct tn_net tn_net;
typedef struct tn_plan tn_plan;
typedef struct tn_ctx tn_ctx;
typedef struct tn_program tn_program;
typedef struct tn_batch tn_batch;

/* ------------------------------------------------------------------ networks (Section 2.1) */

/* Build a network (Eq. 2.1-2.3).
 *   n_tensors  number of tensors |V| >= 1
 *   degree     [n_tensors] degree d_v >= 0 of each tensor (0 = scalar)
 *   dims       concatenation of every tensor's dims n_v (sum of degree entries, each >= 1)
 *   data       concatenation of every tensor's entries, complex128 interleaved (re, im),
 *              row-major; 2 * sum_v |T_v| doubles, each finite and below 2^127 in magnitude
 *              (each tensor's max-abs is tracked in FP32 by the per-step scaling;
 *              intermediates may grow without bound)
 *   n_edges, edges  the edge list; every (u, a) slot must be named exactly once, the dims at both
 *              ends must agree (n_{u,a} = n_{v,b}), and u != v (no self-loops).  Several edges
 *              between the same two tensors are allowed.
 * The arrays are copied; the caller keeps ownership of its buffers.
 * Errors: TN_EINVAL for any violation above or an element count above 2^62; TN_ENOMEM. */
tn_status tn_build(int32_t n_tensors, const int32_t *degree, const int64_t *dims,
                   const double *data, int32_t n_edges, const tn_edge *edges, tn_net **out);

/* Replace the entries of tensor t (same shape), e.g. a new bitstring's bra tensors.
 * data: |T_t| complex128 interleaved, each part finite and below 2^127 in magnitude.  Programs
 * built from this net pick the change up at their next run (the leaves are re-uploaded).
 * Errors: TN_EINVAL. */
tn_status tn_net_set_tensor(tn_net *net, int32_t t, const double *data);

/* Number of tensors, edges, and whether every leg is bound (a closed network). */
tn_status tn_net_info(const tn_net *net, int32_t *n_tensors, int32_t *n_edges, int32_t *closed);
void tn_net_free(tn_net *net);

/* ------------------------------------------------------------------ planning (Sections 3-4) */

typedef struct {
    int32_t k;                  /* number of partitions, 1 <= k <= n_tensors */
    int32_t mode;               /* tn_sa_mode; default TN_SA_DIRECTED */
    double T0, Tf;              /* initial / final temperature of Eq. 4.3-4.4 (log-cost units) */
    int32_t steps_per_temp;     /* N of Algorithm 1 (split as ceil(N/p) per thread) */
    int32_t threads;            /* p of Algorithm 1 (division algorithm); >= 1 */
    double time_limit_s;        /* > 0: time-based cooling, t = elapsed / limit */
    int32_t iterations;         /* used when time_limit_s <= 0: t = i / iterations */
    int32_t restart_threshold;  /* RestartThreshold of Algorithm 1 */
    int32_t fanin_samples;      /* RandomGreedy samples for the fan-in tree (k > 4) */
    uint64_t seed;
    int32_t initial;            /* tn_initial: how the initial partition (Section 4.2) is formed */
    int32_t pad0;
    const int32_t *initial_part;/* TN_INIT_GIVEN: [n_tensors] initial partition in [0, k).
                                   Read during tn_plan_create only. */
    const int32_t *position;    /* TN_INIT_QUBIT_BLOCK: [n_tensors] position hint of each tensor,
                                   >= 0 (for a circuit: the qubit the tensor sits on, a 2-qubit
                                   gate on its lower qubit).  Read during tn_plan_create only. */
    int32_t fanin_device;       /* >= 0: for k > 4 the RandomGreedy fan-in trees of every annealing
                                   step are evaluated on this CUDA device, the chains advancing in
                                   lockstep with one batched launch per step (the plan is the same
                                   as with host evaluation); -1: on the host */
    int32_t pad1;
} tn_plan_opts;

/* Initial partition of the annealing (Section 4.2 starts from a hypergraph partitioner's cut; this
 * library forms one of its own):
 *   TN_INIT_BFS          k balanced regions: breadth-first order from tensor 0 (restarting in
 *                        unvisited components), cut into k contiguous chunks of near-equal size
 *   TN_INIT_QUBIT_BLOCK  k contiguous blocks of positions: tensor t goes to partition
 *                        floor(position[t] * k / P) with P = max(position) + 1 (for grid
 *                        circuits numbered row-major these are blocks of rows)
 *   TN_INIT_GIVEN        initial_part as given */
typedef enum { TN_INIT_BFS = 0, TN_INIT_QUBIT_BLOCK = 1, TN_INIT_GIVEN = 2 } tn_initial;

/* Fill opts with the defaults: k = 1, DIRECTED, T0 = 0.1, Tf = 0.001, N = 8, p = 1,
 * iterations = 200, RestartThreshold = 50, 32 fan-in samples, seed = 0, initial = TN_INIT_BFS,
 * initial_part = position = NULL, fanin_device = -1. */
void tn_plan_opts_default(tn_plan_opts *opts);

/* Plan a contraction (Section 4): initial partition, simulated-annealing refinement
 * (Algorithms 1 and 2) minimising con_dist (Eq. 3.5 with con = con_serial and no communication
 * term, Section 4.4 and 5.2), a Greedy tree per partition and a fan-in tree over the partition
 * results (exhaustive for k <= 4, RandomGreedy above).  With k = 1 the plan is the Greedy tree.
 * Deterministic for a given seed when time_limit_s <= 0.
 * Errors: TN_EINVAL (bad k or options; TN_INIT_GIVEN without initial_part or with an entry outside
 * [0, k); TN_INIT_QUBIT_BLOCK without position or with a negative entry; an initial partition
 * with an empty part), TN_ENOMEM. */
tn_status tn_plan_create(const tn_net *net, const tn_plan_opts *opts, tn_plan **out);

/* Wrap a caller-chosen tree as a plan.  steps: [n_steps][2] (left, right) node ids, where leaves
 * are 0..n-1 and step s creates node n + s; n_steps must be n - 1.  part: [n] partition of each
 * tensor in [0, k) (NULL means k = 1).  Errors: TN_EINVAL if the steps do not form one binary
 * tree over all tensors or the tree does not accept the partition (Eq. 2.7). */
tn_status tn_plan_import(const tn_net *net, int32_t k, const int32_t *part, int32_t n_steps,
                         const int32_t *steps, tn_plan **out);

/* What the program compiler makes of (net, plan, precision) with a given shared-memory budget for
 * subtree programs (see tn_ctx_set_local_budget; here 0 = none and > 0 = that many bytes), without
 * touching a device.  Errors: TN_EINVAL, TN_EUNSUPPORTED (open network). */
typedef struct {
    int32_t global_steps;      /* entries of the global dataflow step list */
    int32_t n_rows, n_tile, n_dot, n_local;   /* global steps per kernel class; subtree programs */
    int32_t n_local_steps;     /* pairwise steps executed inside subtree programs */
    int32_t max_local_smem;    /* largest shared-memory need of a subtree program (bytes) */
    int32_t levels;            /* dependency levels of the global step list */
    int64_t total_tiles;       /* work tiles of one contraction */
    size_t arena_bytes;        /* device memory for intermediates of one contraction */
    double flops, bytes;       /* algorithmic flops (8 * con_serial) and bytes of one contraction */
    int32_t n_warp_progs;      /* warp programs: subtrees of small steps run by one warp each */
    int32_t n_warp_steps;      /* pairwise steps executed inside warp programs */
    int32_t n_chained;         /* ROWS steps run as continuations of a chain (rows_chains of
                                  tn_exec_config, on here) */
    int32_t pad;
} tn_compile_stats;
tn_status tn_plan_compile_stats(const tn_net *net, const tn_plan *plan, tn_precision prec,
                                int32_t local_budget, tn_compile_stats *out);

/* The global step list the compiler produces (same inputs as tn_plan_compile_stats): for each
 * entry 8 int64 {kernel class (0 ROWS, 1 TILE, 2 DOTP, 3 DOTF, 5 subtree program), M, N, K,
 * work tiles, dependency level, program steps (ROWS: the entry that continues it in a chain, -1
 * none), program shared-memory bytes}.  At most cap entries
 * are written to out (may be NULL); *n_out receives the full count.  Errors: as compile_stats. */
tn_status tn_plan_compile_steps(const tn_net *net, const tn_plan *plan, tn_precision prec,
                                int32_t local_budget, int64_t *out, int32_t cap, int32_t *n_out);

/* Exact counts of the plan's tree B (Section 3):
 *   total_ops = con_serial(B) (Eq. 3.2), crit_ops = con_dist(B, K) (Eq. 3.5, con = con_serial,
 *   comm = 0), mem_elems = mem(B) (Eq. 3.1).  Any pointer may be NULL. */
tn_status tn_plan_counts(const tn_plan *plan, tn_u128 *total_ops, tn_u128 *crit_ops,
                         tn_u128 *mem_elems);

/* EvaluateState (Section 4.4) for many candidate states at once: for each of n_states partitions
 * of the network into k parts (parts: [n_states][n_tensors], entries in [0, k), no part empty) the
 * counts of the plan tn_plan_create would assemble from it -- a Greedy tree per partition and the
 * fan-in tree over the partition results (every merge order for k <= 4, else the best of
 * fanin_samples RandomGreedy samples) -- written to con_serial, con_dist and mem ([n_states]
 * each, Eq. 3.2, 3.5, 3.1; any may be NULL).  device >= 0 evaluates the fan-in trees of k > 4 on
 * that CUDA device in one batched launch, device = -1 on the host; both give the same counts,
 * which equal tn_plan_counts of tn_plan_create with the state as TN_INIT_GIVEN and no annealing.
 * saturated ([n_states], may be NULL) is set to 1 for a state whose sizes or costs reach 2^120
 * (its counts are then lower bounds).
 * Errors: TN_EINVAL (bad k or parts), TN_EUNSUPPORTED (device evaluation of k > 256 or of more
 * than 2048 cut legs), TN_ECUDA, TN_ENOMEM. */
tn_status tn_plan_eval_states(const tn_net *net, int32_t k, int32_t fanin_samples, int32_t device,
                              int32_t n_states, const int32_t *parts, tn_u128 *con_serial,
                              tn_u128 *con_dist, tn_u128 *mem, int32_t *saturated);

typedef struct {
    tn_u128 con_serial, con_dist, con_par, mem; /* Eq. 3.2, 3.5, 3.4, 3.1 */
    tn_u128 initial_con_dist;                   /* con_dist of the initial partition */
    int32_t k, n_steps;
    int32_t sa_iterations, sa_accepted, sa_restarts;
    double plan_seconds;
} tn_plan_info;
tn_status tn_plan_get_info(const tn_plan *plan, tn_plan_info *info);

/* Export the plan.  part_of_tensor: [n_tensors]; steps: [n_steps][3] (left, right, out) with the
 * node numbering of tn_plan_import (partition 0's steps first, ..., fan-in steps last);
 * step_part: [n_steps] partition of each step, -1 for fan-in steps.  Any array may be NULL;
 * *n_steps receives n_tensors - 1. */
tn_status tn_plan_export(const tn_plan *plan, int32_t *part_of_tensor, int32_t *steps,
                         int32_t *step_part, int32_t *n_steps);
void tn_plan_free(tn_plan *plan);

/* Slicing on top of partitioning (Section 4.1; Section 6 names it as the way past the memory
 * limit).  Fixing the index of every edge of a set S splits the contraction into prod_{e in S} n(e)
 * slices, each the same network with n(e) = 1 on S, contracted along the plan's tree; the value is
 * the sum of the slices.  tn_plan_slice chooses S greedily for the plan's tree: while its mem
 * (Eq. 3.1) is above target_mem elements and fewer than max_edges are chosen, it slices the leg of
 * the peak-memory step (the step maximising |v| + |c1| + |c2| and its children's legs) that lowers
 * mem the most (ties: fewer total operations, then the smaller edge id).  Writes the chosen edge
 * ids to edges (increasing, at most max_edges), their number to *n_edges, and the counts: slices,
 * per-slice con_serial (Eq. 3.2) and mem, and the total operations of all slices (slices x
 * per-slice; the excess over the unsliced con_serial is the redundant work).  Counts may be NULL.
 * Errors: TN_EINVAL, TN_EUNSUPPORTED (more than 2^100 slices). */
tn_status tn_plan_slice(const tn_net *net, const tn_plan *plan, tn_u128 target_mem, int32_t max_edges,
                        int32_t *edges, int32_t *n_edges, tn_u128 *n_slices, tn_u128 *slice_con,
                        tn_u128 *slice_mem, tn_u128 *total_con);

/* ------------------------------------------------------------------ contraction on the GPU */

/* Create a context on `device` that enqueues on `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream).  hbm_budget_bytes bounds the device memory a program may use (0 = no bound).
 * Errors: TN_ECUDA (no sm_103a device), TN_ENOMEM. */
tn_status tn_ctx_create(int32_t device, void *cuda_stream, size_t hbm_budget_bytes, tn_ctx **out);
void tn_ctx_free(tn_ctx *ctx);

/* Block until all work enqueued on the context's stream has finished.  Errors: TN_ECUDA. */
tn_status tn_ctx_synchronize(tn_ctx *ctx);

/* The CUDA device of the context.  Errors: TN_EINVAL. */
tn_status tn_ctx_device(const tn_ctx *ctx, int32_t *device);

/* How programs and batches made from the context execute their steps.
 *   TN_EXEC_PERSISTENT (default)  one persistent dataflow kernel per run: every step is cut into
 *       work tiles; resident blocks claim tiles in dependency-level order across all jobs, wait
 *       (bounded, ~4 s) for the steps producing their operands, run the tile and publish it.
 *   TN_EXEC_GRAPH  one kernel launch per step and job, recorded once into a CUDA graph.
 * Takes effect for programs and batches created afterwards.  Errors: TN_EINVAL. */
typedef enum { TN_EXEC_PERSISTENT = 0, TN_EXEC_GRAPH = 1 } tn_exec_mode;
tn_status tn_ctx_set_exec_mode(tn_ctx *ctx, int32_t mode);

/* Shared memory (bytes) a CTA-resident subtree program may use.  The compiler runs every maximal
 * subtree of the contraction tree whose sequential working set -- its leaves plus the
 * intermediates alive at any one time -- fits this budget inside one thread block, entirely in
 * shared memory; only the subtree's result goes to device memory.  -1 (default): the largest
 * budget that keeps two blocks per SM; 0: no subtree programs (every step is a global step).
 * Takes effect for programs and batches created afterwards.  Errors: TN_EINVAL. */
tn_status tn_ctx_set_local_budget(tn_ctx *ctx, int32_t bytes);

/* Execution configuration of a context (applies to programs, batches and servers created
 * afterwards; the autotuner below picks one by measurement).
 *   local_budget     as tn_ctx_set_local_budget: shared memory per block program, -1 automatic
 *                    (two blocks per SM), 0 no subtree programs of any kind
 *   big_programs     1: large programs -- maximal subtrees that fit the shared memory of one block
 *                    per SM, each input staged when it is consumed (fan-in chains); 0: none
 *   warp_programs    1: warp programs -- subtrees of small steps run by one warp each; 0: none
 *   tc_min_m/n/k     in the split precisions, a dense step runs on the tensor cores when
 *                    M >= tc_min_m, N >= tc_min_n and K >= tc_min_k
 *   rows_chains      1: a chain of narrow dataflow steps, each consuming the previous one's output
 *                    as its large operand, runs in one block of the persistent kernel with the
 *                    tensor kept in shared memory between the steps (complex64 storage); 0: every
 *                    step writes its output to the arena.  Results are bit-identical either way.
 *   wait_limit_us    how long (microseconds, >= 1) a work tile of the persistent kernel waits for
 *                    the steps producing its operands before it gives up: the tile is skipped, its
 *                    job's status becomes TN_ETIMEOUT, and a launch-wide abort flag makes every
 *                    later wait of the launch give up at once, so the launch ends.  The context
 *                    stays usable.
 *   graph_capture    1: a batch (or program) in the persistent mode records one run -- the reset,
 *                    the leaf conversion and every launch -- into a CUDA graph at creation and
 *                    replays it (one graph launch per run); its per-class kernel times
 *                    (tn_batch_kernel_times) are then those of the last replay.  0: the launches
 *                    are issued one by one every run.
 *   schedule         order of the persistent kernel's work list (every order is a topological one,
 *                    so the claim-in-order scheme stays deadlock-free): 0 by dependency level (all
 *                    jobs' level-1 tiles, then level 2, ...); 1 critical path first: by decreasing
 *                    weight of the path from the step to the root, sum of 2^vc (the path sums of
 *                    Eq. 3.4, whose maximum is con_par), so the steps on the longest weighted
 *                    paths are claimed first.
 *   tc_tile_n        output tile width of the tensor-core steps, complex columns: 64 or 128; 0
 *                    chooses 64 for a step with N <= 64 and 128 otherwise
 * Defaults: {-1, 0, 1, 64, 32, 16, 1, 4000000, 1, 1, 0} (large programs off: on the 24-qubit
 * brickwork benchmark they measured slower than running fan-in chains as dataflow steps; critical
 * path first, about 1 % faster there than the level order).
 * Errors: TN_EINVAL. */
typedef struct {
    int32_t local_budget;
    int32_t big_programs;
    int32_t warp_programs;
    int32_t tc_min_m, tc_min_n, tc_min_k;
    int32_t rows_chains;
    int32_t wait_limit_us;
    int32_t graph_capture;
    int32_t schedule;
    int32_t tc_tile_n;
} tn_exec_config;
tn_status tn_ctx_get_config(const tn_ctx *ctx, tn_exec_config *cfg);
tn_status tn_ctx_set_config(tn_ctx *ctx, const tn_exec_config *cfg);

/* Autotuner: for the batch (n, nets, plans, prec) -- the same arguments as tn_batch_create --
 * build a batch under each candidate configuration (program kinds on and off, block-program
 * budgets for two and three blocks per SM, no programs, ROWS chains off, the critical-path-first
 * work order; in the split precisions also tensor-core thresholds and the tensor-core tile width
 * -- the tile shapes of the dense steps), time `runs` runs of each with CUDA events after warm-up, keep the fastest
 * configuration in the context and return it.  out_ms (may be NULL) receives its mean device time
 * per run; cand_ms (may be NULL, cap entries) the mean time of every candidate in the order tried,
 * with *n_cand the number of candidates (failed ones: a negative time).  Errors: TN_EINVAL, those
 * of tn_batch_create when no candidate builds. */
tn_status tn_ctx_autotune(tn_ctx *ctx, int32_t n, const tn_net *const *nets, const tn_plan *const *plans,
                          tn_precision prec, int32_t runs, tn_exec_config *out_best, double *out_ms,
                          double *cand_ms, int32_t cap, int32_t *n_cand);

typedef struct {
    double device_ms;          /* device time of the contraction (CUDA events) */
    int32_t launches;          /* kernels launched */
    int32_t n_gather, n_tile, n_dot, n_tc;  /* steps per kernel class */
    double flops;              /* algorithmic flops, 8 * con_serial */
    double bytes;              /* algorithmic bytes: sum over steps of (|A|+|B|+|C|) * element size */
    size_t arena_bytes;        /* device memory held for intermediates */
    double h2d_bytes;          /* host-to-device bytes copied by the last run (leaf uploads) */
    int32_t n_local;           /* CTA-resident subtree programs (one block each) */
    int32_t n_local_steps;     /* steps executed inside subtree and warp programs */
    int32_t dyn_smem;          /* dynamic shared memory per block of the contraction kernels */
    int32_t n_warp_progs;      /* warp programs (one warp each) */
    /* the algorithmic bytes above split by the kernel class that executes each step: warp
     * programs, block and large programs, tensor-core GEMM, persistent dataflow kernel */
    double bytes_warp, bytes_block, bytes_tc, bytes_flow;
} tn_run_info;

/* Compile (net, plan, precision) into a device program: per-step layouts, index maps, kernel
 * classes, a static memory plan for all intermediates, the leaves uploaded to the device.
 * The net and plan must outlive the program; tn_net_set_tensor changes are uploaded by the next
 * tn_program_run.
 * Errors: TN_EBUDGET (footprint above the budget), TN_EUNSUPPORTED (open network), TN_ECUDA. */
tn_status tn_program_create(tn_ctx *ctx, const tn_net *net, const tn_plan *plan, tn_precision prec,
                            tn_program **out);

/* Enqueue one contraction on the context's stream without waiting.  d_result is DEVICE memory of
 * at least 32 bytes, receiving {double re, double im, int32 exp2, int32 status}.  The program's
 * leaves and intermediates stay resident between runs.  Errors: TN_ECUDA. */
tn_status tn_program_run(tn_program *prog, void *d_result);

/* Bytes of device memory the program holds (leaves + intermediates + descriptors). */
tn_status tn_program_footprint(const tn_program *prog, size_t *bytes);
tn_status tn_program_last_info(const tn_program *prog, tn_run_info *info);
void tn_program_free(tn_program *prog);

/* One contraction end to end: upload the leaves from the host net, run, read the amplitude back.
 * out_amp: host double[2]; out_exp2: host int32.  info may be NULL.  Blocks until done.
 * The compiled program is cached in the context for the next call with the same net and plan.
 * Errors: as tn_program_create / tn_program_run; TN_ETIMEOUT if a device wait gave up. */
tn_status tn_contract(tn_ctx *ctx, const tn_net *net, const tn_plan *plan, tn_precision prec,
                      double out_amp[2], int32_t *out_exp2, tn_run_info *info);

/* Sliced contraction: the slices of the closed network (n_sliced edges, none an open leg) run as
 * the jobs of a batch of at most max_jobs jobs -- one compiled plan (the plan's tree on the sliced
 * structure), each job's tensors on sliced edges replaced by its slice -- and their values are
 * summed in FP64; the amplitude is returned as for tn_contract, and the number of slices in
 * *n_slices (may be NULL).  Slices are numbered in mixed radix over `sliced` (the first edge
 * slowest); first_slice and slice_count (0 = all) select a range, whose partial sum is returned
 * (for timing a sample of a large slicing).  Blocks until done.
 * Errors: TN_EINVAL, TN_EUNSUPPORTED (more than 2^40 slices), those of tn_batch_create and
 * tn_batch_run, TN_ETIMEOUT. */
tn_status tn_contract_sliced(tn_ctx *ctx, const tn_net *net, const tn_plan *plan, tn_precision prec,
                             int32_t n_sliced, const int32_t *sliced, int32_t max_jobs, int64_t first_slice,
                             int64_t slice_count, double out_amp[2], int32_t *out_exp2, int64_t *n_slices);

/* ------------------------------------------------------------------ batches (many contractions) */

/* A batch holds n independent contractions ("jobs") resident on the device and runs them all in
 * one persistent launch (the k partitions of every job are independent step lists, so they and
 * all the jobs proceed concurrently).  Jobs whose nets have the same structure and share a plan
 * share one compiled step list; they differ only in their leaves (for example one circuit with
 * many bitstrings).  nets[i] and plans[i] must outlive the batch.
 * Errors: TN_EINVAL, TN_EBUDGET, TN_EUNSUPPORTED (open network), TN_ENOMEM, TN_ECUDA. */
tn_status tn_batch_create(tn_ctx *ctx, int32_t n, const tn_net *const *nets,
                          const tn_plan *const *plans, tn_precision prec, tn_batch **out);

/* Enqueue one run of every job on the context's stream (leaves re-uploaded first for nets changed
 * by tn_net_set_tensor).  d_results: NULL, or DEVICE memory of n * 32 bytes that receives one
 * {double re, double im, int32 exp2, int32 status} record per job.  Errors: TN_ECUDA. */
tn_status tn_batch_run(tn_batch *b, void *d_results);

/* Replace the entries of tensor tensor[i] of job job[i] (same shape) for i < count, in the batch's
 * resident copy only (the nets are not modified).  data: the new entries back to back, complex128
 * interleaved, each part finite and below 2^127 in magnitude.  The values are written into pinned
 * host memory (two staging sets used in turn, so the call may overlap a run in flight: it waits
 * only for the copy out of the set it refills, made two runs earlier) and applied on the device by
 * the next tn_batch_run, in two copies and one scatter kernel.  Errors: TN_EINVAL (nothing is
 * staged), TN_ENOMEM, TN_ECUDA. */
tn_status tn_batch_set_tensors(tn_batch *b, int32_t count, const int32_t *job, const int32_t *tensor,
                               const double *data);

/* Wait for the last run and copy its results to the host: amps [n][2], exp2 [n], status [n]
 * (0 ok, TN_ETIMEOUT if a device wait gave up); any pointer may be NULL.  With status == NULL a
 * timed-out job makes the call return TN_ETIMEOUT.  Errors: TN_ECUDA, TN_ETIMEOUT. */
tn_status tn_batch_results(tn_batch *b, double *amps, int32_t *exp2, int32_t *status);
tn_status tn_batch_footprint(const tn_batch *b, size_t *bytes);
tn_status tn_batch_last_info(const tn_batch *b, tn_run_info *info);

/* Mean device duration (CUDA events recorded on the context's stream before the first and after
 * the last contraction kernel of a run) over the last n_runs runs, 1 <= n_runs <= 256; waits for
 * them.
 * Errors: TN_EINVAL, TN_EUNSUPPORTED (graph mode), TN_ECUDA. */
tn_status tn_batch_kernel_ms(const tn_batch *b, int32_t n_runs, double *mean_ms);

/* The same device time split by kernel class (CUDA events recorded between the launches of each
 * run): mean_ms[0] warp programs, [1] block and large programs, [2] tensor-core operand packing,
 * [3] tensor-core GEMM, [4] persistent dataflow launches (summed over the dependency phases).
 * Errors: as tn_batch_kernel_ms. */
tn_status tn_batch_kernel_times(const tn_batch *b, int32_t n_runs, double *mean_ms);
void tn_batch_free(tn_batch *b);

/* Diagnostics, for testing the bounded waits: from the next run on, the persistent work list of
 * the batch leaves out every tile of global step `step` of job `job` (the numbering of
 * tn_plan_compile_steps), so the tiles consuming that step wait for a producer that never runs
 * and give up after the context's wait_limit_us (see tn_exec_config): that job -- and any other
 * job with a tile still waiting when the abort flag rises -- reports TN_ETIMEOUT, every other job
 * completes normally.  Holds accumulate; step = -1 releases every hold of `job`, job = -1 every
 * hold of the batch.  Waits for the batch's stream.
 * Errors: TN_EINVAL (no such job, or the step is not in the persistent work list, or graph
 * execution mode), TN_ECUDA. */
tn_status tn_batch_debug_hold(tn_batch *b, int32_t job, int32_t step);

/* Diagnostics: cycle accounting of the persistent kernel (costs a few atomics per work item; off
 * by default).  tn_batch_profile waits for the stream and returns 16 accumulated SM-cycle sums and
 * item counts since profiling was switched on: [0..4] work items of the dataflow kernel by class
 * (ROWS, TILE, DOTP, DOTF, TC), [5] block programs, [6] large programs, [8] program waves made of
 * small steps only, [9] waves that hold block-wide steps (block programs), [10] warp programs,
 * [12] dependency waits, [13] waves with block-wide steps (large programs).
 * Errors: TN_EINVAL, TN_ECUDA. */
tn_status tn_batch_set_profiling(tn_batch *b, int32_t on);
tn_status tn_batch_profile(tn_batch *b, int64_t *cycles, int64_t *items);

/* One-shot: create a batch, run it once, return the results on the host, free it. */
tn_status tn_batch_contract(tn_ctx *ctx, int32_t n, const tn_net *const *nets,
                            const tn_plan *const *plans, tn_precision prec, double *out_amps,
                            int32_t *out_exp2);

/* Permute the axes of a row-major DEVICE tensor (the transposition of the TTGT scheme realising
 * Eq. 2.4, Section 5.1): output axis t is input axis perm[t], so out has dims[perm[t]] at axis t.
 *   d_in, d_out   device buffers of prod(dims) elements, not overlapping
 *   elem_bytes    1, 2, 4, 8 or 16 (the payload is moved bit for bit)
 *   rank          0..32; dims[rank] >= 1; perm a permutation of 0..rank-1
 * Enqueued on the context's stream, returns without waiting.  Errors: TN_EINVAL, TN_ECUDA. */
tn_status tn_permute(tn_ctx *ctx, const void *d_in, void *d_out, int32_t elem_bytes, int32_t rank,
                     const int64_t *dims, const int32_t *perm);

/* Inner product sum_i a[i] * b[i] (bilinear, no conjugation) of two DEVICE vectors of n complex
 * numbers, accumulated in FP64, without allocating any memory.  The paper has no counterpart: it
 * is the engine's final-reduction kernel offered to callers that cannot allocate device memory
 * while they run -- code whose device memory belongs to a host framework's pool, or serving loops
 * where cudaMalloc / cudaFree would synchronize the device or could fail mid-request.
 *   device       the CUDA device of the vectors; the caller's current device is restored before
 *                the call returns
 *   cuda_stream  cudaStream_t to enqueue on (NULL = legacy default stream); returns without waiting
 *   d_a, d_b     n complex64 (prec = TN_C64) or complex128 (TN_C128) numbers, interleaved
 *   n            0 <= n <= 2^26; larger n is rejected with TN_EINVAL (the scratch holds one FP64
 *                partial sum per 65536 elements, 1024 of them)
 *   d_out        DEVICE double[2] receiving (re, im)
 * Scratch lives in a file-scope device array (16 KB) that every GPU loading the library keeps
 * until the process exits; all calls share it, so calls whose kernels overlap on the GPU (for
 * example on two streams) race and must be ordered by the caller.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  The looked-up address is kept for the life of the
 * process: after a cudaDeviceReset of that device it is stale, so do not call tn_dot_noalloc on a
 * device that was reset.  No cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: TN_EINVAL, TN_ECUDA. */
tn_status tn_dot_noalloc(int32_t device, void *cuda_stream, const void *d_a, const void *d_b,
                         int64_t n, tn_precision prec, double *d_out);

/* ------------------------------------------------------------------ serving */

/* A request loop with continuous batching (the serving pattern of the engine).  Models -- a
 * registered (net, plan) -- stay compiled and resident; a request names a model and replaces some
 * of its tensors (for instance the bra tensors of a bitstring, or the single-qubit slots of an
 * expectation value).  A worker thread admits queued requests into launches as device memory
 * allows -- each request needs its model's per-job bytes from a pool of hbm_budget_bytes
 * allocated at creation -- and keeps up to two launches in flight on two streams, so requests
 * that arrive while one launch runs start in the next one and overlap with it.  A request's
 * result depends only on its own data: it is the same alone and in any mix.
 * The context's device is used; the server owns its streams. */
typedef struct tn_server tn_server;

typedef struct {
    int64_t submitted, completed, rejected;   /* rejected: larger than the whole pool (TN_EBUDGET) */
    int64_t launches, launched_requests;       /* batches launched and the requests they carried */
    int32_t max_in_flight, pad;                /* most launches on the device at once (<= 2) */
    size_t pool_used;                          /* pool bytes held by launches in flight */
} tn_serve_stats;

/* max_batch: most requests per launch.  Errors: TN_EINVAL, TN_ENOMEM (pool), TN_ECUDA. */
tn_status tn_serve_create(tn_ctx *ctx, tn_precision prec, size_t hbm_budget_bytes, int32_t max_batch,
                          tn_server **out);
/* Compile and keep resident a closed network with its plan (copied; the net's current tensor
 * values are the model's defaults).  Thread-safe.  Errors: TN_EINVAL, TN_EUNSUPPORTED, TN_ECUDA. */
tn_status tn_serve_register(tn_server *s, const tn_net *net, const tn_plan *plan, int32_t *model);
/* Device bytes one request of `model` holds while in flight, and its algorithmic flops. */
tn_status tn_serve_model_info(tn_server *s, int32_t model, size_t *job_bytes, double *flops);
/* Queue a request: `count` tensors of the model replaced by `data` (their entries back to back,
 * complex128 interleaved, each part finite and below 2^127 in magnitude; copied).  Thread-safe,
 * returns at once with a ticket.  Errors: TN_EINVAL. */
tn_status tn_serve_submit(tn_server *s, int32_t model, int32_t count, const int32_t *tensors,
                          const double *data, uint64_t *ticket);
/* Wait up to timeout_s (0 = do not wait) for a ticket.  *done = 0 if not finished yet; otherwise
 * the result (value = (re + i im) * 2^exp2) and its latency from submission to completion, and the
 * ticket is released.  Returns TN_EBUDGET for a request that can never fit the pool, TN_ETIMEOUT or
 * TN_ECUDA if its launch failed. */
tn_status tn_serve_poll(tn_server *s, uint64_t ticket, double timeout_s, double out_amp[2],
                        int32_t *out_exp2, double *latency_s, int32_t *done);
tn_status tn_serve_get_stats(tn_server *s, tn_serve_stats *stats);
/* Stops the worker after the launches in flight finish; queued requests are dropped. */
void tn_serve_free(tn_server *s);

/* ------------------------------------------------------------------ diagnostics */

const char *tn_status_str(tn_status s);
const char *tn_last_error(void);   /* thread-local message of the last failure */
const char *tn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TNSA_H */
