// Device step descriptors, job tables and kernel launchers of the contraction engine.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace tn {

// One pairwise contraction (Eq. 2.4 with arbitrary axis orders), written as
//     C[m, n] = sum_k A[offA(m) + kA(k)] * B[kB(k) + nB(n)]
// where m runs over the free legs of A (in A's order), n over the free legs of B (in B's order)
// and k over the shared legs (in A's order).  C is stored row-major [M, N]: its legs are A's free
// legs followed by B's free legs, so no output permutation is ever needed.  Consecutive legs
// that stay consecutive are fused into one "group" (rank reduction); each group is
// (dim, stride in A and/or B).  Group 0 is the innermost (fastest-varying) one.
constexpr int kMaxGroups = 32;

struct Groups {
    int32_t n;           // number of groups
    int32_t pow2;        // 1 if every dim is a power of two (digits by shift / mask)
    int64_t dim[kMaxGroups];
    int64_t sa[kMaxGroups];   // stride in A (m and k groups) or in B (n groups)
    int64_t sb[kMaxGroups];   // stride in B (k groups only)
    int32_t lsb[kMaxGroups];  // pow2: bit position of the group's lowest digit bit
    int64_t mask[kMaxGroups]; // pow2: dim - 1
};

// Kernel classes.  A contraction producing at most 16 outputs from a long shared index is split
// in two steps: DOTP reduces K-chunks into FP64 partials, DOTF sums them in a fixed order.
enum StepKind : int32_t {
    STEP_ROWS = 0, STEP_TILE = 1, STEP_DOTP = 2, STEP_DOTF = 3, STEP_TC = 4,
    STEP_LOCAL = 5      // a whole subtree run by one block in shared memory (tile_rows = program)
};

enum StepFlags : int32_t {
    FLAG_A_LEAF = 1,    // A lives in the job's leaf buffer (else in its arena)
    FLAG_B_LEAF = 2,
    FLAG_ROOT = 4,      // the step produces the network's value: write the job's result record
    FLAG_NO_C = 8,      // no tensor output (DOTP, or the root's DOTF)
    FLAG_TF32 = 16,     // TC: TF32 split (else BF16 split)
    FLAG_A_SMEM = 32,   // ROWS: A is copied whole into shared memory and C leaves through it
    FLAG_CHAIN_CONT = 64, // ROWS (FLAG_A_SMEM): A is the C of the previous step of a chain, which
                          // the persistent kernel keeps in shared memory; no work item of its own
    FLAG_A_MCONT = 128,   // TC: A's row index is its contiguous one (the pack reads rows fastest)
    FLAG_B_NCONT = 256,   // TC: B's column index is its contiguous one
    FLAG_DOT_SMEM_A = 512,  // DOTP (complex64, one tile, M = 1): A, read in a permuted order, is
                            // first copied whole and coalesced into shared memory
    FLAG_DOT_SMEM_B = 1024  // the same for B (N = 1)
};

struct StepDesc {
    int64_t M, N, K;
    int64_t a_off, b_off, c_off;   // element offsets into the leaf buffer or the arena
    int64_t img_a, img_b;          // TC: byte offsets in the arena of the packed operand images
    int32_t node_a, node_b, node_c;
    int32_t kind;
    int32_t flags;
    int32_t ntiles;                // work tiles of this step
    int32_t dep0, dep1;            // steps producing A and B (-1: a leaf); DOTF: dep0 = its DOTP
    int32_t tile_rows;             // ROWS: output rows per tile; DOTP: shared indices per tile;
                                   // TILE: tile shape (0: 64 x 64, kTileNarrow: 128 x 32)
    int32_t part_off;              // DOTP / DOTF: offset of the step's partials (in double2)
    int32_t level;                 // longest path from the leaves (scheduling order)
    int32_t ktab_off;              // DOTP: first entry of its shared-index offset table (-1: none)
    int32_t chain_next;            // ROWS (FLAG_A_SMEM): the step that consumes C next in the same
                                   // block, C kept in shared memory (-1: C goes to the arena)
    int32_t a_lgn;                 // FLAG_CHAIN_CONT: log2 of the previous step's N (the row width
                                   // of A's rotated shared-memory layout)
    Groups m, n, k;
};

// ---- CTA-resident subtree programs -------------------------------------------------------------
// A local step is the same contraction as a StepDesc with every operand in shared memory (int32
// element offsets) and at most kLG fused groups per index class.
constexpr int kLG = 6;
enum LocalMode : uint8_t { LMODE_ROWS = 0, LMODE_GEMM = 1, LMODE_REDUCE = 2 };
enum LocalFlags : int32_t {
    LFLAG_JOB_ROOT = 1,     // (program, step) produces the job's amplitude
    LFLAG_SMALL = 2,        // (step) small enough for one warp
    LFLAG_TAB = 4,          // (small step, M N <= 16, K <= 16) the index maps are tabulated: the
                            // bytes of the group fields from m_dim on hold kTabWords packed
                            // offsets (low 16 bits in A, high 16 in B), outputs then shared indices
    LFLAG_C_OUT = 16        // (warp programs) C is the program's result: written to the job's
                            // arena at root_c_off
};
constexpr int kTabOut = 16, kTabK = 16;

// A wave of a program: steps [first, first + n_small) run one per warp, then n_big steps use the
// whole block; the steps of a wave are independent of each other.
struct LocalWave {
    int32_t first, n_small, n_big;
    int32_t first_in, n_in;             // staging pieces loaded before the wave (lazy programs)
    int32_t pad[3];
};
static_assert(sizeof(LocalWave) % 16 == 0, "waves are staged in 16-byte pieces");

struct LocalStep {
    int32_t M, N, K;
    int32_t a_off, b_off, c_off;        // shared-memory element offsets
    int16_t sa, sb, sc;                 // scale slots of A, B and C
    uint8_t nm, nn, nk, pow2, mode, flags;
    int32_t m_dim[kLG], m_str[kLG];     // free legs of A (stride in A)
    int32_t n_dim[kLG], n_str[kLG];     // free legs of B (stride in B)
    int32_t k_dim[kLG], k_sa[kLG], k_sb[kLG];
    uint8_t m_lsb[kLG], n_lsb[kLG], k_lsb[kLG];
    uint8_t pad[2];
};
static_assert(sizeof(LocalStep) == 224, "LocalStep layout");
static_assert(offsetof(LocalStep, m_lsb) - offsetof(LocalStep, m_dim) >= 4 * (kTabOut + kTabK),
              "the tabulated offsets fit the group fields");

struct LocalProg {
    int32_t first_step, n_steps;        // into the job's LocalStep array
    int32_t first_leaf, n_leaves;       // into the job's LeafRef array
    int32_t n_slots;                    // nodes of the subtree (leaves and intermediates)
    int32_t smem_bytes;                 // dynamic shared memory the program needs
    int32_t root_node, root_slot;
    int32_t root_smem_off, root_size;   // where the subtree's value sits in shared memory
    int64_t root_c_off;                 // and where it goes in the job's arena
    int32_t flags;                      // LFLAG_JOB_ROOT: the subtree is the whole network
    int32_t first_wave, n_waves;        // into the job's LocalWave array
    int32_t kind;                       // ProgKind
};
// Program kinds: PROG_BLOCK -- one block, inputs staged up front, two blocks per SM;
// PROG_WARP -- one warp, steps in plan order; PROG_BIG -- one block per SM, each input staged at
// the wave that consumes it (large subtrees such as fan-in chains).
enum ProgKind : int32_t { PROG_BLOCK = 0, PROG_WARP = 1, PROG_BIG = 2 };

// A staging piece of a program input: `count` (at most 16) elements at element offset global_off
// of the job's leaf buffer (src 0) or of its arena (src 1: a warp program's result), copied to
// shared-memory element offset smem_off.  The first piece of an input has slot >= 0 and also
// copies the max-abs and exponent of node `node` into that scale slot.
struct LeafRef {
    int64_t global_off;
    int32_t count, smem_off, slot, node, src, pad;
};
static_assert(sizeof(LeafRef) == 32, "staging pieces are 32 bytes");

// Everything one contraction (a "job") owns on the device.  Several jobs may share one compiled
// step list (same network structure and plan) and differ only in their leaves.
struct JobPtrs {
    const double2 *leaf64;   // complex128 leaves as uploaded
    const int64_t *leaf_off; // [n_leaves + 1] element offsets of the leaves
    const void *leaf;        // storage-type leaves
    char *arena;             // intermediates
    double2 *partials;       // DOTP partials
    int32_t *exp2;           // [n_nodes] power-of-two exponent of each node's stored values
    uint32_t *maxbits;       // [n_nodes] float bits of max(|Re|, |Im|) of each node's values
    int32_t *done;           // [n_steps] completed tiles of each step (persistent execution)
    void *result;            // DeviceResult
    const StepDesc *steps;   // the job's compiled step list
    const LocalProg *progs;  // CTA-resident subtree programs
    const LocalStep *lsteps;
    const LeafRef *leafrefs;
    const LocalWave *lwaves;
    const int2 *ktab;        // (offset in A, offset in B) of each shared index of tabulated DOTP steps
    int32_t n_steps;
    int32_t n_leaves;
};

// Result record written to device memory at the end of a run.
struct DeviceResult {
    double re, im;
    int32_t exp2;
    int32_t status;          // 0 = ok, 5 = a bounded wait gave up (TN_ETIMEOUT)
    int64_t pad;
};

// A unit of persistent work: tile `tile` of step `step` of job `job`.  Dataflow items also carry
// their dependencies -- the steps producing A and B (-1: none) and how many tiles each has -- so
// that a block can wait on them without first reading the step descriptors.
struct WorkItem {
    uint32_t job, step, tile;
    int32_t dep0 = -1, dep1 = -1;
    uint32_t need0 = 0, need1 = 0;
    uint32_t pad = 0;
};
static_assert(sizeof(WorkItem) == 32, "work items are 32 bytes");

// Launchers (all enqueue on `stream`, return the launch error).
// max_leaf_elems: the largest leaf of any job (selects the conversion for large leaves).
cudaError_t launch_leaf_convert(bool c128, const JobPtrs *jobs_dev, int32_t n_jobs,
                                int32_t max_leaves, int64_t max_leaf_elems, cudaStream_t stream);
cudaError_t launch_step(bool c128, const StepDesc &h_desc, int32_t step, const JobPtrs &job,
                        int32_t dyn_smem, cudaStream_t stream);
cudaError_t launch_finish_leaf(bool c128, const JobPtrs &job, cudaStream_t stream);
// Optional cycle accounting of the persistent kernel: prof[slot] sums SM cycles (block 0's view
// of each work item, thread 0), prof[kProfSlots + slot] counts items.  Slots 0..4: work items by
// StepKind (dependency wait excluded); 5: block programs; 6: large programs; 8: waves of small
// steps; 9: waves with block-wide steps (block programs); 10: warp programs (lane 0's view);
// 12: dependency waits; 13: waves with block-wide steps (large programs); 14: waiting for the
// inputs of large programs; ROWS steps staged through shared memory, by phase: 7 operand staging,
// 11 the multiply-add loop, 15 the epilogue.
constexpr int kProfSlots = 16;

// counter: two zeroed 32-bit words, the work claim counter and the launch-wide abort flag.
// wait_ns: a dependency wait gives up after about this many nanoseconds (TN_ETIMEOUT).
cudaError_t launch_persistent(bool c128, const JobPtrs *jobs_dev, const WorkItem *work,
                              int64_t n_work, uint32_t *counter, int32_t grid,
                              long long wait_ns, long long *prof, cudaStream_t stream);
// Co-resident grid of the persistent kernel.
int32_t persistent_grid(bool c128);

// ---- dense steps on the tensor cores (kernels_tc.cu) ------------------------------------------
// A dense step C [M, N] = A [M, K] B [K, N] (complex64 storage, BF16 or TF32 split) runs as a pack
// launch -- every operand k-block gathered, scaled, split into hi / lo and written as a
// shared-memory image -- and a GEMM launch over output tiles of 128 rows x NC complex columns,
// NC = 64 or 128 per step (StepDesc.tile_rows).  Images: A tile t, k-block kb at
// img_a + (t KB + kb) 2 kTcImgA (hi plane, then lo); B'' likewise with planes of tc_img_b(NC).
constexpr int kTcRows = 128;               // rows of C per GEMM tile (tensor-memory lanes)
constexpr int kTcColsMax = 128;            // complex columns of C per GEMM tile, at most (256 real)
constexpr uint32_t kTcImgA = 128 * 64;     // one plane of an A k-block: 128 rows x 64 bytes
__host__ __device__ constexpr uint32_t tc_img_b(int nc) { return (uint32_t)(2 * nc * 64); }   // 2 NC rows x 64 B
// units: (job, step, unit) with unit < (ceil(M/128) + ceil(N/NC)) KB (tc_pack_units).
cudaError_t launch_tc_pack(bool tf32, const JobPtrs *jobs_dev, const WorkItem *units, int32_t n_units,
                           cudaStream_t stream);
// tiles: (job, step, tile) with tile < ceil(M/128) ceil(N/NC); each completed tile adds one to
// the job's done[step].  abort_flag: a zeroed device int32 (the launch-wide abort flag).
cudaError_t launch_tc_gemm(bool tf32, const JobPtrs *jobs_dev, const WorkItem *tiles, int32_t n_tiles,
                           int32_t *abort_flag, long long wait_ns, cudaStream_t stream);
int64_t tc_pack_units(int64_t M, int64_t N, int64_t K, bool tf32, int nc);
// Bytes of a step's operand images (a_bytes: the A part, may be NULL).
size_t tc_image_bytes(int64_t M, int64_t N, int64_t K, bool tf32, int nc, size_t *a_bytes);
// Subtree programs; items: (job, pseudo-step, 0), the n_warp warp programs first (four per
// block of kWarpThreads), then the n_block block programs (one per block, `dyn_smem` bytes), then
// the n_big large programs (one per block, `dyn_big` bytes).
cudaError_t launch_local(bool c128, const JobPtrs *jobs_dev, const WorkItem *items, int32_t n_warp,
                         int32_t n_block, int32_t n_big, int32_t dyn_smem, int32_t dyn_big, long long *prof,
                         cudaStream_t stream);
// Dynamic shared memory a local program may use so that `blocks_per_sm` persistent blocks fit.
int32_t local_smem_budget(bool c128, int32_t blocks_per_sm);
cudaError_t launch_scatter_updates(const int64_t *hdr, const double2 *vals, int64_t n_upd,
                                   double2 *leaf64, cudaStream_t stream);
cudaError_t launch_permute(const void *src, void *dst, int32_t elem_bytes, int32_t rank,
                           const int64_t *dims, const int32_t *perm, cudaStream_t stream);

// Tiling constants shared by the compiler and the kernels.
constexpr int kThreads = 256;
constexpr int kTileM = 64, kTileN = 64, kTileK = 16;   // CUDA-core GEMM tile
constexpr int kTileNarrow = 1;                          // TILE: tile_rows = 1 selects 128 x 32 tiles
constexpr int kRowsMaxKN = 1024, kRowsMaxK = 64, kRowsMaxN = 16;
constexpr int kDotMaxOut = 4;
// ROWS steps staged through shared memory (complex64): A (M K elements) and then the padded C
// (M (N + 1) elements) share kRowsSmemElems elements of the dataflow kernel's dynamic shared memory.
constexpr int kRowsSmemElems = 9216;
constexpr int kPersistDynSmem = kRowsSmemElems * 8;
// Longest chain of ROWS steps one persistent block runs with the tensor kept in shared memory.
constexpr int kMaxChain = 32;
constexpr int kDotChunk = 8192;                         // shared indices per DOTP tile
// Warp programs: blocks of kWarpThreads, each warp with a private kWarpSlice-byte shared-memory
// slice (step descriptor, scale slots, intermediates).
constexpr int kWarpThreads = 128;
constexpr int kWarpSlice = 8192;

}  // namespace tn
