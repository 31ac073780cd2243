// Device step descriptors and kernel launchers of the contraction engine.
#pragma once

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

enum StepKind : int32_t { STEP_ROWS = 0, STEP_TILE = 1, STEP_DOT = 2, STEP_TC = 3 };

struct StepDesc {
    const void *A;
    const void *B;
    void *C;                 // may be null for the root step (result written to the scalar slot)
    int64_t M, N, K;
    int32_t node_a, node_b, node_c;
    int32_t kind;
    int32_t is_root;
    int32_t pad;
    Groups m, n, k;
};

// Per-node power-of-two scale bookkeeping (spec precision row): the stored values V of
// node v represent V * 2^exp2[v]; maxbits[v] holds the float bit pattern of max(|Re V|, |Im V|)
// (atomicMax on the bit pattern orders non-negative floats correctly).
struct ScaleState {
    int32_t *exp2;
    uint32_t *maxbits;
};

// Result record written to device memory at the end of a run.
struct DeviceResult {
    double re, im;
    int32_t exp2;
    int32_t status;
    int64_t pad;
};

// Launchers (all enqueue on `stream`, return the launch error).
cudaError_t launch_leaf_convert(bool c128, const double *src, void *dst, const int64_t *leaf_off,
                                int32_t n_leaves, ScaleState sc, cudaStream_t stream);
cudaError_t launch_step(bool c128, const StepDesc *d_desc, const StepDesc &h_desc, ScaleState sc,
                        double *dot_partials, int32_t dot_blocks, DeviceResult *result,
                        cudaStream_t stream, int32_t *launches);
cudaError_t launch_finish_leaf(bool c128, const void *leaf, int32_t node, ScaleState sc,
                               DeviceResult *result, cudaStream_t stream);
cudaError_t launch_permute(const void *src, void *dst, int32_t elem_bytes, int32_t rank,
                           const int64_t *dims, const int32_t *perm, cudaStream_t stream);

// Number of blocks of the first phase of the dot kernel (partials buffer: blocks * 16 double2).
int32_t dot_partial_blocks();

}  // namespace tn
