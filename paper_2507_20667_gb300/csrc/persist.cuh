// The persistent dataflow kernel k_persist: every block claims work tiles (job, step, tile) from
// a global list in dependency-level order, waits -- with a bounded spin -- until the steps
// producing its operands have completed all their tiles, runs the tile and publishes its
// completion.  Many independent contractions run in one launch.  Claiming in list order is
// deadlock-free: a tile is claimed only by a running block and waits only on tiles earlier in the
// list, which were claimed by blocks that are running, so the earliest unfinished tile always
// progresses (co-residency of the grid is not needed).  A block claims its next tile while the
// current one runs.  A chain of narrow ROWS steps is one work item, its tensor kept in shared
// memory between the steps.  Each storage type is instantiated in its own translation unit
// (kernels_persist_f32.cu, kernels_persist_f64.cu).
#pragma once

#include "contract_common.cuh"

namespace tn {

namespace {

// Persistent dataflow kernel.  PROF: the variant with cycle accounting (prof non-null).
template <typename T, bool PROF>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1)
    k_persist(const JobPtrs *__restrict__ jobs, const WorkItem *__restrict__ work, int64_t n_work,
              uint32_t *counter, long long wait_ns, long long *prof) {
    int32_t *abort_flag = reinterpret_cast<int32_t *>(counter + 1);
    extern __shared__ __align__(16) char dyn[];
    __shared__ StepDesc d;
    __shared__ __align__(16) char smem[Scratch<T>::bytes];
    __shared__ float red[32];
    __shared__ uint32_t s_item;
    __shared__ int32_t s_ok;
    __shared__ int32_t s_chain[kMaxChain];   // continuation steps of the current ROWS chain
    // Claim-ahead: thread 0 claims the next item while the current one runs, so the claim's round
    // trip is off the critical path.  A block claims items in increasing order and runs them in
    // that order; the earliest unfinished item is therefore always being run (never only held),
    // which keeps the list order deadlock-free.
    uint32_t nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(counter, 1u);
    while (true) {
        if (threadIdx.x == 0) s_item = nxt;
        __syncthreads();
        const uint32_t w = s_item;
        if ((int64_t)w >= n_work) break;
        const WorkItem it = work[w];
        const JobPtrs &j = jobs[it.job];
        // the descriptor's loads are in flight while thread 0 waits for the operands
        int4 dr[kDescRounds];
        desc_fetch(dr, j.steps + it.step);
        long long t0 = 0;
        if (threadIdx.x == 0) {
            if (PROF) t0 = clock64();
            nxt = atomicAdd(counter, 1u);
            const bool ok = wait_deps(j, it, abort_flag, wait_ns);
            if (!ok) atomicExch(&static_cast<DeviceResult *>(j.result)->status, kStatusTimeout);
            s_ok = ok;
            if (PROF) {
                const long long t1 = clock64();
                atomicAdd((unsigned long long *)(prof + 12), (unsigned long long)(t1 - t0));
                atomicAdd((unsigned long long *)(prof + kProfSlots + 12), 1ull);
                t0 = t1;
            }
        }
        desc_store(dr, d);
        __syncthreads();
        int32_t n_chain = 0;
        bool chained = false;
        if constexpr (sizeof(T) == 4) {
            if (s_ok && d.kind == STEP_ROWS && d.chain_next >= 0) {
                n_chain = rows_chain<PROF>(d, j, smem, dyn, red, s_chain, prof);
                chained = true;
            }
        }
        if (s_ok && !chained) run_tile<T>(d, it.tile, j, smem, red, dyn);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(j.done + it.step, 1);
            for (int32_t c = 0; c < n_chain; ++c) atomicAdd(j.done + s_chain[c], 1);
            if (!s_ok) {   // a failed chain still completes its steps, so no consumer waits on them
                int32_t st = d.chain_next;
                for (int32_t c = 0; st >= 0 && c < kMaxChain; ++c) {
                    atomicAdd(j.done + st, 1);
                    st = __ldcg(&j.steps[st].chain_next);
                }
            }
            if (PROF) {
                atomicAdd((unsigned long long *)(prof + d.kind), (unsigned long long)(clock64() - t0));
                atomicAdd((unsigned long long *)(prof + kProfSlots + d.kind), 1ull);
            }
        }
    }
}

}  // namespace

// complex64 instantiation (kernels_persist_f32.cu)
cudaError_t launch_persistent_f32(const JobPtrs *jobs_dev, const WorkItem *work, int64_t n_work, uint32_t *counter,
                                  int32_t grid, long long wait_ns, long long *prof, cudaStream_t stream);
int32_t persistent_blocks_per_sm_f32();

}  // namespace tn
