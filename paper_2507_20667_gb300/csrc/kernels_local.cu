// k_warp (warp programs) and k_local (block and large programs): subtrees of small steps that
// depend on leaves only, run before the dataflow kernel.
#include "contract_common.cuh"

namespace tn {

namespace {

// Warp programs: every warp of the block runs its own program (no block barrier), in its own
// kWarpSlice-byte slice of shared memory, and publishes its pseudo-step as complete.  PROF: the
// variant with cycle accounting (prof non-null), compiled apart.
template <typename T, bool PROF>
__global__ void __launch_bounds__(kWarpThreads, 6) k_warp(const JobPtrs *__restrict__ jobs,
                                                          const WorkItem *__restrict__ items, int32_t n_items,
                                                          long long *prof) {
    extern __shared__ __align__(16) char dyn[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t g = blockIdx.x * (kWarpThreads / 32) + warp;
    if (g >= n_items) return;   // warp-uniform; the kernel has no block barrier
    const WorkItem it = items[g];
    const JobPtrs &j = jobs[it.job];
    const int32_t prog = __ldcg(&j.steps[it.step].tile_rows);
    long long t0 = 0;
    if (PROF && lane == 0) t0 = clock64();
    run_warp_prog<T>(prog, j, dyn + warp * kWarpSlice);
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        atomicAdd(j.done + it.step, 1);
        if (PROF) {
            atomicAdd((unsigned long long *)(prof + 10), (unsigned long long)(clock64() - t0));
            atomicAdd((unsigned long long *)(prof + kProfSlots + 10), 1ull);
        }
    }
}

// All subtree programs of a batch: one block per program (they depend on leaves only).  Each
// publishes its pseudo-step as complete, so the dataflow kernel that runs next never waits on it.
template <typename T, bool PROF>
__global__ void __launch_bounds__(kThreads) k_local(const JobPtrs *__restrict__ jobs,
                                                    const WorkItem *__restrict__ items, long long *prof) {
    extern __shared__ __align__(16) char dyn[];
    __shared__ __align__(16) char smem[Scratch<T>::local];
    const WorkItem it = items[blockIdx.x];
    const JobPtrs &j = jobs[it.job];
    const int32_t prog = __ldcg(&j.steps[it.step].tile_rows);
    long long t0 = 0;
    if (PROF && threadIdx.x == 0) t0 = clock64();
    run_local<T, PROF>(prog, j, dyn, smem, prof);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(j.done + it.step, 1);
        if (PROF) {   // slot 5: block programs, 6: large programs
            const int slot = __ldcg(&j.progs[prog].kind) == PROG_BIG ? 6 : STEP_LOCAL;
            atomicAdd((unsigned long long *)(prof + slot), (unsigned long long)(clock64() - t0));
            atomicAdd((unsigned long long *)(prof + kProfSlots + slot), 1ull);
        }
    }
}

}  // namespace

template <typename T, bool PROF>
cudaError_t launch_local_t(const JobPtrs *jobs_dev, const WorkItem *items, int32_t n_warp, int32_t n_block,
                           int32_t n_big, int32_t dyn_smem, int32_t dyn_big, long long *prof, cudaStream_t stream) {
    if (n_warp > 0) {
        constexpr int per_block = kWarpThreads / 32;
        const int32_t smem = per_block * kWarpSlice;
        cudaError_t e = allow_dyn_smem(k_warp<T, PROF>, smem);
        if (e != cudaSuccess) return e;
        const unsigned grid = (unsigned)((n_warp + per_block - 1) / per_block);
        k_warp<T, PROF><<<grid, kWarpThreads, smem, stream>>>(jobs_dev, items, n_warp, prof);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // block programs, then the large ones (each launch with its own shared-memory size)
    const int32_t counts[2] = {n_block, n_big}, dyn[2] = {dyn_smem, dyn_big};
    const WorkItem *it = items + n_warp;
    for (int q = 0; q < 2; ++q) {
        if (counts[q] <= 0) continue;
        cudaError_t e = allow_dyn_smem(k_local<T, PROF>, dyn[q]);
        if (e != cudaSuccess) return e;
        k_local<T, PROF><<<counts[q], kThreads, dyn[q], stream>>>(jobs_dev, it, prof);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        it += counts[q];
    }
    return cudaSuccess;
}

cudaError_t launch_local(bool c128, const JobPtrs *jobs_dev, const WorkItem *items, int32_t n_warp,
                         int32_t n_block, int32_t n_big, int32_t dyn_smem, int32_t dyn_big, long long *prof,
                         cudaStream_t stream) {
    if (c128)
        return prof ? launch_local_t<double, true>(jobs_dev, items, n_warp, n_block, n_big, dyn_smem, dyn_big, prof,
                                                   stream)
                    : launch_local_t<double, false>(jobs_dev, items, n_warp, n_block, n_big, dyn_smem, dyn_big,
                                                    nullptr, stream);
    return prof ? launch_local_t<float, true>(jobs_dev, items, n_warp, n_block, n_big, dyn_smem, dyn_big, prof, stream)
                : launch_local_t<float, false>(jobs_dev, items, n_warp, n_block, n_big, dyn_smem, dyn_big, nullptr,
                                               stream);
}

int32_t local_smem_budget(bool c128, int32_t blocks_per_sm) {
    int dev = 0, per_sm = 0, per_block = 0, reserved = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) return 0;
    cudaFuncAttributes fa;
    cudaError_t e = c128 ? cudaFuncGetAttributes(&fa, k_local<double, false>)
                          : cudaFuncGetAttributes(&fa, k_local<float, false>);
    if (e != cudaSuccess) return 0;
    int32_t b = per_sm / blocks_per_sm - reserved - (int32_t)fa.sharedSizeBytes;
    if (b > per_block - (int32_t)fa.sharedSizeBytes) b = per_block - (int32_t)fa.sharedSizeBytes;
    return b > 0 ? (b / 16) * 16 : 0;
}

}  // namespace tn
