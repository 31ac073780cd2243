// k_persist for complex64 storage.
#include "persist.cuh"

namespace tn {

cudaError_t launch_persistent_f32(const JobPtrs *jobs_dev, const WorkItem *work, int64_t n_work, uint32_t *counter,
                                  int32_t grid, long long wait_ns, long long *prof, cudaStream_t stream) {
    auto kern = prof ? k_persist<float, true> : k_persist<float, false>;
    const cudaError_t e = allow_dyn_smem(kern, kPersistDynSmem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, kThreads, kPersistDynSmem, stream>>>(jobs_dev, work, n_work, counter, wait_ns, prof);
    return cudaGetLastError();
}

int32_t persistent_blocks_per_sm_f32() {
    int per_sm = 0;
    cudaError_t e = allow_dyn_smem(k_persist<float, false>, kPersistDynSmem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<float, false>, kThreads, kPersistDynSmem);
    return e == cudaSuccess ? per_sm : 0;
}

}  // namespace tn
