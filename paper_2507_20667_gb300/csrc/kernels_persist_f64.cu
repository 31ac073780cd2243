// k_persist for complex128 storage, and the launchers of both storage types.
#include "persist.cuh"

namespace tn {

int32_t persistent_grid(bool c128) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (c128) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<double, false>, kThreads, 0) !=
            cudaSuccess)
            return 0;
    } else {
        per_sm = persistent_blocks_per_sm_f32();
    }
    return sms * per_sm;
}

cudaError_t launch_persistent(bool c128, const JobPtrs *jobs_dev, const WorkItem *work, int64_t n_work,
                              uint32_t *counter, int32_t grid, long long wait_ns, long long *prof,
                              cudaStream_t stream) {
    if (n_work <= 0) return cudaSuccess;
    if (grid > n_work) grid = (int32_t)n_work;
    if (!c128) return launch_persistent_f32(jobs_dev, work, n_work, counter, grid, wait_ns, prof, stream);
    if (prof)
        k_persist<double, true><<<(unsigned)grid, kThreads, 0, stream>>>(jobs_dev, work, n_work, counter, wait_ns,
                                                                        prof);
    else
        k_persist<double, false><<<(unsigned)grid, kThreads, 0, stream>>>(jobs_dev, work, n_work, counter, wait_ns,
                                                                         nullptr);
    return cudaGetLastError();
}

}  // namespace tn
