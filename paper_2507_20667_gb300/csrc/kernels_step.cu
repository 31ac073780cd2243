// k_step: one step of one job, one block per work tile (the graph execution mode).
#include "contract_common.cuh"

namespace tn {

namespace {

template <typename T>
__global__ void __launch_bounds__(kThreads) k_step(const StepDesc *__restrict__ steps, int32_t step,
                                                   JobPtrs job) {
    extern __shared__ __align__(16) char dyn[];
    __shared__ StepDesc d;
    __shared__ __align__(16) char smem[Scratch<T>::bytes];
    __shared__ float red[32];
    load_desc(d, steps + step);
    run_item<T>(d, blockIdx.x, job, smem, red, dyn, nullptr);
}

}  // namespace

cudaError_t launch_step(bool c128, const StepDesc &h, int32_t step, const JobPtrs &job, int32_t dyn_smem,
                        cudaStream_t stream) {
    if (h.ntiles <= 0 || h.kind == STEP_TC) return cudaErrorInvalidValue;   // TC: launch_tc_pack / _gemm
    const int32_t dyn = h.kind == STEP_LOCAL
                            ? dyn_smem
                            : ((h.flags & (FLAG_A_SMEM | FLAG_DOT_SMEM_A | FLAG_DOT_SMEM_B)) ? kPersistDynSmem : 0);
    cudaError_t e = c128 ? allow_dyn_smem(k_step<double>, dyn) : allow_dyn_smem(k_step<float>, dyn);
    if (e != cudaSuccess) return e;
    if (c128) k_step<double><<<(unsigned)h.ntiles, kThreads, dyn, stream>>>(job.steps, step, job);
    else k_step<float><<<(unsigned)h.ntiles, kThreads, dyn, stream>>>(job.steps, step, job);
    return cudaGetLastError();
}

}  // namespace tn
