// Device helpers shared by the translation units of the contraction kernels (kernels_contract.cu,
// kernels_step.cu, kernels_local.cu, kernels_persist_f32.cu, kernels_persist_f64.cu).
#pragma once

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"
#include "local_ops.cuh"
#include "tile_ops.cuh"

namespace tn {

namespace {

constexpr int32_t kStatusTimeout = 5;

__device__ __forceinline__ uint32_t ld_acquire(const int32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until the steps producing a work item's operands have completed all their tiles; false if
// the wait gave up.  Both counters are read together (one round trip when they are done).  The
// first wait that gives up raises the launch-wide abort flag, after which every wait returns at
// once, so a broken dependency costs one time-out, not one per waiting tile.
__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__device__ bool wait_deps(const JobPtrs &j, const WorkItem &it, int32_t *abort_flag, long long limit_ns) {
    const bool d0 = it.dep0 >= 0, d1 = it.dep1 >= 0;
    uint32_t c0 = d0 ? ld_acquire(j.done + it.dep0) : 0u, c1 = d1 ? ld_acquire(j.done + it.dep1) : 0u;
    if ((!d0 || c0 >= it.need0) && (!d1 || c1 >= it.need1)) return true;
    const long long t0 = global_ns();
    unsigned ns = 32;
    while (true) {
        if (d0 && c0 < it.need0) c0 = ld_acquire(j.done + it.dep0);
        if (d1 && c1 < it.need1) c1 = ld_acquire(j.done + it.dep1);
        if ((!d0 || c0 >= it.need0) && (!d1 || c1 >= it.need1)) return true;
        if (ld_acquire(abort_flag)) return false;
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        // the global timer counts nanoseconds whatever the SM clock
        if (global_ns() - t0 > limit_ns) {
            atomicExch(abort_flag, 1);
            return false;
        }
    }
}

template <typename T>
__device__ __forceinline__ void run_item(const StepDesc &d, int64_t tile, const JobPtrs &j, char *smem,
                                         float *red, char *dyn, long long *prof) {
    if (d.kind == STEP_LOCAL) {
        if (__ldcg(&j.progs[d.tile_rows].kind) == PROG_WARP) {
            if (threadIdx.x < 32) run_warp_prog<T>(d.tile_rows, j, dyn);   // graph mode: warp 0
            __syncthreads();
        } else {
            run_local<T>(d.tile_rows, j, dyn, smem, prof);
        }
    } else {
        run_tile<T>(d, tile, j, smem, red, dyn);
    }
}

// Static plus dynamic shared memory above 48 KB per block needs an opt-in for the dynamic part;
// it is set whenever a kernel takes dynamic shared memory (a cheap host call).
template <typename K>
inline cudaError_t allow_dyn_smem(K kernel, int32_t bytes) {
    if (bytes <= 0) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

}  // namespace tn
