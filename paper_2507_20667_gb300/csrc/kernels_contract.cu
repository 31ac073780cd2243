// Contraction kernels for sm_103a.
//
//  * k_leaf_convert  complex128 leaves -> storage type, with each leaf's max-abs (one thread/leaf)
//  * k_step          one step of one job, one block per work tile (graph execution mode);
//    k_step_tc       the same for tensor-core steps
//  * k_warp          warp programs: subtrees of small steps, one warp each, four per block
//  * k_local         one block per CTA-resident subtree program (all operands in shared memory);
//                    block programs and large programs are two launches of it
//  * k_persist       persistent dataflow kernel: every block claims work tiles (job, step, tile)
//                    from a global list in dependency-level order, waits -- with a bounded spin --
//                    until the steps producing its operands have completed all their tiles, runs
//                    the tile and publishes its completion.  Many independent contractions run in
//                    one launch.  Claiming in list order is deadlock-free: a tile is claimed only
//                    by a running block and waits only on tiles earlier in the list, which were
//                    claimed by blocks that are running, so the earliest unfinished tile always
//                    progresses (co-residency of the grid is not needed).  A block claims its
//                    next tile while the current one runs.  A chain of narrow ROWS steps is one
//                    work item, its tensor kept in shared memory between the steps.
// Dense tensor-core steps run in their own pack and GEMM launches (kernels_tc.cu).
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

// One thread per leaf: the leaf's complex128 entries are read in bursts of 8 independent loads,
// converted to the storage type, and reduced to the leaf's max-abs (gate tensors have at most 16
// entries, so a leaf costs one or two memory latencies).
template <typename T>
__global__ void __launch_bounds__(128) k_leaf_convert(const JobPtrs *__restrict__ jobs) {
    using C = cx_t<T>;
    const JobPtrs &j = jobs[blockIdx.y];
    const int32_t leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= j.n_leaves) return;
    const int64_t b = j.leaf_off[leaf], e = j.leaf_off[leaf + 1];
    C *dst = static_cast<C *>(const_cast<void *>(j.leaf));
    float mx = 0.f;
    constexpr int U = 8;
    for (int64_t i0 = b; i0 < e; i0 += U) {
        double2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u < e) v[u] = j.leaf64[i0 + u];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u < e) {
                const C w = cmake((T)v[u].x, (T)v[u].y);
                dst[i0 + u] = w;
                mx = fmaxf(mx, absmax2(w));
            }
    }
    j.maxbits[leaf] = __float_as_uint(mx);
    j.exp2[leaf] = 0;
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

// Warp programs: every warp of the block runs its own program (no block barrier), in its own
// kWarpSlice-byte slice of shared memory, and publishes its pseudo-step as complete.
template <typename T>
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
    if (prof && lane == 0) t0 = clock64();
    run_warp_prog<T>(prog, j, dyn + warp * kWarpSlice);
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        atomicAdd(j.done + it.step, 1);
        if (prof) {
            atomicAdd((unsigned long long *)(prof + 10), (unsigned long long)(clock64() - t0));
            atomicAdd((unsigned long long *)(prof + kProfSlots + 10), 1ull);
        }
    }
}

// All subtree programs of a batch: one block per program (they depend on leaves only).  Each
// publishes its pseudo-step as complete, so the dataflow kernel that runs next never waits on it.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_local(const JobPtrs *__restrict__ jobs,
                                                    const WorkItem *__restrict__ items, long long *prof) {
    extern __shared__ __align__(16) char dyn[];
    __shared__ __align__(16) char smem[Scratch<T>::local];
    const WorkItem it = items[blockIdx.x];
    const JobPtrs &j = jobs[it.job];
    const int32_t prog = __ldcg(&j.steps[it.step].tile_rows);
    long long t0 = 0;
    if (prof && threadIdx.x == 0) t0 = clock64();
    run_local<T>(prog, j, dyn, smem, prof);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(j.done + it.step, 1);
        if (prof) {   // slot 5: block programs, 6: large programs
            const int slot = __ldcg(&j.progs[prog].kind) == PROG_BIG ? 6 : STEP_LOCAL;
            atomicAdd((unsigned long long *)(prof + slot), (unsigned long long)(clock64() - t0));
            atomicAdd((unsigned long long *)(prof + kProfSlots + slot), 1ull);
        }
    }
}

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

// Scatter staged tensor updates {dst offset, count, src offset} into the complex128 leaves.
__global__ void __launch_bounds__(128) k_scatter_updates(const int64_t *__restrict__ hdr,
                                                         const double2 *__restrict__ vals,
                                                         int64_t n_upd, double2 *__restrict__ leaf64) {
    for (int64_t u = blockIdx.x * 4 + (threadIdx.x >> 5); u < n_upd; u += (int64_t)gridDim.x * 4) {
        const int64_t dst = hdr[3 * u], cnt = hdr[3 * u + 1], src = hdr[3 * u + 2];
        for (int64_t i = threadIdx.x & 31; i < cnt; i += 32) leaf64[dst + i] = vals[src + i];
    }
}

template <typename T>
__global__ void k_finish_leaf(JobPtrs j) {
    const cx_t<T> v = static_cast<const cx_t<T> *>(j.leaf)[0];
    DeviceResult *r = static_cast<DeviceResult *>(j.result);
    r->re = (double)v.x;
    r->im = (double)v.y;
    r->exp2 = 0;
}

}  // namespace

cudaError_t launch_leaf_convert(bool c128, const JobPtrs *jobs_dev, int32_t n_jobs,
                                int32_t max_leaves, cudaStream_t stream) {
    if (n_jobs <= 0 || max_leaves <= 0) return cudaSuccess;
    dim3 grid((unsigned)((max_leaves + 127) / 128), (unsigned)n_jobs);
    if (c128) k_leaf_convert<double><<<grid, 128, 0, stream>>>(jobs_dev);
    else k_leaf_convert<float><<<grid, 128, 0, stream>>>(jobs_dev);
    return cudaGetLastError();
}

// Static plus dynamic shared memory above 48 KB per block needs an opt-in for the dynamic part;
// it is set whenever a kernel takes dynamic shared memory (a cheap host call).
template <typename K>
cudaError_t allow_dyn_smem(K kernel, int32_t bytes) {
    if (bytes <= 0) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_step(bool c128, const StepDesc &h, int32_t step, const JobPtrs &job, int32_t dyn_smem,
                        cudaStream_t stream) {
    if (h.ntiles <= 0 || h.kind == STEP_TC) return cudaErrorInvalidValue;   // TC: launch_tc_pack / _gemm
    const int32_t dyn = h.kind == STEP_LOCAL ? dyn_smem : ((h.flags & FLAG_A_SMEM) ? kPersistDynSmem : 0);
    cudaError_t e = c128 ? allow_dyn_smem(k_step<double>, dyn) : allow_dyn_smem(k_step<float>, dyn);
    if (e != cudaSuccess) return e;
    if (c128) k_step<double><<<(unsigned)h.ntiles, kThreads, dyn, stream>>>(job.steps, step, job);
    else k_step<float><<<(unsigned)h.ntiles, kThreads, dyn, stream>>>(job.steps, step, job);
    return cudaGetLastError();
}

cudaError_t launch_finish_leaf(bool c128, const JobPtrs &job, cudaStream_t stream) {
    if (c128) k_finish_leaf<double><<<1, 1, 0, stream>>>(job);
    else k_finish_leaf<float><<<1, 1, 0, stream>>>(job);
    return cudaGetLastError();
}

cudaError_t launch_scatter_updates(const int64_t *hdr, const double2 *vals, int64_t n_upd,
                                   double2 *leaf64, cudaStream_t stream) {
    if (n_upd <= 0) return cudaSuccess;
    int64_t blocks = (n_upd + 3) / 4;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_scatter_updates<<<(unsigned)blocks, 128, 0, stream>>>(hdr, vals, n_upd, leaf64);
    return cudaGetLastError();
}

int32_t persistent_grid(bool c128) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cudaError_t e;
    if (c128) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<double, false>, kThreads, 0);
    } else {
        e = allow_dyn_smem(k_persist<float, false>, kPersistDynSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<float, false>, kThreads, kPersistDynSmem);
    }
    if (e != cudaSuccess) return 0;
    return sms * per_sm;
}

cudaError_t launch_local(bool c128, const JobPtrs *jobs_dev, const WorkItem *items, int32_t n_warp,
                         int32_t n_block, int32_t n_big, int32_t dyn_smem, int32_t dyn_big, long long *prof,
                         cudaStream_t stream) {
    if (n_warp > 0) {
        constexpr int per_block = kWarpThreads / 32;
        const int32_t smem = per_block * kWarpSlice;
        cudaError_t e = c128 ? allow_dyn_smem(k_warp<double>, smem) : allow_dyn_smem(k_warp<float>, smem);
        if (e != cudaSuccess) return e;
        const unsigned grid = (unsigned)((n_warp + per_block - 1) / per_block);
        if (c128) k_warp<double><<<grid, kWarpThreads, smem, stream>>>(jobs_dev, items, n_warp, prof);
        else k_warp<float><<<grid, kWarpThreads, smem, stream>>>(jobs_dev, items, n_warp, prof);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // block programs, then the large ones (each launch with its own shared-memory size)
    const int32_t counts[2] = {n_block, n_big}, dyn[2] = {dyn_smem, dyn_big};
    const WorkItem *it = items + n_warp;
    for (int q = 0; q < 2; ++q) {
        if (counts[q] <= 0) continue;
        cudaError_t e = c128 ? allow_dyn_smem(k_local<double>, dyn[q]) : allow_dyn_smem(k_local<float>, dyn[q]);
        if (e != cudaSuccess) return e;
        if (c128) k_local<double><<<counts[q], kThreads, dyn[q], stream>>>(jobs_dev, it, prof);
        else k_local<float><<<counts[q], kThreads, dyn[q], stream>>>(jobs_dev, it, prof);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        it += counts[q];
    }
    return cudaSuccess;
}

int32_t local_smem_budget(bool c128, int32_t blocks_per_sm) {
    int dev = 0, per_sm = 0, per_block = 0, reserved = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) return 0;
    cudaFuncAttributes fa;
    cudaError_t e = c128 ? cudaFuncGetAttributes(&fa, k_local<double>) : cudaFuncGetAttributes(&fa, k_local<float>);
    if (e != cudaSuccess) return 0;
    int32_t b = per_sm / blocks_per_sm - reserved - (int32_t)fa.sharedSizeBytes;
    if (b > per_block - (int32_t)fa.sharedSizeBytes) b = per_block - (int32_t)fa.sharedSizeBytes;
    return b > 0 ? (b / 16) * 16 : 0;
}

cudaError_t launch_persistent(bool c128, const JobPtrs *jobs_dev, const WorkItem *work, int64_t n_work,
                              uint32_t *counter, int32_t grid, long long wait_ns, long long *prof,
                              cudaStream_t stream) {
    if (n_work <= 0) return cudaSuccess;
    if (grid > n_work) grid = (int32_t)n_work;
    if (c128) {
        if (prof)
            k_persist<double, true><<<(unsigned)grid, kThreads, 0, stream>>>(jobs_dev, work, n_work, counter,
                                                                            wait_ns, prof);
        else
            k_persist<double, false><<<(unsigned)grid, kThreads, 0, stream>>>(jobs_dev, work, n_work, counter,
                                                                             wait_ns, nullptr);
    } else {
        auto kern = prof ? k_persist<float, true> : k_persist<float, false>;
        const cudaError_t e = allow_dyn_smem(kern, kPersistDynSmem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)grid, kThreads, kPersistDynSmem, stream>>>(jobs_dev, work, n_work, counter, wait_ns, prof);
    }
    return cudaGetLastError();
}

}  // namespace tn
