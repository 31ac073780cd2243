// Contraction kernels for sm_103a, in five translation units that compile in parallel:
//
//  * kernels_contract.cu    k_leaf_convert: complex128 leaves -> storage type, with each leaf's
//                           max-abs (one thread per small leaf; blocks per slice of a large leaf);
//                           k_scatter_updates, k_finish_leaf
//  * kernels_step.cu        k_step: one step of one job, one block per work tile (graph mode)
//  * kernels_local.cu       k_warp: warp programs (subtrees of small steps, one warp each);
//                           k_local: one block per CTA-resident subtree program (all operands in
//                           shared memory), block programs and large programs in two launches
//  * kernels_persist_*.cu   k_persist: the persistent dataflow kernel (complex64, complex128)
// Dense tensor-core steps run in their own pack and GEMM launches (kernels_tc.cu).
#include "contract_common.cuh"

namespace tn {

namespace {

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

// Leaves of more than kLeafSmall entries (dense operands): blocks (leaf, job, slice) stream the
// leaf with coalesced loads, slice z taking every gridDim.z-th run of blockDim.x entries, and
// merge their max-abs into the leaf's (zeroed) slot with an atomic max on the float bits.
constexpr int64_t kLeafSmall = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_leaf_convert_wide(const JobPtrs *__restrict__ jobs) {
    using C = cx_t<T>;
    __shared__ float red[32];
    const JobPtrs &j = jobs[blockIdx.y];
    const int32_t leaf = blockIdx.x;
    if (leaf >= j.n_leaves) return;   // block-uniform
    const int64_t b = j.leaf_off[leaf], e = j.leaf_off[leaf + 1];
    C *dst = static_cast<C *>(const_cast<void *>(j.leaf));
    float mx = 0.f;
    const int64_t stride = (int64_t)gridDim.z * blockDim.x;
    for (int64_t i = b + (int64_t)blockIdx.z * blockDim.x + threadIdx.x; i < e; i += stride) {
        const double2 v = j.leaf64[i];
        const C w = cmake((T)v.x, (T)v.y);
        dst[i] = w;
        mx = fmaxf(mx, absmax2(w));
    }
    mx = warp_max(mx);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
        if (mx > 0.f) atomicMax(j.maxbits + leaf, __float_as_uint(mx));
        if (blockIdx.z == 0) j.exp2[leaf] = 0;
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
                                int32_t max_leaves, int64_t max_leaf_elems, cudaStream_t stream) {
    if (n_jobs <= 0 || max_leaves <= 0) return cudaSuccess;
    if (max_leaf_elems > kLeafSmall) {
        // about 64 entries per thread for the largest leaf, at most 1024 slices
        const int64_t z = std::min<int64_t>(1024, std::max<int64_t>(1, (max_leaf_elems + 256 * 64 - 1) / (256 * 64)));
        const dim3 grid((unsigned)max_leaves, (unsigned)n_jobs, (unsigned)z);
        if (c128) k_leaf_convert_wide<double><<<grid, 256, 0, stream>>>(jobs_dev);
        else k_leaf_convert_wide<float><<<grid, 256, 0, stream>>>(jobs_dev);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((max_leaves + 127) / 128), (unsigned)n_jobs);
    if (c128) k_leaf_convert<double><<<grid, 128, 0, stream>>>(jobs_dev);
    else k_leaf_convert<float><<<grid, 128, 0, stream>>>(jobs_dev);
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

}  // namespace tn
