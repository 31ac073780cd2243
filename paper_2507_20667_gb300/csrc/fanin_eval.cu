// Batched evaluation of fan-in trees on the GPU (Section 4.4, EvaluateState; the RandomGreedy
// samples of Algorithm 1's DoSteps are the planner's hot loop for large k).  One block per
// (state, sample): the block runs one Greedy pass over the state's k partition results, every
// thread scoring a share of the live pairs with the shared integer objective (fanin_core.cuh),
// a block reduction picking the best pair with the host planner's tie rule, and thread 0 then
// evaluates the merge sequence (con_dist of Eq. 3.5, the fan-in's con and mem) in 128-bit
// integers.  The host keeps, per state, the best sample (smallest con_dist, then con, then the
// lowest sample index), exactly as the host planner does.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fanin_core.cuh"
#include "tn_internal.hpp"

namespace tn {

namespace {

constexpr int kThreadsF = 256;

struct DevJob {
    int32_t k, W, unit, pad;
    uint64_t seed;
    int64_t roots;   // offset (uint64 words) of the roots' leg sets [k][W]
    int64_t con;     // offset (u128) of the partition results' con [k]
    int64_t dims;    // offset (int64) of the compact edge dimensions [64 W] (unit: unused)
};

struct DevOut {
    fanin::u128 con_dist, con, mem;
    int32_t sat, pad[3];
};

struct Best {
    fanin::i128 score;
    int32_t i, j;
};

__device__ __forceinline__ bool best_less(const Best &a, const Best &b) {   // b comes before a
    if (a.i < 0) return b.i >= 0;
    if (b.i < 0) return false;
    return fanin::pair_before(b.score, b.i, b.j, a.score, a.i, a.j);
}

__global__ void __launch_bounds__(kThreadsF) k_fanin_samples(const DevJob *__restrict__ jobs,
                                                             const uint64_t *__restrict__ roots,
                                                             const fanin::u128 *__restrict__ cons,
                                                             const int64_t *__restrict__ dims, int32_t samples,
                                                             DevOut *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    const DevJob jb = jobs[blockIdx.x];
    const int s = blockIdx.y;
    const int k = jb.k, W = jb.W, nn = 2 * k - 1;
    // shared layout: size [nn] u128, cost [nn] u128, con [k] u128, legs [nn W] u64, steps [2(k-1)] i16,
    // parent [nn] i16, alive list [k] i16, alive flags [nn] u8
    fanin::u128 *size = reinterpret_cast<fanin::u128 *>(sm);
    fanin::u128 *cost = size + nn;
    fanin::u128 *con = cost + nn;
    uint64_t *legs = reinterpret_cast<uint64_t *>(con + k);
    int16_t *steps = reinterpret_cast<int16_t *>(legs + (size_t)nn * W);
    int16_t *parent = steps + 2 * (k - 1) + 2;
    int16_t *al = parent + nn;
    uint8_t *alive = reinterpret_cast<uint8_t *>(al + k);
    __shared__ Best red[kThreadsF / 32];
    __shared__ int32_t s_m, s_bi, s_bj;
    __shared__ int32_t s_sat;
    const fanin::Dims d{W, jb.unit, dims + jb.dims};
    for (int x = threadIdx.x; x < k * W; x += blockDim.x) legs[x] = roots[jb.roots + x];
    for (int x = threadIdx.x; x < k; x += blockDim.x) con[x] = cons[jb.con + x];
    if (threadIdx.x == 0) {
        bool sat = false;
        for (int i = 0; i < k; ++i) {
            size[i] = fanin::set_size(legs + (size_t)i * W, legs + (size_t)i * W, 0, d, sat);
            alive[i] = 1;
            al[i] = (int16_t)i;
        }
        s_m = k;
        s_sat = sat;
    }
    __syncthreads();
    const bool noisy = s > 0;
    const uint64_t seed = noisy ? fanin::sample_seed(jb.seed, s) : 0;
    for (int it = 0; it < k - 1; ++it) {
        const int m = s_m;
        const int npairs = m * (m - 1) / 2;
        Best mine{0, -1, -1};
        bool sat = false;
        // pair p -> (a, b), a < b over the alive list, rows a = 0, 1, ...
        int a = 0, rowlen = m - 1, base = 0;
        for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
            while (p >= base + rowlen) {
                base += rowlen;
                ++a;
                --rowlen;
            }
            const int b = a + 1 + (p - base);
            const int i = al[a], j = al[b];
            const uint64_t *li = legs + (size_t)i * W, *lj = legs + (size_t)j * W;
            if (!fanin::intersects(li, lj, W)) continue;
            const fanin::i128 obj =
                (fanin::i128)size[i] + (fanin::i128)size[j] - (fanin::i128)fanin::set_size(li, lj, 1, d, sat);
            const Best cand{fanin::pair_score(obj, noisy, seed, (uint32_t)i, (uint32_t)j), i, j};
            if (best_less(mine, cand)) mine = cand;
        }
        if (sat) s_sat = 1;
        // block reduction (score descending, then i, then j ascending)
        for (int o = 16; o > 0; o >>= 1) {
            Best other;
            const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)(uint64_t)mine.score, o);
            const unsigned long long hi =
                __shfl_down_sync(0xffffffffu, (unsigned long long)(uint64_t)(mine.score >> 64), o);
            other.score = (fanin::i128)(((fanin::u128)hi << 64) | (fanin::u128)lo);
            other.i = __shfl_down_sync(0xffffffffu, mine.i, o);
            other.j = __shfl_down_sync(0xffffffffu, mine.j, o);
            if (best_less(mine, other)) mine = other;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            Best b = red[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (best_less(b, red[w])) b = red[w];
            int bi = b.i, bj = b.j;
            const int next = k + it;
            if (bi < 0) {   // no connected pair: the two smallest (size, then id)
                int x = -1, y = -1;
                for (int v = 0; v < next; ++v) {
                    if (!alive[v]) continue;
                    if (x < 0 || size[v] < size[x]) {
                        y = x;
                        x = v;
                    } else if (y < 0 || size[v] < size[y]) {
                        y = v;
                    }
                }
                bi = x < y ? x : y;
                bj = x < y ? y : x;
            }
            s_bi = bi;
            s_bj = bj;
            steps[2 * it] = (int16_t)bi;
            steps[2 * it + 1] = (int16_t)bj;
            alive[bi] = alive[bj] = 0;
            alive[next] = 1;
            int q = 0;
            for (int v = 0; v < m; ++v)
                if (al[v] != bi && al[v] != bj) al[q++] = al[v];
            al[q++] = (int16_t)next;
            s_m = q;
        }
        __syncthreads();
        const int next = k + it;
        for (int w = threadIdx.x; w < W; w += blockDim.x)
            legs[(size_t)next * W + w] = legs[(size_t)s_bi * W + w] ^ legs[(size_t)s_bj * W + w];
        __syncthreads();
        if (threadIdx.x == 0) {
            bool sat2 = false;
            size[next] = fanin::set_size(legs + (size_t)next * W, legs + (size_t)next * W, 0, d, sat2);
            if (sat2) s_sat = 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const fanin::Counts c = fanin::eval_steps(k, con, steps, d, legs, size, parent, cost);
        DevOut &o = out[(size_t)blockIdx.x * samples + s];
        o.con_dist = c.con_dist;
        o.con = c.con;
        o.mem = c.mem;
        o.sat = (c.sat || s_sat) ? 1 : 0;
    }
}

size_t smem_for(int k, int W) {
    const size_t nn = 2 * (size_t)k - 1;
    size_t b = (2 * nn + k) * sizeof(fanin::u128) + nn * W * sizeof(uint64_t) + (2 * (size_t)k + nn + k) * 2 + nn;
    return (b + 15) / 16 * 16;
}

}  // namespace

// Evaluate the fan-in trees of many states on `device`: for every input its RandomGreedy samples
// (k > 4 only) in one launch; result[i] = the best sample's counts and index.
tn_status fanin_eval_device(int32_t device, const std::vector<FaninInput> &ins, int32_t samples,
                            std::vector<FaninBest> &result, FaninWorkspace &ws) {
    result.assign(ins.size(), FaninBest());
    if (ins.empty()) return TN_OK;
    samples = std::max(samples, 1);
    std::vector<DevJob> jobs(ins.size());
    size_t n_roots = 0, n_con = 0, n_dims = 0, smem = 0;
    for (size_t q = 0; q < ins.size(); ++q) {
        const FaninInput &in = ins[q];
        if (in.k < 5 || in.k > fanin::kMaxK || in.W < 1 || in.W > fanin::kMaxWords)
            return fail(TN_EUNSUPPORTED, "the GPU fan-in evaluator takes 5 <= k <= 256 and at most 2048 cut legs");
        jobs[q] = DevJob{in.k, in.W, in.unit ? 1 : 0, 0, in.seed, (int64_t)n_roots, (int64_t)n_con, (int64_t)n_dims};
        n_roots += in.roots.size();
        n_con += in.part_con.size();
        n_dims += in.dims.size();
        smem = std::max(smem, smem_for(in.k, in.W));
    }
    if (smem > 200 * 1024) return fail(TN_EUNSUPPORTED, "fan-in problem too large for shared memory");
    const size_t b_jobs = jobs.size() * sizeof(DevJob), b_roots = std::max<size_t>(n_roots, 1) * 8,
                 b_con = std::max<size_t>(n_con, 1) * 16, b_dims = std::max<size_t>(n_dims, 1) * 8,
                 b_out = ins.size() * (size_t)samples * sizeof(DevOut);
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_jobs = 0, o_roots = al(b_jobs), o_con = o_roots + al(b_roots), o_dims = o_con + al(b_con),
                 o_out = o_dims + al(b_dims), total = o_out + al(b_out);
    if (cudaSetDevice(device) != cudaSuccess) return fail(TN_ECUDA, "cudaSetDevice");
    if (!ws.stream) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fail(TN_ECUDA, "cudaStreamCreate");
        ws.stream = st;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(ws.stream);
    if (total > ws.cap) {
        if (ws.d_buf) cudaFree(ws.d_buf);
        if (ws.h_buf) cudaFreeHost(ws.h_buf);
        ws.d_buf = nullptr;
        ws.h_buf = nullptr;
        ws.cap = 0;
        if (cudaMalloc(&ws.d_buf, total * 2) != cudaSuccess || cudaMallocHost(&ws.h_buf, total * 2) != cudaSuccess)
            return fail(TN_ENOMEM, "fan-in evaluator buffers");
        ws.cap = total * 2;
    }
    char *h = static_cast<char *>(ws.h_buf);
    std::memcpy(h + o_jobs, jobs.data(), b_jobs);
    size_t r = 0, c = 0, dd = 0;
    for (const FaninInput &in : ins) {
        std::memcpy(h + o_roots + r * 8, in.roots.data(), in.roots.size() * 8);
        std::memcpy(h + o_con + c * 16, in.part_con.data(), in.part_con.size() * 16);
        if (!in.dims.empty()) std::memcpy(h + o_dims + dd * 8, in.dims.data(), in.dims.size() * 8);
        r += in.roots.size();
        c += in.part_con.size();
        dd += in.dims.size();
    }
    char *d = static_cast<char *>(ws.d_buf);
    cudaError_t e = cudaMemcpyAsync(d, h, o_out, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fanin_samples, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        dim3 grid((unsigned)ins.size(), (unsigned)samples);
        k_fanin_samples<<<grid, kThreadsF, smem, stream>>>(
            reinterpret_cast<const DevJob *>(d + o_jobs), reinterpret_cast<const uint64_t *>(d + o_roots),
            reinterpret_cast<const fanin::u128 *>(d + o_con), reinterpret_cast<const int64_t *>(d + o_dims), samples,
            reinterpret_cast<DevOut *>(d + o_out));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + o_out, d + o_out, b_out, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(TN_ECUDA, std::string("fan-in evaluator: ") + cudaGetErrorString(e));
    const DevOut *o = reinterpret_cast<const DevOut *>(h + o_out);
    for (size_t q = 0; q < ins.size(); ++q) {
        FaninBest &b = result[q];
        for (int s = 0; s < samples; ++s) {
            const DevOut &x = o[q * (size_t)samples + s];
            fanin::Counts cs{x.con_dist, x.con, x.mem, x.sat != 0};
            if (s == 0 || fanin::better(cs, b.counts)) {
                b.counts = cs;
                b.sample = s;
            }
            b.counts.sat = b.counts.sat || x.sat;
        }
    }
    return TN_OK;
}

void fanin_workspace_free(FaninWorkspace &ws) {
    if (ws.d_buf) cudaFree(ws.d_buf);
    if (ws.h_buf) cudaFreeHost(ws.h_buf);
    if (ws.stream) cudaStreamDestroy(static_cast<cudaStream_t>(ws.stream));
    ws = FaninWorkspace();
}

}  // namespace tn
