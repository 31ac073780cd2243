// Axis permutation of a row-major tensor (the "T" of TTGT, Section 5.1): out axis t = in axis
// perm[t].  Moves bytes only, so it is exact for any payload.  Axes that stay adjacent and in
// order are fused first.  When the innermost axis survives the permutation, each thread copies
// one element along it (coalesced on both sides); otherwise a 32 x 32 tile of (output-innermost,
// input-innermost) is staged in shared memory so that both the reads and the writes are
// coalesced.
#include <cstdint>
#include <vector>

#include "kernels.cuh"

namespace tn {

namespace {

constexpr int kMaxRank = 32;

struct PermPlan {
    int32_t rank;                 // fused output rank
    int64_t odim[kMaxRank];       // output dims, axis 0 slowest
    int64_t istride[kMaxRank];    // input stride of each output axis
    int64_t ostride[kMaxRank];    // output stride of each output axis
    int32_t a;                    // output-innermost axis (index into the arrays above)
    int32_t b;                    // axis that is innermost in the input (-1 if same as a)
    int64_t total;
};

template <typename E>
__global__ void __launch_bounds__(256) k_perm_gather(const E *__restrict__ in, E *__restrict__ out,
                                                     PermPlan p) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = i, src = 0;
        for (int32_t t = p.rank - 1; t >= 0; --t) {
            int64_t dgt = rem % p.odim[t];
            rem /= p.odim[t];
            src += dgt * p.istride[t];
        }
        out[i] = in[src];
    }
}

template <typename E>
__global__ void __launch_bounds__(256) k_perm_tile(const E *__restrict__ in, E *__restrict__ out,
                                                   PermPlan p, int64_t tiles_a, int64_t tiles_b) {
    __shared__ E tile[32][33];
    const int64_t da = p.odim[p.a], db = p.odim[p.b];
    int64_t blk = blockIdx.x;
    const int64_t ta = blk % tiles_a;
    blk /= tiles_a;
    const int64_t tb = blk % tiles_b;
    int64_t batch = blk / tiles_b;
    int64_t ibase = 0, obase = 0;
    for (int32_t t = p.rank - 1; t >= 0; --t) {
        if (t == p.a || t == p.b) continue;
        int64_t dgt = batch % p.odim[t];
        batch /= p.odim[t];
        ibase += dgt * p.istride[t];
        obase += dgt * p.ostride[t];
    }
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    const int64_t a0 = ta * 32, b0 = tb * 32;
    // read: consecutive threads walk the input-innermost axis b (input stride 1)
    for (int r = ty; r < 32; r += 8) {
        int64_t ai = a0 + r, bi = b0 + tx;
        if (ai < da && bi < db) tile[r][tx] = in[ibase + ai * p.istride[p.a] + bi];
    }
    __syncthreads();
    // write: consecutive threads walk the output-innermost axis a (output stride 1)
    for (int r = ty; r < 32; r += 8) {
        int64_t bi = b0 + r, ai = a0 + tx;
        if (ai < da && bi < db) out[obase + bi * p.ostride[p.b] + ai] = tile[tx][r];
    }
}

template <typename E>
cudaError_t perm_launch(const void *src, void *dst, const PermPlan &p, cudaStream_t st) {
    const E *in = static_cast<const E *>(src);
    E *out = static_cast<E *>(dst);
    if (p.total == 0) return cudaSuccess;
    if (p.b < 0) {
        int64_t blocks = (p.total + 255) / 256;
        if (blocks > 152 * 32) blocks = 152 * 32;
        k_perm_gather<E><<<(unsigned)blocks, 256, 0, st>>>(in, out, p);
    } else {
        int64_t da = p.odim[p.a], db = p.odim[p.b];
        int64_t ta = (da + 31) / 32, tb = (db + 31) / 32;
        int64_t batch = p.total / (da * db);
        int64_t blocks = ta * tb * batch;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        k_perm_tile<E><<<(unsigned)blocks, 256, 0, st>>>(in, out, p, ta, tb);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_permute(const void *src, void *dst, int32_t elem_bytes, int32_t rank,
                           const int64_t *dims, const int32_t *perm, cudaStream_t stream) {
    // input strides
    std::vector<int64_t> istr(rank);
    int64_t acc = 1;
    for (int32_t t = rank - 1; t >= 0; --t) { istr[t] = acc; acc *= dims[t]; }
    const int64_t total = acc;
    // output axes (dims of 1 dropped), fused when adjacent in the input in the same order
    std::vector<int64_t> od, is;
    for (int32_t t = 0; t < rank; ++t) {
        int64_t d = dims[perm[t]], s = istr[perm[t]];
        if (d == 1) continue;
        if (!od.empty() && is.back() == d * s) {
            od.back() *= d;
            is.back() = s;
        } else {
            od.push_back(d);
            is.push_back(s);
        }
    }
    PermPlan p{};
    p.total = total;
    p.rank = (int32_t)od.size();
    if (p.rank > kMaxRank) return cudaErrorInvalidValue;
    acc = 1;
    for (int32_t t = p.rank - 1; t >= 0; --t) {
        p.odim[t] = od[t];
        p.istride[t] = is[t];
        p.ostride[t] = acc;
        acc *= od[t];
    }
    p.a = p.rank - 1;
    p.b = -1;
    if (p.rank >= 2 && p.istride[p.a] != 1) {
        for (int32_t t = 0; t < p.rank; ++t)
            if (p.istride[t] == 1) p.b = t;
    }
    if (p.rank == 0) { p.rank = 1; p.odim[0] = 1; p.istride[0] = 1; p.ostride[0] = 1; p.a = 0; }
    switch (elem_bytes) {
        case 1: return perm_launch<uint8_t>(src, dst, p, stream);
        case 2: return perm_launch<uint16_t>(src, dst, p, stream);
        case 4: return perm_launch<uint32_t>(src, dst, p, stream);
        case 8: return perm_launch<uint64_t>(src, dst, p, stream);
        case 16: return perm_launch<uint4>(src, dst, p, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tn
