// Axis permutation of a row-major tensor (the "T" of TTGT, Section 5.1): out axis t = in axis
// perm[t].  Moves bytes only, so it is exact for any payload.  Axes that stay adjacent and in
// order are fused first.  When the innermost axis survives the permutation, the tensor is a set
// of contiguous rows moved as wholes: a group of lanes per row, whose first lane computes the
// row's source offset and broadcasts it with a shuffle, copies the row in 16-byte vectors when both
// ends are 16-byte aligned (element by element otherwise).  Otherwise a tile of
// (output-innermost, input-innermost) is staged in shared memory so that both the reads and the
// writes are coalesced: 64 x 64 for elements of up to 8 bytes (contiguous runs of 512 bytes on
// both sides for 8-byte elements, instead of 256), 32 x 32 otherwise.
#include <algorithm>
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
    int32_t pow2;                 // every output dim is a power of two: digits by shift and mask
    int32_t lg[kMaxRank];         // log2 of each output dim (pow2 only)
};

// Input offset of output row r (all axes but the innermost, p.a); the digits come out by shift
// and mask when every dim is a power of two.
__device__ __forceinline__ int64_t row_src(const PermPlan &p, int64_t r) {
    int64_t src = 0;
    if (p.pow2) {
        for (int32_t t = p.rank - 1; t >= 0; --t) {
            if (t == p.a) continue;
            src += (r & (p.odim[t] - 1)) * p.istride[t];
            r >>= p.lg[t];
        }
    } else {
        for (int32_t t = p.rank - 1; t >= 0; --t) {
            if (t == p.a) continue;
            const int64_t dgt = r % p.odim[t];
            r /= p.odim[t];
            src += dgt * p.istride[t];
        }
    }
    return src;
}

// Row copy: the output is rows of length odim[a] (the fused innermost axis, stride 1 on both
// sides).  A group of G lanes (G = 16-byte vectors per row, at most 32, a power of two) moves one
// row: its first lane computes the row's source offset and shares it with a shuffle, and the group
// copies the row in 16-byte vectors (element by element when a row is not 16-byte aligned).
template <typename E>
__global__ void __launch_bounds__(256) k_perm_rows(const E *__restrict__ in, E *__restrict__ out, PermPlan p,
                                                   int32_t G) {
    const int lane = threadIdx.x & 31, sub = lane & (G - 1), grp = lane / G;
    const int64_t len = p.odim[p.a], rows = p.total / len;
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 5) * (32 / G);
    const bool vec = (len * (int64_t)sizeof(E)) % 16 == 0 && sizeof(E) <= 16 &&
                     (reinterpret_cast<uintptr_t>(in) % 16) == 0 && (reinterpret_cast<uintptr_t>(out) % 16) == 0;
    constexpr int per = 16 / sizeof(E) > 0 ? 16 / (int)sizeof(E) : 1;   // elements per 16-byte vector
    const int64_t first = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / G) + grp;
    // every lane runs the same number of iterations (the shuffle needs the whole warp)
    const int64_t iters = (rows + groups - 1) / groups;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t r = first + it * groups;
        int64_t src = 0;
        if (sub == 0 && r < rows) src = row_src(p, r);
        src = __shfl_sync(0xffffffffu, src, lane - sub);
        if (r >= rows) continue;
        const E *ip = in + src;
        E *op = out + r * len;
        if (vec) {
            const uint4 *iv = reinterpret_cast<const uint4 *>(ip);
            uint4 *ov = reinterpret_cast<uint4 *>(op);
            const int64_t nv = len / per;
            for (int64_t i = sub; i < nv; i += G) ov[i] = __ldg(iv + i);
        } else {
            for (int64_t i = sub; i < len; i += G) op[i] = __ldg(ip + i);
        }
    }
}

// Short rows (fewer than 64 bytes): one thread per row, copying it element by element; the
// threads of a warp write consecutive rows, so the writes stay coalesced.
template <typename E>
__global__ void __launch_bounds__(256) k_perm_short_rows(const E *__restrict__ in, E *__restrict__ out,
                                                         PermPlan p) {
    const int64_t len = p.odim[p.a], rows = p.total / len;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = row_src(p, r);
        for (int64_t i = 0; i < len; ++i) out[r * len + i] = __ldg(in + src + i);
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

// Grouped tile, for permutations of many short axes (the bit permutations of qubit tensors): the
// output's innermost axes whose sizes multiply to at most 64 (or 32) form group A, the input's
// innermost axes (outside A) group B.  A block moves PA x PB tiles of (A index, B index), each for
// one index of the remaining axes, through shared memory: it reads with consecutive threads along B
// (contiguous in the input) and writes with consecutive threads along A (contiguous in the output).
constexpr int kGroupMax = 64;   // largest group: the edge of the large tile

struct GroupTile {
    int32_t pa, pb;                           // sizes of the two groups (products of their dims)
    int32_t nrest;
    int64_t in_a[kGroupMax], out_a[kGroupMax];   // offsets of each A index in the input / output
    int64_t in_b[kGroupMax], out_b[kGroupMax];   // same for B
    int64_t rdim[kMaxRank], rin[kMaxRank], rout[kMaxRank];   // remaining axes, outermost first
};

// TE: tile edge (groups of at most TE elements); kTiles tiles per block, TE * TE / 256 elements of
// each per thread.
template <typename E, int TE, int kTiles>
__global__ void __launch_bounds__(256) k_perm_group_tile(const E *__restrict__ in, E *__restrict__ out,
                                                         const GroupTile g, int64_t n_tiles) {
    constexpr int kPer = TE * TE / 256;
    static_assert(kPer * 256 == TE * TE && TE <= kGroupMax && TE + kTiles <= 256, "tile split");
    __shared__ E tile[TE][TE + 1];
    __shared__ int64_t s_in_a[TE], s_out_a[TE], s_in_b[TE], s_out_b[TE], s_ib[kTiles], s_ob[kTiles];
    const int tid = threadIdx.x;
    // the offset tables move from the parameters to shared memory once (the arithmetic loops index
    // them per thread), and the next kTiles threads decompose the block's tile indices
    if (tid < TE) {
        s_in_a[tid] = tid < g.pa ? g.in_a[tid] : 0;
        s_out_a[tid] = tid < g.pa ? g.out_a[tid] : 0;
        s_in_b[tid] = tid < g.pb ? g.in_b[tid] : 0;
        s_out_b[tid] = tid < g.pb ? g.out_b[tid] : 0;
    } else if (tid < TE + kTiles) {
        int64_t blk = (int64_t)blockIdx.x * kTiles + (tid - TE), ib = 0, ob = 0;
        for (int32_t t = g.nrest - 1; t >= 0; --t) {
            const int64_t dgt = blk % g.rdim[t];
            blk /= g.rdim[t];
            ib += dgt * g.rin[t];
            ob += dgt * g.rout[t];
        }
        s_ib[tid - TE] = ib;
        s_ob[tid - TE] = ob;
    }
    __syncthreads();
    // every read of the block's tiles is issued first (kTiles x kPer loads in flight per thread),
    // then each tile goes through shared memory in turn
    const int n = g.pa * g.pb;                       // at most TE * TE: kPer per thread
    int nq = kTiles;
    if ((int64_t)blockIdx.x * kTiles + nq > n_tiles) nq = (int)(n_tiles - (int64_t)blockIdx.x * kTiles);
    E v[kTiles][kPer];
#pragma unroll
    for (int q = 0; q < kTiles; ++q)
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int e = tid + u * 256;
            if (q < nq && e < n) {
                const int b = e % g.pb, a = e / g.pb;
                v[q][u] = __ldg(in + s_ib[q] + s_in_a[a] + s_in_b[b]);
            }
        }
#pragma unroll
    for (int q = 0; q < kTiles; ++q) {
        if (q >= nq) break;   // block-uniform
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int e = tid + u * 256;
            if (e < n) tile[e / g.pb][e % g.pb] = v[q][u];
        }
        __syncthreads();
        const int64_t ob = s_ob[q];
        for (int e = tid; e < n; e += blockDim.x) {
            const int a = e % g.pa, b = e / g.pa;
            out[ob + s_out_a[a] + s_out_b[b]] = tile[a][b];
        }
        __syncthreads();
    }
}

// Builds the grouped tile of plan p with groups of at most `lim` elements (lim <= kGroupMax); false
// when it does not apply (groups smaller than 8 elements).
bool group_tile(const PermPlan &p, GroupTile &g, int64_t lim) {
    std::vector<char> in_a(p.rank, 0), in_b(p.rank, 0);
    int64_t pa = 1, pb = 1;
    std::vector<int32_t> ga, gb;   // innermost first
    for (int32_t t = p.rank - 1; t >= 0 && pa * p.odim[t] <= lim; --t) {
        pa *= p.odim[t];
        ga.push_back(t);
        in_a[t] = 1;
    }
    // input order: axes by decreasing input stride; group B takes the innermost ones outside A
    std::vector<int32_t> by_in(p.rank);
    for (int32_t t = 0; t < p.rank; ++t) by_in[t] = t;
    std::sort(by_in.begin(), by_in.end(), [&](int32_t x, int32_t y) { return p.istride[x] < p.istride[y]; });
    for (int32_t t : by_in) {
        if (in_a[t]) continue;
        if (pb * p.odim[t] > lim) break;
        pb *= p.odim[t];
        gb.push_back(t);
        in_b[t] = 1;
    }
    if (pa < 8 || pb < 8) return false;
    g.pa = (int32_t)pa;
    g.pb = (int32_t)pb;
    auto offsets = [&](const std::vector<int32_t> &axes, int64_t *oin, int64_t *oout, int64_t n) {
        for (int64_t idx = 0; idx < n; ++idx) {
            int64_t rem = idx, si = 0, so = 0;
            for (int32_t t : axes) {   // innermost first
                const int64_t d = rem % p.odim[t];
                rem /= p.odim[t];
                si += d * p.istride[t];
                so += d * p.ostride[t];
            }
            oin[idx] = si;
            oout[idx] = so;
        }
    };
    offsets(ga, g.in_a, g.out_a, pa);
    offsets(gb, g.in_b, g.out_b, pb);
    g.nrest = 0;
    for (int32_t t = 0; t < p.rank; ++t) {
        if (in_a[t] || in_b[t]) continue;
        g.rdim[g.nrest] = p.odim[t];
        g.rin[g.nrest] = p.istride[t];
        g.rout[g.nrest] = p.ostride[t];
        g.nrest++;
    }
    return true;
}

template <typename E>
cudaError_t perm_launch(const void *src, void *dst, const PermPlan &p, cudaStream_t st) {
    const E *in = static_cast<const E *>(src);
    E *out = static_cast<E *>(dst);
    if (p.total == 0) return cudaSuccess;
    if (p.b >= 0 && p.odim[p.a] < 32) {
        GroupTile g;
        // the 64 x 64 tile (33 KB of shared memory for 8-byte elements) when it is at least half
        // full, else the 32 x 32 tile, four per block
        if constexpr (sizeof(E) <= 8) {
            if (group_tile(p, g, 64) && (int64_t)g.pa * g.pb >= 2048) {
                const int64_t tiles = p.total / ((int64_t)g.pa * g.pb);
                if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
                k_perm_group_tile<E, 64, 1><<<(unsigned)tiles, 256, 0, st>>>(in, out, g, tiles);
                return cudaGetLastError();
            }
        }
        if (group_tile(p, g, 32)) {
            const int64_t tiles = p.total / ((int64_t)g.pa * g.pb), blocks = (tiles + 3) / 4;
            if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
            k_perm_group_tile<E, 32, 4><<<(unsigned)blocks, 256, 0, st>>>(in, out, g, tiles);
            return cudaGetLastError();
        }
    }
    if (p.b < 0) {
        const int64_t rows = p.total / p.odim[p.a];
        if (p.odim[p.a] * (int64_t)sizeof(E) < 64) {
            int64_t blocks = (rows + 255) / 256;
            if (blocks > 152 * 16) blocks = 152 * 16;
            k_perm_short_rows<E><<<(unsigned)blocks, 256, 0, st>>>(in, out, p);
        } else {
            // G lanes per row (its 16-byte vectors, rounded up to a power of two, at most 32)
            const int64_t nvec = (p.odim[p.a] * (int64_t)sizeof(E) + 15) / 16;
            int32_t G = 1;
            while (G < 32 && G < nvec) G *= 2;
            const int64_t per_block = 8 * (32 / G);
            int64_t blocks = (rows + per_block - 1) / per_block;
            if (blocks > 152 * 8) blocks = 152 * 8;
            k_perm_rows<E><<<(unsigned)blocks, 256, 0, st>>>(in, out, p, G);
        }
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
    p.pow2 = 1;
    for (int32_t t = 0; t < p.rank; ++t) {
        int32_t l = 0;
        while ((int64_t(1) << l) < p.odim[t]) ++l;
        p.lg[t] = l;
        if ((int64_t(1) << l) != p.odim[t]) p.pow2 = 0;
    }
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
