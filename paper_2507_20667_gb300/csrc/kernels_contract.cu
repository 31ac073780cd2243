// CUDA-core contraction kernels for sm_103a: the gather-fused row kernel for tiny bonds, a tiled
// complex GEMM with gathered operand loads, and the FP64-accumulating dot kernel that produces
// the final amplitude.  Every kernel reads its operands through the step's index maps, applies
// the per-node power-of-two scales and records the output's max-abs for the next step.
#include <cstdint>

#include "kernels.cuh"

namespace tn {

namespace {

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

template <typename T> using cx_t = typename Cx<T>::t;

__device__ __forceinline__ float2 cmake(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ double2 cmake(double r, double i) { return make_double2(r, i); }

template <typename C>
__device__ __forceinline__ void cfma(C &acc, const C &a, const C &b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// frexp-style exponent of the float with bit pattern `bits` (0 for zero): x = f * 2^e, f in
// [0.5, 1).  Subnormal maxima are treated as 2^-126.
__device__ __forceinline__ int32_t scale_exponent(uint32_t bits) {
    if (bits == 0u) return 0;
    int32_t e = (int32_t)((bits >> 23) & 0xffu);
    return e == 0 ? -126 : e - 126;
}

template <typename T>
__device__ __forceinline__ T pow2(int32_t e) {
    return (T)ldexp(1.0, e);
}

__device__ __forceinline__ float absmax2(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }
__device__ __forceinline__ float absmax2(double2 v) {
    return (float)fmax(fabs(v.x), fabs(v.y));
}

// Offset contributed by the digits of `idx` over a group list (stride `sa`).
__device__ __forceinline__ int64_t group_off(const Groups &g, int64_t idx) {
    int64_t off = 0;
    if (g.pow2) {
        for (int32_t i = 0; i < g.n; ++i) off += ((idx >> g.lsb[i]) & g.mask[i]) * g.sa[i];
    } else {
        for (int32_t i = 0; i < g.n; ++i) {
            int64_t d = idx % g.dim[i];
            idx /= g.dim[i];
            off += d * g.sa[i];
        }
    }
    return off;
}

// Offsets in A and B of a shared-leg multi-index.
__device__ __forceinline__ void group_off2(const Groups &g, int64_t idx, int64_t &oa, int64_t &ob) {
    oa = 0;
    ob = 0;
    if (g.pow2) {
        for (int32_t i = 0; i < g.n; ++i) {
            int64_t d = (idx >> g.lsb[i]) & g.mask[i];
            oa += d * g.sa[i];
            ob += d * g.sb[i];
        }
    } else {
        for (int32_t i = 0; i < g.n; ++i) {
            int64_t d = idx % g.dim[i];
            idx /= g.dim[i];
            oa += d * g.sa[i];
            ob += d * g.sb[i];
        }
    }
}

__device__ __forceinline__ void load_desc(StepDesc &dst, const StepDesc *src) {
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(StepDesc) / sizeof(int4)); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide max of non-negative values, then one atomicMax on the bit pattern.
__device__ __forceinline__ void publish_max(float v, uint32_t *slot) {
    __shared__ float red[32];
    v = warp_max(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
        v = warp_max(v);
        if (lane == 0 && v > 0.f) atomicMax(slot, __float_as_uint(v));
    }
}

static_assert(sizeof(StepDesc) % sizeof(int4) == 0, "descriptor must be a multiple of 16 bytes");

// ------------------------------------------------------------------------------ leaf convert
// complex128 leaves -> storage type, with each leaf's max-abs; one block per leaf.
template <typename T>
__global__ void __launch_bounds__(128) k_leaf_convert(const double2 *__restrict__ src,
                                                      cx_t<T> *__restrict__ dst,
                                                      const int64_t *__restrict__ off,
                                                      ScaleState sc) {
    const int32_t leaf = blockIdx.x;
    const int64_t b = off[leaf], e = off[leaf + 1];
    float mx = 0.f;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        double2 v = src[i];
        cx_t<T> w = cmake((T)v.x, (T)v.y);
        dst[i] = w;
        mx = fmaxf(mx, absmax2(w));
    }
    __shared__ float red[32];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        sc.maxbits[leaf] = __float_as_uint(m);
        sc.exp2[leaf] = 0;
    }
}

// ------------------------------------------------------------------------------ rows kernel
// Tiny-bond contraction (N <= NT <= 16, K <= 64): B (K x N) is staged in shared memory, each
// thread owns one output row m, reads its K entries of A through the index map and writes N
// consecutive outputs.  HBM traffic is one read of A and one write of C.
constexpr int kRowsMaxKN = 1024;
constexpr int kRowsMaxK = 64;

template <typename T, int NT>
__global__ void __launch_bounds__(256) k_rows(const StepDesc *__restrict__ dd, ScaleState sc) {
    using C = cx_t<T>;
    __shared__ StepDesc d;
    __shared__ C Bs[kRowsMaxKN];
    __shared__ int64_t kA[kRowsMaxK];
    load_desc(d, dd);
    const int64_t M = d.M;
    const int32_t N = (int32_t)d.N, K = (int32_t)d.K;
    const int32_t eA = scale_exponent(sc.maxbits[d.node_a]);
    const int32_t eB = scale_exponent(sc.maxbits[d.node_b]);
    const T sA = pow2<T>(-eA), sB = pow2<T>(-eB);
    const C *__restrict__ A = static_cast<const C *>(d.A);
    const C *__restrict__ B = static_cast<const C *>(d.B);
    C *__restrict__ Cp = static_cast<C *>(d.C);
    for (int32_t i = threadIdx.x; i < K * N; i += blockDim.x) {
        int32_t k = i / N, n = i - k * N;
        int64_t oa, ob;
        group_off2(d.k, k, oa, ob);
        ob += group_off(d.n, n);
        C v = B[ob];
        Bs[i] = cmake(v.x * sB, v.y * sB);
        if (n == 0) kA[k] = oa;
    }
    __syncthreads();
    float mx = 0.f;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const int64_t offA = group_off(d.m, m);
        C acc[NT];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n] = cmake((T)0, (T)0);
        for (int32_t k = 0; k < K; ++k) {
            const C a = A[offA + kA[k]];
#pragma unroll
            for (int n = 0; n < NT; ++n)
                if (n < N) cfma(acc[n], a, Bs[k * N + n]);
        }
        C *out = Cp + m * N;
#pragma unroll
        for (int n = 0; n < NT; ++n)
            if (n < N) {
                C v = cmake(acc[n].x * sA, acc[n].y * sA);
                out[n] = v;
                mx = fmaxf(mx, absmax2(v));
            }
    }
    publish_max(mx, &sc.maxbits[d.node_c]);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        sc.exp2[d.node_c] = sc.exp2[d.node_a] + eA + sc.exp2[d.node_b] + eB;
}

// ------------------------------------------------------------------------------ tile kernel
// General contraction on CUDA cores: 64 x 64 output tile per block, K in chunks of 16, operand
// tiles gathered through the index maps into shared memory, 4 x 4 outputs per thread.
constexpr int TM = 64, TN = 64, TK = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_tile(const StepDesc *__restrict__ dd, ScaleState sc) {
    using C = cx_t<T>;
    __shared__ StepDesc d;
    __shared__ C As[TK][TM];
    __shared__ C Bs[TK][TN];
    __shared__ int64_t rowA[TM], colB[TN], kAo[TK], kBo[TK];
    load_desc(d, dd);
    const int64_t M = d.M, N = d.N, K = d.K;
    const int64_t tiles_n = (N + TN - 1) / TN;
    const int64_t tile = blockIdx.x;
    const int64_t m0 = (tile / tiles_n) * TM, n0 = (tile % tiles_n) * TN;
    const int32_t eA = scale_exponent(sc.maxbits[d.node_a]);
    const int32_t eB = scale_exponent(sc.maxbits[d.node_b]);
    const T sA = pow2<T>(-eA), sB = pow2<T>(-eB);
    const C *__restrict__ A = static_cast<const C *>(d.A);
    const C *__restrict__ B = static_cast<const C *>(d.B);
    C *__restrict__ Cp = static_cast<C *>(d.C);
    const int tid = threadIdx.x;
    if (tid < TM) rowA[tid] = (m0 + tid < M) ? group_off(d.m, m0 + tid) : -1;
    else if (tid < TM + TN) {
        int c = tid - TM;
        colB[c] = (n0 + c < N) ? group_off(d.n, n0 + c) : -1;
    }
    const int tx = tid & 15, ty = tid >> 4;
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cmake((T)0, (T)0);
    for (int64_t k0 = 0; k0 < K; k0 += TK) {
        __syncthreads();
        if (tid < TK) {
            int64_t oa = -1, ob = -1;
            if (k0 + tid < K) group_off2(d.k, k0 + tid, oa, ob);
            kAo[tid] = oa;
            kBo[tid] = ob;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < (TM * TK) / 256; ++r) {
            int i = tid + r * 256;
            int row = i % TM, kk = i / TM;
            C v = cmake((T)0, (T)0);
            if (rowA[row] >= 0 && kAo[kk] >= 0) {
                v = A[rowA[row] + kAo[kk]];
                v = cmake(v.x * sA, v.y * sA);
            }
            As[kk][row] = v;
        }
#pragma unroll
        for (int r = 0; r < (TN * TK) / 256; ++r) {
            int i = tid + r * 256;
            int col = i % TN, kk = i / TN;
            C v = cmake((T)0, (T)0);
            if (colB[col] >= 0 && kBo[kk] >= 0) {
                v = B[kBo[kk] + colB[col]];
                v = cmake(v.x * sB, v.y * sB);
            }
            Bs[kk][col] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
    }
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t n = n0 + tx + 16 * j;
            if (n < N) {
                Cp[m * N + n] = acc[i][j];
                mx = fmaxf(mx, absmax2(acc[i][j]));
            }
        }
    }
    publish_max(mx, &sc.maxbits[d.node_c]);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        sc.exp2[d.node_c] = sc.exp2[d.node_a] + eA + sc.exp2[d.node_b] + eB;
}

// ------------------------------------------------------------------------------ dot kernel
// Small outputs (M * N <= 16) with any K: every block reduces a slice of K into FP64 partials
// (products formed in the storage precision, summed in runs of 32 in that precision and then in
// FP64); a one-block second pass sums the partials in a fixed order.  The root step of a closed
// network (M = N = 1) always runs here, which gives the FP64 final reduction.
constexpr int kDotMaxOut = 16;
constexpr int kDotBlocks = 4 * 152;
constexpr int kDotThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const StepDesc *__restrict__ dd,
                                                             ScaleState sc,
                                                             double2 *__restrict__ partials) {
    using C = cx_t<T>;
    __shared__ StepDesc d;
    __shared__ int64_t rowA[kDotMaxOut], colB[kDotMaxOut];
    __shared__ double2 red[kDotThreads / 32][kDotMaxOut];
    load_desc(d, dd);
    const int32_t M = (int32_t)d.M, N = (int32_t)d.N;
    const int64_t K = d.K;
    if (threadIdx.x < M) rowA[threadIdx.x] = group_off(d.m, threadIdx.x);
    if (threadIdx.x < N) colB[threadIdx.x] = group_off(d.n, threadIdx.x);
    __syncthreads();
    const int32_t eA = scale_exponent(sc.maxbits[d.node_a]);
    const int32_t eB = scale_exponent(sc.maxbits[d.node_b]);
    const T sA = pow2<T>(-eA), sB = pow2<T>(-eB);
    const C *__restrict__ A = static_cast<const C *>(d.A);
    const C *__restrict__ B = static_cast<const C *>(d.B);
    const int32_t MN = M * N;
    double2 acc[kDotMaxOut];
    C run[kDotMaxOut];
#pragma unroll
    for (int i = 0; i < kDotMaxOut; ++i) { acc[i] = make_double2(0, 0); run[i] = cmake((T)0, (T)0); }
    int cnt = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t oa, ob;
        group_off2(d.k, k, oa, ob);
#pragma unroll
        for (int i = 0; i < kDotMaxOut; ++i) {
            if (i < MN) {
                int m = i / N, n = i - m * N;
                C a = A[oa + rowA[m]], b = B[ob + colB[n]];
                a = cmake(a.x * sA, a.y * sA);
                b = cmake(b.x * sB, b.y * sB);
                cfma(run[i], a, b);
            }
        }
        if (++cnt == 32) {
#pragma unroll
            for (int i = 0; i < kDotMaxOut; ++i) {
                acc[i].x += (double)run[i].x;
                acc[i].y += (double)run[i].y;
                run[i] = cmake((T)0, (T)0);
            }
            cnt = 0;
        }
    }
#pragma unroll
    for (int i = 0; i < kDotMaxOut; ++i) {
        acc[i].x += (double)run[i].x;
        acc[i].y += (double)run[i].y;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kDotMaxOut; ++i) {
        if (i >= MN) break;
        double x = acc[i].x, y = acc[i].y;
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
        if (lane == 0) red[warp][i] = make_double2(x, y);
    }
    __syncthreads();
    if (threadIdx.x < MN) {
        double2 s = make_double2(0, 0);
        for (int w = 0; w < kDotThreads / 32; ++w) { s.x += red[w][threadIdx.x].x; s.y += red[w][threadIdx.x].y; }
        partials[(int64_t)blockIdx.x * kDotMaxOut + threadIdx.x] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_dot_final(const StepDesc *__restrict__ dd, ScaleState sc,
                                                   const double2 *__restrict__ partials,
                                                   int32_t nblocks, DeviceResult *result) {
    using C = cx_t<T>;
    __shared__ StepDesc d;
    __shared__ double2 red[8][kDotMaxOut];
    load_desc(d, dd);
    const int32_t MN = (int32_t)(d.M * d.N);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < MN; ++i) {
        double x = 0, y = 0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            double2 p = partials[(int64_t)b * kDotMaxOut + i];
            x += p.x;
            y += p.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
        if (lane == 0) red[warp][i] = make_double2(x, y);
    }
    __syncthreads();
    const int32_t eA = scale_exponent(sc.maxbits[d.node_a]);
    const int32_t eB = scale_exponent(sc.maxbits[d.node_b]);
    const int32_t e_out = sc.exp2[d.node_a] + eA + sc.exp2[d.node_b] + eB;
    if (threadIdx.x < MN) {
        double2 s = make_double2(0, 0);
        for (int w = 0; w < 8; ++w) { s.x += red[w][threadIdx.x].x; s.y += red[w][threadIdx.x].y; }
        if (d.is_root && result) {
            result->re = s.x;
            result->im = s.y;
            result->exp2 = e_out;
            result->status = 0;
        }
        if (d.C) {
            C v = cmake((T)s.x, (T)s.y);
            static_cast<C *>(d.C)[threadIdx.x] = v;
            atomicMax(&sc.maxbits[d.node_c], __float_as_uint(absmax2(v)));
        }
    }
    if (threadIdx.x == 0) sc.exp2[d.node_c] = e_out;
}

// A network of a single tensor of degree 0: the result is the leaf itself.
template <typename T>
__global__ void k_finish_leaf(const cx_t<T> *leaf, int32_t node, ScaleState sc,
                              DeviceResult *result) {
    cx_t<T> v = leaf[0];
    result->re = (double)v.x;
    result->im = (double)v.y;
    result->exp2 = sc.exp2[node];
    result->status = 0;
}

template <typename T, int NT>
void rows_launch(const StepDesc *d, const StepDesc &h, ScaleState sc, cudaStream_t st) {
    int64_t blocks = (h.M + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_rows<T, NT><<<(unsigned)blocks, 256, 0, st>>>(d, sc);
}

template <typename T>
cudaError_t step_launch(const StepDesc *d, const StepDesc &h, ScaleState sc, double *partials,
                        int32_t dot_blocks, DeviceResult *result, cudaStream_t st,
                        int32_t *launches) {
    switch (h.kind) {
        case STEP_ROWS:
            if (h.N <= 1) rows_launch<T, 1>(d, h, sc, st);
            else if (h.N <= 2) rows_launch<T, 2>(d, h, sc, st);
            else if (h.N <= 4) rows_launch<T, 4>(d, h, sc, st);
            else if (h.N <= 8) rows_launch<T, 8>(d, h, sc, st);
            else rows_launch<T, 16>(d, h, sc, st);
            *launches += 1;
            break;
        case STEP_TILE: {
            int64_t tiles = ((h.M + TM - 1) / TM) * ((h.N + TN - 1) / TN);
            k_tile<T><<<(unsigned)tiles, 256, 0, st>>>(d, sc);
            *launches += 1;
            break;
        }
        case STEP_DOT: {
            int64_t blocks = (h.K + kDotThreads - 1) / kDotThreads;
            if (blocks > dot_blocks) blocks = dot_blocks;
            if (blocks < 1) blocks = 1;
            k_dot_partial<T><<<(unsigned)blocks, kDotThreads, 0, st>>>(
                d, sc, reinterpret_cast<double2 *>(partials));
            k_dot_final<T><<<1, 256, 0, st>>>(d, sc, reinterpret_cast<double2 *>(partials),
                                              (int32_t)blocks, result);
            *launches += 2;
            break;
        }
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

int32_t dot_partial_blocks() { return kDotBlocks; }

cudaError_t launch_leaf_convert(bool c128, const double *src, void *dst, const int64_t *leaf_off,
                                int32_t n_leaves, ScaleState sc, cudaStream_t stream) {
    if (n_leaves <= 0) return cudaSuccess;
    if (c128)
        k_leaf_convert<double><<<n_leaves, 128, 0, stream>>>(
            reinterpret_cast<const double2 *>(src), static_cast<double2 *>(dst), leaf_off, sc);
    else
        k_leaf_convert<float><<<n_leaves, 128, 0, stream>>>(
            reinterpret_cast<const double2 *>(src), static_cast<float2 *>(dst), leaf_off, sc);
    return cudaGetLastError();
}

cudaError_t launch_step(bool c128, const StepDesc *d_desc, const StepDesc &h_desc, ScaleState sc,
                        double *dot_partials, int32_t dot_blocks, DeviceResult *result,
                        cudaStream_t stream, int32_t *launches) {
    if (c128)
        return step_launch<double>(d_desc, h_desc, sc, dot_partials, dot_blocks, result, stream,
                                   launches);
    return step_launch<float>(d_desc, h_desc, sc, dot_partials, dot_blocks, result, stream,
                              launches);
}

cudaError_t launch_finish_leaf(bool c128, const void *leaf, int32_t node, ScaleState sc,
                               DeviceResult *result, cudaStream_t stream) {
    if (c128)
        k_finish_leaf<double><<<1, 1, 0, stream>>>(static_cast<const double2 *>(leaf), node, sc, result);
    else
        k_finish_leaf<float><<<1, 1, 0, stream>>>(static_cast<const float2 *>(leaf), node, sc, result);
    return cudaGetLastError();
}

}  // namespace tn
