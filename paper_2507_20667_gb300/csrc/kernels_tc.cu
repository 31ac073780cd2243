// Dense contraction steps on the tcgen05 tensor cores in a split precision (BF16 or TF32 hi/lo),
// as two grouped launches per dependency phase:
//
//  * k_tc_pack   gathers an operand of a dense step through the step's index maps (the TTGT
//                transposition of Eq. 2.4, fused), scales it exactly by its power-of-two operand
//                scale, splits every real value x into hi = r(x) and lo = r(x - hi) (r rounding to
//                BF16 or TF32), and writes the k-blocks as ready-made shared-memory images: K-major,
//                64-byte rows, 64-byte swizzle, hi plane then lo plane.  A complex [M, K] operand
//                is the real [M, 2K] matrix of (Re, Im) pairs; the B operand is written as B'',
//                whose rows 2n and 2n+1 hold (Re B, -Im B) and (Im B, Re B) pairs, so that
//                A_real B''^T is C [M, N] with (Re, Im) interleaved (the real 4M form).  Tails
//                (rows, columns, shared indices past the step's extent) are zero.
//  * k_tc_gemm   one CTA per SM, warp-specialised: warp 0 streams the k-block images of a
//                128-row x NC-complex-column tile (NC = 64 or 128) with bulk copies into a 4-stage
//                shared-memory ring (mbarrier transaction counts), warp 1 issues the MMAs -- per
//                k-block hi*hi, hi*lo and lo*hi, each as two K-slices -- and releases each stage
//                with tcgen05.commit, and warps 2-9 add the accumulator into FP32 registers
//                (tcgen05.ld), write complex64 C, publish the tile's max-abs and mark the tile
//                complete.  The tensor-memory accumulator holds at most kSegBlocks k-blocks: a long
//                shared index is summed in segments, each accumulated by the tensor cores into one
//                of two 128 x 2NC FP32 buffers and then added, rounding to nearest, into the
//                epilogue's registers while the next segment accumulates in the other buffer.  The
//                tensor cores' own accumulation does not round to nearest (measured: the product
//                drifts toward zero by about 2^-25 of its value per accumulated MMA), so bounding
//                the MMAs per buffer bounds that drift whatever K is.  The producer runs up to four
//                k-blocks ahead of the MMAs, across tile boundaries, and a tile's epilogue overlaps
//                the next tile's MMAs.
//
// Every mbarrier wait is bounded and gives up when the launch-wide abort flag rises; a role that
// gives up marks its job TN_ETIMEOUT, and before the CTA exits the producer waits (bounded) for
// its bulk copies in flight and the MMA warp for its MMAs, then tensor memory is freed.
#include <cstdint>

#include "kernels.cuh"
#include "tc_ops.cuh"
#include "tile_ops.cuh"

namespace tn {

namespace {

constexpr int32_t kStatusTimeout = 5;
constexpr int kPackThreads = 256;
constexpr int kEpiWarps = 8;
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;   // warp 0 producer, warp 1 MMA issuer, warps 2-9 epilogue
constexpr int kStages = 4;
constexpr uint32_t kStageBytes = 2 * kTcImgA + 2 * tc_img_b(kTcColsMax);   // A hi, A lo, B'' hi, B'' lo
constexpr uint32_t kAccBuf = 256;                              // 128 x 256 FP32 accumulator buffer
constexpr uint32_t kAccCols = 2 * kAccBuf;                     // two buffers: all 512 TMEM columns
constexpr int kSegBlocks = 8;                                  // k-blocks per accumulation segment
constexpr int kBarBytes = 256;
constexpr int kGemmSmem = kStages * (int)kStageBytes + kBarBytes + 1024;   // + alignment slack
static_assert(kStageBytes % 1024 == 0, "stage images keep 1024-byte alignment");
static_assert((2 * kStages + 5) * 8 + 12 <= kBarBytes, "barrier area");
static_assert(2 * kTcColsMax <= (int)kAccBuf, "a tile's accumulator fits one buffer");
static_assert(kGemmSmem <= 227 * 1024, "shared memory per CTA");

template <bool TF32> struct TcK { static constexpr int KC = TF32 ? 8 : 16; };   // complex k per k-block

// Store the complex pair (re, im) as real columns 2kk, 2kk+1 of row r of a k-block image: hi plane
// at img, lo plane at img + plane.
template <bool TF32>
__device__ __forceinline__ void put_pair(char *img, uint32_t plane, uint32_t r, uint32_t kk, float re, float im) {
    if constexpr (TF32) {
        const float h0 = round_tf32(re), h1 = round_tf32(im);
        const uint32_t off = sw64_off(r, 8 * kk);
        *reinterpret_cast<float2 *>(img + off) = make_float2(h0, h1);
        *reinterpret_cast<float2 *>(img + plane + off) = make_float2(round_tf32(re - h0), round_tf32(im - h1));
    } else {
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(re, h0, l0);
        split_bf16(im, h1, l1);
        const uint32_t off = sw64_off(r, 4 * kk);
        __nv_bfloat162 h, l;
        h.x = h0; h.y = h1;
        l.x = l0; l.y = l1;
        *reinterpret_cast<__nv_bfloat162 *>(img + off) = h;
        *reinterpret_cast<__nv_bfloat162 *>(img + plane + off) = l;
    }
}

// One pack unit: k-block kb of row tile t of operand A (unit < MT*KB) or column tile t of B''.
template <bool TF32>
__global__ void __launch_bounds__(kPackThreads) k_tc_pack(const JobPtrs *__restrict__ jobs,
                                                          const WorkItem *__restrict__ units) {
    constexpr int KC = TcK<TF32>::KC;
    constexpr int PER = kTcRows * KC / kPackThreads;
    static_assert(PER * kPackThreads == kTcRows * KC, "pack split");
    __shared__ StepDesc d;
    constexpr int LD = KC + 1;            // padded row: no bank conflicts when rows are fastest
    __shared__ float2 tile[kTcRows * LD];
    __shared__ int64_t roff[kTcRows];
    __shared__ int64_t koff[KC];
    const WorkItem u = units[blockIdx.x];
    const JobPtrs &j = jobs[u.job];
    load_desc(d, j.steps + u.step);
    const int64_t M = d.M, N = d.N, K = d.K;
    const int NC = d.tile_rows;
    const int64_t KB = (K + KC - 1) / KC, MT = (M + kTcRows - 1) / kTcRows;
    const bool side_a = (int64_t)u.tile < MT * KB;
    const int64_t v = side_a ? (int64_t)u.tile : (int64_t)u.tile - MT * KB;
    const int64_t t = v / KB, kb = v % KB;
    const int rows = side_a ? kTcRows : NC;   // operand rows of the unit (B: complex columns)
    const int64_t extent = side_a ? M : N, r0 = t * rows, k0 = kb * KC;
    const Groups &g = side_a ? d.m : d.n;
    for (int i = threadIdx.x; i < kTcRows; i += kPackThreads)
        roff[i] = (i < rows && r0 + i < extent) ? group_off(g, r0 + i) : -1;
    for (int i = threadIdx.x; i < KC; i += kPackThreads) {
        int64_t oa = -1, ob = -1;
        if (k0 + i < K) group_off2(d.k, k0 + i, oa, ob);
        koff[i] = side_a ? oa : ob;
    }
    int32_t eA, eB;
    step_scales(d, j, eA, eB);
    const float s = pow2<float>(side_a ? -eA : -eB);
    const float2 *__restrict__ X = operand<float2>(d, j, side_a);
    __syncthreads();
    // gather, rows fastest when the operand's row index is its contiguous one
    const bool rows_fast = (d.flags & (side_a ? FLAG_A_MCONT : FLAG_B_NCONT)) != 0;
    float2 x[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = threadIdx.x + q * kPackThreads;
        const int r = rows_fast ? (e % kTcRows) : (e / KC), kk = rows_fast ? (e / kTcRows) : (e % KC);
        x[q] = (roff[r] >= 0 && koff[kk] >= 0) ? __ldcg(X + roff[r] + koff[kk]) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = threadIdx.x + q * kPackThreads;
        const int r = rows_fast ? (e % kTcRows) : (e / KC), kk = rows_fast ? (e / kTcRows) : (e % KC);
        tile[r * LD + kk] = make_float2(x[q].x * s, x[q].y * s);
    }
    __syncthreads();
    // split and write, shared index fastest (a warp covers whole 64-byte rows)
    const uint32_t plane = side_a ? kTcImgA : tc_img_b(NC);
    char *img = j.arena + (side_a ? d.img_a : d.img_b) + (size_t)(t * KB + kb) * 2 * plane;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = threadIdx.x + q * kPackThreads;
        const int r = e / KC, kk = e % KC;
        if (r >= rows) continue;   // a B unit of NC = 64 columns fills half the tile
        const float2 y = tile[r * LD + kk];
        if (side_a) {
            put_pair<TF32>(img, plane, (uint32_t)r, (uint32_t)kk, y.x, y.y);
        } else {
            put_pair<TF32>(img, plane, 2u * r, (uint32_t)kk, y.x, -y.y);
            put_pair<TF32>(img, plane, 2u * r + 1u, (uint32_t)kk, y.y, y.x);
        }
    }
    if (u.tile == 0 && threadIdx.x == 0) write_exponent(d, j, eA, eB);
}

// Geometry of one GEMM tile, read by every role from the step descriptor.
struct TileGeo {
    int64_t M, N, KB, mt, nt;
    int NC;
    const char *img_a, *img_b;
};

template <bool TF32>
__device__ __forceinline__ TileGeo tile_geo(const JobPtrs &j, const WorkItem &w) {
    constexpr int KC = TcK<TF32>::KC;
    const StepDesc *d = j.steps + w.step;
    TileGeo g;
    g.M = __ldcg(&d->M);
    g.N = __ldcg(&d->N);
    g.KB = (__ldcg(&d->K) + KC - 1) / KC;
    g.NC = __ldcg(&d->tile_rows);
    const int64_t NT = (g.N + g.NC - 1) / g.NC;
    g.mt = (int64_t)w.tile / NT;
    g.nt = (int64_t)w.tile % NT;
    g.img_a = j.arena + __ldcg(&d->img_a) + (size_t)(g.mt * g.KB) * 2 * kTcImgA;
    g.img_b = j.arena + __ldcg(&d->img_b) + (size_t)(g.nt * g.KB) * 2 * tc_img_b(g.NC);
    return g;
}

__device__ __forceinline__ void mark_timeout(const JobPtrs &j) {
    atomicExch(&static_cast<DeviceResult *>(j.result)->status, kStatusTimeout);
}

// Wait for a phase without regard to the abort flag (used only to drain operations this CTA
// started itself before it exits); bounded all the same.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity, long long limit_ns) {
    const long long t0 = tc_global_ns();
    while (!mbar_try(bar, parity))
        if (tc_global_ns() - t0 > limit_ns) return;
}

template <bool TF32>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_tc_gemm(const JobPtrs *__restrict__ jobs, const WorkItem *__restrict__ tiles, int32_t n_tiles,
              int32_t *abort_flag, long long wait_ns) {
    extern __shared__ __align__(1024) char dyn_raw[];
    char *ring = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(dyn_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;    // [2] a segment is accumulated in buffer b
    uint64_t *acc_empty = acc_full + 2;      // [2] the epilogue has read buffer b
    uint64_t *drain = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    // epilogue-warp tickets, counted per buffer of a tile's last segment: kEpiWarps per completed
    // tile.  Every ticket of a tile precedes, on its buffer's counter, every ticket of a later tile:
    // that tile's last segment reuses the buffer only after all warps released its previous use,
    // which each warp does after its tickets of the earlier tiles.
    uint32_t *tickets = tmem_slot + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full + b, 1);
            mbar_init(acc_empty + b, kEpiWarps);
            tickets[b] = 0;
        }
        mbar_init(drain, 1);
        mbar_init_fence();
    }
    if (warp == 1) tmem_alloc(tmem_slot, kAccCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- producer: bulk copies of the k-block images into the ring
        uint32_t it = 0;
        bool ok = true;
        for (int32_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const WorkItem w = tiles[t];
            const JobPtrs &j = jobs[w.job];
            const TileGeo g = tile_geo<TF32>(j, w);
            for (int64_t kb = 0; kb < g.KB; ++kb, ++it) {
                const uint32_t s = it % kStages;
                if (!mbar_wait(empty + s, ((it / kStages) & 1u) ^ 1u, wait_ns, abort_flag)) {
                    mark_timeout(j);
                    ok = false;
                    break;
                }
                char *st = ring + s * kStageBytes;
                const uint32_t bb = 2 * tc_img_b(g.NC);
                mbar_arrive_expect_tx(full + s, 2 * kTcImgA + bb);
                bulk_g2s(st, g.img_a + (size_t)kb * 2 * kTcImgA, 2 * kTcImgA, full + s);
                bulk_g2s(st + 2 * kTcImgA, g.img_b + (size_t)kb * bb, bb, full + s);
            }
        }
        // the copies this CTA started land before it exits
        const uint32_t first = it > (uint32_t)kStages ? it - kStages : 0u;
        for (uint32_t i = first; i < it; ++i) mbar_drain(full + i % kStages, (i / kStages) & 1u, wait_ns);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: segment sg accumulates into buffer sg % 2
        uint32_t it = 0, sg = 0;
        bool ok = true;
        for (int32_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const WorkItem w = tiles[t];
            const JobPtrs &j = jobs[w.job];
            const TileGeo g = tile_geo<TF32>(j, w);
            const uint32_t idesc = TF32 ? idesc_tf32(kTcRows, 2 * g.NC) : idesc_bf16(kTcRows, 2 * g.NC);
            for (int64_t kb0 = 0; kb0 < g.KB && ok; kb0 += kSegBlocks, ++sg) {
                const uint32_t b = sg & 1u;
                if (!mbar_wait(acc_empty + b, ((sg >> 1) & 1u) ^ 1u, wait_ns, abort_flag)) {
                    mark_timeout(j);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dst = tmem + b * kAccBuf;
                const int64_t kb1 = kb0 + kSegBlocks < g.KB ? kb0 + kSegBlocks : g.KB;
                for (int64_t kb = kb0; kb < kb1; ++kb, ++it) {
                    const uint32_t s = it % kStages;
                    if (!mbar_wait(full + s, (it / kStages) & 1u, wait_ns, abort_flag)) {
                        mark_timeout(j);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(ring + s * kStageBytes);
                    const uint64_t ah = smem_desc_sw64(a), al = smem_desc_sw64(a + kTcImgA);
                    const uint64_t bh = smem_desc_sw64(a + 2 * kTcImgA),
                                   bl = smem_desc_sw64(a + 2 * kTcImgA + tc_img_b(g.NC));
#pragma unroll
                    for (int h = 0; h < 2; ++h) {   // two 32-byte K-slices of the 64-byte rows
                        const uint64_t adv = (uint64_t)(h * 32 >> 4);
                        const uint32_t acc = (kb > kb0 || h > 0) ? 1u : 0u;
                        if constexpr (TF32) {
                            tc_mma_tf32(dst, ah + adv, bh + adv, idesc, acc);
                            tc_mma_tf32(dst, ah + adv, bl + adv, idesc, 1u);
                            tc_mma_tf32(dst, al + adv, bh + adv, idesc, 1u);
                        } else {
                            tc_mma_bf16(dst, ah + adv, bh + adv, idesc, acc);
                            tc_mma_bf16(dst, ah + adv, bl + adv, idesc, 1u);
                            tc_mma_bf16(dst, al + adv, bh + adv, idesc, 1u);
                        }
                    }
                    tc_commit(empty + s);   // the stage is free once these MMAs have read it
                }
                if (!ok) break;
                tc_commit(acc_full + b);    // the segment's partial sums are complete
            }
        }
        // every MMA this CTA issued completes before tensor memory is freed
        tc_commit(drain);
        mbar_drain(drain, 0u, wait_ns);
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its 32 rows of the tile), and
        // half (w - 2) / 4 of the tile's 2 NC FP32 columns
        const uint32_t quarter = (uint32_t)(warp & 3);
        const int half = (warp - 2) >> 2;
        uint32_t sg = 0;
        for (int32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            const WorkItem w = tiles[t];
            const JobPtrs &j = jobs[w.job];
            const TileGeo g = tile_geo<TF32>(j, w);
            const StepDesc *d = j.steps + w.step;
            const int nch = g.NC / 16;   // 16-column chunks of a half: 4 or 8
            float sum[8 * 16];
#pragma unroll
            for (int i = 0; i < 8 * 16; ++i) sum[i] = 0.f;
            bool ok = true;
            uint32_t b = 0;
            for (int64_t kb0 = 0; kb0 < g.KB; kb0 += kSegBlocks, ++sg) {
                b = sg & 1u;
                if (!mbar_wait(acc_full + b, (sg >> 1) & 1u, wait_ns, abort_flag)) {
                    mark_timeout(j);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem + ((32u * quarter) << 16) + b * kAccBuf + (uint32_t)(half * g.NC);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (c < nch) {
                        float v[16];
                        tc_ld16(base + (uint32_t)(16 * c), v);
#pragma unroll
                        for (int p = 0; p < 16; ++p) sum[16 * c + p] += v[p];
                    }
                }
                if (kb0 + kSegBlocks < g.KB) {   // not the tile's last segment: release the buffer now
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acc_empty + b);
                }
            }
            if (!ok) break;
            const int64_t m = g.mt * kTcRows + 32 * quarter + lane;
            const int64_t N = g.N;
            float2 *__restrict__ Cp = reinterpret_cast<float2 *>(j.arena) + __ldcg(&d->c_off);
            float mx = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c >= nch || m >= g.M) continue;
                const float *v = sum + 16 * c;
                const int64_t n0 = g.nt * g.NC + half * (g.NC / 2) + 8 * c;
                float2 *row = Cp + m * N;
                if (n0 + 8 <= N && ((m * N + n0) & 1) == 0) {
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        *reinterpret_cast<float4 *>(row + n0 + 2 * p) =
                            make_float4(v[4 * p], v[4 * p + 1], v[4 * p + 2], v[4 * p + 3]);
#pragma unroll
                    for (int p = 0; p < 16; ++p) mx = fmaxf(mx, fabsf(v[p]));
                } else {
#pragma unroll
                    for (int p = 0; p < 8; ++p)
                        if (n0 + p < N) {
                            row[n0 + p] = make_float2(v[2 * p], v[2 * p + 1]);
                            mx = fmaxf(mx, fmaxf(fabsf(v[2 * p]), fabsf(v[2 * p + 1])));
                        }
                }
            }
            mx = warp_max(mx);
            if (lane == 0) {
                if (mx > 0.f) atomicMax(j.maxbits + __ldcg(&d->node_c), __float_as_uint(mx));
                // the last epilogue warp to finish the tile publishes it (no block barrier: a warp
                // that gave up on a wait must not hold the others)
                __threadfence();
                if (atomicAdd(tickets + b, 1u) % (uint32_t)kEpiWarps == (uint32_t)kEpiWarps - 1u) {
                    __threadfence();
                    atomicAdd(j.done + w.step, 1);
                }
            }
            // release the last segment's buffer only after the ticket (see tickets above)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + b);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kAccCols);
}

template <typename K>
cudaError_t allow_smem(K kernel, int32_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

cudaError_t launch_tc_pack(bool tf32, const JobPtrs *jobs_dev, const WorkItem *units, int32_t n_units,
                           cudaStream_t stream) {
    if (n_units <= 0) return cudaSuccess;
    if (tf32) k_tc_pack<true><<<(unsigned)n_units, kPackThreads, 0, stream>>>(jobs_dev, units);
    else k_tc_pack<false><<<(unsigned)n_units, kPackThreads, 0, stream>>>(jobs_dev, units);
    return cudaGetLastError();
}

cudaError_t launch_tc_gemm(bool tf32, const JobPtrs *jobs_dev, const WorkItem *tiles, int32_t n_tiles,
                           int32_t *abort_flag, long long wait_ns, cudaStream_t stream) {
    if (n_tiles <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int32_t grid = n_tiles < sms ? n_tiles : sms;
    if (tf32) {
        e = allow_smem(k_tc_gemm<true>, kGemmSmem);
        if (e != cudaSuccess) return e;
        k_tc_gemm<true><<<(unsigned)grid, kGemmThreads, kGemmSmem, stream>>>(jobs_dev, tiles, n_tiles, abort_flag,
                                                                           wait_ns);
    } else {
        e = allow_smem(k_tc_gemm<false>, kGemmSmem);
        if (e != cudaSuccess) return e;
        k_tc_gemm<false><<<(unsigned)grid, kGemmThreads, kGemmSmem, stream>>>(jobs_dev, tiles, n_tiles, abort_flag,
                                                                            wait_ns);
    }
    return cudaGetLastError();
}

int64_t tc_pack_units(int64_t M, int64_t N, int64_t K, bool tf32, int nc) {
    const int64_t KC = tf32 ? 8 : 16, KB = (K + KC - 1) / KC;
    return ((M + kTcRows - 1) / kTcRows + (N + nc - 1) / nc) * KB;
}

size_t tc_image_bytes(int64_t M, int64_t N, int64_t K, bool tf32, int nc, size_t *a_bytes) {
    const int64_t KC = tf32 ? 8 : 16, KB = (K + KC - 1) / KC;
    const size_t a = (size_t)((M + kTcRows - 1) / kTcRows) * (size_t)KB * 2 * kTcImgA;
    const size_t b = (size_t)((N + nc - 1) / nc) * (size_t)KB * 2 * tc_img_b(nc);
    if (a_bytes) *a_bytes = a;
    return a + b;
}

}  // namespace tn
