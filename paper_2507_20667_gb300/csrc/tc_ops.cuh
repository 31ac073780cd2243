// Dense complex contraction steps on the 5th-generation tensor cores (tcgen05, sm_103a), in a
// split precision: every real operand x is written as hi + lo with hi = r(x) and lo = r(x - hi),
// r rounding to BF16 (kind::f16) or to TF32 (kind::tf32), and the product is accumulated in FP32 as
// hi*hi + hi*lo + lo*hi (the lo*lo term is dropped).
//
// Complex arithmetic uses the real 4M form.  A complex [M, K] is the real [M, 2K] matrix whose row
// holds (Re, Im) pairs; B'' is the real [2N, 2K] matrix whose rows 2n and 2n+1 hold (Re B, -Im B)
// and (Im B, Re B) pairs.  Then A_real * B''^T is the complex C [M, N] with (Re, Im) interleaved,
// i.e. exactly the complex64 storage of C.
//
// One work tile = 128 rows of C x 64 complex columns (128 real columns).  Per K-block (32 complex
// indices for BF16, 16 for TF32: one 128-byte row of the operand tile either way) the block
// gathers A and B through the step's index maps (scaled exactly by the power-of-two operand
// scales), splits them and stores four 16 KB operand tiles in the canonical K-major,
// 128-byte-swizzled shared-memory layout; one thread issues 12 tcgen05.mma (3 products x 4 slices
// of 32 bytes of K) into a 128 x 128 FP32 accumulator in tensor memory and commits them to an
// mbarrier; every wait on it is bounded.  The epilogue reads the accumulator with tcgen05.ld.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "tile_ops.cuh"

namespace tn {

constexpr int kTcM = 128;          // rows of C per tile (TMEM lanes)
constexpr int kTcNc = 64;          // complex columns of C per tile
constexpr int kTcN = 2 * kTcNc;    // real columns (MMA N)
constexpr int kTcKc = 32;          // complex shared indices per K-block (BF16; TF32 takes 16)
constexpr int kTcTileBytes = kTcM * 128;           // one 128-row operand tile: 16 KB
constexpr int kTcSmem = 4 * kTcTileBytes + 1024;   // A hi, A lo, B hi, B lo (+ alignment slack)
constexpr uint32_t kTcCols = 128;                  // TMEM columns (FP32 accumulator)

// ---- PTX wrappers -----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the phase with parity `parity` of `bar` to complete: false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit_cycles) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit_cycles) return false;
    }
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes, 8-row
// atoms 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// Instruction descriptors (FP32 accumulator, A and B both K-major, M x N): kind::f16 with BF16
// operands (format 1), kind::tf32 with TF32 operands (format 2).
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t m, uint32_t n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Byte offset of byte b (0..127) of row r in a K-major 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw128_off(uint32_t r, uint32_t b) {
    return r * 128u + ((((b >> 4) ^ (r & 7u)) << 4) | (b & 15u));
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Round to TF32 (10 explicit mantissa bits), nearest with ties away from zero.
__device__ __forceinline__ float round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Store the complex pair (re, im) as the real columns 2kk, 2kk+1 of row r: hi part and lo part.
template <bool TF32>
__device__ __forceinline__ void put_pair(char *hi_tile, char *lo_tile, uint32_t r, uint32_t kk, float re, float im) {
    if constexpr (TF32) {
        const float h0 = round_tf32(re), h1 = round_tf32(im);
        const uint32_t off = sw128_off(r, 8 * kk);
        *reinterpret_cast<float2 *>(hi_tile + off) = make_float2(h0, h1);
        *reinterpret_cast<float2 *>(lo_tile + off) = make_float2(round_tf32(re - h0), round_tf32(im - h1));
    } else {
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(re, h0, l0);
        split_bf16(im, h1, l1);
        const uint32_t off = sw128_off(r, 4 * kk);
        __nv_bfloat162 h, l;
        h.x = h0; h.y = h1;
        l.x = l0; l.y = l1;
        *reinterpret_cast<__nv_bfloat162 *>(hi_tile + off) = h;
        *reinterpret_cast<__nv_bfloat162 *>(lo_tile + off) = l;
    }
}

struct TcState {
    uint32_t tmem;       // TMEM base address of this block's accumulator
    uint64_t *bar;       // mbarrier in shared memory
    uint32_t phase;      // parity of the next phase to wait for
    int32_t *abort_flag; // launch-wide abort flag
    bool pending;        // a wait gave up: MMAs of phase `phase` may still be in flight
};

constexpr long long kTcWaitLimit = 8000000000LL;   // cycles (~4 s at 2 GHz)

// One tensor-core work tile of step d (complex64 storage; BF16 split, or TF32 split when the step
// has FLAG_TF32).  Returns false if a wait on the tensor core gave up (the caller reports
// TN_ETIMEOUT).
template <bool TF32>
__device__ bool tile_tc_impl(const StepDesc &d, int64_t tile, const JobPtrs &j, char *smem_raw, char *scratch,
                             float *red, TcState &tc) {
    using C = float2;
    constexpr int KC = TF32 ? kTcKc / 2 : kTcKc;   // complex indices per 128-byte operand row
    // 1024-byte aligned operand tiles
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    char *Ah = base, *Al = base + kTcTileBytes, *Bh = base + 2 * kTcTileBytes, *Bl = base + 3 * kTcTileBytes;
    int64_t *rowA = reinterpret_cast<int64_t *>(scratch);
    int64_t *colB = rowA + kTcM;
    int64_t *kAo = colB + kTcNc;
    int64_t *kBo = kAo + kTcKc;
    const int64_t M = d.M, N = d.N, K = d.K;
    const int64_t tiles_n = (N + kTcNc - 1) / kTcNc;
    const int64_t m0 = (tile / tiles_n) * kTcM, n0 = (tile % tiles_n) * kTcNc;
    int32_t eA, eB;
    step_scales(d, j, eA, eB);
    const float sA = pow2<float>(-eA), sB = pow2<float>(-eB);
    const C *__restrict__ A = operand<C>(d, j, true);
    const C *__restrict__ B = operand<C>(d, j, false);
    C *__restrict__ Cp = reinterpret_cast<C *>(j.arena) + d.c_off;
    const int tid = threadIdx.x;
    for (int i = tid; i < kTcM; i += blockDim.x) rowA[i] = (m0 + i < M) ? group_off(d.m, m0 + i) : -1;
    for (int i = tid; i < kTcNc; i += blockDim.x) colB[i] = (n0 + i < N) ? group_off(d.n, n0 + i) : -1;
    const uint32_t idesc = TF32 ? idesc_tf32(kTcM, kTcN) : idesc_bf16(kTcM, kTcN);
    bool ok = true;
    uint32_t acc = 0;
    for (int64_t k0 = 0; k0 < K && ok; k0 += KC) {
        __syncthreads();   // previous K-block's offsets are no longer read
        for (int i = tid; i < KC; i += blockDim.x) {
            int64_t oa = -1, ob = -1;
            if (k0 + i < K) group_off2(d.k, k0 + i, oa, ob);
            kAo[i] = oa;
            kBo[i] = ob;
        }
        __syncthreads();
        // The block's kThreads threads gather the K-block: every load is issued first (RA + RB
        // independent loads in flight per thread), then the values are split and stored.
        // A: 128 rows x KC complex k;  B'': rows 2n = (Re B, -Im B), 2n+1 = (Im B, Re B)
        constexpr int RA = kTcM * KC / kThreads, RB = kTcNc * KC / kThreads;
        static_assert(RA * kThreads == kTcM * KC && RB * kThreads == kTcNc * KC, "gather split");
        C va[RA], vb[RB];
#pragma unroll
        for (int q = 0; q < RA; ++q) {
            const int e = tid + q * kThreads, r = e / KC, kk = e - r * KC;
            va[q] = (rowA[r] >= 0 && kAo[kk] >= 0) ? ldc(A + rowA[r] + kAo[kk]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int e = tid + q * kThreads, nn = e / KC, kk = e - nn * KC;
            vb[q] = (colB[nn] >= 0 && kBo[kk] >= 0) ? ldc(B + kBo[kk] + colB[nn]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < RA; ++q) {
            const int e = tid + q * kThreads, r = e / KC, kk = e - r * KC;
            put_pair<TF32>(Ah, Al, r, kk, va[q].x * sA, va[q].y * sA);
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int e = tid + q * kThreads, nn = e / KC, kk = e - nn * KC;
            const float re = vb[q].x * sB, im = vb[q].y * sB;
            put_pair<TF32>(Bh, Bl, 2 * nn, kk, re, -im);
            put_pair<TF32>(Bh, Bl, 2 * nn + 1, kk, im, re);
        }
        fence_async_smem();   // make the generic-proxy stores visible to the tensor core
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint64_t ah = smem_desc_sw128(smem_u32(Ah)), al = smem_desc_sw128(smem_u32(Al));
            const uint64_t bh = smem_desc_sw128(smem_u32(Bh)), bl = smem_desc_sw128(smem_u32(Bl));
#pragma unroll
            for (int s = 0; s < 4; ++s) {   // 32 bytes of K per MMA: advance inside the atom
                const uint64_t adv = (uint64_t)(s * 32 >> 4);
                if constexpr (TF32) {
                    tc_mma_tf32(tc.tmem, ah + adv, bh + adv, idesc, acc);
                    acc = 1;
                    tc_mma_tf32(tc.tmem, ah + adv, bl + adv, idesc, 1);
                    tc_mma_tf32(tc.tmem, al + adv, bh + adv, idesc, 1);
                } else {
                    tc_mma_bf16(tc.tmem, ah + adv, bh + adv, idesc, acc);
                    acc = 1;
                    tc_mma_bf16(tc.tmem, ah + adv, bl + adv, idesc, 1);
                    tc_mma_bf16(tc.tmem, al + adv, bh + adv, idesc, 1);
                }
            }
            tc_commit(tc.bar);
        }
        acc = 1;
        // all threads wait for the MMAs (the operand tiles are rewritten next)
        ok = mbar_wait(tc.bar, tc.phase, kTcWaitLimit);
        if (ok) {
            tc.phase ^= 1u;
        } else {
            tc.pending = true;
            atomicExch(tc.abort_flag, 1);
        }
        tc_fence_after();
    }
    if (!ok) return false;
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows), column half w / 4
    float mx = 0.f;
    {
        const int warp = tid >> 5, lane = tid & 31;
        const int row = 32 * (warp & 3) + lane;
        const int half = warp >> 2;
        const int64_t m = m0 + row;
        for (int q = 0; q < 4; ++q) {
            float v[16];
            const uint32_t col = (uint32_t)(half * 64 + q * 16);
            tc_ld16(tc.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + col, v);
            if (m < M) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int64_t n = n0 + (col >> 1) + c;
                    if (n < N) {
                        const C out = make_float2(v[2 * c], v[2 * c + 1]);
                        Cp[m * N + n] = out;
                        mx = fmaxf(mx, absmax2(out));
                    }
                }
            }
        }
    }
    tc_fence_before();   // TMEM reads complete before the next tile's MMAs overwrite it
    publish_max(mx, j.maxbits + d.node_c, red);
    tc_fence_after();
    if (tile == 0 && threadIdx.x == 0) write_exponent(d, j, eA, eB);
    return true;
}

__device__ __forceinline__ bool tile_tc(const StepDesc &d, int64_t tile, const JobPtrs &j, char *smem_raw,
                                        char *scratch, float *red, TcState &tc) {
    if (d.flags & FLAG_TF32) return tile_tc_impl<true>(d, tile, j, smem_raw, scratch, red, tc);
    return tile_tc_impl<false>(d, tile, j, smem_raw, scratch, red, tc);
}

}  // namespace tn
