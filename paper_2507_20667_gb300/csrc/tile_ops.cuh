// Tile-level device functions of the contraction kernels.  One call computes one work tile of
// one step; the per-step kernels map blocks to tiles, the persistent kernel claims tiles from a
// global work list.  All operand loads bypass L1 (ld.global.cg): inside one persistent launch an
// arena address is rewritten by later steps, so an SM must never see a stale L1 line.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace tn {

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

template <typename C> __device__ __forceinline__ C ldc(const C *p) { return __ldcg(p); }

template <typename C> __device__ __forceinline__ C cscale(C v, decltype(C::x) s) {
    return cmake(v.x * s, v.y * s);
}

// frexp-style exponent of the float with bit pattern `bits` (0 for zero): x = f * 2^e with f in
// [0.5, 1).  Subnormal maxima are treated as 2^-126.
__device__ __forceinline__ int32_t scale_exponent(uint32_t bits) {
    if (bits == 0u) return 0;
    int32_t e = (int32_t)((bits >> 23) & 0xffu);
    // a max-abs of 2^126 or more keeps e = 126, so that the scale 2^-e stays a normal float (the
    // scaled values then stay below 4); the exponent bookkeeping uses the same e
    return e == 0 ? -126 : (e - 126 > 126 ? 126 : e - 126);
}

// Exact 2^e built from the IEEE-754 exponent field (e within the normal range of T; the scale
// exponents used here stay in [-128, 128]).
template <typename T> __device__ __forceinline__ T pow2(int32_t e);
template <> __device__ __forceinline__ float pow2<float>(int32_t e) {
    e = e < -126 ? -126 : (e > 127 ? 127 : e);
    return __int_as_float((e + 127) << 23);
}
template <> __device__ __forceinline__ double pow2<double>(int32_t e) {
    e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
    return __longlong_as_double((long long)(e + 1023) << 52);
}

__device__ __forceinline__ float absmax2(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }
__device__ __forceinline__ float absmax2(double2 v) { return (float)fmax(fabs(v.x), fabs(v.y)); }

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

// Copy a descriptor into shared memory (all threads), followed by a barrier.
__device__ __forceinline__ void load_desc(StepDesc &dst, const StepDesc *src) {
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(StepDesc) / sizeof(int4)); i += blockDim.x)
        d[i] = __ldcg(s + i);
    __syncthreads();
}
static_assert(sizeof(StepDesc) % sizeof(int4) == 0, "descriptor must be a multiple of 16 bytes");

// The same copy in two halves, so that the loads can be in flight while thread 0 waits on the
// step's dependencies: desc_fetch issues them (one 16-byte piece per thread and round), desc_store
// writes the pieces to shared memory (the caller then synchronises).
constexpr int kDescPieces = (int)(sizeof(StepDesc) / sizeof(int4));
constexpr int kDescRounds = (kDescPieces + kThreads - 1) / kThreads;
__device__ __forceinline__ void desc_fetch(int4 (&r)[kDescRounds], const StepDesc *src) {
    const int4 *s = reinterpret_cast<const int4 *>(src);
#pragma unroll
    for (int q = 0; q < kDescRounds; ++q) {
        const int i = threadIdx.x + q * kThreads;
        if (i < kDescPieces) r[q] = __ldcg(s + i);
    }
}
__device__ __forceinline__ void desc_store(const int4 (&r)[kDescRounds], StepDesc &dst) {
    int4 *d = reinterpret_cast<int4 *>(&dst);
#pragma unroll
    for (int q = 0; q < kDescRounds; ++q) {
        const int i = threadIdx.x + q * kThreads;
        if (i < kDescPieces) d[i] = r[q];
    }
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide max of non-negative values, then one atomicMax on the bit pattern (non-negative
// floats order like their bit patterns).  Ends with a barrier.
__device__ __forceinline__ void publish_max(float v, uint32_t *slot, float *red) {
    v = warp_max(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
        v = warp_max(v);
        if (lane == 0 && v > 0.f) atomicMax(slot, __float_as_uint(v));
    }
    __syncthreads();
}

template <typename C>
__device__ __forceinline__ const C *operand(const StepDesc &d, const JobPtrs &j, bool is_a) {
    const bool leaf = is_a ? (d.flags & FLAG_A_LEAF) : (d.flags & FLAG_B_LEAF);
    const int64_t off = is_a ? d.a_off : d.b_off;
    return leaf ? static_cast<const C *>(j.leaf) + off : reinterpret_cast<const C *>(j.arena) + off;
}

__device__ __forceinline__ void step_scales(const StepDesc &d, const JobPtrs &j, int32_t &eA, int32_t &eB) {
    eA = scale_exponent(__ldcg(j.maxbits + d.node_a));
    eB = scale_exponent(__ldcg(j.maxbits + d.node_b));
}

__device__ __forceinline__ void write_exponent(const StepDesc &d, const JobPtrs &j, int32_t eA, int32_t eB) {
    j.exp2[d.node_c] = __ldcg(j.exp2 + d.node_a) + eA + __ldcg(j.exp2 + d.node_b) + eB;
}

// Shared-memory scratch needed by any tile function, per element type.
template <typename T> struct Scratch {
    using C = cx_t<T>;
    static constexpr int TK_MM = sizeof(T) == 4 ? 8 : 4;   // shared-index chunk of local_mm
    static constexpr int rows = kRowsMaxKN * sizeof(C) + kRowsMaxK * sizeof(int64_t);
    // GEMM operand tiles and index arrays: 64 x 64, and for complex64 also 128 x 32 (the larger)
    static constexpr int tile_cols = sizeof(T) == 4 ? 2 * kTileM + kTileN / 2 : kTileM + kTileN;
    static constexpr int tile = kTileK * tile_cols * sizeof(C) + (tile_cols + 4 * kTileK) * sizeof(int64_t);
    static constexpr int dot = (kThreads / 32) * kDotMaxOut * sizeof(double2) + 2 * kDotMaxOut * sizeof(int64_t);
    // subtree programs: the register-tiled GEMM's operand tiles and offsets, or the REDUCE mode's
    // offset table and FP64 partials
    static constexpr int mm = (TK_MM * (257 + 65) * (int)sizeof(C) + (256 + 64) * 4 + TK_MM * 8 + 15) / 16 * 16;
    static constexpr int local = mm > 1024 * 8 + (kThreads / 32) * 16 ? mm : 1024 * 8 + (kThreads / 32) * 16;
    static constexpr int m1 = rows > tile ? rows : tile;
    static constexpr int m2 = dot > local ? dot : local;
    static constexpr int bytes = m1 > m2 ? m1 : m2;
};

// ------------------------------------------------------------------------------ ROWS
// Tiny-bond contraction (N <= NT <= 16, K <= 64): B (K x N) is staged in shared memory, each
// thread owns output rows m, reads their K entries of A through the index map and writes N
// consecutive outputs.  The K entries of a row are loaded in bursts of KC independent loads, so
// a row pays one memory latency per burst instead of one per entry.  HBM traffic: one read of A,
// one write of C.
template <typename T, int NT>
__device__ void tile_rows(const StepDesc &d, int64_t tile, const JobPtrs &j, char *smem, float *red) {
    using C = cx_t<T>;
    constexpr int KC = 8;
    C *Bs = reinterpret_cast<C *>(smem);
    int64_t *kA = reinterpret_cast<int64_t *>(smem + kRowsMaxKN * sizeof(C));
    const int32_t N = (int32_t)d.N, K = (int32_t)d.K;
    int32_t eA, eB;
    step_scales(d, j, eA, eB);
    const T sA = pow2<T>(-eA), sB = pow2<T>(-eB);
    const C *__restrict__ A = operand<C>(d, j, true);
    const C *__restrict__ B = operand<C>(d, j, false);
    C *__restrict__ Cp = reinterpret_cast<C *>(j.arena) + d.c_off;
    for (int32_t i = threadIdx.x; i < K * N; i += blockDim.x) {
        int32_t k = i / N, n = i - k * N;
        int64_t oa, ob;
        group_off2(d.k, k, oa, ob);
        ob += group_off(d.n, n);
        Bs[i] = cscale(ldc(B + ob), sB);
        if (n == 0) kA[k] = oa;
    }
    __syncthreads();
    const int64_t m_begin = tile * (int64_t)d.tile_rows;
    const int64_t m_end = min(d.M, m_begin + (int64_t)d.tile_rows);
    float mx = 0.f;
    for (int64_t m = m_begin + threadIdx.x; m < m_end; m += blockDim.x) {
        const C *Arow = A + group_off(d.m, m);
        C acc[NT];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n] = cmake((T)0, (T)0);
        for (int32_t k0 = 0; k0 < K; k0 += KC) {
            C a[KC];
#pragma unroll
            for (int kk = 0; kk < KC; ++kk)
                a[kk] = (k0 + kk < K) ? ldc(Arow + kA[k0 + kk]) : cmake((T)0, (T)0);
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                if (k0 + kk >= K) break;
                const C av = cscale(a[kk], sA);
                const C *Bk = Bs + (k0 + kk) * N;
#pragma unroll
                for (int n = 0; n < NT; ++n)
                    if (n < N) cfma(acc[n], av, Bk[n]);
            }
        }
        C *out = Cp + m * N;
#pragma unroll
        for (int n = 0; n < NT; ++n)
            if (n < N) {
                out[n] = acc[n];
                mx = fmaxf(mx, absmax2(acc[n]));
            }
    }
    publish_max(mx, j.maxbits + d.node_c, red);
    if (tile == 0 && threadIdx.x == 0) write_exponent(d, j, eA, eB);
}

// Rotated shared-memory layout of a chained ROWS step's C (N a power of two): element (m, n) of
// the dense row-major [M, N] tensor, dense index i = m N + n, sits at m N + ((n + (m >> r)) mod N)
// with r = max(0, 4 - log2 N).  The threads of a warp each write their own row m; the rotation puts
// their N-th outputs in 16 different 8-byte bank pairs.  The next step maps its dense A index
// through the same function.
__device__ __forceinline__ int32_t rot_index(int32_t i, int32_t lgn) {
    const int32_t mask = (1 << lgn) - 1, r = lgn >= 4 ? 0 : 4 - lgn;
    return (i & ~mask) | ((i + (i >> (lgn + r))) & mask);
}

// Block-wide max of non-negative values, returned to every thread.  Ends with a barrier.
__device__ __forceinline__ float block_max(float v, float *red) {
    v = warp_max(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
    v = warp_max(v);
    __syncthreads();
    return v;
}

// ROWS step whose A fits in shared memory (complex64, FLAG_A_SMEM; the tile covers all M rows):
// A is copied whole with 16-byte cp.async (coalesced) -- or, for a continuation of a chain
// (A_ROT), is already in shared memory in the rotated layout of width 2^a_lgn -- and B densely and
// scaled into the scratch area; each thread owns R = 32 / NT rows with their accumulators in
// registers, reading A from shared memory (a row starts its shared index at m mod K when k is
// contiguous in A, which keeps a warp's reads in different banks).  C then either stays in shared
// memory in the rotated layout (c_in_smem: the next step of the chain consumes it; cmax receives
// the block's max-abs of C) or is written into the same shared memory with padded rows and leaves
// it in coalesced order.  HBM traffic: one read of A, one write of C, both coalesced (neither
// for the inner steps of a chain).  Ends with a barrier.
// Phase cycle accounting of the profiling variant of the dataflow kernel (PROF), compiled out of
// the other one.
template <bool PROF>
__device__ __forceinline__ void prof_phase(long long *prof, int slot, long long &t) {
    if (PROF && threadIdx.x == 0) {
        const long long t1 = clock64();
        atomicAdd((unsigned long long *)(prof + slot), (unsigned long long)(t1 - t));
        atomicAdd((unsigned long long *)(prof + kProfSlots + slot), 1ull);
        t = t1;
    }
}

template <int NT, bool A_ROT, bool PROF>
__device__ void rows_smem_core(const StepDesc &d, const JobPtrs &j, char *smem, char *dyn, float *red,
                               float sA, float sB, bool c_in_smem, float &cmax, long long *prof) {
    long long tp = 0;
    if (PROF && threadIdx.x == 0) tp = clock64();
    using C = float2;
    constexpr int R = 32 / NT;
    C *As = reinterpret_cast<C *>(dyn);
    // [K][PB] scaled B, PB = N + 1 rounded up to even: rows start on 16 bytes and are read two
    // entries per load
    C *Bd = reinterpret_cast<C *>(smem);
    int32_t *kat = reinterpret_cast<int32_t *>(Bd + 16 * (NT + 2));   // [K] offsets in A
    const int32_t M = (int32_t)d.M, N = (int32_t)d.N, K = (int32_t)d.K, PB = (N + 2) & ~1, MK = M * K;
    const int32_t PC = N + 1;   // padded C rows (M (N + 1) elements fit by construction)
    const C *__restrict__ A = operand<C>(d, j, true);
    const C *__restrict__ B = operand<C>(d, j, false);
    C *__restrict__ Cp = reinterpret_cast<C *>(j.arena) + d.c_off;
    const int tid = threadIdx.x;
    if (!A_ROT) {
        for (int32_t i = tid; 2 * i + 1 < MK; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(As + 2 * i)),
                         "l"(A + 2 * i)
                         : "memory");
        if ((MK & 1) && tid == 0)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(As + MK - 1)),
                         "l"(A + MK - 1)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int32_t i = tid; i < K * N; i += blockDim.x) {
        const int32_t k = i / N, n = i - k * N;
        int64_t oa, ob;
        group_off2(d.k, k, oa, ob);
        ob += group_off(d.n, n);
        Bd[k * PB + n] = cscale(ldc(B + ob), sB);
        if (n == 0) kat[k] = (int32_t)oa;
    }
    if (!A_ROT) asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    prof_phase<PROF>(prof, 7, tp);
    const int32_t lga = d.a_lgn;
    const bool skew = d.k.n > 0 && d.k.sa[0] == 1;
    const int32_t step = blockDim.x;
    C acc[R][NT];
    int32_t rows[R];
    // rows m0 + r * step of this thread (one pass: M <= R * blockDim by construction)
    const int32_t m0 = tid;
    const int32_t sh = skew ? m0 % K : 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int32_t m = m0 + r * step;
        rows[r] = m < M ? (int32_t)group_off(d.m, m) : -1;
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[r][n] = make_float2(0.f, 0.f);
    }
#pragma unroll 1
    for (int32_t kk = 0; kk < K; ++kk) {
        int32_t k = kk + sh;
        if (k >= K) k -= K;
        const int32_t ko = kat[k];
        C av[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int32_t ia = rows[r] + ko;
            if (A_ROT) ia = rot_index(ia, lga);
            av[r] = rows[r] >= 0 ? cscale(As[ia], sA) : make_float2(0.f, 0.f);
        }
        const float4 *Bk = reinterpret_cast<const float4 *>(Bd + k * PB);
#pragma unroll
        for (int n2 = 0; n2 < NT / 2; ++n2) {
            if (2 * n2 >= N) break;
            const float4 bb = Bk[n2];
            const C b0 = make_float2(bb.x, bb.y), b1 = make_float2(bb.z, bb.w);
#pragma unroll
            for (int r = 0; r < R; ++r) cfma(acc[r][2 * n2], av[r], b0);
            if (2 * n2 + 1 < N) {
#pragma unroll
                for (int r = 0; r < R; ++r) cfma(acc[r][2 * n2 + 1], av[r], b1);
            }
        }
    }
    __syncthreads();   // every thread is done reading A
    prof_phase<PROF>(prof, 11, tp);
    float mx = 0.f;
    if (c_in_smem) {
        const int32_t lgn = __ffs(N) - 1, rs = lgn >= 4 ? 0 : 4 - lgn;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int32_t m = m0 + r * step;
            if (m >= M) continue;
#pragma unroll
            for (int n = 0; n < NT; ++n)
                if (n < N) {
                    As[m * N + ((n + (m >> rs)) & (N - 1))] = acc[r][n];
                    mx = fmaxf(mx, absmax2(acc[r][n]));
                }
        }
        cmax = block_max(mx, red);
        prof_phase<PROF>(prof, 15, tp);
        return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int32_t m = m0 + r * step;
        if (m >= M) continue;
#pragma unroll
        for (int n = 0; n < NT; ++n)
            if (n < N) {
                As[m * PC + n] = acc[r][n];
                mx = fmaxf(mx, absmax2(acc[r][n]));
            }
    }
    __syncthreads();
    for (int32_t i = tid; i < M * N; i += blockDim.x) {
        const int32_t m = i / N;
        Cp[i] = As[m * PC + (i - m * N)];
    }
    publish_max(mx, j.maxbits + d.node_c, red);
    prof_phase<PROF>(prof, 15, tp);
}

template <bool A_ROT, bool PROF>
__device__ __forceinline__ void rows_smem_any(const StepDesc &d, const JobPtrs &j, char *smem, char *dyn,
                                              float *red, float sA, float sB, bool c_in_smem, float &cmax,
                                              long long *prof) {
    if (d.N <= 4) rows_smem_core<4, A_ROT, PROF>(d, j, smem, dyn, red, sA, sB, c_in_smem, cmax, prof);
    else if (d.N <= 8) rows_smem_core<8, A_ROT, PROF>(d, j, smem, dyn, red, sA, sB, c_in_smem, cmax, prof);
    else rows_smem_core<16, A_ROT, PROF>(d, j, smem, dyn, red, sA, sB, c_in_smem, cmax, prof);
}

// A ROWS step staged through shared memory on its own.
__device__ __forceinline__ void tile_rows_smem(const StepDesc &d, const JobPtrs &j, char *smem, char *dyn,
                                               float *red) {
    int32_t eA, eB;
    step_scales(d, j, eA, eB);
    float cmax = 0.f;
    rows_smem_any<false, false>(d, j, smem, dyn, red, pow2<float>(-eA), pow2<float>(-eB), false, cmax, nullptr);
    if (threadIdx.x == 0) write_exponent(d, j, eA, eB);
}

// A chain of ROWS steps linked by chain_next, run by one block of the persistent kernel: the first
// step reads A from the arena, each later one takes the previous step's C, kept in shared memory,
// as its A, and the last writes its C to the arena.  The per-step power-of-two scaling is
// unchanged: a continuation's A exponent comes from the block max of the previous C, which is the
// value the separate steps would publish, so results are bit-identical to running the steps one
// by one; the exponents of the inner nodes stay in registers and only the last node's max-abs and
// exponent are written.  d is the block's shared descriptor and is overwritten with each step's;
// thread 0 writes the indices of the continuation steps to chain[].  Returns their count.
template <bool PROF>
__device__ __forceinline__ int32_t rows_chain(StepDesc &d, const JobPtrs &j, char *smem, char *dyn, float *red,
                                              int32_t *chain, long long *prof) {
    int32_t eA, eB;
    step_scales(d, j, eA, eB);
    int32_t xa = __ldcg(j.exp2 + d.node_a), xb = __ldcg(j.exp2 + d.node_b);
    int32_t n = 0;
    while (true) {
        const int32_t next = d.chain_next;
        int4 dr[kDescRounds];
        if (next >= 0) desc_fetch(dr, j.steps + next);
        float cmax = 0.f;
        const float sA = pow2<float>(-eA), sB = pow2<float>(-eB);
        if (n == 0) rows_smem_any<false, PROF>(d, j, smem, dyn, red, sA, sB, next >= 0, cmax, prof);
        else rows_smem_any<true, PROF>(d, j, smem, dyn, red, sA, sB, next >= 0, cmax, prof);
        const int32_t xc = xa + eA + xb + eB;
        if (next < 0) {
            if (threadIdx.x == 0) j.exp2[d.node_c] = xc;
            return n;
        }
        desc_store(dr, d);   // the step ended with a barrier: nobody reads the old descriptor
        __syncthreads();
        if (threadIdx.x == 0) chain[n] = next;
        ++n;
        xa = xc;
        eA = scale_exponent(__float_as_uint(cmax));
        eB = scale_exponent(__ldcg(j.maxbits + d.node_b));
        xb = __ldcg(j.exp2 + d.node_b);
    }
}

template <typename T>
__device__ __forceinline__ void tile_rows_dispatch(const StepDesc &d, int64_t tile, const JobPtrs &j,
                                                   char *smem, float *red, char *dyn) {
    if constexpr (sizeof(T) == 4) {
        if (d.flags & FLAG_A_SMEM) {
            tile_rows_smem(d, j, smem, dyn, red);
            return;
        }
    }
    if (d.N <= 1) tile_rows<T, 1>(d, tile, j, smem, red);
    else if (d.N <= 2) tile_rows<T, 2>(d, tile, j, smem, red);
    else if (d.N <= 4) tile_rows<T, 4>(d, tile, j, smem, red);
    else if (d.N <= 8) tile_rows<T, 8>(d, tile, j, smem, red);
    else tile_rows<T, 16>(d, tile, j, smem, red);
}

// ------------------------------------------------------------------------------ TILE (GEMM)
// General contraction on CUDA cores: a TM x TN output tile (64 x 64, or 128 x 32 for narrow N),
// K in chunks of kTileK, operand tiles gathered through the index maps into shared memory, 4 x 4
// outputs per thread.  The gathers of chunk c + 1 are issued into registers before chunk c is
// computed, so their latency overlaps the arithmetic.
template <typename T, int TM, int TN>
__device__ void tile_gemm(const StepDesc &d, int64_t tile, const JobPtrs &j, char *smem, float *red) {
    using C = cx_t<T>;
    constexpr int TX = TN / 4, TY = TM / 4;
    static_assert(TX * TY == kThreads, "one 4 x 4 register tile per thread");
    constexpr int RA = TM * kTileK / kThreads, RB = TN * kTileK / kThreads;
    static_assert(RA * kThreads == TM * kTileK && RB * kThreads == TN * kTileK, "operand tile split");
    C(*As)[TM] = reinterpret_cast<C(*)[TM]>(smem);
    C(*Bs)[TN] = reinterpret_cast<C(*)[TN]>(smem + kTileK * TM * sizeof(C));
    int64_t *rowA = reinterpret_cast<int64_t *>(smem + kTileK * (TM + TN) * sizeof(C));
    int64_t *colB = rowA + TM;
    int64_t(*kAo)[kTileK] = reinterpret_cast<int64_t(*)[kTileK]>(colB + TN);   // [2][kTileK]
    int64_t(*kBo)[kTileK] = kAo + 2;
    const int64_t M = d.M, N = d.N, K = d.K;
    const int64_t tiles_n = (N + TN - 1) / TN;
    const int64_t m0 = (tile / tiles_n) * TM, n0 = (tile % tiles_n) * TN;
    int32_t eA, eB;
    step_scales(d, j, eA, eB);
    const T sA = pow2<T>(-eA), sB = pow2<T>(-eB);
    const C *__restrict__ A = operand<C>(d, j, true);
    const C *__restrict__ B = operand<C>(d, j, false);
    C *__restrict__ Cp = reinterpret_cast<C *>(j.arena) + d.c_off;
    const int tid = threadIdx.x;
    for (int i = tid; i < TM + TN; i += kThreads) {
        if (i < TM) rowA[i] = (m0 + i < M) ? group_off(d.m, m0 + i) : -1;
        else colB[i - TM] = (n0 + i - TM < N) ? group_off(d.n, n0 + i - TM) : -1;
    }
    const int64_t nch = (K + kTileK - 1) / kTileK;
    auto koffs = [&](int64_t c) {
        if (tid < kTileK) {
            const int64_t k = c * kTileK + tid;
            int64_t oa = -1, ob = -1;
            if (k < K) group_off2(d.k, k, oa, ob);
            kAo[c & 1][tid] = oa;
            kBo[c & 1][tid] = ob;
        }
    };
    C ra[RA], rb[RB];
    auto gather = [&](int64_t c) {
        const int64_t *ka = kAo[c & 1], *kb = kBo[c & 1];
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const int i = tid + r * kThreads, row = i % TM, kk = i / TM;
            ra[r] = (rowA[row] >= 0 && ka[kk] >= 0) ? ldc(A + rowA[row] + ka[kk]) : cmake((T)0, (T)0);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int i = tid + r * kThreads, col = i % TN, kk = i / TN;
            rb[r] = (colB[col] >= 0 && kb[kk] >= 0) ? ldc(B + kb[kk] + colB[col]) : cmake((T)0, (T)0);
        }
    };
    koffs(0);
    __syncthreads();
    gather(0);
    const int tx = tid % TX, ty = tid / TX;
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = cmake((T)0, (T)0);
    for (int64_t c = 0; c < nch; ++c) {
        __syncthreads();   // the previous chunk's arithmetic is done with As / Bs
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const int i = tid + r * kThreads;
            As[i / TM][i % TM] = cscale(ra[r], sA);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int i = tid + r * kThreads;
            Bs[i / TN][i % TN] = cscale(rb[r], sB);
        }
        if (c + 1 < nch) koffs(c + 1);
        __syncthreads();
        if (c + 1 < nch) gather(c + 1);
#pragma unroll
        for (int kk = 0; kk < kTileK; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + TY * i];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) b[jj] = Bs[kk][tx + TX * jj];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) cfma(acc[i][jj], a[i], b[jj]);
        }
    }
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + TY * i;
        if (m >= M) continue;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            int64_t n = n0 + tx + TX * jj;
            if (n < N) {
                Cp[m * N + n] = acc[i][jj];
                mx = fmaxf(mx, absmax2(acc[i][jj]));
            }
        }
    }
    publish_max(mx, j.maxbits + d.node_c, red);
    if (tile == 0 && threadIdx.x == 0) write_exponent(d, j, eA, eB);
}

// ------------------------------------------------------------------------------ DOT
// Small outputs (M * N <= kDotMaxOut) with a long shared index.  DOTP: each tile reduces
// kDotChunk shared indices; products are formed in the storage precision, summed per thread in
// bursts of 8 in that precision and then in FP64.  DOTF: one tile sums the partials in a fixed order, so results are
// reproducible.  The root step of a closed network (M = N = 1) always takes this path: the final
// reduction of the amplitude is FP64.
template <typename T>
__device__ void tile_dotp(const StepDesc &d, int64_t tile, const JobPtrs &j, char *smem, char *dyn) {
    using C = cx_t<T>;
    double2(*red)[kDotMaxOut] = reinterpret_cast<double2(*)[kDotMaxOut]>(smem);
    int64_t *rowA = reinterpret_cast<int64_t *>(smem + (kThreads / 32) * kDotMaxOut * sizeof(double2));
    int64_t *colB = rowA + kDotMaxOut;
    const int32_t M = (int32_t)d.M, N = (int32_t)d.N;
    const int32_t MN = M * N;
    if (threadIdx.x < M) rowA[threadIdx.x] = group_off(d.m, threadIdx.x);
    if (threadIdx.x < N) colB[threadIdx.x] = group_off(d.n, threadIdx.x);
    __syncthreads();
    int32_t eA, eB;
    step_scales(d, j, eA, eB);
    const T sA = pow2<T>(-eA), sB = pow2<T>(-eB);
    const C *__restrict__ A = operand<C>(d, j, true);
    const C *__restrict__ B = operand<C>(d, j, false);
    // an operand whose offsets are permuted along k (complex64 only) is copied whole -- K elements,
    // 16-byte aligned in the arena -- with coalesced 16-byte copies, then gathered from shared
    // memory with plain loads (Xs)
    const bool sm_a = sizeof(T) == 4 && (d.flags & FLAG_DOT_SMEM_A) != 0;
    const bool sm_b = sizeof(T) == 4 && (d.flags & FLAG_DOT_SMEM_B) != 0;
    C *Xs = reinterpret_cast<C *>(dyn);
    if (sm_a || sm_b) {
        const C *src = sm_a ? A : B;
        const int32_t K = (int32_t)d.K;
        for (int32_t i = threadIdx.x; 2 * i + 1 < K; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(Xs + 2 * i)),
                         "l"(src + 2 * i)
                         : "memory");
        if ((K & 1) && threadIdx.x == 0) Xs[K - 1] = ldc(src + K - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
    }
    double2 acc[kDotMaxOut];
#pragma unroll
    for (int i = 0; i < kDotMaxOut; ++i) acc[i] = make_double2(0, 0);
    const int64_t k_begin = tile * (int64_t)d.tile_rows;
    const int64_t k_end = min(d.K, k_begin + (int64_t)d.tile_rows);
    // bursts of U shared indices per thread: offsets first, then U independent load pairs; each
    // burst is summed in the storage precision and then added in FP64
    constexpr int U = 8;
    for (int64_t kb = k_begin; kb < k_end; kb += (int64_t)U * blockDim.x) {
        int64_t oa[U], ob[U];
        if (d.ktab_off >= 0) {   // tabulated offsets: one coalesced 8-byte load per index
            const int2 *tab = j.ktab + d.ktab_off;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = kb + (int64_t)u * blockDim.x + threadIdx.x;
                oa[u] = -1;
                ob[u] = 0;
                if (k < k_end) {
                    const int2 t = __ldg(tab + k);
                    oa[u] = t.x;
                    ob[u] = t.y;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = kb + (int64_t)u * blockDim.x + threadIdx.x;
                oa[u] = -1;
                ob[u] = 0;
                if (k < k_end) group_off2(d.k, k, oa[u], ob[u]);
            }
        }
        C run[kDotMaxOut];
#pragma unroll
        for (int i = 0; i < kDotMaxOut; ++i) run[i] = cmake((T)0, (T)0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (oa[u] < 0) continue;
#pragma unroll
            for (int i = 0; i < kDotMaxOut; ++i) {
                if (i < MN) {
                    const int m = i / N, n = i - m * N;
                    const C av = sm_a ? Xs[oa[u] + rowA[m]] : ldc(A + oa[u] + rowA[m]);
                    const C bv = sm_b ? Xs[ob[u] + colB[n]] : ldc(B + ob[u] + colB[n]);
                    const C a = cscale(av, sA), b = cscale(bv, sB);
                    cfma(run[i], a, b);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kDotMaxOut; ++i) {
            acc[i].x += (double)run[i].x;
            acc[i].y += (double)run[i].y;
        }
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
        for (int w = 0; w < kThreads / 32; ++w) { s.x += red[w][threadIdx.x].x; s.y += red[w][threadIdx.x].y; }
        j.partials[d.part_off + tile * kDotMaxOut + threadIdx.x] = s;
    }
    __syncthreads();
}

template <typename T>
__device__ void tile_dotf(const StepDesc &d, const JobPtrs &j, char *smem) {
    using C = cx_t<T>;
    double2(*red)[kDotMaxOut] = reinterpret_cast<double2(*)[kDotMaxOut]>(smem);
    const int32_t MN = (int32_t)(d.M * d.N);
    const int32_t nparts = d.tile_rows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < MN; ++i) {
        double x = 0, y = 0;
        for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
            double2 p = __ldcg(j.partials + d.part_off + (int64_t)b * kDotMaxOut + i);
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
    int32_t eA, eB;
    step_scales(d, j, eA, eB);
    const int32_t e_out = __ldcg(j.exp2 + d.node_a) + eA + __ldcg(j.exp2 + d.node_b) + eB;
    if (threadIdx.x < MN) {
        double2 s = make_double2(0, 0);
        for (int w = 0; w < kThreads / 32; ++w) { s.x += red[w][threadIdx.x].x; s.y += red[w][threadIdx.x].y; }
        if (d.flags & FLAG_ROOT) {
            DeviceResult *r = static_cast<DeviceResult *>(j.result);
            r->re = s.x;
            r->im = s.y;
            r->exp2 = e_out;
        }
        if (!(d.flags & FLAG_NO_C)) {
            C v = cmake((T)s.x, (T)s.y);
            (reinterpret_cast<C *>(j.arena) + d.c_off)[threadIdx.x] = v;
            atomicMax(j.maxbits + d.node_c, __float_as_uint(absmax2(v)));
        }
    }
    if (threadIdx.x == 0) j.exp2[d.node_c] = e_out;
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void run_tile(const StepDesc &d, int64_t tile, const JobPtrs &j, char *smem,
                                         float *red, char *dyn) {
    switch (d.kind) {
        case STEP_ROWS: tile_rows_dispatch<T>(d, tile, j, smem, red, dyn); break;
        case STEP_TILE:
            if constexpr (sizeof(T) == 4) {
                if (d.tile_rows == kTileNarrow) {
                    tile_gemm<T, 2 * kTileM, kTileN / 2>(d, tile, j, smem, red);
                    break;
                }
            }
            tile_gemm<T, kTileM, kTileN>(d, tile, j, smem, red);
            break;
        case STEP_DOTP: tile_dotp<T>(d, tile, j, smem, dyn); break;
        case STEP_DOTF: tile_dotf<T>(d, j, smem); break;
        default: break;
    }
}

}  // namespace tn
