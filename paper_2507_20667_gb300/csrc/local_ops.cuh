// CTA-resident subtree programs.  A subtree of the contraction tree whose sequential working set
// (its leaves plus the intermediates alive at any one time) fits a shared-memory budget runs
// entirely inside one thread block: the block stages the subtree's leaves into shared memory,
// executes its pairwise steps in plan order with one barrier per step, and writes only the
// subtree's result to global memory.  This replaces hundreds of tiny global work tiles -- each a
// claim, a dependency wait and a global round trip -- by on-chip work.
#pragma once

#include <cstdint>

#include "kernels.cuh"
#include "tile_ops.cuh"

namespace tn {

__device__ __forceinline__ int32_t lgroup_off(int32_t n, const int32_t *dim, const int32_t *str,
                                              const uint8_t *lsb, bool pow2, int32_t idx) {
    int32_t off = 0;
    if (pow2) {
        for (int32_t i = 0; i < n; ++i) off += ((idx >> lsb[i]) & (dim[i] - 1)) * str[i];
    } else {
        for (int32_t i = 0; i < n; ++i) {
            const int32_t d = idx % dim[i];
            idx /= dim[i];
            off += d * str[i];
        }
    }
    return off;
}

__device__ __forceinline__ void lgroup_off2(const LocalStep &s, int32_t idx, int32_t &oa, int32_t &ob) {
    oa = 0;
    ob = 0;
    if (s.pow2) {
        for (int32_t i = 0; i < s.nk; ++i) {
            const int32_t d = (idx >> s.k_lsb[i]) & (s.k_dim[i] - 1);
            oa += d * s.k_sa[i];
            ob += d * s.k_sb[i];
        }
    } else {
        for (int32_t i = 0; i < s.nk; ++i) {
            const int32_t d = idx % s.k_dim[i];
            idx /= s.k_dim[i];
            oa += d * s.k_sa[i];
            ob += d * s.k_sb[i];
        }
    }
}

// A power-of-two group list held in registers: offset(idx) = sum ((idx >> lsb) & mask) * stride.
struct RegGroups {
    int32_t n;
    int32_t lsb[kLG], mask[kLG], str[kLG];
};

__device__ __forceinline__ RegGroups reg_groups(int32_t n, const int32_t *dim, const int32_t *str,
                                                const uint8_t *lsb) {
    RegGroups g;
    g.n = n;
#pragma unroll
    for (int i = 0; i < kLG; ++i) {
        g.lsb[i] = i < n ? lsb[i] : 0;
        g.mask[i] = i < n ? dim[i] - 1 : 0;
        g.str[i] = i < n ? str[i] : 0;
    }
    return g;
}

__device__ __forceinline__ int32_t reg_off(const RegGroups &g, int32_t idx) {
    int32_t off = 0;
#pragma unroll
    for (int i = 0; i < kLG; ++i) off += ((idx >> g.lsb[i]) & g.mask[i]) * g.str[i];
    return off;
}

constexpr int kKTab = 1024;   // shared indices whose offsets are tabulated per step

struct LocalSmem {
    LocalStep *desc;     // all step descriptors of the program, in execution order
    LocalWave *waves;
    uint32_t *smax;      // [n_slots] max-abs bit pattern of each node of the program
    int32_t *sexp;       // [n_slots] power-of-two exponent of each node
    char *data;          // leaves, then the arena of intermediates
};

// Shared-memory layout of a program (the host computes the same sizes in local_fit).
__device__ __host__ __forceinline__ size_t local_fixed_bytes(int32_t n_steps, int32_t n_waves, int32_t n_slots) {
    return (size_t)n_steps * sizeof(LocalStep) + (size_t)n_waves * sizeof(LocalWave) +
           ((8 * (size_t)n_slots + 15) / 16) * 16;
}

__device__ __forceinline__ LocalSmem local_layout(char *dyn, const LocalProg &P) {
    LocalSmem L;
    L.desc = reinterpret_cast<LocalStep *>(dyn);
    L.waves = reinterpret_cast<LocalWave *>(dyn + (size_t)P.n_steps * sizeof(LocalStep));
    L.smax = reinterpret_cast<uint32_t *>(L.waves + P.n_waves);
    L.sexp = reinterpret_cast<int32_t *>(L.smax + P.n_slots);
    L.data = dyn + local_fixed_bytes(P.n_steps, P.n_waves, P.n_slots);
    return L;
}

// Copies a program's inputs into shared memory: one staging piece (at most 16 elements of a leaf
// or of a program's result) per thread, its elements loaded in bursts of LB independent loads;
// the first piece of each input also copies the input's max-abs and exponent.
template <typename T, int LB = 16>
__device__ __forceinline__ void stage_inputs(const JobPtrs &j, const LeafRef *refs, int32_t n_refs, int32_t t0,
                                             int32_t stride, cx_t<T> *data, uint32_t *smax, int32_t *sexp) {
    using C = cx_t<T>;
    for (int32_t l = t0; l < n_refs; l += stride) {
        const LeafRef r = refs[l];
        if (r.slot >= 0) {
            smax[r.slot] = __ldcg(j.maxbits + r.node);
            sexp[r.slot] = __ldcg(j.exp2 + r.node);
        }
        const C *src = (r.src ? reinterpret_cast<const C *>(j.arena) : static_cast<const C *>(j.leaf)) + r.global_off;
        for (int32_t i0 = 0; i0 < r.count; i0 += LB) {
            C v[LB];
#pragma unroll
            for (int u = 0; u < LB; ++u)
                if (i0 + u < r.count) v[u] = __ldcg(src + i0 + u);
#pragma unroll
            for (int u = 0; u < LB; ++u)
                if (i0 + u < r.count) data[r.smem_off + i0 + u] = v[u];
        }
    }
}

// Asynchronous copies (cp.async) of program inputs into shared memory, so that a large program's
// next wave of inputs is in flight while the current wave computes.
__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// stage_inputs with asynchronous copies (the caller commits, waits and synchronises); the scale
// slots are written at once.
template <typename T>
__device__ __forceinline__ void stage_inputs_async(const JobPtrs &j, const LeafRef *refs, int32_t n_refs, int32_t t0,
                                                   int32_t stride, cx_t<T> *data, uint32_t *smax, int32_t *sexp) {
    using C = cx_t<T>;
    for (int32_t l = t0; l < n_refs; l += stride) {
        const LeafRef r = refs[l];
        if (r.slot >= 0) {
            smax[r.slot] = __ldcg(j.maxbits + r.node);
            sexp[r.slot] = __ldcg(j.exp2 + r.node);
        }
        const C *src = (r.src ? reinterpret_cast<const C *>(j.arena) : static_cast<const C *>(j.leaf)) + r.global_off;
        for (int32_t i = 0; i < r.count; ++i) {
            if constexpr (sizeof(C) == 8) cp_async8(data + r.smem_off + i, src + i);
            else cp_async16(data + r.smem_off + i, src + i);
        }
    }
}

// Error-free transformations (Knuth's TwoSum; the FMA form of Dekker's TwoProduct, as used by
// Ogita, Rump and Oishi for accurate dot products), written with round-to-nearest intrinsics so
// that the compiler neither contracts nor reorders them: a + b = s + err and a * b = p + err
// exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// A sum kept as an unevaluated pair hi + lo (about 44 significant bits); adds x = xh + xl.
__device__ __forceinline__ void df_add(float &hi, float &lo, float xh, float xl) {
    float s, t;
    two_sum(hi, xh, s, t);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(xl, t));
}

// A small step computed by one warp: C = A * B with A, B and C at any address (shared memory, or
// global memory in warp programs).  S lanes share an output (S a power of two, S <= 32 / outputs,
// S <= K) and split its shared index; their partial sums are combined with xor shuffles.  The
// shared-index offsets are computed once per 32 indices -- lane l holds (kA, kB) of index k0 + l,
// packed in 16 bits each (program operands have fewer than 2^16 elements) -- and are broadcast
// with a shuffle.  The operand scales 2^-eA and 2^-eB are applied together on the B side when
// their product is a normal number (products then round exactly as with separate scaling), else
// separately.  In complex64 each output is accumulated as hi + lo pairs from exact products and
// exact pairwise sums, and rounded once when it is stored: these steps are most of a circuit's
// steps, and with plain FP32 multiply-adds their several roundings per output (rather than the one
// of storing it) tripled the error of small amplitudes; the extra arithmetic costs about 3 % of
// the time of a batch of 24-qubit brickwork amplitudes, where these steps are latency-bound.
// Returns the warp-wide max-abs of C (every lane).
template <typename T>
__device__ __forceinline__ float small_core(const LocalStep &s, const cx_t<T> *A, const cx_t<T> *B, cx_t<T> *Cp,
                                            int32_t eA, int32_t eB) {
    using C = cx_t<T>;
    const int lane = threadIdx.x & 31;
    const int32_t es = eA + eB;
    const bool fold = es > -120 && es < 120;
    const T sA = fold ? (T)1 : pow2<T>(-eA);
    const T sB = fold ? pow2<T>(-es) : pow2<T>(-eB);
    const int32_t N = s.N, K = s.K, O = s.M * s.N;
    const bool tab = (s.flags & LFLAG_TAB) != 0;
    const uint32_t *tbl = reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(&s) +
                                                             offsetof(LocalStep, m_dim));
    int32_t S = 1;
    while (S * 2 * O <= 32 && S < K) S *= 2;
    const int32_t sub = lane & (S - 1), per_pass = 32 / S;
    const bool p2 = s.pow2;
    float mx = 0.f;
    for (int32_t o0 = 0; o0 < O; o0 += per_pass) {
        const int32_t o = o0 + lane / S;
        const bool act = o < O;
        int32_t oa = 0, ob = 0;
        if (act && tab) {
            const uint32_t t = tbl[o];
            oa = (int32_t)(t & 0xffffu);
            ob = (int32_t)(t >> 16);
        } else if (act) {
            const int32_t m = o / N, n = o - m * N;
            oa = lgroup_off(s.nm, s.m_dim, s.m_str, s.m_lsb, p2, m);
            ob = lgroup_off(s.nn, s.n_dim, s.n_str, s.n_lsb, p2, n);
        }
        C acc = cmake((T)0, (T)0);
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;   // complex64: the sums as hi + lo pairs
        for (int32_t k0 = 0; k0 < K; k0 += 32) {
            uint32_t packed = 0;
            if (k0 + lane < K) {
                if (tab) {
                    packed = tbl[kTabOut + lane];   // K <= kTabK: one pass, k0 = 0
                } else {
                    int32_t ka, kb;
                    lgroup_off2(s, k0 + lane, ka, kb);
                    packed = (uint32_t)ka | ((uint32_t)kb << 16);
                }
            }
            const int32_t kn = min(32, K - k0);
            for (int32_t kk = 0; kk < kn; kk += S) {
                const int32_t k = kk + sub;
                const uint32_t p = __shfl_sync(0xffffffffu, packed, k & 31);
                if (act && k < kn) {
                    const C a = A[oa + (int32_t)(p & 0xffffu)];
                    const C b = B[ob + (int32_t)(p >> 16)];
                    const C as = fold ? a : cscale(a, sA), bs = cscale(b, sB);
                    if constexpr (sizeof(T) == 4) {
                        // exact products, then exact sums of pairs: Re and Im of a * b as hi + lo
                        const float p1 = __fmul_rn(as.x, bs.x), e1 = __fmaf_rn(as.x, bs.x, -p1);
                        const float p2 = __fmul_rn(as.y, bs.y), e2 = __fmaf_rn(as.y, bs.y, -p2);
                        const float p3 = __fmul_rn(as.x, bs.y), e3 = __fmaf_rn(as.x, bs.y, -p3);
                        const float p4 = __fmul_rn(as.y, bs.x), e4 = __fmaf_rn(as.y, bs.x, -p4);
                        float s1, t1, s2, t2;
                        two_sum(p1, -p2, s1, t1);
                        two_sum(p3, p4, s2, t2);
                        df_add(rh, rl, s1, __fadd_rn(__fsub_rn(e1, e2), t1));
                        df_add(ih, il, s2, __fadd_rn(__fadd_rn(e3, e4), t2));
                    } else {
                        cfma(acc, as, bs);
                    }
                }
            }
        }
        if constexpr (sizeof(T) == 4) {
            for (int32_t off = S >> 1; off > 0; off >>= 1) {
                const float orh = __shfl_xor_sync(0xffffffffu, rh, off), orl = __shfl_xor_sync(0xffffffffu, rl, off);
                const float oih = __shfl_xor_sync(0xffffffffu, ih, off), oil = __shfl_xor_sync(0xffffffffu, il, off);
                df_add(rh, rl, orh, orl);
                df_add(ih, il, oih, oil);
            }
            acc = cmake(__fadd_rn(rh, rl), __fadd_rn(ih, il));   // one rounding of each sum
        } else {
            for (int32_t off = S >> 1; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
        }
        if (act && sub == 0) {
            Cp[o] = acc;
            mx = fmaxf(mx, absmax2(acc));
        }
    }
    // non-negative floats order like their bit patterns
    return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
}

// A small step of a block program, run by one warp; the warp publishes the output's max-abs and
// exponent itself.
template <typename T>
__device__ __forceinline__ void local_small(const LocalStep &s, const LocalSmem &L) {
    using C = cx_t<T>;
    const int32_t eA = scale_exponent(L.smax[s.sa]), eB = scale_exponent(L.smax[s.sb]);
    const float mx = small_core<T>(s, reinterpret_cast<const C *>(L.data) + s.a_off,
                                   reinterpret_cast<const C *>(L.data) + s.b_off,
                                   reinterpret_cast<C *>(L.data) + s.c_off, eA, eB);
    if ((threadIdx.x & 31) == 0) {
        L.smax[s.sc] = __float_as_uint(mx);
        L.sexp[s.sc] = L.sexp[s.sa] + eA + L.sexp[s.sb] + eB;
    }
}

// Shared-memory slice of a warp program: the current step's descriptor, the scale slots of its
// intermediates, then the intermediates (the host computes the same sizes).
__device__ __host__ __forceinline__ size_t warp_fixed_bytes(int32_t n_slots) {
    return sizeof(LocalStep) + ((8 * (size_t)n_slots + 15) / 16) * 16;
}

// Runs warp program `prog` of job `j` in the calling warp, `slice` being its kWarpSlice bytes of
// shared memory.  The warp stages the program's leaves into the slice, then runs the steps in
// plan order with every operand in shared memory; the last step writes the program's result (and
// its max-abs and exponent) to global memory.  Each step's descriptor is prefetched while the
// previous step runs.
template <typename T>
__device__ void run_warp_prog(int32_t prog, const JobPtrs &j, char *slice) {
    using C = cx_t<T>;
    const int lane = threadIdx.x & 31;
    const LocalProg &P = j.progs[prog];
    const int32_t n_steps = P.n_steps, first = P.first_step, n_slots = P.n_slots;
    const int64_t root_c_off = P.root_c_off;
    const int32_t root_node = P.root_node;
    LocalStep *desc = reinterpret_cast<LocalStep *>(slice);
    uint32_t *smax = reinterpret_cast<uint32_t *>(slice + sizeof(LocalStep));
    int32_t *sexp = reinterpret_cast<int32_t *>(smax + n_slots);
    C *data = reinterpret_cast<C *>(slice + warp_fixed_bytes(n_slots));
    constexpr int kPieces = (int)(sizeof(LocalStep) / sizeof(int4));
    static_assert(kPieces <= 32, "one descriptor piece per lane");
    const int4 *dsrc = reinterpret_cast<const int4 *>(j.lsteps + first);
    int4 nxt = make_int4(0, 0, 0, 0);
    if (lane < kPieces) nxt = __ldg(dsrc + lane);
    stage_inputs<T>(j, j.leafrefs + P.first_leaf, P.n_leaves, lane, 32, data, smax, sexp);
    for (int32_t si = 0; si < n_steps; ++si) {
        __syncwarp();   // staging / the previous step are done with the slice and the descriptor
        if (lane < kPieces) reinterpret_cast<int4 *>(desc)[lane] = nxt;
        __syncwarp();
        if (si + 1 < n_steps && lane < kPieces) nxt = __ldg(dsrc + (int64_t)(si + 1) * kPieces + lane);
        const LocalStep &s = *desc;
        const int32_t eA = scale_exponent(smax[s.sa]), eB = scale_exponent(smax[s.sb]);
        const int32_t e = sexp[s.sa] + eA + sexp[s.sb] + eB;
        const bool out = s.flags & LFLAG_C_OUT;
        C *Cp = out ? reinterpret_cast<C *>(j.arena) + root_c_off : data + s.c_off;
        const float mx = small_core<T>(s, data + s.a_off, data + s.b_off, Cp, eA, eB);
        if (lane == 0) {
            if (out) {
                j.maxbits[root_node] = __float_as_uint(mx);
                j.exp2[root_node] = e;
            } else {
                smax[s.sc] = __float_as_uint(mx);
                sexp[s.sc] = e;
            }
        }
    }
}

// Block-wide steps of block programs (all operands in shared memory).  Modes:
//   LMODE_ROWS / LMODE_GEMM   row by row (local_rows, N and K <= 16) or register-tiled
//                             (local_mm, tile shape chosen by N)
//   LMODE_REDUCE              few outputs, long K: S threads per output split K, FP64 partial sums,
//                             shuffle / shared-memory reduction; the job's root (the amplitude)
//                             always takes this mode
// Shared-index offsets of a step, tabulated in shared memory when K <= kKTab.
__device__ __forceinline__ void build_ktab(const LocalStep &s, int2 *kt) {
    if (s.K > kKTab) return;
    for (int32_t k = threadIdx.x; k < s.K; k += blockDim.x) {
        int32_t ka, kb;
        lgroup_off2(s, k, ka, kb);
        kt[k] = make_int2(ka, kb);
    }
}

__device__ __forceinline__ int2 kofs(const LocalStep &s, const int2 *kt, int32_t k) {
    if (s.K <= kKTab) return kt[k];
    int32_t ka, kb;
    lgroup_off2(s, k, ka, kb);
    return make_int2(ka, kb);
}

// Block-wide contraction with every operand in shared memory, register-tiled: the block's 256
// threads form TX x TY with RM x RN outputs each, covering a (TY*RM) x (TX*RN) output tile.  The
// shared index runs in chunks of TK: the chunk's A and B entries are gathered through the index
// maps (scaled exactly) into padded, transposed tiles of the scratch area -- so that the
// arithmetic loop reads them without bank conflicts -- and each thread accumulates its outputs in
// registers.  The gather maps consecutive threads along whichever index is contiguous in the
// operand (k or m for A, k or n for B).
template <typename T, int TX, int TY, int RM, int RN, int TK>
__device__ void local_mm(const LocalStep &s, const LocalSmem &L, T sA, T sB, float &mx, char *scratch) {
    using C = cx_t<T>;
    static_assert(TX * TY == kThreads, "256 threads");
    constexpr int TM = TY * RM, TN = TX * RN, PA = TM + 1, PB = TN + 1;
    C *As = reinterpret_cast<C *>(scratch);              // [TK][PA]
    C *Bs = As + TK * PA;                                // [TK][PB]
    int32_t *ra = reinterpret_cast<int32_t *>(Bs + TK * PB);   // [TM] row offsets in A
    int32_t *cb = ra + TM;                                      // [TN] column offsets in B
    int2 *kt = reinterpret_cast<int2 *>(cb + TN);               // [TK] shared-index offsets
    const C *A = reinterpret_cast<const C *>(L.data) + s.a_off;
    const C *B = reinterpret_cast<const C *>(L.data) + s.b_off;
    C *Cp = reinterpret_cast<C *>(L.data) + s.c_off;
    const int32_t M = s.M, N = s.N, K = s.K;
    const bool p2 = s.pow2;
    const bool a_k_inner = s.nk > 0 && s.k_sa[0] == 1;   // k contiguous in A
    const bool b_k_inner = s.nk > 0 && s.k_sb[0] == 1;   // k contiguous in B
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    for (int32_t m0 = 0; m0 < M; m0 += TM)
        for (int32_t n0 = 0; n0 < N; n0 += TN) {
            __syncthreads();   // the previous tile is done with the scratch
            for (int i = tid; i < TM + TN; i += kThreads) {
                if (i < TM) ra[i] = m0 + i < M ? lgroup_off(s.nm, s.m_dim, s.m_str, s.m_lsb, p2, m0 + i) : -1;
                else cb[i - TM] = n0 + i - TM < N ? lgroup_off(s.nn, s.n_dim, s.n_str, s.n_lsb, p2, n0 + i - TM) : -1;
            }
            C acc[RM][RN];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int jj = 0; jj < RN; ++jj) acc[i][jj] = cmake((T)0, (T)0);
            for (int32_t k0 = 0; k0 < K; k0 += TK) {
                if (tid < TK) {
                    int2 o = make_int2(-1, -1);
                    if (k0 + tid < K) lgroup_off2(s, k0 + tid, o.x, o.y);
                    kt[tid] = o;
                }
                __syncthreads();
                for (int e = tid; e < TM * TK; e += kThreads) {
                    const int row = a_k_inner ? e / TK : e % TM, kk = a_k_inner ? e % TK : e / TM;
                    const int2 o = kt[kk];
                    As[kk * PA + row] = (ra[row] >= 0 && o.x >= 0) ? cscale(A[ra[row] + o.x], sA) : cmake((T)0, (T)0);
                }
                for (int e = tid; e < TN * TK; e += kThreads) {
                    const int col = b_k_inner ? e / TK : e % TN, kk = b_k_inner ? e % TK : e / TN;
                    const int2 o = kt[kk];
                    Bs[kk * PB + col] = (cb[col] >= 0 && o.x >= 0) ? cscale(B[o.y + cb[col]], sB) : cmake((T)0, (T)0);
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < TK; ++kk) {
                    C a[RM], b[RN];
#pragma unroll
                    for (int i = 0; i < RM; ++i) a[i] = As[kk * PA + ty + TY * i];
#pragma unroll
                    for (int jj = 0; jj < RN; ++jj) b[jj] = Bs[kk * PB + tx + TX * jj];
#pragma unroll
                    for (int i = 0; i < RM; ++i)
#pragma unroll
                        for (int jj = 0; jj < RN; ++jj) cfma(acc[i][jj], a[i], b[jj]);
                }
                __syncthreads();   // the chunk's tiles and offsets are rewritten next
            }
#pragma unroll
            for (int i = 0; i < RM; ++i) {
                const int32_t m = m0 + ty + TY * i;
                if (m >= M) continue;
#pragma unroll
                for (int jj = 0; jj < RN; ++jj) {
                    const int32_t n = n0 + tx + TX * jj;
                    if (n < N) {
                        Cp[m * N + n] = acc[i][jj];
                        mx = fmaxf(mx, absmax2(acc[i][jj]));
                    }
                }
            }
        }
}

// Block-wide narrow contraction (N <= NT <= 16, K <= 16) with every operand in shared memory.
// NS neighbouring threads share a set of R rows (m, m + blockDim / NS, ...), R = 32 / NT (16 / NT
// for complex128), and each of them holds the R x NT / NS accumulators of its own columns in
// registers; NS > 1 only when the rows alone would leave at least half the block idle.  Per shared
// index a thread reads its rows' A entries and its part of one row of B from a dense, scaled,
// padded copy in the scratch area, and every B entry feeds R complex multiply-adds.  No barrier
// inside the loop.  When k is the contiguous index of A, a thread starts its k loop at m mod K, so
// that the threads of a warp read different banks of A (the padded B rows keep their B reads apart
// too).
template <typename T, int NT, int NS>
__device__ void local_rows(const LocalStep &s, const LocalSmem &L, T sA, T sB, float &mx, char *scratch) {
    using C = cx_t<T>;
    constexpr int R = (sizeof(T) == 4 ? 32 : 16) / NT > 0 ? (sizeof(T) == 4 ? 32 : 16) / NT : 1;
    // NS neighbouring threads share each row: thread g of them holds columns [g NC, g NC + NC)
    constexpr int NC = NT / NS;
    const C *A = reinterpret_cast<const C *>(L.data) + s.a_off;
    const C *B = reinterpret_cast<const C *>(L.data) + s.b_off;
    C *Cp = reinterpret_cast<C *>(L.data) + s.c_off;
    // [K][PB] scaled B; complex64 rows are padded to an even length, so they start on 16 bytes and
    // are read two entries per load
    constexpr bool PAIRS = sizeof(T) == 4 && NC % 2 == 0;
    const int32_t N = s.N, K = s.K, M = s.M, PB = sizeof(T) == 4 ? (N + 2) & ~1 : N + 1;
    C *Bd = reinterpret_cast<C *>(scratch);
    int32_t *kat = reinterpret_cast<int32_t *>(Bd + 16 * (NT + 2));          // [K] offsets in A
    const bool p2 = s.pow2;
    for (int32_t i = threadIdx.x; i < K * N; i += blockDim.x) {
        const int32_t k = i / N, n = i - k * N;
        int32_t ka, kb;
        lgroup_off2(s, k, ka, kb);
        kb += lgroup_off(s.nn, s.n_dim, s.n_str, s.n_lsb, p2, n);
        Bd[k * PB + n] = cscale(B[kb], sB);
        if (n == 0) kat[k] = ka;
    }
    __syncthreads();
    const int32_t g = (int32_t)threadIdx.x % NS, c0 = g * NC;
    if (c0 >= N) return;   // no column of this group (the caller's barrier follows)
    const bool skew = s.nk > 0 && s.k_sa[0] == 1;
    const int32_t step = (int32_t)blockDim.x / NS;
    for (int32_t m0 = (int32_t)threadIdx.x / NS; m0 < M; m0 += step * R) {
        int32_t offA[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int32_t m = m0 + r * step;
            offA[r] = m < M ? lgroup_off(s.nm, s.m_dim, s.m_str, s.m_lsb, p2, m) : -1;
        }
        const int32_t sh = skew ? m0 % K : 0;   // rows of a warp start at different k
        C acc[R][NC];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int n = 0; n < NC; ++n) acc[r][n] = cmake((T)0, (T)0);
#pragma unroll 1
        for (int32_t kk = 0; kk < K; ++kk) {
            int32_t k = kk + sh;
            if (k >= K) k -= K;
            const int32_t ko = kat[k];
            C av[R];
#pragma unroll
            for (int r = 0; r < R; ++r) av[r] = offA[r] >= 0 ? cscale(A[offA[r] + ko], sA) : cmake((T)0, (T)0);
            const C *Bk = Bd + k * PB + c0;
            if constexpr (PAIRS) {
                const float4 *Bk4 = reinterpret_cast<const float4 *>(Bk);
#pragma unroll
                for (int n2 = 0; n2 < NC / 2; ++n2) {
                    if (c0 + 2 * n2 >= N) break;
                    const float4 bb = Bk4[n2];
                    const C b0 = cmake(bb.x, bb.y), b1 = cmake(bb.z, bb.w);
#pragma unroll
                    for (int r = 0; r < R; ++r) cfma(acc[r][2 * n2], av[r], b0);
                    if (c0 + 2 * n2 + 1 < N) {
#pragma unroll
                        for (int r = 0; r < R; ++r) cfma(acc[r][2 * n2 + 1], av[r], b1);
                    }
                }
            } else {
#pragma unroll
                for (int n = 0; n < NC; ++n) {
                    if (c0 + n >= N) break;
                    const C b = Bk[n];
#pragma unroll
                    for (int r = 0; r < R; ++r) cfma(acc[r][n], av[r], b);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (offA[r] < 0) continue;
            C *out = Cp + (m0 + r * step) * N + c0;
#pragma unroll
            for (int n = 0; n < NC; ++n)
                if (c0 + n < N) {
                    out[n] = acc[r][n];
                    mx = fmaxf(mx, absmax2(acc[r][n]));
                }
        }
    }
}

// Narrow block-wide step: NS threads share a row when the rows alone would leave threads idle.
template <typename T, int NT>
__device__ __forceinline__ void local_rows_any(const LocalStep &s, const LocalSmem &L, T sA, T sB, float &mx,
                                               char *scratch) {
    constexpr int R = (sizeof(T) == 4 ? 32 : 16) / NT > 0 ? (sizeof(T) == 4 ? 32 : 16) / NT : 1;
    const int32_t busy = (s.M + R - 1) / R;   // threads with a row when NS = 1
    if constexpr (NT >= 8) {
        if (4 * busy <= (int32_t)blockDim.x) return local_rows<T, NT, 4>(s, L, sA, sB, mx, scratch);
    }
    if (2 * busy <= (int32_t)blockDim.x) return local_rows<T, NT, 2>(s, L, sA, sB, mx, scratch);
    local_rows<T, NT, 1>(s, L, sA, sB, mx, scratch);
}

// Scratch bytes of local_mm: the largest tile set (TK = 8 for complex64, 4 for complex128).
template <typename T> struct LocalMmScratch {
    static constexpr int TK = sizeof(T) == 4 ? 8 : 4;
    static constexpr int bytes = TK * (257 + 65) * (int)sizeof(cx_t<T>) + (256 + 64) * 4 + TK * 8;
};

// Block-wide steps: narrow ones (N, K <= 16) row by row, the rest register-tiled.
template <typename T>
__device__ __forceinline__ void local_mm_dispatch(const LocalStep &s, const LocalSmem &L, T sA, T sB, float &mx,
                                                  char *scratch) {
    constexpr int TK = LocalMmScratch<T>::TK;
    if (s.N <= 16 && s.K <= 16) {
        if (s.N <= 4) local_rows_any<T, 4>(s, L, sA, sB, mx, scratch);
        else if (s.N <= 8) local_rows_any<T, 8>(s, L, sA, sB, mx, scratch);
        else local_rows_any<T, 16>(s, L, sA, sB, mx, scratch);
    } else if (s.N <= 4) local_mm<T, 1, 256, 1, 4, TK>(s, L, sA, sB, mx, scratch);
    else if (s.N <= 8) local_mm<T, 2, 128, 2, 4, TK>(s, L, sA, sB, mx, scratch);
    else if (s.N <= 16) local_mm<T, 4, 64, 4, 4, TK>(s, L, sA, sB, mx, scratch);
    else if (s.N <= 32) local_mm<T, 8, 32, 4, 4, TK>(s, L, sA, sB, mx, scratch);
    else local_mm<T, 16, 16, 4, 4, TK>(s, L, sA, sB, mx, scratch);
}

// REDUCE: threads are grouped S per output (S a power of two, S <= blockDim); each group splits K
// and sums in FP64; groups of up to 32 lanes reduce with shuffles, larger ones through `red64`.
template <typename T>
__device__ __forceinline__ void local_reduce(const LocalStep &s, const LocalSmem &L, T sA, T sB, float &mx,
                                             double2 *red64, const JobPtrs &j, int32_t e_out, const int2 *kt) {
    using C = cx_t<T>;
    const C *A = reinterpret_cast<const C *>(L.data) + s.a_off;
    const C *B = reinterpret_cast<const C *>(L.data) + s.b_off;
    C *Cp = reinterpret_cast<C *>(L.data) + s.c_off;
    const int32_t O = s.M * s.N, K = s.K, N = s.N;
    int32_t S = 1;
    while (S * 2 * O <= (int32_t)blockDim.x && S < K) S *= 2;
    const int32_t groups = blockDim.x / S;
    for (int32_t o0 = 0; o0 < O; o0 += groups) {
        const int32_t o = o0 + threadIdx.x / S, sub = threadIdx.x % S;
        double2 acc = make_double2(0, 0);
        if (o < O) {
            const int32_t m = o / N, n = o - m * N;
            const int32_t offA = lgroup_off(s.nm, s.m_dim, s.m_str, s.m_lsb, s.pow2, m);
            const int32_t offB = lgroup_off(s.nn, s.n_dim, s.n_str, s.n_lsb, s.pow2, n);
            C run = cmake((T)0, (T)0);
            int cnt = 0;
            for (int32_t k = sub; k < K; k += S) {
                const int2 ko = kofs(s, kt, k);
                cfma(run, cscale(A[offA + ko.x], sA), cscale(B[ko.y + offB], sB));
                if (++cnt == 32) {
                    acc.x += (double)run.x;
                    acc.y += (double)run.y;
                    run = cmake((T)0, (T)0);
                    cnt = 0;
                }
            }
            acc.x += (double)run.x;
            acc.y += (double)run.y;
        }
        // reduce the S partials of each output
        const int32_t w = S < 32 ? S : 32;
        for (int off = w / 2; off > 0; off >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, off, w);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, off, w);
        }
        if (S > 32) {
            // one partial per warp, then the first lane of each group sums its warps
            if ((threadIdx.x & 31) == 0) red64[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (sub == 0) {
                acc = make_double2(0, 0);
                for (int32_t q = 0; q < S / 32; ++q) {
                    const double2 p = red64[(threadIdx.x >> 5) + q];
                    acc.x += p.x;
                    acc.y += p.y;
                }
            }
            __syncthreads();
        }
        if (sub == 0 && o < O) {
            if (s.flags & LFLAG_JOB_ROOT) {
                DeviceResult *r = static_cast<DeviceResult *>(j.result);
                r->re = acc.x;
                r->im = acc.y;
                r->exp2 = e_out;
            } else {
                const C v = cmake((T)acc.x, (T)acc.y);
                Cp[o] = v;
                mx = fmaxf(mx, absmax2(v));
            }
        }
    }
}

// Runs local program `prog` of job `j` in the calling block.  `dyn` is the block's dynamic shared
// memory, laid out by local_layout().
template <typename T, bool PROF = false>
__device__ void run_local(int32_t prog, const JobPtrs &j, char *dyn, char *scratch, long long *prof) {
    // scratch: the block's static tile scratch -- dense B / offset tables, then FP64 partials
    double2 *red64 = reinterpret_cast<double2 *>(scratch + kKTab * sizeof(int2));
    using C = cx_t<T>;
    const LocalProg P = j.progs[prog];
    const LocalSmem L = local_layout(dyn, P);
    C *data = reinterpret_cast<C *>(L.data);
    // stage the descriptors and waves, zero the slots, then stage the leaves (one warp per leaf)
    {
        const int nd = P.n_steps * (int)(sizeof(LocalStep) / 16);
        const int4 *src = reinterpret_cast<const int4 *>(j.lsteps + P.first_step);
        int4 *dst = reinterpret_cast<int4 *>(L.desc);
#pragma unroll 4
        for (int i = threadIdx.x; i < nd; i += blockDim.x) dst[i] = __ldcg(src + i);
        const int4 *wsrc = reinterpret_cast<const int4 *>(j.lwaves + P.first_wave);
        int4 *wdst = reinterpret_cast<int4 *>(L.waves);
        const int nw4 = P.n_waves * (int)(sizeof(LocalWave) / 16);
        for (int i = threadIdx.x; i < nw4; i += blockDim.x) wdst[i] = __ldcg(wsrc + i);
    }
    for (int32_t i = threadIdx.x; i < P.n_slots; i += blockDim.x) { L.smax[i] = 0u; L.sexp[i] = 0; }
    __syncthreads();
    stage_inputs<T>(j, j.leafrefs + P.first_leaf, P.n_leaves, threadIdx.x, blockDim.x, data, L.smax, L.sexp);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    long long tp = 0;
    if (PROF && threadIdx.x == 0) tp = clock64();
    // large programs: each wave's inputs are copied asynchronously one wave ahead (the compiler
    // places them clear of the previous wave's operands and results)
    const bool lazy = P.kind == PROG_BIG;
    if (lazy && P.n_waves > 0) {
        const LocalWave W0 = L.waves[0];
        stage_inputs_async<T>(j, j.leafrefs + W0.first_in, W0.n_in, threadIdx.x, blockDim.x, data, L.smax, L.sexp);
        cp_async_commit();
    }
    for (int32_t w = 0; w < P.n_waves; ++w) {
        const LocalWave W = L.waves[w];
        if (lazy) {
            if (w + 1 < P.n_waves) {
                const LocalWave W1 = L.waves[w + 1];
                stage_inputs_async<T>(j, j.leafrefs + W1.first_in, W1.n_in, threadIdx.x, blockDim.x, data, L.smax,
                                      L.sexp);
            }
            cp_async_commit();
            cp_async_wait_prev();   // this wave's inputs have landed (the next wave's may be in flight)
            __syncthreads();
            if (PROF && threadIdx.x == 0) {   // slot 14: waiting for the inputs of large programs
                const long long t1 = clock64();
                atomicAdd((unsigned long long *)(prof + 14), (unsigned long long)(t1 - tp));
                atomicAdd((unsigned long long *)(prof + kProfSlots + 14), 1ull);
            }
        }
        // independent small steps: one warp each
        for (int32_t i = warp; i < W.n_small; i += nw) local_small<T>(L.desc[W.first + i], L);
        // big steps: the whole block, one after the other
        for (int32_t i = 0; i < W.n_big; ++i) {
            const LocalStep &s = L.desc[W.first + W.n_small + i];
            const int32_t eA = scale_exponent(L.smax[s.sa]), eB = scale_exponent(L.smax[s.sb]);
            const T sA = pow2<T>(-eA), sB = pow2<T>(-eB);
            const int32_t e_out = L.sexp[s.sa] + eA + L.sexp[s.sb] + eB;
            float mx = 0.f;
            const int2 *kt = reinterpret_cast<const int2 *>(scratch);
            if (s.mode != LMODE_REDUCE) {
                local_mm_dispatch<T>(s, L, sA, sB, mx, scratch);
            } else {
                build_ktab(s, reinterpret_cast<int2 *>(scratch));
                __syncthreads();
                local_reduce<T>(s, L, sA, sB, mx, red64, j, e_out, kt);
            }
            mx = warp_max(mx);
            if (lane == 0 && mx > 0.f) atomicMax(L.smax + s.sc, __float_as_uint(mx));
            if (threadIdx.x == 0) L.sexp[s.sc] = e_out;
            __syncthreads();   // scratch (dense B / offset table) is reused by the next big step
        }
        __syncthreads();
        if (PROF && threadIdx.x == 0) {
            const long long t1 = clock64();
            // 8: waves of small steps only, 9: waves with block-wide steps, 13: those of large programs
            const int slot = W.n_big ? (P.kind == PROG_BIG ? 13 : 9) : 8;
            atomicAdd((unsigned long long *)(prof + slot), (unsigned long long)(t1 - tp));
            atomicAdd((unsigned long long *)(prof + kProfSlots + slot), 1ull);
            tp = t1;
        }
    }
    if (lazy) cp_async_wait_all();
    // publish the program's result (unless it was the job's amplitude, already written)
    if (!(P.flags & LFLAG_JOB_ROOT)) {
        C *out = reinterpret_cast<C *>(j.arena) + P.root_c_off;
        for (int32_t i = threadIdx.x; i < P.root_size; i += blockDim.x) out[i] = data[P.root_smem_off + i];
        if (threadIdx.x == 0) {
            j.maxbits[P.root_node] = L.smax[P.root_slot];
            j.exp2[P.root_node] = L.sexp[P.root_slot];
        }
    }
    __syncthreads();
}

}  // namespace tn
