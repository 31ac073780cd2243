// The fan-in (reduction) tree over the k partition results (Section 4.4, EvaluateState): the
// pieces that the host planner and the batched GPU evaluator share, so that both make the same
// choices bit for bit.  Leg sets are bitsets over compact edge ids; sizes (Eq. 2.3) and 2^vc
// (Eq. 3.3) are exact integer products saturating at 2^120; the RandomGreedy perturbation of a
// pair's objective is integer arithmetic on a counter-based hash, so no floating-point rounding
// can make the two disagree.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define TN_HD __host__ __device__ __forceinline__
#else
#define TN_HD inline
#endif

namespace tn {
namespace fanin {

using u128 = unsigned __int128;
using i128 = __int128;

constexpr u128 kCap = ((u128)1) << 120;
constexpr int kMaxK = 256;          // partitions the GPU evaluator accepts
constexpr int kMaxWords = 32;       // 2048 compact edge ids

TN_HD int popc64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __popcll(x);
#else
    return __builtin_popcountll(x);
#endif
}
TN_HD int ctz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __ffsll((long long)x) - 1;
#else
    return __builtin_ctzll(x);
#endif
}

// Dimensions of the compact edge ids: unit = every dimension is 2 (a size is 2^popcount).
struct Dims {
    int32_t W;               // 64-bit words per leg set
    int32_t unit;
    const int64_t *dim;      // [64 W] when !unit
};

// Size of the leg set op(a, b) (op 0: a, 1: a XOR b -- Eq. 2.6, 2: a OR b -- E(v) of Eq. 3.3).
TN_HD u128 set_size(const uint64_t *a, const uint64_t *b, int op, const Dims &d, bool &sat) {
    if (d.unit) {
        int e = 0;
        for (int w = 0; w < d.W; ++w) e += popc64(op == 0 ? a[w] : op == 1 ? (a[w] ^ b[w]) : (a[w] | b[w]));
        if (e > 120) {
            sat = true;
            return kCap;
        }
        return ((u128)1) << e;
    }
    u128 p = 1;
    for (int w = 0; w < d.W; ++w) {
        uint64_t x = op == 0 ? a[w] : op == 1 ? (a[w] ^ b[w]) : (a[w] | b[w]);
        while (x) {
            const int bit = ctz64(x);
            x &= x - 1;
            p *= (u128)d.dim[w * 64 + bit];
            if (p > kCap) {
                sat = true;
                p = kCap;
            }
        }
    }
    return p;
}

TN_HD bool intersects(const uint64_t *a, const uint64_t *b, int W) {
    for (int w = 0; w < W; ++w)
        if (a[w] & b[w]) return true;
    return false;
}

TN_HD uint64_t mix64(uint64_t h, uint64_t v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h * 0xff51afd7ed558ccdull;
}

// Counter-based 64-bit hash (the splitmix64 finaliser) of a sample seed and a pair of node ids.
TN_HD uint64_t pair_hash(uint64_t seed, uint32_t i, uint32_t j) {
    uint64_t z = seed ^ (((uint64_t)i << 32) | (uint64_t)j);
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Score of merging nodes i < j in a RandomGreedy sample: the memory-reduction objective of
// Eq. 4.5, |A| + |B| - |A x B|, perturbed in a noisy sample by a uniform factor in [-1/2, 1/2) of
// max(|obj|, 1) (capped at 2^100) that is fixed per pair for the whole sample:
// obj + (u m / 2^21 rounded toward zero), u a 21-bit signed draw.  Exact integer arithmetic.
TN_HD i128 pair_score(i128 obj, bool noisy, uint64_t seed, uint32_t i, uint32_t j) {
    if (!noisy) return obj;
    const int64_t u = (int64_t)(pair_hash(seed, i, j) >> 43) - (int64_t)(1 << 20);   // [-2^20, 2^20)
    i128 m = obj < 0 ? -obj : obj;
    if (m < 1) m = 1;
    const i128 cap = ((i128)1) << 100;
    if (m > cap) m = cap;
    const i128 x = (i128)u * m;                          // |x| <= 2^120
    const i128 q = x < 0 ? -((-x) >> 21) : (x >> 21);
    return obj + q;
}

// Pair order of a Greedy pass: higher score first, then the lexicographically smaller (i, j).
TN_HD bool pair_before(i128 sa, int ia, int ja, i128 sb, int ib, int jb) {
    if (sa != sb) return sa > sb;
    if (ia != ib) return ia < ib;
    return ja < jb;
}

// Counts of a fan-in merge sequence over k roots (local ids 0..k-1, new nodes k, k+1, ...):
// con_dist (Eq. 3.5 with con = con_serial and no communication term), the fan-in's own con and
// mem (Eq. 3.1 over its nodes).  legs: [(2k-1) W] with the roots' sets in the first k rows (the
// rest is overwritten); size: [2k-1]; parent: [2k-1]; cost: [2k-1].
struct Counts {
    u128 con_dist, con, mem;
    bool sat;
};
TN_HD Counts eval_steps(int k, const u128 *part_con, const int16_t *steps, const Dims &d, uint64_t *legs, u128 *size,
                        int16_t *parent, u128 *cost) {
    Counts r;
    r.con_dist = 0;
    r.con = 0;
    r.mem = 0;
    r.sat = false;
    const int W = d.W;
    for (int i = 0; i < 2 * k - 1; ++i) {
        parent[i] = -1;
        cost[i] = 0;
    }
    for (int i = 0; i < k; ++i) size[i] = set_size(legs + (size_t)i * W, legs + (size_t)i * W, 0, d, r.sat);
    for (int s = 0; s < k - 1; ++s) {
        const int a = steps[2 * s], b = steps[2 * s + 1], o = k + s;
        uint64_t *lo = legs + (size_t)o * W;
        const uint64_t *la = legs + (size_t)a * W, *lb = legs + (size_t)b * W;
        cost[o] = set_size(la, lb, 2, d, r.sat);
        for (int w = 0; w < W; ++w) lo[w] = la[w] ^ lb[w];
        size[o] = set_size(lo, lo, 0, d, r.sat);
        parent[a] = parent[b] = (int16_t)o;
        r.con += cost[o];
        const u128 m = size[o] + size[a] + size[b];
        if (m > r.mem) r.mem = m;
    }
    for (int i = 0; i < k; ++i) {
        u128 c = part_con[i];
        for (int v = parent[i]; v >= 0; v = parent[v]) c += cost[v];
        if (c > r.con_dist) r.con_dist = c;
    }
    return r;
}

// Seed of sample s (s >= 1) of a state whose fan-in seed is `seed`.
TN_HD uint64_t sample_seed(uint64_t seed, int s) { return mix64(seed, (uint64_t)s); }

// Best of two evaluated fan-in trees: smaller con_dist, then smaller con (then the earlier one).
TN_HD bool better(const Counts &a, const Counts &b) {
    if (a.con_dist != b.con_dist) return a.con_dist < b.con_dist;
    return a.con < b.con;
}

}  // namespace fanin
}  // namespace tn
