/*
 * Oracle contractor -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct complex128 contraction of a tensor network along a given
 * contraction tree.  Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this file's library; the engine never does.  It shares no code with the engine.
 *
 * What it computes: the pairwise contraction of Eq. 2.4 (Section 2.2), generalised to any axis
 * order as the text after Eq. 2.4 allows.  For a step (S, T) the shared legs are the edges that
 * appear in both operands (the intersection in Eq. 2.6); the result carries the remaining legs of
 * S in S's order followed by the remaining legs of T in T's order, and
 *     R[i, k] = sum over all shared multi-indices j of S[i, j] * T[j, k]
 * evaluated element by element with a mixed-radix counter -- no permutation passes, no blocking,
 * no BLAS.  OpenMP splits the output elements across threads; each output element is one
 * sequential sum, so the result does not depend on the thread count.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int rank;
    int *legs;         /* edge id of each axis, axis 0 slowest */
    int64_t size;
    cplx *val;
} otensor;

static int64_t edge_dim(const int64_t *edim, int e) { return edim[e]; }

/* Returns 0 on success, negative on bad input, -100 on allocation failure. */
int oracle_contract(int n_tensors, const int32_t *degree, const int64_t *dims,
                    const double *data, int n_edges, const int32_t *edges,
                    int n_steps, const int32_t *steps,
                    double *out, int64_t out_cap, int32_t *out_legs, int32_t *out_rank)
{
    int n_nodes = n_tensors + n_steps;
    otensor *T = (otensor *)calloc((size_t)n_nodes, sizeof(otensor));
    int64_t *edim = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_edges > 0 ? n_edges : 1));
    int64_t *dim_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_tensors + 1));
    if (!T || !edim || !dim_off) return -100;

    dim_off[0] = 0;
    for (int t = 0; t < n_tensors; ++t) dim_off[t + 1] = dim_off[t] + degree[t];

    /* leaves: legs(v) = edge(v) in axis order (Eq. 2.2) */
    const double *p = data;
    for (int t = 0; t < n_tensors; ++t) {
        T[t].rank = degree[t];
        T[t].legs = (int *)malloc(sizeof(int) * (size_t)(degree[t] > 0 ? degree[t] : 1));
        for (int a = 0; a < degree[t]; ++a) T[t].legs[a] = -1;
        int64_t sz = 1;
        for (int a = 0; a < degree[t]; ++a) sz *= dims[dim_off[t] + a];
        T[t].size = sz;
        T[t].val = (cplx *)malloc(sizeof(cplx) * (size_t)sz);
        for (int64_t i = 0; i < sz; ++i) T[t].val[i] = p[2 * i] + I * p[2 * i + 1];
        p += 2 * sz;
    }
    for (int e = 0; e < n_edges; ++e) {
        int u = edges[4 * e], a = edges[4 * e + 1], v = edges[4 * e + 2], b = edges[4 * e + 3];
        if (u < 0 || u >= n_tensors || a < 0 || a >= degree[u]) return -1;
        T[u].legs[a] = e;
        edim[e] = dims[dim_off[u] + a];
        if (v >= 0) {
            if (v >= n_tensors || b < 0 || b >= degree[v]) return -1;
            if (dims[dim_off[v] + b] != edim[e]) return -2;
            T[v].legs[b] = e;
        }
    }
    for (int t = 0; t < n_tensors; ++t)
        for (int a = 0; a < T[t].rank; ++a)
            if (T[t].legs[a] < 0) return -3;

    for (int s = 0; s < n_steps; ++s) {
        int l = steps[2 * s], r = steps[2 * s + 1], o = n_tensors + s;
        if (l < 0 || r < 0 || l >= o || r >= o || l == r || !T[l].val || !T[r].val) return -4;
        otensor *S = &T[l], *U = &T[r];

        /* row-major strides of both operands */
        int64_t *sS = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S->rank + 1));
        int64_t *sU = (int64_t *)malloc(sizeof(int64_t) * (size_t)(U->rank + 1));
        int64_t acc = 1;
        for (int a = S->rank - 1; a >= 0; --a) { sS[a] = acc; acc *= edge_dim(edim, S->legs[a]); }
        acc = 1;
        for (int a = U->rank - 1; a >= 0; --a) { sU[a] = acc; acc *= edge_dim(edim, U->legs[a]); }

        /* classify legs: output legs (free of S then free of U) and shared legs */
        int maxr = S->rank + U->rank;
        int *olegs = (int *)malloc(sizeof(int) * (size_t)(maxr + 1));
        int64_t *odim = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxr + 1));
        int64_t *ostrS = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxr + 1));
        int64_t *ostrU = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxr + 1));
        int64_t *jdim = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxr + 1));
        int64_t *jstrS = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxr + 1));
        int64_t *jstrU = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxr + 1));
        int orank = 0, jrank = 0;
        for (int a = 0; a < S->rank; ++a) {
            int e = S->legs[a], bpos = -1;
            for (int b = 0; b < U->rank; ++b) if (U->legs[b] == e) bpos = b;
            if (bpos < 0) {
                olegs[orank] = e; odim[orank] = edim[e]; ostrS[orank] = sS[a]; ostrU[orank] = 0;
                ++orank;
            } else {
                jdim[jrank] = edim[e]; jstrS[jrank] = sS[a]; jstrU[jrank] = sU[bpos]; ++jrank;
            }
        }
        for (int b = 0; b < U->rank; ++b) {
            int e = U->legs[b], apos = -1;
            for (int a = 0; a < S->rank; ++a) if (S->legs[a] == e) apos = a;
            if (apos < 0) {
                olegs[orank] = e; odim[orank] = edim[e]; ostrS[orank] = 0; ostrU[orank] = sU[b];
                ++orank;
            }
        }
        int64_t osize = 1, jsize = 1;
        for (int a = 0; a < orank; ++a) osize *= odim[a];
        for (int a = 0; a < jrank; ++a) jsize *= jdim[a];
        cplx *R = (cplx *)malloc(sizeof(cplx) * (size_t)osize);
        if (!R) return -100;

        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < osize; ++i) {
            /* decode output multi-index (last leg fastest) into operand offsets */
            int64_t rem = i, offS = 0, offU = 0;
            for (int a = orank - 1; a >= 0; --a) {
                int64_t d = rem % odim[a];
                rem /= odim[a];
                offS += d * ostrS[a];
                offU += d * ostrU[a];
            }
            cplx sum = 0;
            for (int64_t j = 0; j < jsize; ++j) {
                int64_t rj = j, jS = 0, jU = 0;
                for (int a = jrank - 1; a >= 0; --a) {
                    int64_t d = rj % jdim[a];
                    rj /= jdim[a];
                    jS += d * jstrS[a];
                    jU += d * jstrU[a];
                }
                sum += S->val[offS + jS] * U->val[offU + jU];
            }
            R[i] = sum;
        }

        T[o].rank = orank;
        T[o].legs = (int *)malloc(sizeof(int) * (size_t)(orank > 0 ? orank : 1));
        memcpy(T[o].legs, olegs, sizeof(int) * (size_t)orank);
        T[o].size = osize;
        T[o].val = R;
        free(S->val); S->val = NULL;
        free(U->val); U->val = NULL;
        free(sS); free(sU); free(olegs); free(odim); free(ostrS); free(ostrU);
        free(jdim); free(jstrS); free(jstrU);
    }

    /* the result is the one remaining tensor */
    int root = -1, alive = 0;
    for (int t = 0; t < n_nodes; ++t)
        if (T[t].val) { root = t; ++alive; }
    if (alive != 1) return -5;
    if (T[root].size > out_cap) return -6;
    for (int64_t i = 0; i < T[root].size; ++i) {
        out[2 * i] = creal(T[root].val[i]);
        out[2 * i + 1] = cimag(T[root].val[i]);
    }
    *out_rank = T[root].rank;
    for (int a = 0; a < T[root].rank; ++a) out_legs[a] = T[root].legs[a];

    for (int t = 0; t < n_nodes; ++t) { free(T[t].legs); free(T[t].val); }
    free(T); free(edim); free(dim_off);
    return 0;
}
