// Slicing on top of partitioning (Section 4.1; named in Section 6 as the way past the memory
// limit).  Fixing the index of a set S of edges splits the contraction into prod_{e in S} n(e)
// independent slices: every slice is the same network with the sliced edges of dimension 1 and
// the tensors touching them cut to one index, contracted along the same tree, and the amplitude
// is the sum of the slices' values.  A slice's memory (Eq. 3.1) and operation count (Eq. 3.2) are
// those of the tree with n(e) = 1 on S; the slices together repeat work that the unsliced tree
// shares, which the counts report as redundant operations.
//
// tn_plan_slice picks S greedily: while the tree's mem exceeds the target, slice the leg of the
// peak-memory step (Eq. 3.1's maximising node and its children) that lowers mem most (ties:
// fewer total operations, then the smaller edge id).  tn_contract_sliced runs the slices as the
// jobs of batches (one compiled plan, leaves replaced per job) and sums them in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tn_internal.hpp"

namespace tn {
namespace {

struct TreeCounts {
    u128 con = 0, mem = 0;
    int32_t peak = -1;      // node maximising |v| + |c1| + |c2|
    bool ovf = false;
};

// Counts of the plan's tree with edge dimensions `dim` (Eq. 3.1, 3.2).
TreeCounts tree_counts(const Net &net, const Plan &plan, const std::vector<int64_t> &dim,
                       std::vector<Legs> *legs_out = nullptr) {
    const int32_t n = net.n, nn = 2 * n - 1;
    std::vector<Legs> legs(nn);
    std::vector<u128> size(nn, 0);
    TreeCounts r;
    for (int32_t t = 0; t < n; ++t) {
        legs[t] = net.legs[t];
        size[t] = legs_size(legs[t], dim, r.ovf);
    }
    for (int32_t s = 0; s < n - 1; ++s) {
        const int32_t a = plan.steps[s][0], b = plan.steps[s][1], o = n + s;
        legs_symdiff(legs[a], legs[b], legs[o]);
        size[o] = legs_size(legs[o], dim, r.ovf);
        r.con += union_size(legs[a], legs[b], dim, r.ovf);
        const u128 m = size[o] + size[a] + size[b];
        if (m > r.mem) {
            r.mem = m;
            r.peak = o;
        }
    }
    if (legs_out) *legs_out = std::move(legs);
    return r;
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

tn_status tn_plan_slice(const tn_net *net, const tn_plan *plan, tn_u128 target_mem, int32_t max_edges,
                        int32_t *edges, int32_t *n_edges, tn_u128 *n_slices, tn_u128 *slice_con,
                        tn_u128 *slice_mem, tn_u128 *total_con) {
    if (!net || !plan || !n_edges || max_edges < 0 || (max_edges > 0 && !edges))
        return fail(TN_EINVAL, "NULL argument or negative max_edges");
    const Net &nt = net->impl;
    const Plan &pl = plan->impl;
    if (pl.n != nt.n || (int32_t)pl.steps.size() != nt.n - 1) return fail(TN_EINVAL, "the plan is not of this net");
    const u128 target = ((u128)target_mem.hi << 64) | (u128)target_mem.lo;
    std::vector<int64_t> dim = nt.edim;
    std::vector<int32_t> chosen;
    u128 slices = 1;
    std::vector<Legs> legs;
    TreeCounts cur = tree_counts(nt, pl, dim, &legs);
    while (cur.mem > target && (int32_t)chosen.size() < max_edges && cur.peak >= 0) {
        const int32_t o = cur.peak, s = o - nt.n;
        Legs cand;
        for (int32_t v : {o, pl.steps[s][0], pl.steps[s][1]}) cand.insert(cand.end(), legs[v].begin(), legs[v].end());
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        int32_t best = -1;
        TreeCounts best_c;
        u128 best_total = 0;
        for (int32_t e : cand) {
            if (dim[e] <= 1) continue;
            const int64_t keep = dim[e];
            dim[e] = 1;
            const TreeCounts c = tree_counts(nt, pl, dim);
            dim[e] = keep;
            const u128 total = c.con * slices * (u128)keep;
            if (best < 0 || c.mem < best_c.mem || (c.mem == best_c.mem && total < best_total)) {
                best = e;
                best_c = c;
                best_total = total;
            }
        }
        if (best < 0) break;   // the peak step has no leg left to slice
        slices *= (u128)dim[best];
        dim[best] = 1;
        chosen.push_back(best);
        cur = tree_counts(nt, pl, dim, &legs);
        if (slices > ((u128)1 << 100)) return fail(TN_EUNSUPPORTED, "more than 2^100 slices");
    }
    std::sort(chosen.begin(), chosen.end());
    for (size_t i = 0; i < chosen.size(); ++i) edges[i] = chosen[i];
    *n_edges = (int32_t)chosen.size();
    if (n_slices) *n_slices = to_abi(slices);
    if (slice_con) *slice_con = to_abi(cur.con);
    if (slice_mem) *slice_mem = to_abi(cur.mem);
    if (total_con) *total_con = to_abi(cur.con * slices);
    return TN_OK;
}

tn_status tn_contract_sliced(tn_ctx *ctx, const tn_net *net, const tn_plan *plan, tn_precision prec,
                             int32_t n_sliced, const int32_t *sliced, int32_t max_jobs, int64_t first_slice,
                             int64_t slice_count, double out_amp[2], int32_t *out_exp2, int64_t *n_slices_out) {
    if (!ctx || !net || !plan || !out_amp || !out_exp2 || n_sliced < 0 || (n_sliced > 0 && !sliced) || max_jobs < 1)
        return fail(TN_EINVAL, "NULL argument, negative n_sliced or max_jobs < 1");
    const Net &nt = net->impl;
    const Plan &pl = plan->impl;
    if (pl.n != nt.n || (int32_t)pl.steps.size() != nt.n - 1) return fail(TN_EINVAL, "the plan is not of this net");
    std::vector<char> is_sliced(nt.n_edges, 0);
    std::vector<int64_t> radix;
    int64_t n_slices = 1;
    for (int32_t i = 0; i < n_sliced; ++i) {
        const int32_t e = sliced[i];
        if (e < 0 || e >= nt.n_edges || is_sliced[e]) return fail(TN_EINVAL, "bad or repeated sliced edge");
        if (nt.edges[e].v < 0) return fail(TN_EINVAL, "an open leg cannot be sliced");
        is_sliced[e] = 1;
        radix.push_back(nt.edim[e]);
        if (n_slices > ((int64_t)1 << 40) / nt.edim[e]) return fail(TN_EUNSUPPORTED, "more than 2^40 slices");
        n_slices *= nt.edim[e];
    }
    // the sliced structure: sliced axes of dimension 1
    std::vector<int32_t> degree(nt.degree);
    std::vector<int64_t> dims(nt.dims);
    std::vector<int32_t> touched;   // tensors with a sliced axis
    for (int32_t t = 0; t < nt.n; ++t) {
        bool any = false;
        for (int32_t a = 0; a < nt.degree[t]; ++a)
            if (is_sliced[nt.axis_edge[t][a]]) {
                dims[nt.dim_off[t] + a] = 1;
                any = true;
            }
        if (any) touched.push_back(t);
    }
    // slice index of a sliced edge: its position in `sliced` (mixed radix, first edge slowest)
    std::vector<int32_t> slot(nt.n_edges, -1);
    for (int32_t i = 0; i < n_sliced; ++i) slot[sliced[i]] = i;
    // element offsets of the sliced tensors' entries, per slice: entries of slice sigma of tensor
    // t are the entries whose sliced axes hold sigma's indices, in row-major order
    auto slice_of = [&](int32_t t, const std::vector<int64_t> &sigma, std::vector<double> &dst) {
        const int32_t d = nt.degree[t];
        std::vector<int64_t> stride(d, 1), idx(d, 0), full(d);
        for (int32_t a = d - 1; a >= 0; --a) {
            full[a] = nt.dims[nt.dim_off[t] + a];
            if (a + 1 < d) stride[a] = stride[a + 1] * full[a + 1];
        }
        int64_t base = 0, count = 1;
        std::vector<int32_t> free_axes;
        for (int32_t a = 0; a < d; ++a) {
            const int32_t e = nt.axis_edge[t][a];
            if (is_sliced[e]) base += sigma[slot[e]] * stride[a];
            else { free_axes.push_back(a); count *= full[a]; }
        }
        const double *src = nt.data.data() + 2 * nt.data_off[t];
        for (int64_t q = 0; q < count; ++q) {
            int64_t rem = q, off = base;
            for (int32_t i = (int32_t)free_axes.size() - 1; i >= 0; --i) {
                const int32_t a = free_axes[i];
                off += (rem % full[a]) * stride[a];
                rem /= full[a];
            }
            dst.push_back(src[2 * off]);
            dst.push_back(src[2 * off + 1]);
        }
    };
    // the structure net holds slice 0's entries; the plan is the same tree on it
    std::vector<double> data;
    data.reserve(nt.data.size());
    std::vector<int64_t> sigma(n_sliced, 0);
    for (int32_t t = 0; t < nt.n; ++t) {
        if (std::binary_search(touched.begin(), touched.end(), t)) slice_of(t, sigma, data);
        else data.insert(data.end(), nt.data.begin() + 2 * nt.data_off[t], nt.data.begin() + 2 * nt.data_off[t + 1]);
    }
    tn_net *snet = nullptr;
    tn_status s = tn_build(nt.n, degree.data(), dims.data(), data.data(), nt.n_edges, nt.edges.data(), &snet);
    if (s != TN_OK) return s;
    std::vector<int32_t> steps(2 * (size_t)(nt.n - 1));
    for (int32_t i = 0; i + 1 < nt.n; ++i) {
        steps[2 * i] = pl.steps[i][0];
        steps[2 * i + 1] = pl.steps[i][1];
    }
    tn_plan *splan = nullptr;
    s = tn_plan_import(snet, pl.k, pl.part.data(), nt.n - 1, steps.data(), &splan);
    if (s != TN_OK) { tn_net_free(snet); return s; }
    if (first_slice < 0 || first_slice >= n_slices || slice_count < 0)
        return fail(TN_EINVAL, "first_slice outside [0, slices) or negative slice_count");
    const int64_t end = slice_count == 0 ? n_slices : std::min<int64_t>(n_slices, first_slice + slice_count);
    const int64_t per = std::min<int64_t>(end - first_slice, max_jobs);
    std::vector<const tn_net *> nets(per, snet);
    std::vector<const tn_plan *> plans(per, splan);
    tn_batch *b = nullptr;
    s = tn_batch_create(ctx, (int32_t)per, nets.data(), plans.data(), prec, &b);
    if (s != TN_OK) { tn_plan_free(splan); tn_net_free(snet); return s; }
    // FP64 sum of the slices' values m 2^e: the running sum is kept as (double, exponent)
    double acc_re = 0, acc_im = 0;
    int32_t acc_e = INT32_MIN;
    auto add = [&](double re, double im, int32_t e) {
        if (re == 0 && im == 0) return;
        if (acc_e == INT32_MIN) { acc_re = re; acc_im = im; acc_e = e; return; }
        if (e > acc_e) {
            acc_re = std::ldexp(acc_re, acc_e - e);
            acc_im = std::ldexp(acc_im, acc_e - e);
            acc_e = e;
        }
        acc_re += std::ldexp(re, e - acc_e);
        acc_im += std::ldexp(im, e - acc_e);
    };
    std::vector<double> amps(2 * per);
    std::vector<int32_t> ex(per), st(per);
    std::vector<int32_t> jobs, tens;
    std::vector<double> vals;
    for (int64_t first = first_slice; first < end && s == TN_OK; first += per) {
        const int64_t cnt = std::min<int64_t>(per, end - first);
        jobs.clear();
        tens.clear();
        vals.clear();
        for (int64_t j = 0; j < per; ++j) {
            // slice number first + j (jobs past the last slice repeat slice 0 and are not summed)
            int64_t rem = first + j < end ? first + j : first;
            for (int32_t i = n_sliced - 1; i >= 0; --i) {
                sigma[i] = rem % radix[i];
                rem /= radix[i];
            }
            for (int32_t t : touched) {
                jobs.push_back((int32_t)j);
                tens.push_back(t);
                slice_of(t, sigma, vals);
            }
        }
        if (!jobs.empty()) s = tn_batch_set_tensors(b, (int32_t)jobs.size(), jobs.data(), tens.data(), vals.data());
        if (s == TN_OK) s = tn_batch_run(b, nullptr);
        if (s == TN_OK) s = tn_batch_results(b, amps.data(), ex.data(), st.data());
        for (int64_t j = 0; s == TN_OK && j < cnt; ++j) {
            if (st[j] != 0) s = fail(TN_ETIMEOUT, "a slice's device wait gave up");
            else add(amps[2 * j], amps[2 * j + 1], ex[j]);
        }
    }
    tn_batch_free(b);
    tn_plan_free(splan);
    tn_net_free(snet);
    if (s != TN_OK) return s;
    // normalise the mantissa into [0.5, 1) in magnitude
    int32_t e2 = acc_e == INT32_MIN ? 0 : acc_e;
    const double mx = std::max(std::fabs(acc_re), std::fabs(acc_im));
    if (mx > 0) {
        int sh = 0;
        std::frexp(mx, &sh);
        acc_re = std::ldexp(acc_re, -sh);
        acc_im = std::ldexp(acc_im, -sh);
        e2 += sh;
    }
    out_amp[0] = acc_re;
    out_amp[1] = acc_im;
    *out_exp2 = e2;
    if (n_slices_out) *n_slices_out = n_slices;
    return TN_OK;
}

}  // extern "C"
