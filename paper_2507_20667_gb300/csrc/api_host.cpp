// Host-side entry points of the C ABI: networks, plans, diagnostics.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <string>

#include "tn_internal.hpp"

namespace tn {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

tn_status fail(tn_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

uint64_t next_uid() {
    static std::atomic<uint64_t> counter{1};
    return counter.fetch_add(1);
}

}  // namespace tn

using namespace tn;

extern "C" {

const char *tn_status_str(tn_status s) {
    switch (s) {
        case TN_OK: return "ok";
        case TN_EINVAL: return "invalid argument";
        case TN_ENOMEM: return "out of memory";
        case TN_EBUDGET: return "device memory budget exceeded";
        case TN_ECUDA: return "CUDA error";
        case TN_ETIMEOUT: return "device wait timed out";
        case TN_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *tn_last_error(void) { return g_last_error.c_str(); }

const char *tn_version(void) { return "tnsa-gb300 0.1 (sm_103a)"; }

tn_status tn_build(int32_t n_tensors, const int32_t *degree, const int64_t *dims,
                   const double *data, int32_t n_edges, const tn_edge *edges, tn_net **out) {
    if (!out) return fail(TN_EINVAL, "out is NULL");
    if (n_tensors < 1) return fail(TN_EINVAL, "n_tensors must be >= 1");
    if (!degree || (n_edges > 0 && !edges) || n_edges < 0)
        return fail(TN_EINVAL, "NULL degree or edges");
    tn_net *h = new (std::nothrow) tn_net;
    if (!h) return fail(TN_ENOMEM, "allocating the network");
    try {
        Net &net = h->impl;
        net.n = n_tensors;
        net.n_edges = n_edges;
        net.degree.assign(degree, degree + n_tensors);
        net.dim_off.assign(n_tensors + 1, 0);
        net.data_off.assign(n_tensors + 1, 0);
        for (int32_t t = 0; t < n_tensors; ++t) {
            if (degree[t] < 0) { delete h; return fail(TN_EINVAL, "negative degree"); }
            net.dim_off[t + 1] = net.dim_off[t] + degree[t];
        }
        const int64_t nd = net.dim_off[n_tensors];
        if (nd > 0 && !dims) { delete h; return fail(TN_EINVAL, "NULL dims"); }
        net.dims.assign(dims, dims + nd);
        for (int32_t t = 0; t < n_tensors; ++t) {
            int64_t sz = 1;
            for (int64_t a = net.dim_off[t]; a < net.dim_off[t + 1]; ++a) {
                if (net.dims[a] < 1) { delete h; return fail(TN_EINVAL, "dims must be >= 1"); }
                if (sz > (((int64_t)1) << 62) / net.dims[a]) {
                    delete h;
                    return fail(TN_EINVAL, "tensor element count above 2^62");
                }
                sz *= net.dims[a];
            }
            net.data_off[t + 1] = net.data_off[t] + sz;
            if (net.data_off[t + 1] > (((int64_t)1) << 62)) {
                delete h;
                return fail(TN_EINVAL, "total element count above 2^62");
            }
        }
        if (!data) { delete h; return fail(TN_EINVAL, "NULL data"); }
        if (!entries_in_range(data, 2 * (size_t)net.data_off[n_tensors])) {
            delete h;
            return fail(TN_EINVAL, "tensor entries must be finite and below 2^127 in magnitude");
        }
        net.data.assign(data, data + 2 * net.data_off[n_tensors]);
        net.edges.assign(edges, edges + n_edges);
        net.edim.assign(n_edges, 0);
        net.axis_edge.resize(n_tensors);
        for (int32_t t = 0; t < n_tensors; ++t) net.axis_edge[t].assign(degree[t], -1);
        for (int32_t e = 0; e < n_edges; ++e) {
            const tn_edge &x = edges[e];
            if (x.u < 0 || x.u >= n_tensors || x.a < 0 || x.a >= degree[x.u]) {
                delete h;
                return fail(TN_EINVAL, "edge " + std::to_string(e) + ": (u, a) out of range");
            }
            if (x.v < -1 || x.v >= n_tensors) {
                delete h;
                return fail(TN_EINVAL, "edge " + std::to_string(e) + ": v out of range");
            }
            if (x.v == x.u) {
                delete h;
                return fail(TN_EINVAL, "edge " + std::to_string(e) + ": self-loop");
            }
            if (net.axis_edge[x.u][x.a] >= 0) {
                delete h;
                return fail(TN_EINVAL, "edge " + std::to_string(e) + ": axis (u, a) named twice");
            }
            net.axis_edge[x.u][x.a] = e;
            net.edim[e] = net.dims[net.dim_off[x.u] + x.a];
            if (x.v >= 0) {
                if (x.b < 0 || x.b >= degree[x.v]) {
                    delete h;
                    return fail(TN_EINVAL, "edge " + std::to_string(e) + ": (v, b) out of range");
                }
                if (net.axis_edge[x.v][x.b] >= 0) {
                    delete h;
                    return fail(TN_EINVAL, "edge " + std::to_string(e) + ": axis (v, b) named twice");
                }
                if (net.dims[net.dim_off[x.v] + x.b] != net.edim[e]) {
                    delete h;
                    return fail(TN_EINVAL, "edge " + std::to_string(e) + ": n_{u,a} != n_{v,b}");
                }
                net.axis_edge[x.v][x.b] = e;
            } else {
                net.closed = false;
            }
        }
        net.legs.resize(n_tensors);
        for (int32_t t = 0; t < n_tensors; ++t) {
            for (int32_t a = 0; a < degree[t]; ++a)
                if (net.axis_edge[t][a] < 0) {
                    delete h;
                    return fail(TN_EINVAL, "tensor " + std::to_string(t) + " axis " +
                                               std::to_string(a) + " is not named by any edge");
                }
            net.legs[t] = net.axis_edge[t];
            std::sort(net.legs[t].begin(), net.legs[t].end());
        }
    } catch (const std::bad_alloc &) {
        delete h;
        return fail(TN_ENOMEM, "allocating the network");
    }
    h->impl.uid = next_uid();
    *out = h;
    return TN_OK;
}

tn_status tn_net_set_tensor(tn_net *h, int32_t t, const double *data) {
    if (!h || !data) return fail(TN_EINVAL, "NULL argument");
    Net &net = h->impl;
    if (t < 0 || t >= net.n) return fail(TN_EINVAL, "tensor index out of range");
    if (!entries_in_range(data, 2 * (size_t)(net.data_off[t + 1] - net.data_off[t])))
        return fail(TN_EINVAL, "tensor entries must be finite and below 2^127 in magnitude");
    std::memcpy(&net.data[2 * net.data_off[t]], data,
                sizeof(double) * 2 * (size_t)(net.data_off[t + 1] - net.data_off[t]));
    net.version++;
    return TN_OK;
}

tn_status tn_net_info(const tn_net *h, int32_t *n_tensors, int32_t *n_edges, int32_t *closed) {
    if (!h) return fail(TN_EINVAL, "NULL net");
    if (n_tensors) *n_tensors = h->impl.n;
    if (n_edges) *n_edges = h->impl.n_edges;
    if (closed) *closed = h->impl.closed ? 1 : 0;
    return TN_OK;
}

void tn_net_free(tn_net *net) { delete net; }

void tn_plan_opts_default(tn_plan_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->k = 1;
    o->mode = TN_SA_DIRECTED;
    o->T0 = 0.1;
    o->Tf = 0.001;
    o->steps_per_temp = 8;
    o->threads = 1;
    o->time_limit_s = 0;
    o->iterations = 200;
    o->restart_threshold = 50;
    o->fanin_samples = 32;
    o->seed = 0;
    o->initial = TN_INIT_BFS;
    o->pad0 = 0;
    o->initial_part = nullptr;
    o->position = nullptr;
    o->fanin_device = -1;
    o->pad1 = 0;
}

tn_status tn_plan_create(const tn_net *net, const tn_plan_opts *opts, tn_plan **out) {
    if (!net || !opts || !out) return fail(TN_EINVAL, "NULL argument");
    tn_plan *p = new (std::nothrow) tn_plan;
    if (!p) return fail(TN_ENOMEM, "allocating the plan");
    tn_status s;
    try {
        s = plan_run(net->impl, *opts, p->impl);
    } catch (const std::bad_alloc &) {
        s = fail(TN_ENOMEM, "planner allocation");
    }
    if (s != TN_OK) { delete p; return s; }
    p->impl.uid = next_uid();
    *out = p;
    return TN_OK;
}

tn_status tn_plan_import(const tn_net *net, int32_t k, const int32_t *part, int32_t n_steps,
                         const int32_t *steps, tn_plan **out) {
    if (!net || !out || (n_steps > 0 && !steps)) return fail(TN_EINVAL, "NULL argument");
    const Net &nt = net->impl;
    if (k < 1 || k > nt.n) return fail(TN_EINVAL, "k must satisfy 1 <= k <= n_tensors");
    if (!part && k != 1) return fail(TN_EINVAL, "part may be NULL only when k = 1");
    if (n_steps != nt.n - 1) return fail(TN_EINVAL, "n_steps must be n_tensors - 1");
    tn_plan *p = new (std::nothrow) tn_plan;
    if (!p) return fail(TN_ENOMEM, "allocating the plan");
    Plan &pl = p->impl;
    pl.n = nt.n;
    pl.k = k;
    pl.part.assign(nt.n, 0);
    if (part) pl.part.assign(part, part + nt.n);
    pl.steps.resize(n_steps);
    for (int32_t s = 0; s < n_steps; ++s)
        pl.steps[s] = {steps[2 * s], steps[2 * s + 1], nt.n + s};
    tn_status s = plan_finalize(nt, pl);
    if (s != TN_OK) { delete p; return s; }
    pl.init_con_dist = pl.con_dist;
    pl.uid = next_uid();
    *out = p;
    return TN_OK;
}

tn_status tn_plan_counts(const tn_plan *p, tn_u128 *total_ops, tn_u128 *crit_ops,
                         tn_u128 *mem_elems) {
    if (!p) return fail(TN_EINVAL, "NULL plan");
    if (total_ops) *total_ops = to_abi(p->impl.con_serial);
    if (crit_ops) *crit_ops = to_abi(p->impl.con_dist);
    if (mem_elems) *mem_elems = to_abi(p->impl.mem);
    return TN_OK;
}

tn_status tn_plan_eval_states(const tn_net *net, int32_t k, int32_t fanin_samples, int32_t device,
                              int32_t n_states, const int32_t *parts, tn_u128 *con_serial,
                              tn_u128 *con_dist, tn_u128 *mem, int32_t *saturated) {
    if (!net) return fail(TN_EINVAL, "NULL net");
    std::vector<StateCounts> out;
    tn_status s = eval_states(net->impl, k, fanin_samples, device, n_states, parts, out);
    if (s != TN_OK) return s;
    for (int32_t q = 0; q < n_states; ++q) {
        if (con_serial) con_serial[q] = to_abi(out[q].con_serial);
        if (con_dist) con_dist[q] = to_abi(out[q].con_dist);
        if (mem) mem[q] = to_abi(out[q].mem);
        if (saturated) saturated[q] = out[q].saturated ? 1 : 0;
    }
    return TN_OK;
}

tn_status tn_plan_get_info(const tn_plan *p, tn_plan_info *info) {
    if (!p || !info) return fail(TN_EINVAL, "NULL argument");
    const Plan &pl = p->impl;
    info->con_serial = to_abi(pl.con_serial);
    info->con_dist = to_abi(pl.con_dist);
    info->con_par = to_abi(pl.con_par);
    info->mem = to_abi(pl.mem);
    info->initial_con_dist = to_abi(pl.init_con_dist);
    info->k = pl.k;
    info->n_steps = (int32_t)pl.steps.size();
    info->sa_iterations = pl.sa_iterations;
    info->sa_accepted = pl.sa_accepted;
    info->sa_restarts = pl.sa_restarts;
    info->plan_seconds = pl.plan_seconds;
    return TN_OK;
}

tn_status tn_plan_export(const tn_plan *p, int32_t *part_of_tensor, int32_t *steps,
                         int32_t *step_part, int32_t *n_steps) {
    if (!p) return fail(TN_EINVAL, "NULL plan");
    const Plan &pl = p->impl;
    if (part_of_tensor) std::copy(pl.part.begin(), pl.part.end(), part_of_tensor);
    if (steps)
        for (size_t s = 0; s < pl.steps.size(); ++s)
            for (int c = 0; c < 3; ++c) steps[3 * s + c] = pl.steps[s][c];
    if (step_part) std::copy(pl.step_part.begin(), pl.step_part.end(), step_part);
    if (n_steps) *n_steps = (int32_t)pl.steps.size();
    return TN_OK;
}

void tn_plan_free(tn_plan *p) { delete p; }

}  // extern "C"
