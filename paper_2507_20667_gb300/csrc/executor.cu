// Program compiler and runtime: turns (network, plan, precision) into a device program -- per-step
// layouts and fused index maps, kernel classes, a static memory plan for every intermediate --
// and runs it as one CUDA graph on the context's stream.
#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "tn_internal.hpp"

using namespace tn;

struct tn_ctx {
    int32_t device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    tn_program *cached = nullptr;      // program reused by tn_contract, keyed by the unique ids
    uint64_t cached_net = 0, cached_plan = 0;   // of the net and plan (never by address)
    tn_precision cached_prec = TN_C64;
};

struct tn_program {
    tn_ctx *ctx = nullptr;
    const tn_net *net = nullptr;
    uint64_t uploaded_version = ~0ull;
    tn_precision prec = TN_C64;
    bool c128 = false;
    int32_t n = 0, n_nodes = 0;
    int32_t elem = 8;
    // device memory (one allocation, carved)
    void *d_block = nullptr;
    double *d_leaf64 = nullptr;
    void *d_leaf = nullptr;
    int64_t *d_leaf_off = nullptr;
    char *d_arena = nullptr;
    StepDesc *d_desc = nullptr;
    int32_t *d_exp2 = nullptr;
    uint32_t *d_maxbits = nullptr;
    double *d_partials = nullptr;
    DeviceResult *d_res = nullptr;
    size_t footprint = 0, arena_bytes = 0;
    // host
    std::vector<StepDesc> desc;
    std::vector<std::array<int64_t, 3>> where;   // operand locations: leaf index (< 0: -1 - t) or
                                                 // arena byte offset (>= 0); C of the root: unused
    std::vector<int64_t> leaf_off;
    double *h_pinned = nullptr;
    DeviceResult *h_res = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    tn_run_info info{};
    bool ran = false;
};

namespace {

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess)                                                             \
            return fail(TN_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));     \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

int32_t ilog2(int64_t x) {
    int32_t r = 0;
    while ((((int64_t)1) << r) < x) ++r;
    return r;
}

// Build a fused group list from legs listed outermost -> innermost with their strides.
bool make_groups(const std::vector<int64_t> &dim, const std::vector<int64_t> &sa,
                 const std::vector<int64_t> &sb, bool two, Groups &g) {
    std::memset(&g, 0, sizeof(g));
    int32_t n = 0;
    for (int32_t i = (int32_t)dim.size() - 1; i >= 0; --i) {   // innermost first
        if (dim[i] == 1) continue;
        if (n > 0 && sa[i] == g.sa[n - 1] * g.dim[n - 1] &&
            (!two || sb[i] == g.sb[n - 1] * g.dim[n - 1])) {
            g.dim[n - 1] *= dim[i];
            continue;
        }
        if (n == kMaxGroups) return false;
        g.dim[n] = dim[i];
        g.sa[n] = sa[i];
        g.sb[n] = two ? sb[i] : 0;
        ++n;
    }
    g.n = n;
    g.pow2 = 1;
    int32_t bit = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (!is_pow2(g.dim[i])) g.pow2 = 0;
        g.lsb[i] = bit;
        g.mask[i] = g.dim[i] - 1;
        bit += ilog2(g.dim[i]);
    }
    return true;
}

struct FreeList {
    std::map<size_t, size_t> blocks;   // offset -> size
    size_t top = 0, high = 0;
    size_t alloc(size_t sz) {
        for (auto it = blocks.begin(); it != blocks.end(); ++it)
            if (it->second >= sz) {
                size_t off = it->first, rest = it->second - sz;
                blocks.erase(it);
                if (rest) blocks[off + sz] = rest;
                return off;
            }
        size_t off = top;
        top += sz;
        high = std::max(high, top);
        return off;
    }
    void release(size_t off, size_t sz) {
        auto it = blocks.emplace(off, sz).first;
        auto nx = std::next(it);
        if (nx != blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            blocks.erase(nx);
        }
        if (it != blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                blocks.erase(it);
                it = pv;
            }
        }
        if (it->first + it->second == top) {   // give the tail back
            top = it->first;
            blocks.erase(it);
        }
    }
};

tn_status compile(tn_program *p, const Net &net, const Plan &plan) {
    const int32_t n = net.n, nn = 2 * n - 1;
    p->n = n;
    p->n_nodes = nn;
    std::vector<std::vector<int32_t>> layout(nn);
    std::vector<int64_t> size(nn, 1);
    for (int32_t t = 0; t < n; ++t) {
        layout[t] = net.axis_edge[t];
        size[t] = net.data_off[t + 1] - net.data_off[t];
    }
    p->leaf_off.assign(net.data_off.begin(), net.data_off.end());
    const size_t esz = (size_t)p->elem;
    std::vector<size_t> arena_off(nn, (size_t)-1);
    FreeList fl;
    p->desc.assign(n - 1, StepDesc{});
    double flops = 0, bytes = 0;
    int32_t counts[4] = {0, 0, 0, 0};
    for (int32_t s = 0; s < n - 1; ++s) {
        const int32_t l = plan.steps[s][0], r = plan.steps[s][1], o = n + s;
        const bool root = (s == n - 2);
        const int32_t a = size[l] >= size[r] ? l : r, b = (a == l) ? r : l;
        const auto &LA = layout[a], &LB = layout[b];
        auto in = [](const std::vector<int32_t> &v, int32_t e) {
            return std::find(v.begin(), v.end(), e) != v.end();
        };
        std::vector<int64_t> strA(LA.size()), strB(LB.size());
        int64_t acc = 1;
        for (int32_t i = (int32_t)LA.size() - 1; i >= 0; --i) { strA[i] = acc; acc *= net.edim[LA[i]]; }
        acc = 1;
        for (int32_t i = (int32_t)LB.size() - 1; i >= 0; --i) { strB[i] = acc; acc *= net.edim[LB[i]]; }
        std::vector<int64_t> md, ms, nd, ns, kd, ksa, ksb, none;
        std::vector<int32_t> out;
        int64_t M = 1, N = 1, K = 1;
        for (size_t i = 0; i < LA.size(); ++i) {
            int32_t e = LA[i];
            auto jt = std::find(LB.begin(), LB.end(), e);
            if (jt == LB.end()) {
                md.push_back(net.edim[e]); ms.push_back(strA[i]); out.push_back(e); M *= net.edim[e];
            } else {
                kd.push_back(net.edim[e]); ksa.push_back(strA[i]); ksb.push_back(strB[jt - LB.begin()]);
                K *= net.edim[e];
            }
        }
        for (size_t i = 0; i < LB.size(); ++i) {
            int32_t e = LB[i];
            if (!in(LA, e)) {
                nd.push_back(net.edim[e]); ns.push_back(strB[i]); out.push_back(e); N *= net.edim[e];
            }
        }
        layout[o] = out;
        size[o] = M * N;
        StepDesc &d = p->desc[s];
        d.M = M;
        d.N = N;
        d.K = K;
        d.node_a = a;
        d.node_b = b;
        d.node_c = o;
        d.is_root = root ? 1 : 0;
        if (!make_groups(md, ms, none, false, d.m) || !make_groups(nd, ns, none, false, d.n) ||
            !make_groups(kd, ksa, ksb, true, d.k))
            return fail(TN_EUNSUPPORTED, "step " + std::to_string(s) + " has more than 32 leg groups");
        if (root) {
            if (M * N != 1) return fail(TN_EUNSUPPORTED, "open networks are not supported by tn_contract");
            d.kind = STEP_DOT;
        } else if (M * N <= 16 && K > 64) {
            d.kind = STEP_DOT;
        } else if (N <= 16 && K <= 64 && K * N <= 1024) {
            d.kind = STEP_ROWS;
        } else {
            d.kind = STEP_TILE;
        }
        counts[d.kind]++;
        flops += 8.0 * (double)M * (double)N * (double)K;
        bytes += (double)(size[a] + size[b] + size[o]) * (double)esz;
        // memory plan: allocate the output, then release the inputs
        if (!root) arena_off[o] = fl.alloc(align_up((size_t)size[o] * esz, 256));
        for (int32_t x : {l, r})
            if (x >= n) fl.release(arena_off[x], align_up((size_t)size[x] * esz, 256));
    }
    p->arena_bytes = std::max(fl.high, (size_t)256);
    p->info.n_gather = counts[STEP_ROWS];
    p->info.n_tile = counts[STEP_TILE];
    p->info.n_dot = counts[STEP_DOT];
    p->info.n_tc = counts[STEP_TC];
    p->info.flops = flops;
    p->info.bytes = bytes;
    p->info.arena_bytes = p->arena_bytes;
    // operand locations, resolved to device addresses once the arena exists
    p->where.resize(n - 1);
    for (int32_t s = 0; s < n - 1; ++s) {
        const StepDesc &d = p->desc[s];
        auto loc = [&](int32_t v) -> int64_t { return v < n ? -1 - (int64_t)v : (int64_t)arena_off[v]; };
        p->where[s] = {loc(d.node_a), loc(d.node_b), d.is_root ? 0 : loc(d.node_c)};
    }
    return TN_OK;
}

tn_status upload_leaves(tn_program *p) {
    const Net &net = p->net->impl;
    const size_t bytes = sizeof(double) * net.data.size();
    if (bytes) {
        std::memcpy(p->h_pinned, net.data.data(), bytes);
        CK(cudaMemcpyAsync(p->d_leaf64, p->h_pinned, bytes, cudaMemcpyHostToDevice, p->ctx->stream));
    }
    p->uploaded_version = net.version;
    return TN_OK;
}

tn_status record_graph(tn_program *p) {
    cudaStream_t st = p->ctx->stream;
    ScaleState sc{p->d_exp2, p->d_maxbits};
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int32_t launches = 0;
    cudaError_t err = cudaMemsetAsync(p->d_maxbits, 0, sizeof(uint32_t) * p->n_nodes, st);
    if (err == cudaSuccess)
        err = launch_leaf_convert(p->c128, p->d_leaf64, p->d_leaf, p->d_leaf_off, p->n, sc, st);
    launches += 1;
    for (size_t s = 0; err == cudaSuccess && s < p->desc.size(); ++s)
        err = launch_step(p->c128, p->d_desc + s, p->desc[s], sc, p->d_partials,
                          dot_partial_blocks(), p->d_res, st, &launches);
    if (err == cudaSuccess && p->n == 1) {
        err = launch_finish_leaf(p->c128, p->d_leaf, 0, sc, p->d_res, st);
        launches += 1;
    }
    cudaGraph_t g = nullptr;
    cudaError_t err2 = cudaStreamEndCapture(st, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(TN_ECUDA, std::string("recording the program: ") + cudaGetErrorString(err));
    }
    if (err2 != cudaSuccess) return fail(TN_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(err2));
    err = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return fail(TN_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(err));
    p->info.launches = launches;
    return TN_OK;
}

void program_destroy(tn_program *p) {
    if (!p) return;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->d_block) cudaFree(p->d_block);
    if (p->h_pinned) cudaFreeHost(p->h_pinned);
    if (p->h_res) cudaFreeHost(p->h_res);
    delete p;
}

}  // namespace

extern "C" {

tn_status tn_ctx_create(int32_t device, void *cuda_stream, size_t hbm_budget_bytes, tn_ctx **out) {
    if (!out) return fail(TN_EINVAL, "out is NULL");
    int count = 0;
    CK(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(TN_ECUDA, "no such CUDA device");
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(TN_ECUDA, "this build targets sm_103a (GB300); device is sm_" +
                                  std::to_string(prop.major) + std::to_string(prop.minor));
    CK(cudaSetDevice(device));
    tn_ctx *c = new (std::nothrow) tn_ctx;
    if (!c) return fail(TN_ENOMEM, "allocating the context");
    c->device = device;
    c->budget = hbm_budget_bytes;
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return fail(TN_ECUDA, cudaGetErrorString(e)); }
        c->own_stream = true;
    }
    *out = c;
    return TN_OK;
}

void tn_ctx_free(tn_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    program_destroy(c->cached);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

tn_status tn_ctx_synchronize(tn_ctx *c) {
    if (!c) return fail(TN_EINVAL, "NULL ctx");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    return TN_OK;
}

tn_status tn_program_create(tn_ctx *ctx, const tn_net *net, const tn_plan *plan, tn_precision prec,
                            tn_program **out) {
    if (!ctx || !net || !plan || !out) return fail(TN_EINVAL, "NULL argument");
    if (prec < TN_C128 || prec > TN_BF16_SPLIT) return fail(TN_EINVAL, "unknown precision");
    const Net &nt = net->impl;
    const Plan &pl = plan->impl;
    if (pl.n != nt.n) return fail(TN_EINVAL, "plan and network do not match");
    if (!nt.closed) return fail(TN_EUNSUPPORTED, "open networks are not supported by tn_contract");
    CK(cudaSetDevice(ctx->device));
    tn_program *p = new (std::nothrow) tn_program;
    if (!p) return fail(TN_ENOMEM, "allocating the program");
    p->ctx = ctx;
    p->net = net;
    p->prec = prec;
    p->c128 = (prec == TN_C128);
    p->elem = p->c128 ? 16 : 8;
    tn_status s = compile(p, nt, pl);
    if (s != TN_OK) { program_destroy(p); return s; }
    // one device allocation, carved into the program's buffers
    const size_t n_el = (size_t)nt.data_off[nt.n];
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max(bytes, (size_t)16), 256); return o; };
    const size_t o_leaf64 = carve(16 * n_el);
    const size_t o_leaf = carve((size_t)p->elem * n_el);
    const size_t o_loff = carve(sizeof(int64_t) * (nt.n + 1));
    const size_t o_desc = carve(sizeof(StepDesc) * p->desc.size());
    const size_t o_exp = carve(sizeof(int32_t) * p->n_nodes);
    const size_t o_max = carve(sizeof(uint32_t) * p->n_nodes);
    const size_t o_part = carve(sizeof(double) * 2 * 16 * (size_t)dot_partial_blocks());
    const size_t o_res = carve(sizeof(DeviceResult));
    const size_t o_arena = carve(p->arena_bytes);
    p->footprint = off;
    if (ctx->budget && p->footprint > ctx->budget) {
        program_destroy(p);
        return fail(TN_EBUDGET, "program needs " + std::to_string(off) + " bytes of device memory");
    }
    cudaError_t e = cudaMalloc(&p->d_block, off);
    if (e != cudaSuccess) {
        program_destroy(p);
        return fail(e == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA, cudaGetErrorString(e));
    }
    char *base = static_cast<char *>(p->d_block);
    p->d_leaf64 = reinterpret_cast<double *>(base + o_leaf64);
    p->d_leaf = base + o_leaf;
    p->d_leaf_off = reinterpret_cast<int64_t *>(base + o_loff);
    p->d_desc = reinterpret_cast<StepDesc *>(base + o_desc);
    p->d_exp2 = reinterpret_cast<int32_t *>(base + o_exp);
    p->d_maxbits = reinterpret_cast<uint32_t *>(base + o_max);
    p->d_partials = reinterpret_cast<double *>(base + o_part);
    p->d_res = reinterpret_cast<DeviceResult *>(base + o_res);
    p->d_arena = base + o_arena;
    // resolve descriptor operand addresses
    for (size_t i = 0; i < p->desc.size(); ++i) {
        StepDesc &d = p->desc[i];
        auto resolve = [&](int64_t w) -> char * {
            if (w < 0) return static_cast<char *>(p->d_leaf) + (size_t)p->elem * (size_t)p->leaf_off[-1 - w];
            return p->d_arena + w;
        };
        d.A = resolve(p->where[i][0]);
        d.B = resolve(p->where[i][1]);
        d.C = d.is_root ? nullptr : resolve(p->where[i][2]);
    }
    cudaStream_t st = ctx->stream;
    if (cudaMallocHost(&p->h_pinned, std::max((size_t)16, sizeof(double) * nt.data.size())) != cudaSuccess ||
        cudaMallocHost(&p->h_res, sizeof(DeviceResult)) != cudaSuccess) {
        program_destroy(p);
        return fail(TN_ENOMEM, "pinned staging buffer");
    }
    e = cudaMemcpyAsync(p->d_leaf_off, p->leaf_off.data(), sizeof(int64_t) * (nt.n + 1),
                        cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !p->desc.empty())
        e = cudaMemcpyAsync(p->d_desc, p->desc.data(), sizeof(StepDesc) * p->desc.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_exp2, 0, sizeof(int32_t) * p->n_nodes, st);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
    if (e != cudaSuccess) { program_destroy(p); return fail(TN_ECUDA, cudaGetErrorString(e)); }
    s = upload_leaves(p);
    if (s == TN_OK) s = record_graph(p);
    if (s == TN_OK) {
        e = cudaStreamSynchronize(st);   // descriptor and leaf uploads read host buffers
        if (e != cudaSuccess) s = fail(TN_ECUDA, cudaGetErrorString(e));
    }
    if (s != TN_OK) { program_destroy(p); return s; }
    *out = p;
    return TN_OK;
}

tn_status tn_program_run(tn_program *p, void *d_result) {
    if (!p || !d_result) return fail(TN_EINVAL, "NULL argument");
    CK(cudaSetDevice(p->ctx->device));
    cudaStream_t st = p->ctx->stream;
    if (p->uploaded_version != p->net->impl.version) {
        CK(cudaStreamSynchronize(st));   // the pinned staging buffer may still be in flight
        tn_status s = upload_leaves(p);
        if (s != TN_OK) return s;
    }
    CK(cudaEventRecord(p->ev0, st));
    CK(cudaGraphLaunch(p->gexec, st));
    CK(cudaEventRecord(p->ev1, st));
    if (d_result != (void *)p->d_res)
        CK(cudaMemcpyAsync(d_result, p->d_res, sizeof(DeviceResult), cudaMemcpyDeviceToDevice, st));
    p->ran = true;
    return TN_OK;
}

tn_status tn_program_footprint(const tn_program *p, size_t *bytes) {
    if (!p || !bytes) return fail(TN_EINVAL, "NULL argument");
    *bytes = p->footprint;
    return TN_OK;
}

tn_status tn_program_last_info(const tn_program *pc, tn_run_info *info) {
    if (!pc || !info) return fail(TN_EINVAL, "NULL argument");
    tn_program *p = const_cast<tn_program *>(pc);
    if (p->ran) {
        CK(cudaSetDevice(p->ctx->device));
        CK(cudaEventSynchronize(p->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->info.device_ms = ms;
    }
    *info = p->info;
    return TN_OK;
}

void tn_program_free(tn_program *p) {
    if (!p) return;
    cudaSetDevice(p->ctx->device);
    cudaStreamSynchronize(p->ctx->stream);
    if (p->ctx->cached == p) p->ctx->cached = nullptr;
    program_destroy(p);
}

tn_status tn_contract(tn_ctx *ctx, const tn_net *net, const tn_plan *plan, tn_precision prec,
                      double out_amp[2], int32_t *out_exp2, tn_run_info *info) {
    if (!ctx || !net || !plan || !out_amp || !out_exp2) return fail(TN_EINVAL, "NULL argument");
    CK(cudaSetDevice(ctx->device));
    if (!(ctx->cached && ctx->cached_net == net->impl.uid && ctx->cached_plan == plan->impl.uid &&
          ctx->cached_prec == prec)) {
        if (ctx->cached) {
            cudaStreamSynchronize(ctx->stream);
            program_destroy(ctx->cached);
            ctx->cached = nullptr;
        }
        tn_program *p = nullptr;
        tn_status s = tn_program_create(ctx, net, plan, prec, &p);
        if (s != TN_OK) return s;
        ctx->cached = p;
        ctx->cached_net = net->impl.uid;
        ctx->cached_plan = plan->impl.uid;
        ctx->cached_prec = prec;
    }
    tn_program *p = ctx->cached;
    p->net = net;                  // the same net (by id); refresh the address
    p->uploaded_version = ~0ull;   // end to end: the leaves are copied from the host every call
    tn_status s = tn_program_run(p, p->d_res);
    if (s != TN_OK) return s;
    CK(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(DeviceResult), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const DeviceResult r = *p->h_res;
    if (r.status != 0) return fail(TN_ETIMEOUT, "device reported status " + std::to_string(r.status));
    out_amp[0] = r.re;
    out_amp[1] = r.im;
    *out_exp2 = r.exp2;
    if (info) {
        tn_status si = tn_program_last_info(p, info);
        if (si != TN_OK) return si;
    }
    return TN_OK;
}

tn_status tn_permute(tn_ctx *ctx, const void *d_in, void *d_out, int32_t elem_bytes, int32_t rank,
                     const int64_t *dims, const int32_t *perm) {
    if (!ctx || (!d_in && rank > 0) || !d_out || (rank > 0 && (!dims || !perm)))
        return fail(TN_EINVAL, "NULL argument");
    if (rank < 0 || rank > 32) return fail(TN_EINVAL, "rank must be in [0, 32]");
    if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16)
        return fail(TN_EINVAL, "elem_bytes must be 1, 2, 4, 8 or 16");
    std::vector<int> seen(rank, 0);
    for (int32_t t = 0; t < rank; ++t) {
        if (perm[t] < 0 || perm[t] >= rank || seen[perm[t]]) return fail(TN_EINVAL, "perm is not a permutation");
        seen[perm[t]] = 1;
        if (dims[t] < 1) return fail(TN_EINVAL, "dims must be >= 1");
    }
    CK(cudaSetDevice(ctx->device));
    CK(launch_permute(d_in, d_out, elem_bytes, rank, dims, perm, ctx->stream));
    return TN_OK;
}

}  // extern "C"
