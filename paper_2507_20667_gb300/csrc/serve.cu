// Serving loop: continuous batching of contraction requests over resident models.
//
// A model is a registered (network, plan): compiled once, its step tables kept on the device, its
// leaves kept on the host as the base values of its requests.  A request names a model and
// overrides some leaves (the bra tensors of a bitstring, the Z slots of an expectation value).
// A worker thread admits queued requests into launches as device memory allows (each request
// needs its model's per-job bytes from a pool sized to the HBM budget), and keeps up to two
// launches in flight on two streams: requests that arrive while one launch runs start in the next
// one, which overlaps with it on the device.  Each launch is the batch path: leaf upload, leaf
// conversion, subtree programs, the persistent dataflow kernel, result read-back.  A request's
// result depends only on its own job, so it is the same alone and in any mix.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "compile.cuh"
#include "kernels.cuh"
#include "tn_internal.hpp"

using namespace tn;

namespace {

constexpr size_t kMaxModels = 1 << 16;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// First-fit allocator over [0, size) with coalescing.
struct Arena {
    std::map<size_t, size_t> free_;   // offset -> size
    size_t size_ = 0, used_ = 0;
    void reset(size_t size) { free_.clear(); free_[0] = size; size_ = size; used_ = 0; }
    bool alloc(size_t sz, size_t &off) {
        sz = align256(std::max<size_t>(sz, 256));
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= sz) {
                off = it->first;
                const size_t rest = it->second - sz;
                free_.erase(it);
                if (rest) free_[off + sz] = rest;
                used_ += sz;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t sz) {
        sz = align256(std::max<size_t>(sz, 256));
        used_ -= sz;
        auto it = free_.emplace(off, sz).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Model {
    Compiled c;
    void *dev = nullptr;              // step tables
    std::vector<double> leaves;       // base complex128 leaves (interleaved)
    std::vector<int64_t> leaf_off;
    std::vector<PhaseTemplate> ph;    // per dependency phase: dataflow items, TC units and tiles
    size_t n_items = 0;               // work items of all phases (dataflow, pack, GEMM)
    std::vector<int32_t> local_steps; // pseudo-steps of block programs
    std::vector<int32_t> warp_steps;  // pseudo-steps of warp programs
    std::vector<int32_t> big_steps;   // pseudo-steps of large programs
    size_t o_leaf = 0, o_arena = 0, o_part = 0, o_exp = 0, job_bytes = 0;
};

struct Request {
    uint64_t ticket;
    int32_t model;
    std::vector<int32_t> tensors;
    std::vector<double> data;
    double t_submit;
};

struct Result {
    double re = 0, im = 0;
    int32_t exp2 = 0, status = TN_OK;
    double latency = 0;
};

struct Flight {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<Request> reqs;
    std::vector<std::pair<size_t, size_t>> blocks;   // pool (offset, size) to release
    char *h_stage = nullptr;
    size_t h_cap = 0;
    DeviceResult *h_res = nullptr;
    size_t res_cap = 0;
};

}  // namespace

struct tn_server {
    tn_ctx *ctx = nullptr;
    int32_t device = 0;
    tn_precision prec = TN_C64;
    bool c128 = false;
    int32_t elem = 8;
    int32_t max_batch = 64;
    CompileOpts copt;                 // compiler options (from the context's configuration)
    long long wait_ns = 4000000000LL; // dependency-wait limit of the persistent kernel
    char *pool = nullptr;
    size_t pool_bytes = 0;
    Arena arena;
    std::vector<std::unique_ptr<Model>> models;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    Flight fl[2];
    std::thread worker;
    std::atomic<bool> stop{false};
    int32_t dyn_smem = 0, dyn_big = 0, grid = 0;
    bool any_tc = false;
    std::string worker_error;
    tn_serve_stats stats{};
};

namespace {

// Harvest a finished launch: results to the map, memory back to the pool.
void harvest(tn_server *S, Flight &f) {
    const double t = now_s();
    std::lock_guard<std::mutex> lock(S->mu);
    for (size_t i = 0; i < f.reqs.size(); ++i) {
        Result r;
        r.re = f.h_res[i].re;
        r.im = f.h_res[i].im;
        r.exp2 = f.h_res[i].exp2;
        r.status = f.h_res[i].status ? TN_ETIMEOUT : TN_OK;
        r.latency = t - f.reqs[i].t_submit;
        S->results[f.reqs[i].ticket] = r;
        S->stats.completed++;
    }
    for (auto &b : f.blocks) S->arena.release(b.first, b.second);
    f.blocks.clear();
    f.reqs.clear();
    f.busy = false;
    S->cv.notify_all();
}

// Enqueue one launch for the requests in f.reqs (their job blocks already allocated in f.blocks).
cudaError_t launch(tn_server *S, Flight &f, const std::vector<size_t> &job_off, size_t meta_off) {
    const int32_t n = (int32_t)f.reqs.size();
    // meta layout: leaf64 | JobPtrs | work items | local items | reset region
    int64_t leaf_total = 0;
    std::vector<int64_t> l64(n);
    for (int32_t i = 0; i < n; ++i) {
        l64[i] = leaf_total;
        leaf_total += S->models[f.reqs[i].model]->leaf_off.back();
    }
    std::vector<WorkItem> work, local, packs, gemms;
    int32_t n_phases = 1;
    for (int32_t i = 0; i < n; ++i) n_phases = std::max(n_phases, (int32_t)S->models[f.reqs[i].model]->ph.size());
    // per phase: the TC units and tiles of all jobs, then the jobs' dataflow items merged level by
    // level (all jobs' level-1 tiles first, ...)
    struct Range { size_t w0, nw, p0, np, g0, ng; };
    std::vector<Range> ranges(n_phases);
    for (int32_t p = 0; p < n_phases; ++p) {
        Range &r = ranges[p];
        r.p0 = packs.size();
        r.g0 = gemms.size();
        r.w0 = work.size();
        int32_t max_level = 0;
        for (int32_t i = 0; i < n; ++i) {
            const Model &m = *S->models[f.reqs[i].model];
            if (p >= (int32_t)m.ph.size()) continue;
            for (WorkItem w : m.ph[p].pack) { w.job = (uint32_t)i; packs.push_back(w); }
            for (WorkItem w : m.ph[p].gemm) { w.job = (uint32_t)i; gemms.push_back(w); }
            for (int32_t lv : m.ph[p].level) max_level = std::max(max_level, lv);
        }
        std::vector<size_t> cursor(n, 0);
        for (int32_t lv = 0; lv <= max_level; ++lv)
            for (int32_t i = 0; i < n; ++i) {
                const Model &m = *S->models[f.reqs[i].model];
                if (p >= (int32_t)m.ph.size()) continue;
                const PhaseTemplate &pt = m.ph[p];
                size_t &c = cursor[i];
                while (c < pt.work.size() && pt.level[c] == lv) {
                    WorkItem w = pt.work[c++];
                    w.job = (uint32_t)i;
                    work.push_back(w);
                }
            }
        r.np = packs.size() - r.p0;
        r.ng = gemms.size() - r.g0;
        r.nw = work.size() - r.w0;
    }
    // warp programs first, then block programs (launch_local's item order)
    for (int32_t i = 0; i < n; ++i)
        for (int32_t s : S->models[f.reqs[i].model]->warp_steps) local.push_back({(uint32_t)i, (uint32_t)s, 0u});
    const int32_t n_warp = (int32_t)local.size();
    for (int32_t i = 0; i < n; ++i)
        for (int32_t s : S->models[f.reqs[i].model]->local_steps) local.push_back({(uint32_t)i, (uint32_t)s, 0u});
    const int32_t n_block = (int32_t)local.size() - n_warp;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t s : S->models[f.reqs[i].model]->big_steps) local.push_back({(uint32_t)i, (uint32_t)s, 0u});
    const int32_t n_big = (int32_t)local.size() - n_warp - n_block;
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off = align256(off + std::max<size_t>(bytes, 16)); return o; };
    const size_t o_l64 = carve(sizeof(double2) * (size_t)leaf_total);
    const size_t o_jobs = carve(sizeof(JobPtrs) * (size_t)n);
    const size_t o_work = carve(sizeof(WorkItem) * work.size());
    const size_t o_local = carve(sizeof(WorkItem) * local.size());
    const size_t o_pack = carve(sizeof(WorkItem) * packs.size());
    const size_t o_gemm = carve(sizeof(WorkItem) * gemms.size());
    const size_t upload_bytes = off;
    const size_t o_reset = off;
    const size_t o_res = carve(sizeof(DeviceResult) * (size_t)n);
    std::vector<size_t> o_max(n), o_done(n);
    for (int32_t i = 0; i < n; ++i) {
        const Model &m = *S->models[f.reqs[i].model];
        o_max[i] = carve(sizeof(uint32_t) * (size_t)m.c.n_nodes);
        o_done[i] = carve(sizeof(int32_t) * m.c.steps.size());
    }
    const size_t o_counter = carve(3 * sizeof(uint32_t) * (size_t)n_phases);   // per phase: claim, abort x 2
    const size_t reset_bytes = off - o_reset;
    char *meta = S->pool + meta_off;
    // host staging
    if (upload_bytes > f.h_cap) {
        if (f.h_stage) cudaFreeHost(f.h_stage);
        f.h_stage = nullptr;
        f.h_cap = 0;
        cudaError_t e = cudaMallocHost(&f.h_stage, upload_bytes * 2);
        if (e != cudaSuccess) return e;
        f.h_cap = upload_bytes * 2;
    }
    if ((size_t)n > f.res_cap) {
        if (f.h_res) cudaFreeHost(f.h_res);
        f.h_res = nullptr;
        f.res_cap = 0;
        cudaError_t e = cudaMallocHost(&f.h_res, sizeof(DeviceResult) * (size_t)n * 2);
        if (e != cudaSuccess) return e;
        f.res_cap = (size_t)n * 2;
    }
    double *stage_l64 = reinterpret_cast<double *>(f.h_stage + o_l64);
    JobPtrs *jobs = reinterpret_cast<JobPtrs *>(f.h_stage + o_jobs);
    for (int32_t i = 0; i < n; ++i) {
        const Request &r = f.reqs[i];
        const Model &m = *S->models[r.model];
        double *dst = stage_l64 + 2 * l64[i];
        std::memcpy(dst, m.leaves.data(), sizeof(double) * m.leaves.size());
        size_t src = 0;
        for (int32_t t : r.tensors) {
            const int64_t cnt = m.leaf_off[t + 1] - m.leaf_off[t];
            std::memcpy(dst + 2 * m.leaf_off[t], r.data.data() + src, sizeof(double) * 2 * (size_t)cnt);
            src += 2 * (size_t)cnt;
        }
        char *job = S->pool + job_off[i];
        JobPtrs &j = jobs[i];
        std::memset(&j, 0, sizeof(j));
        j.leaf64 = reinterpret_cast<const double2 *>(meta + o_l64) + l64[i];
        j.leaf_off = m.c.d_leaf_off;
        j.leaf = job + m.o_leaf;
        j.arena = job + m.o_arena;
        j.partials = reinterpret_cast<double2 *>(job + m.o_part);
        j.exp2 = reinterpret_cast<int32_t *>(job + m.o_exp);
        j.maxbits = reinterpret_cast<uint32_t *>(meta + o_max[i]);
        j.done = reinterpret_cast<int32_t *>(meta + o_done[i]);
        j.result = reinterpret_cast<DeviceResult *>(meta + o_res) + i;
        j.steps = m.c.d_steps;
        j.progs = m.c.d_progs;
        j.lsteps = m.c.d_lsteps;
        j.leafrefs = m.c.d_leafrefs;
        j.lwaves = m.c.d_lwaves;
        j.ktab = m.c.d_ktab;
        j.n_steps = (int32_t)m.c.steps.size();
        j.n_leaves = m.c.n;
    }
    if (!work.empty()) std::memcpy(f.h_stage + o_work, work.data(), sizeof(WorkItem) * work.size());
    if (!local.empty()) std::memcpy(f.h_stage + o_local, local.data(), sizeof(WorkItem) * local.size());
    if (!packs.empty()) std::memcpy(f.h_stage + o_pack, packs.data(), sizeof(WorkItem) * packs.size());
    if (!gemms.empty()) std::memcpy(f.h_stage + o_gemm, gemms.data(), sizeof(WorkItem) * gemms.size());
    int32_t max_leaves = 0;
    int64_t max_leaf_elems = 0;
    for (int32_t i = 0; i < n; ++i) {
        const Model &m = *S->models[f.reqs[i].model];
        max_leaves = std::max(max_leaves, m.c.n);
        for (size_t t = 0; t + 1 < m.leaf_off.size(); ++t) max_leaf_elems = std::max(max_leaf_elems, m.leaf_off[t + 1] - m.leaf_off[t]);
    }
    const JobPtrs *d_jobs = reinterpret_cast<const JobPtrs *>(meta + o_jobs);
    cudaError_t e = cudaMemcpyAsync(meta, f.h_stage, upload_bytes, cudaMemcpyHostToDevice, f.st);
    if (e == cudaSuccess) e = cudaMemsetAsync(meta + o_reset, 0, reset_bytes, f.st);
    if (e == cudaSuccess) e = launch_leaf_convert(S->c128, d_jobs, n, max_leaves, max_leaf_elems, f.st);
    if (e == cudaSuccess)
        e = launch_local(S->c128, d_jobs, reinterpret_cast<const WorkItem *>(meta + o_local), n_warp, n_block,
                         n_big, S->dyn_smem, S->dyn_big, nullptr, f.st);
    const bool tf32 = S->prec == TN_TF32_SPLIT;
    for (int32_t p = 0; e == cudaSuccess && p < n_phases; ++p) {
        const Range &r = ranges[p];
        uint32_t *cnt = reinterpret_cast<uint32_t *>(meta + o_counter) + 3 * p;
        if (r.np > 0)
            e = launch_tc_pack(tf32, d_jobs, reinterpret_cast<const WorkItem *>(meta + o_pack) + r.p0, (int32_t)r.np, f.st);
        if (e == cudaSuccess && r.ng > 0)
            e = launch_tc_gemm(tf32, d_jobs, reinterpret_cast<const WorkItem *>(meta + o_gemm) + r.g0, (int32_t)r.ng,
                               reinterpret_cast<int32_t *>(cnt + 2), S->wait_ns, f.st);
        if (e == cudaSuccess && r.nw > 0)
            e = launch_persistent(S->c128, d_jobs, reinterpret_cast<const WorkItem *>(meta + o_work) + r.w0,
                                  (int64_t)r.nw, cnt, S->grid, S->wait_ns, nullptr, f.st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f.h_res, meta + o_res, sizeof(DeviceResult) * (size_t)n, cudaMemcpyDeviceToHost, f.st);
    if (e == cudaSuccess) e = cudaEventRecord(f.ev, f.st);
    return e;
}

// Bytes of the per-launch metadata block for a set of requests (see launch()).
size_t meta_bytes(tn_server *S, const std::vector<Request> &reqs) {
    size_t b = 0;
    for (const Request &r : reqs) {
        const Model &m = *S->models[r.model];
        b += sizeof(double2) * (size_t)m.leaf_off.back() + sizeof(JobPtrs) +
             sizeof(WorkItem) * (m.n_items + m.local_steps.size() + m.warp_steps.size() + m.big_steps.size()) +
             sizeof(DeviceResult) + 3 * sizeof(uint32_t) * m.ph.size() +
             sizeof(uint32_t) * (size_t)m.c.n_nodes + sizeof(int32_t) * m.c.steps.size() + 5 * 256;
    }
    return b + 16 * 256;
}

void worker_loop(tn_server *S) {
    cudaSetDevice(S->device);
    while (!S->stop.load()) {
        for (Flight &f : S->fl)
            if (f.busy && cudaEventQuery(f.ev) == cudaSuccess) harvest(S, f);
        Flight *f = nullptr;
        for (Flight &x : S->fl)
            if (!x.busy) { f = &x; break; }
        std::vector<Request> take;
        std::vector<size_t> job_off;
        size_t meta_off = 0;
        bool launched = false;
        if (f) {
            std::unique_lock<std::mutex> lock(S->mu);
            while (!S->queue.empty() && (int32_t)take.size() < S->max_batch) {
                Request &r = S->queue.front();
                const Model &m = *S->models[r.model];
                if (m.job_bytes >= S->pool_bytes || m.job_bytes + meta_bytes(S, {r}) > S->pool_bytes) {
                    Result res;
                    res.status = TN_EBUDGET;
                    res.latency = now_s() - r.t_submit;
                    S->results[r.ticket] = res;
                    S->stats.rejected++;
                    S->queue.pop_front();
                    S->cv.notify_all();
                    continue;
                }
                size_t off;
                if (!S->arena.alloc(m.job_bytes, off)) break;   // wait for memory to free up
                f->blocks.push_back({off, m.job_bytes});
                job_off.push_back(off);
                take.push_back(std::move(r));
                S->queue.pop_front();
            }
            if (!take.empty()) {
                const size_t mb = meta_bytes(S, take);
                if (S->arena.alloc(mb, meta_off)) {
                    f->blocks.push_back({meta_off, mb});
                } else {   // no room for the metadata: put the requests back, retry later
                    for (auto &b : f->blocks) S->arena.release(b.first, b.second);
                    f->blocks.clear();
                    for (auto it = take.rbegin(); it != take.rend(); ++it) S->queue.push_front(std::move(*it));
                    take.clear();
                }
            }
        }
        if (!take.empty()) {
            f->reqs = std::move(take);
            cudaError_t e = launch(S, *f, job_off, meta_off);
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lock(S->mu);
                S->worker_error = cudaGetErrorString(e);
                for (Request &r : f->reqs) {
                    Result res;
                    res.status = TN_ECUDA;
                    S->results[r.ticket] = res;
                }
                for (auto &b : f->blocks) S->arena.release(b.first, b.second);
                f->blocks.clear();
                f->reqs.clear();
                S->cv.notify_all();
            } else {
                f->busy = true;
                launched = true;
                std::lock_guard<std::mutex> lock(S->mu);
                S->stats.launches++;
                S->stats.launched_requests += (int64_t)f->reqs.size();
                int32_t inflight = 0;
                for (Flight &x : S->fl) inflight += x.busy ? 1 : 0;
                S->stats.max_in_flight = std::max(S->stats.max_in_flight, inflight);
            }
        }
        if (!launched) {
            bool any_busy = S->fl[0].busy || S->fl[1].busy;
            std::unique_lock<std::mutex> lock(S->mu);
            if (any_busy || !S->queue.empty())
                S->cv.wait_for(lock, std::chrono::microseconds(50));
            else
                S->cv.wait_for(lock, std::chrono::milliseconds(2));
        }
    }
    for (Flight &f : S->fl)
        if (f.busy) {
            cudaEventSynchronize(f.ev);
            harvest(S, f);
        }
}

}  // namespace

extern "C" {

tn_status tn_serve_create(tn_ctx *ctx, tn_precision prec, size_t hbm_budget_bytes, int32_t max_batch,
                          tn_server **out) {
    if (!ctx || !out) return fail(TN_EINVAL, "NULL argument");
    if (prec < TN_C128 || prec > TN_BF16_SPLIT) return fail(TN_EINVAL, "unknown precision");
    if (hbm_budget_bytes < (1u << 20)) return fail(TN_EINVAL, "the budget must be at least 1 MiB");
    if (max_batch < 1) return fail(TN_EINVAL, "max_batch must be >= 1");
    int32_t dev = 0;
    tn_status s = tn_ctx_device(ctx, &dev);
    if (s != TN_OK) return s;
    if (cudaSetDevice(dev) != cudaSuccess) return fail(TN_ECUDA, "cudaSetDevice");
    tn_server *S = new (std::nothrow) tn_server;
    if (!S) return fail(TN_ENOMEM, "allocating the server");
    S->ctx = ctx;
    ctx_retain(ctx);
    S->device = dev;
    S->prec = prec;
    S->c128 = prec == TN_C128;
    S->elem = S->c128 ? 16 : 8;
    S->max_batch = max_batch;
    tn_exec_config cfg;
    s = tn_ctx_get_config(ctx, &cfg);
    if (s != TN_OK) {
        delete S;
        ctx_release(ctx);
        return s;
    }
    S->copt = compile_opts(cfg, prec, S->c128);
    S->wait_ns = (long long)cfg.wait_limit_us * 1000;
    // full co-resident grids: a second launch's blocks start as the first one's retire
    S->grid = std::max(1, persistent_grid(S->c128));
    cudaError_t e = cudaMalloc(&S->pool, hbm_budget_bytes);
    if (e != cudaSuccess) {
        delete S;
        ctx_release(ctx);
        return fail(e == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA, cudaGetErrorString(e));
    }
    S->pool_bytes = hbm_budget_bytes;
    S->arena.reset(hbm_budget_bytes);
    for (Flight &f : S->fl) {
        if (cudaStreamCreateWithFlags(&f.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming) != cudaSuccess) {
            tn_serve_free(S);
            return fail(TN_ECUDA, "creating streams");
        }
    }
    S->models.reserve(kMaxModels);   // never reallocated: the worker reads it concurrently
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return TN_OK;
}

tn_status tn_serve_register(tn_server *S, const tn_net *net, const tn_plan *plan, int32_t *model) {
    if (!S || !net || !plan || !model) return fail(TN_EINVAL, "NULL argument");
    if (plan->impl.n != net->impl.n) return fail(TN_EINVAL, "plan and network do not match");
    if (!net->impl.closed) return fail(TN_EUNSUPPORTED, "open networks are not supported");
    if (net->impl.n < 2) return fail(TN_EUNSUPPORTED, "a served network needs at least two tensors");
    if (cudaSetDevice(S->device) != cudaSuccess) return fail(TN_ECUDA, "cudaSetDevice");
    std::unique_ptr<Model> m(new (std::nothrow) Model);
    if (!m) return fail(TN_ENOMEM, "allocating the model");
    // a model whose exact memory count (Eq. 3.1) exceeds the pool can never run: keep it as a
    // placeholder whose requests are refused with TN_EBUDGET
    if ((double)plan->impl.mem * (double)S->elem > (double)S->pool_bytes) {
        m->job_bytes = SIZE_MAX / 4;
        m->c.n = net->impl.n;
        m->leaf_off = net->impl.data_off;
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->models.size() >= kMaxModels) return fail(TN_EINVAL, "too many models");
        *model = (int32_t)S->models.size();
        S->models.push_back(std::move(m));
        return TN_OK;
    }
    tn_status s = compile(m->c, net->impl, plan->impl, S->copt);
    if (s != TN_OK) return s;
    m->leaves = net->impl.data;
    m->leaf_off = net->impl.data_off;
    phase_templates(m->c, m->ph);
    for (const PhaseTemplate &pt : m->ph) m->n_items += pt.work.size() + pt.pack.size() + pt.gemm.size();
    for (size_t st = 0; st < m->c.steps.size(); ++st)
        if (m->c.steps[st].kind == STEP_LOCAL)
        {
            const int32_t kind = m->c.progs[m->c.steps[st].tile_rows].kind;
            (kind == PROG_WARP ? m->warp_steps : kind == PROG_BIG ? m->big_steps : m->local_steps)
                .push_back((int32_t)st);
        }
    // per-request device bytes: storage leaves, arena, partials, exponents
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off = align256(off + std::max<size_t>(bytes, 16)); return o; };
    m->o_leaf = carve((size_t)S->elem * (size_t)m->leaf_off.back());
    m->o_arena = carve(m->c.arena_bytes);
    m->o_part = carve(sizeof(double2) * (size_t)m->c.n_partials);
    m->o_exp = carve(sizeof(int32_t) * (size_t)m->c.n_nodes);
    m->job_bytes = off;
    // resident step tables
    const Compiled &c = m->c;
    size_t t = 0;
    auto tcarve = [&](size_t bytes) { size_t o = t; t = align256(t + std::max<size_t>(bytes, 16)); return o; };
    const size_t a = tcarve(sizeof(StepDesc) * c.steps.size()), b = tcarve(sizeof(int64_t) * c.leaf_off.size());
    const size_t p = tcarve(sizeof(LocalProg) * c.progs.size()), q = tcarve(sizeof(LocalStep) * c.lsteps.size());
    const size_t r = tcarve(sizeof(LeafRef) * c.leafrefs.size()), w = tcarve(sizeof(LocalWave) * c.lwaves.size());
    const size_t kt = tcarve(sizeof(int2) * c.ktab.size());
    cudaError_t e = cudaMalloc(&m->dev, t);
    if (e != cudaSuccess) return fail(TN_ENOMEM, cudaGetErrorString(e));
    char *d = static_cast<char *>(m->dev);
    m->c.d_steps = reinterpret_cast<StepDesc *>(d + a);
    m->c.d_leaf_off = reinterpret_cast<int64_t *>(d + b);
    m->c.d_progs = reinterpret_cast<LocalProg *>(d + p);
    m->c.d_lsteps = reinterpret_cast<LocalStep *>(d + q);
    m->c.d_leafrefs = reinterpret_cast<LeafRef *>(d + r);
    m->c.d_lwaves = reinterpret_cast<LocalWave *>(d + w);
    m->c.d_ktab = reinterpret_cast<int2 *>(d + kt);
    e = cudaMemcpy(m->c.d_steps, c.steps.data(), sizeof(StepDesc) * c.steps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(m->c.d_leaf_off, c.leaf_off.data(), sizeof(int64_t) * c.leaf_off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !c.progs.empty())
        e = cudaMemcpy(m->c.d_progs, c.progs.data(), sizeof(LocalProg) * c.progs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !c.lsteps.empty())
        e = cudaMemcpy(m->c.d_lsteps, c.lsteps.data(), sizeof(LocalStep) * c.lsteps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !c.leafrefs.empty())
        e = cudaMemcpy(m->c.d_leafrefs, c.leafrefs.data(), sizeof(LeafRef) * c.leafrefs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !c.lwaves.empty())
        e = cudaMemcpy(m->c.d_lwaves, c.lwaves.data(), sizeof(LocalWave) * c.lwaves.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !c.ktab.empty())
        e = cudaMemcpy(m->c.d_ktab, c.ktab.data(), sizeof(int2) * c.ktab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->dev);
        return fail(TN_ECUDA, cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->models.size() >= kMaxModels) {
        cudaFree(m->dev);
        return fail(TN_EINVAL, "too many models");
    }
    // the subtree-program kernel's shared memory covers every registered model
    S->dyn_smem = std::max(S->dyn_smem, c.dyn_smem);
    S->dyn_big = std::max(S->dyn_big, c.dyn_big);
    *model = (int32_t)S->models.size();
    S->models.push_back(std::move(m));
    return TN_OK;
}

tn_status tn_serve_model_info(tn_server *S, int32_t model, size_t *job_bytes, double *flops) {
    if (!S) return fail(TN_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(S->mu);
    if (model < 0 || model >= (int32_t)S->models.size()) return fail(TN_EINVAL, "unknown model");
    if (job_bytes) *job_bytes = S->models[model]->job_bytes;
    if (flops) *flops = S->models[model]->c.flops;
    return TN_OK;
}

tn_status tn_serve_submit(tn_server *S, int32_t model, int32_t count, const int32_t *tensors,
                          const double *data, uint64_t *ticket) {
    if (!S || !ticket || (count > 0 && (!tensors || !data)) || count < 0) return fail(TN_EINVAL, "bad argument");
    Request r;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (model < 0 || model >= (int32_t)S->models.size()) return fail(TN_EINVAL, "unknown model");
        const Model &m = *S->models[model];
        size_t vals = 0;
        for (int32_t i = 0; i < count; ++i) {
            if (tensors[i] < 0 || tensors[i] >= m.c.n) return fail(TN_EINVAL, "tensor index out of range");
            vals += 2 * (size_t)(m.leaf_off[tensors[i] + 1] - m.leaf_off[tensors[i]]);
        }
        r.tensors.assign(tensors, tensors + count);
        if (!entries_in_range(data, vals))
            return fail(TN_EINVAL, "tensor entries must be finite and below 2^127 in magnitude");
        r.data.assign(data, data + vals);
        r.model = model;
        r.ticket = S->next_ticket++;
        r.t_submit = now_s();
        *ticket = r.ticket;
        S->queue.push_back(std::move(r));
        S->stats.submitted++;
    }
    S->cv.notify_all();
    return TN_OK;
}

tn_status tn_serve_poll(tn_server *S, uint64_t ticket, double timeout_s, double out_amp[2], int32_t *out_exp2,
                        double *latency_s, int32_t *done) {
    if (!S || !done) return fail(TN_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lock(S->mu);
    auto ready = [&] { return S->results.count(ticket) > 0; };
    if (timeout_s > 0) S->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), ready);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) {
        *done = 0;
        return TN_OK;
    }
    const Result r = it->second;
    S->results.erase(it);
    *done = 1;
    if (out_amp) { out_amp[0] = r.re; out_amp[1] = r.im; }
    if (out_exp2) *out_exp2 = r.exp2;
    if (latency_s) *latency_s = r.latency;
    if (r.status != TN_OK) return fail((tn_status)r.status, r.status == TN_EBUDGET
                                                                 ? "the request does not fit the server's budget"
                                                                 : "the request failed on the device");
    return TN_OK;
}

tn_status tn_serve_get_stats(tn_server *S, tn_serve_stats *st) {
    if (!S || !st) return fail(TN_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    *st = S->stats;
    st->pool_used = S->arena.used_;
    return TN_OK;
}

void tn_serve_free(tn_server *S) {
    if (!S) return;
    S->stop.store(true);
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (Flight &f : S->fl) {
        if (f.st) cudaStreamSynchronize(f.st);
        if (f.ev) cudaEventDestroy(f.ev);
        if (f.st) cudaStreamDestroy(f.st);
        if (f.h_stage) cudaFreeHost(f.h_stage);
        if (f.h_res) cudaFreeHost(f.h_res);
    }
    for (auto &m : S->models)
        if (m->dev) cudaFree(m->dev);
    if (S->pool) cudaFree(S->pool);
    tn_ctx *ctx = S->ctx;
    delete S;
    ctx_release(ctx);
}

}  // extern "C"
