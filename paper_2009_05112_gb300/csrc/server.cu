// server.cu -- vp_server_*: integration requests that arrive over time,
// iterated together.
//
// Every server step runs one adaptive iteration (§2, §3) of every admitted
// request through the same kernels as a batch: per kernel instantiation one
// persistent sampling launch over a queue of (request, sample range) tasks,
// then the per-hypercube estimate, the reallocation and the per-axis
// refinement over all requests at once.  The estimate kernel also applies each
// request's stop rule (the §2.5 combination of its iterations j >= discard
// reaching sdev <= rtol |mean|) and writes one flag per request, the only
// thing the host reads back per step.  Finished requests leave between steps;
// queued ones join when their state fits in the memory budget.
//
// Memory: one reservation of mem_budget bytes made at creation, handed out to
// requests by a first-fit allocator with coalescing; descriptor and group
// tables sized for max_active requests.  Nothing is allocated per step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "host.h"

using namespace vp;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit sub-allocation of [0, size) in 256-byte multiples; freed ranges
// merge with their free neighbours.
class Pool {
  public:
    void reset(size_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Req {
    uint64_t id = 0, tag = 0;
    Member mb;
    double rtol = 0.0;
    int discard = 0, min_meas = 1;
    size_t bytes = 0, off = 0;
    double t_submit = 0.0, t_admit = 0.0;
    Desc d;
};

// one sampling launch per (kind, precision, bucket, exactness)
constexpr int kGroupSlots = 4 * 2 * kNumBuckets * 2;
int group_slot(int kind, int prec, int bucket, bool exact) {
    return ((kind * 2 + prec) * kNumBuckets + bucket) * 2 + (exact ? 1 : 0);
}

}  // namespace

struct vp_server {
    int device = 0, n_sm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the refinement (a8) runs on a side stream beside the estimate and the
    // reallocation (a6, a7)
    cudaStream_t side = nullptr;
    cudaEvent_t efork = nullptr, ejoin = nullptr;
    size_t budget = 0;
    int max_active = 0;
    DevMem pool_mem, tables;
    Pool pool;
    Desc *d_desc = nullptr, *d_new = nullptr;
    uint32_t *d_tree = nullptr, *d_axis = nullptr, *d_new_tree = nullptr, *d_done = nullptr;
    const double *d_inv = nullptr;
    uint32_t *h_done = nullptr;  // pinned
    Group slots[kGroupSlots];
    std::vector<int> live;  // slots with members
    // the running set (touched by the stepping thread only)
    std::vector<std::unique_ptr<Req>> active;
    std::vector<Desc> h_desc;
    std::vector<uint32_t> h_tree, h_axis;
    uint32_t n_tree_total = 0, n_axis_total = 0;
    int max_ng = 1;
    bool any_refine = false, dirty = true;
    // shared with submitting and polling threads (under mu)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::unique_ptr<Req>> queue;
    std::deque<vp_served> finished;
    uint64_t next_id = 0;
    int64_t n_finished = 0, steps = 0, n_eval = 0, n_active = 0;
    size_t peak = 0;
    double busy = 0.0;
    std::thread worker;
    bool running = false, stop = false;
    vp_status werr = VP_OK;
    std::string werr_msg;
    std::mutex step_mu;  // one step at a time
};

static vp_status admit(vp_server *S) {
    std::vector<Req *> fresh;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        while (!S->queue.empty() && (int)S->active.size() < S->max_active) {
            Req *r = S->queue.front().get();
            size_t off = 0;
            if (!S->pool.alloc(r->bytes, &off)) break;  // first come, first served
            r->off = off;
            S->active.push_back(std::move(S->queue.front()));
            S->queue.pop_front();
            fresh.push_back(r);
        }
        S->peak = std::max(S->peak, S->pool.used());
    }
    if (fresh.empty()) return VP_OK;
    cudaStream_t st = S->stream;
    std::vector<Desc> nd;
    std::vector<uint32_t> nt(1, 0u);
    const double t = now_s();
    for (Req *r : fresh) {
        r->t_admit = t;
        r->mb.base = (char *)S->pool_mem.ptr + r->off;
        CU(cudaMemsetAsync(r->mb.base, 0, r->bytes, st));
        fill_desc(r->mb, S->d_inv, r->d);
        r->d.rtol = r->rtol;
        r->d.discard = r->discard;
        r->d.min_meas = r->min_meas;
        r->d.stop_it = r->mb.hist_cap;
        r->d.done_out = nullptr;  // set when the running set is laid out
        vp_status ust = upload_member_init(r->mb, r->d, st);
        if (ust != VP_OK) return ust;
        nd.push_back(r->d);
        nt.push_back(nt.back() + r->mb.n_tree);
    }
    // first allocation of the newcomers: d_h = 1 -> the equal split
    const int n_new = (int)fresh.size();
    CU(cudaMemcpyAsync(S->d_new, nd.data(), n_new * sizeof(Desc), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(S->d_new_tree, nt.data(), (n_new + 1) * 4, cudaMemcpyHostToDevice, st));
    CU(launch_estimate(S->d_new, S->d_new_tree, n_new, nt.back(), 2, st));
    CU(launch_alloc(S->d_new, S->d_new_tree, n_new, nt.back(), st, 1));
    S->dirty = true;
    return VP_OK;
}

// Descriptors, block prefixes and launch groups of the running set.
static vp_status layout(vp_server *S) {
    const int n = (int)S->active.size();
    cudaStream_t st = S->stream;
    S->h_desc.resize(n);
    S->h_tree.assign(n + 1, 0u);
    S->h_axis.assign(n + 1, 0u);
    S->any_refine = false;
    S->max_ng = 1;
    for (int s = 0; s < kGroupSlots; ++s) S->slots[s].members.clear();
    std::vector<const Member *> mp(n);
    for (int i = 0; i < n; ++i) {
        const Req &r = *S->active[i];
        const Member &mb = r.mb;
        mp[i] = &mb;
        S->h_desc[i] = r.d;
        S->h_desc[i].done_out = S->d_done + i;
        S->h_tree[i + 1] = S->h_tree[i] + mb.n_tree;
        S->h_axis[i + 1] = S->h_axis[i] + mb.p.dim;
        S->max_ng = std::max(S->max_ng, mb.p.n_g);
        if (mb.p.alpha > 0.0 && mb.p.n_g > 1) S->any_refine = true;
        // FP64 kernels are guarded; so is the per-axis form (strata that differ)
        const bool exact = mb.exact && mb.p.precision == VP_FP32 && mb.uniform;
        S->slots[group_slot(mb.kind, mb.p.precision, mb.bucket, exact)].members.push_back(i);
    }
    S->n_tree_total = S->h_tree[n];
    S->n_axis_total = S->h_axis[n];
    S->live.clear();
    for (int s = 0; s < kGroupSlots; ++s) {
        Group &g = S->slots[s];
        if (g.members.empty()) continue;
        vp_status gst = group_config_many(mp, g, S->n_sm);
        if (gst != VP_OK) return gst;
        CU(cudaMemcpyAsync(g.d_members, g.members.data(), g.members.size() * 4,
                           cudaMemcpyHostToDevice, st));
        S->live.push_back(s);
    }
    CU(cudaMemcpyAsync(S->d_desc, S->h_desc.data(), n * sizeof(Desc), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(S->d_tree, S->h_tree.data(), (n + 1) * 4, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(S->d_axis, S->h_axis.data(), (n + 1) * 4, cudaMemcpyHostToDevice, st));
    S->dirty = false;
    return VP_OK;
}

// Results of the requests whose flag is set; their memory goes back to the pool.
static vp_status retire(vp_server *S) {
    const int n = (int)S->active.size();
    std::vector<vp_served> out;
    std::vector<double> I, V;
    int64_t evals = 0;
    for (int i = 0; i < n; ++i) {
        if (!(S->h_done[i] & kDoneStop)) continue;
        Req &r = *S->active[i];
        // (copies to pageable memory return when complete)
        State sv;
        CU(cudaMemcpyAsync(&sv, r.d.st, sizeof sv, cudaMemcpyDeviceToHost, S->stream));
        const int nit = (int)std::min<uint32_t>(sv.t, (uint32_t)r.mb.hist_cap);
        I.resize(nit);
        V.resize(nit);
        if (nit) {
            CU(cudaMemcpyAsync(I.data(), r.d.hist_i, nit * 8, cudaMemcpyDeviceToHost, S->stream));
            CU(cudaMemcpyAsync(V.data(), r.d.hist_var, nit * 8, cudaMemcpyDeviceToHost, S->stream));
        }
        vp_served o;
        memset(&o, 0, sizeof o);
        o.id = r.id;
        o.tag = r.tag;
        o.status = (sv.status & kStatusNonFinite) ? VP_ENONFINITE : VP_OK;
        o.converged = (S->h_done[i] & kDoneConverged) ? 1 : 0;
        o.n_iter = (int)sv.t;
        combine(I.data(), V.data(), nit, r.discard, &o.r);
        o.r.n_eval = (int64_t)sv.n_eval_total;
        o.r.last_i = sv.last_i;
        o.r.last_sdev = std::sqrt(sv.last_var);
        o.t_submit = r.t_submit;
        o.t_admit = r.t_admit;
        out.push_back(o);
        evals += o.r.n_eval;
    }
    if (out.empty()) return VP_OK;
    const double t = now_s();
    std::vector<std::unique_ptr<Req>> keep;
    keep.reserve(n);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &o : out) {
            o.t_done = t;
            S->finished.push_back(o);
        }
        S->n_finished += (int64_t)out.size();
        S->n_eval += evals;
        for (int i = 0; i < n; ++i) {
            if (S->h_done[i] & kDoneStop) S->pool.release(S->active[i]->off, S->active[i]->bytes);
            else keep.push_back(std::move(S->active[i]));
        }
    }
    S->active.swap(keep);
    S->dirty = true;
    S->cv_done.notify_all();
    return VP_OK;
}

static vp_status server_step(vp_server *S, int *n_active) {
    std::lock_guard<std::mutex> step_lock(S->step_mu);
    NvtxRange nv("vp.server_step");
    const double t0 = now_s();
    cudaStream_t st = S->stream;
    vp_status rs = admit(S);
    if (rs != VP_OK) return rs;
    const int n = (int)S->active.size();
    if (n > 0) {
        if (S->dirty) {
            rs = layout(S);
            if (rs != VP_OK) return rs;
        }
        for (int s : S->live) {
            Group &g = S->slots[s];
            CU(launch_chunks(S->d_desc, g.d_members, (int)g.members.size(), g.d_chunk_base, g.d_head,
                             g.task, st));
        }
        for (int s : S->live) {
            rs = launch_group(S->d_desc, S->slots[s], st);
            if (rs != VP_OK) return rs;
        }
        if (S->any_refine) {
            CU(cudaEventRecord(S->efork, st));
            CU(cudaStreamWaitEvent(S->side, S->efork, 0));
            CU(launch_refine(S->d_desc, S->d_axis, n, S->n_axis_total, S->max_ng, S->side));
            CU(cudaEventRecord(S->ejoin, S->side));
        }
        CU(launch_estimate(S->d_desc, S->d_tree, n, S->n_tree_total, 0, st));
        CU(launch_alloc(S->d_desc, S->d_tree, n, S->n_tree_total, st, 0));
        if (S->any_refine) CU(cudaStreamWaitEvent(st, S->ejoin, 0));
        CU(cudaMemcpyAsync(S->h_done, S->d_done, n * 4, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        rs = retire(S);
        if (rs != VP_OK) return rs;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->n_active = (int64_t)S->active.size();
        if (n > 0) {
            S->steps += 1;
            S->busy += now_s() - t0;
        }
    }
    if (n_active) *n_active = (int)S->active.size();
    return VP_OK;
}

static void worker_main(vp_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || S->n_active > 0; });
            if (S->stop) return;
        }
        vp_status st = server_step(S, nullptr);
        if (st != VP_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->werr = st;
            S->werr_msg = g_err;
            S->stop = true;
            S->cv_done.notify_all();
            return;
        }
    }
}

static void server_free(vp_server *S) {
    if (S->stream) cudaStreamSynchronize(S->stream);
    dev_free(S->pool_mem, S->stream);
    dev_free(S->tables, S->stream);
    if (S->stream) cudaStreamSynchronize(S->stream);
    if (S->h_done) cudaFreeHost(S->h_done);
    if (S->side) {
        cudaStreamSynchronize(S->side);
        cudaStreamDestroy(S->side);
    }
    if (S->efork) cudaEventDestroy(S->efork);
    if (S->ejoin) cudaEventDestroy(S->ejoin);
    if (S->own_stream && S->stream) cudaStreamDestroy(S->stream);
}

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
#define CHECK_SRV(s) \
    if (!(s)) return fail(VP_EINVAL, "NULL server")

static vp_status server_init(vp_server *S, const vp_server_config *cfg, void *stream) {
    S->budget = cfg && cfg->mem_budget > 0 ? (size_t)cfg->mem_budget : ((size_t)256 << 20);
    S->max_active = cfg && cfg->max_active > 0 ? cfg->max_active : 4096;
    if (cfg && (cfg->mem_budget < 0 || cfg->max_active < 0 || cfg->max_active > 65536))
        return fail(VP_EINVAL, "mem_budget must be >= 0 and max_active 0..65536");
    S->budget = align256(S->budget);
    CU(cudaGetDevice(&S->device));
    CU(cudaDeviceGetAttribute(&S->n_sm, cudaDevAttrMultiProcessorCount, S->device));
    if (stream) {
        S->stream = (cudaStream_t)stream;
    } else {
        CU(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
        S->own_stream = true;
    }
    CU(cudaStreamCreateWithFlags(&S->side, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&S->efork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&S->ejoin, cudaEventDisableTiming));
    // tables: descriptors (running set, newcomers), block prefixes, flags, 1/n,
    // and the group slots' member lists, task prefixes and queue heads
    const size_t A = (size_t)S->max_active;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_desc = take(A * sizeof(Desc)), o_new = take(A * sizeof(Desc));
    const size_t o_tree = take((A + 1) * 4), o_axis = take((A + 1) * 4), o_ntree = take((A + 1) * 4);
    const size_t o_done = take(A * 4), o_inv = take(kInvTabWords * sizeof(double));
    size_t o_slot[kGroupSlots][3];
    for (int s = 0; s < kGroupSlots; ++s) {
        o_slot[s][0] = take(A * 4);
        o_slot[s][1] = take((A + 1) * 8);
        o_slot[s][2] = take(16);
    }
    vp_status st = dev_alloc(S->tables, off, S->stream);
    if (st != VP_OK) return st;
    char *T = (char *)S->tables.ptr;
    CU(cudaMemsetAsync(T, 0, off, S->stream));
    S->d_desc = (Desc *)(T + o_desc);
    S->d_new = (Desc *)(T + o_new);
    S->d_tree = (uint32_t *)(T + o_tree);
    S->d_axis = (uint32_t *)(T + o_axis);
    S->d_new_tree = (uint32_t *)(T + o_ntree);
    S->d_done = (uint32_t *)(T + o_done);
    S->d_inv = (const double *)(T + o_inv);
    for (int kind = 0; kind < 4; ++kind)
        for (int prec = 0; prec < 2; ++prec)
            for (int b = 0; b < kNumBuckets; ++b)
                for (int ex = 0; ex < 2; ++ex) {
                    const int s = group_slot(kind, prec, b, ex != 0);
                    Group &g = S->slots[s];
                    g.kind = kind;
                    g.prec = prec;
                    g.bucket = b;
                    g.exact = ex != 0;
                    g.d_members = (uint32_t *)(T + o_slot[s][0]);
                    g.d_chunk_base = (uint64_t *)(T + o_slot[s][1]);
                    g.d_head = (uint32_t *)(T + o_slot[s][2]);
                }
    std::vector<double> inv;
    inv_table(inv);
    CU(cudaMemcpyAsync((void *)S->d_inv, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, S->stream));
    st = dev_alloc(S->pool_mem, S->budget, S->stream);
    if (st != VP_OK) return st;
    S->pool.reset(S->budget);
    CU(cudaMallocHost(&S->h_done, A * 4));
    CU(cudaStreamSynchronize(S->stream));
    return VP_OK;
}

extern "C" vp_status vp_server_create(const vp_server_config *cfg, void *stream, vp_server **out) {
    if (!out) return fail(VP_EINVAL, "NULL out");
    *out = nullptr;
    vp_server *S = new (std::nothrow) vp_server();
    if (!S) return fail(VP_ENOMEM, "host allocation failed");
    vp_status st = server_init(S, cfg, stream);
    if (st != VP_OK) {
        std::string keep = g_err;
        server_free(S);
        delete S;
        g_err = keep;
        return st;
    }
    *out = S;
    return VP_OK;
}

extern "C" vp_status vp_server_submit(vp_server *S, const vp_request *q, uint64_t *id) {
    CHECK_SRV(S);
    if (!q) return fail(VP_EINVAL, "NULL request");
    std::unique_ptr<Req> r(new (std::nothrow) Req());
    if (!r) return fail(VP_ENOMEM, "host allocation failed");
    vp_status st = validate(&q->p, &q->f, r->mb);
    if (st != VP_OK) return st;
    if (r->mb.n_out > 1) return fail(VP_EINVAL, "served requests take no extra outputs");
    if (!(q->rtol > 0.0 && std::isfinite(q->rtol))) return fail(VP_EINVAL, "rtol must be finite and > 0");
    if (q->discard < 0) return fail(VP_EINVAL, "discard must be >= 0");
    if (q->min_meas < 1) return fail(VP_EINVAL, "min_meas must be >= 1");
    if (r->mb.hist_cap <= q->discard) return fail(VP_EINVAL, "max_it must exceed discard");
    r->rtol = q->rtol;
    r->discard = q->discard;
    r->min_meas = q->min_meas;
    r->tag = q->tag;
    r->bytes = align256(member_layout(r->mb, 0));
    if (r->bytes > S->budget)
        return fail(VP_ENOMEM, "request needs %zu bytes of device state; the budget is %zu", r->bytes,
                    S->budget);
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->werr != VP_OK) {
        g_err = S->werr_msg;
        return S->werr;
    }
    r->id = S->next_id++;
    if (id) *id = r->id;
    S->queue.push_back(std::move(r));
    S->cv_work.notify_one();
    return VP_OK;
}

extern "C" vp_status vp_server_step(vp_server *S, int *n_active) {
    CHECK_SRV(S);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->running) return fail(VP_EINVAL, "the server's worker thread is running");
    }
    return server_step(S, n_active);
}

extern "C" vp_status vp_server_start(vp_server *S) {
    CHECK_SRV(S);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->running) return VP_OK;
    if (S->werr != VP_OK) {
        g_err = S->werr_msg;
        return S->werr;
    }
    S->stop = false;
    S->running = true;
    S->worker = std::thread(worker_main, S);
    return VP_OK;
}

extern "C" vp_status vp_server_stop(vp_server *S) {
    CHECK_SRV(S);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->running) return VP_OK;
        S->stop = true;
        S->cv_work.notify_all();
    }
    S->worker.join();
    std::lock_guard<std::mutex> lk(S->mu);
    S->running = false;
    if (S->werr != VP_OK) {
        g_err = S->werr_msg;
        return S->werr;
    }
    return VP_OK;
}

extern "C" vp_status vp_server_poll(vp_server *S, int max, vp_served *out, int *n) {
    CHECK_SRV(S);
    if (!n || (max > 0 && !out) || max < 0) return fail(VP_EINVAL, "bad poll arguments");
    std::lock_guard<std::mutex> lk(S->mu);
    int k = 0;
    while (k < max && !S->finished.empty()) {
        out[k++] = S->finished.front();
        S->finished.pop_front();
    }
    *n = k;
    if (S->werr != VP_OK) {
        g_err = S->werr_msg;
        return S->werr;
    }
    return VP_OK;
}

extern "C" vp_status vp_server_wait(vp_server *S, int64_t finished, double timeout_s) {
    CHECK_SRV(S);
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(std::max(0.0, timeout_s)));
    const bool ok = S->cv_done.wait_until(lk, until, [&] {
        return S->n_finished >= finished || S->werr != VP_OK;
    });
    if (S->werr != VP_OK) {
        g_err = S->werr_msg;
        return S->werr;
    }
    if (!ok) return fail(VP_ETIMEOUT, "%lld of %lld requests finished", (long long)S->n_finished,
                         (long long)finished);
    return VP_OK;
}

extern "C" vp_status vp_server_get_stats(vp_server *S, vp_server_stats *o) {
    CHECK_SRV(S);
    if (!o) return fail(VP_EINVAL, "NULL out");
    std::lock_guard<std::mutex> lk(S->mu);
    o->submitted = (int64_t)S->next_id;
    o->finished = S->n_finished;
    o->queued = (int64_t)S->queue.size();
    o->active = S->n_active;
    o->steps = S->steps;
    o->bytes_in_use = (int64_t)S->pool.used();
    o->bytes_peak = (int64_t)S->peak;
    o->mem_budget = (int64_t)S->budget;
    o->n_eval = S->n_eval;
    o->busy_s = S->busy;
    return VP_OK;
}

extern "C" double vp_server_clock(void) { return now_s(); }

extern "C" vp_status vp_server_destroy(vp_server *S) {
    if (!S) return VP_OK;
    vp_server_stop(S);
    server_free(S);
    delete S;
    return VP_OK;
}
