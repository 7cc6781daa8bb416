// Request server (lc_serve_*): continuous batching of k-NN requests on one GPU.
//
// The index stays resident on the device.  Requests (batches of queries, each with its own k,
// efSearch and mode) wait in arrival order.  Whenever a stream slot is free, the oldest waiting
// request starts, together with every later waiting request that has the same search
// parameters up to efSearch (same k, shortlist, mode, beam, codebook precision, caps and table
// sizes, and an efSearch of the same power-of-two class): their queries are concatenated into
// one launch series in which each query walks with its own request's efSearch (the per-query
// efSearch path of lc_search_ex), so each query's result is exactly what lc_search returns for
// its request alone.  Under light load a request runs alone as soon as it arrives; under heavy
// load the requests that queued while the slots were busy run as a few large launches, which
// keeps the GPU as full as one large batch.  Each launch's device state (queries, per-query
// efSearch, results, search scratch) is sub-allocated first-fit from one arena of the caller's
// budget; the merge is cut short where the arena has no room, and the oldest request waits
// until it fits.  A request whose state alone can never fit is rejected at submission.
// Completion is observed by lc_serve_poll, which invokes each request's callback on the
// polling thread.  The paper has no serving component; this is the library's own.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <thread>

#include "lc_device.h"

namespace {

// Largest merged launch (queries), unless max_request is larger.  Measured at saturation (512-query
// requests, 4 launch slots, up to 96 outstanding): 8,192 / 16,384 / 32,768 gave 12.7 / 13.4 /
// 10.5M queries/s on the 1M workload and 9.0 / 9.5 / 8.2M on the 10M one (the largest cap
// leaves too few requests queued behind a launch to keep the slots busy).
constexpr int MERGE_QUERIES = 16384;

struct Req {
    uint64_t id = 0;
    int nq = 0;
    lc_search_params sp{};
    lc_request_cb cb = nullptr;
    void *user = nullptr;
    std::vector<float> q;
    int efp = 0;                         // max(ef, k)
};

// One launch series: the queries of one or more requests of the same parameter group.
struct Batch {
    std::vector<Req *> reqs;
    int nq = 0;
    lc_search_params sp{};               // the group's parameters; ef = the largest of the batch
    lc::SearchPlan plan;
    size_t need = 0, off = 0;
    // byte offsets of the batch's arrays inside its block
    size_t o_q = 0, o_ef = 0, o_ids = 0, o_d = 0, o_st = 0, o_yq = 0, o_sl = 0, o_sp = 0, o_ord = 0, o_tab = 0, o_hdr = 0;
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

int ceil_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Requests merge only within one group: every search parameter equal except efSearch, whose
// ef' = max(ef, k) must lie in the same power-of-two class (the launch's per-query state is
// sized by the largest ef' of the batch, so mixing small and large walks would shrink the
// number of small walks in flight).
bool same_group(const Req &a, const Req &b)
{
    const lc_search_params &x = a.sp, &y = b.sp;
    return x.k == y.k && x.shortlist == y.shortlist && x.lut_prec == y.lut_prec && x.mode == y.mode &&
           (x.mode != LC_MODE_BATCHED || x.beam == y.beam) && x.visited_log == y.visited_log &&
           x.max_dist == y.max_dist && x.warps == y.warps && x.walk_full == y.walk_full &&
           x.spill_log == y.spill_log && ceil_pow2(std::max(a.efp, 16)) == ceil_pow2(std::max(b.efp, 16));
}

void layout(Batch &b, int d)
{
    const size_t nq = (size_t)b.nq, k = (size_t)b.plan.k;
    size_t o = 0;
    b.o_q = o;   o += al(nq * d * 4);
    b.o_ef = o;  o += al(nq * 4);
    b.o_ids = o; o += al(nq * k * 4);
    b.o_d = o;   o += al(nq * k * 4);
    b.o_st = o;  o += al(nq * 3 * 4);
    b.o_yq = o;  o += al(b.plan.yq_elems * 4);
    b.o_sl = o;  o += al(b.plan.sl_elems * 4);
    b.o_sp = o;  o += al(b.plan.spill_elems * 4);
    b.o_ord = o; o += al(b.plan.ord_elems * 4);
    b.o_tab = o; o += al(b.plan.tab_elems * 2);
    b.o_hdr = o; o += 256;                    // status word and query counter
    b.need = o;
}

}  // namespace

struct lc_server {
    lc_index *ix = nullptr;
    lc::DeviceIndex *dv = nullptr;
    int device = 0;
    size_t budget = 0;
    unsigned char *arena = nullptr;
    std::map<size_t, size_t> free_blocks;      // offset -> size, coalesced
    int max_request = 0;
    int max_merge = 0;                         // queries per launch
    size_t out_cap = 0;                        // result elements (queries x k) per launch
    // pinned staging per slot: queries, per-query efSearch, ids, dists, stats, status word
    size_t h_q = 0, h_ef = 0, h_ids = 0, h_d = 0, h_st = 0, h_word = 0, h_total = 0;
    struct Slot {
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
        unsigned char *host = nullptr;
        Batch *b = nullptr;
    };
    std::vector<Slot> slots;
    std::deque<Req *> queue;
    uint64_t next_id = 1;
};

namespace {

bool arena_alloc(lc_server *s, size_t need, size_t *off)
{
    for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
        if (it->second < need) continue;
        *off = it->first;
        size_t rest = it->second - need, at = it->first + need;
        s->free_blocks.erase(it);
        if (rest) s->free_blocks[at] = rest;
        return true;
    }
    return false;
}

size_t arena_largest(const lc_server *s)
{
    size_t m = 0;
    for (const auto &f : s->free_blocks) m = std::max(m, f.second);
    return m;
}

void arena_free(lc_server *s, size_t off, size_t size)
{
    if (size == 0) return;
    auto it = s->free_blocks.emplace(off, size).first;
    auto nx = std::next(it);
    if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_blocks.erase(nx);
    }
    if (it != s->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_blocks.erase(it);
        }
    }
}

// Launch parameters and device state of a batch of requests (the first request's group).
lc_status plan_batch(lc_server *s, Batch &b)
{
    b.sp = b.reqs[0]->sp;
    int efb = 0;
    b.nq = 0;
    for (const Req *r : b.reqs) {
        efb = std::max(efb, r->efp);
        b.nq += r->nq;
    }
    b.sp.ef = efb;                              // the bound of the per-query efSearch
    lc_status rs = lc::plan_search(s->dv, b.nq, &b.sp, &b.plan, true);
    if (rs != LC_OK) return rs;
    layout(b, s->dv->d);
    return LC_OK;
}

void deliver(lc_server *s, lc_server::Slot &sl, lc_status status)
{
    Batch *b = sl.b;
    const size_t k = (size_t)b->plan.k;
    const int32_t *ids = reinterpret_cast<const int32_t *>(sl.host + s->h_ids);
    const float *ds = reinterpret_cast<const float *>(sl.host + s->h_d);
    const int32_t *st = reinterpret_cast<const int32_t *>(sl.host + s->h_st);
    const int32_t *word = reinterpret_cast<const int32_t *>(sl.host + s->h_word);
    size_t q0 = 0;
    for (Req *r : b->reqs) {
        lc_status rs = status;
        if (rs == LC_OK && *word) {
            // the launch saw an overflow: the requests whose queries overflowed report it
            for (int i = 0; i < r->nq; i++)
                if (st[(q0 + i) * 3] < 0) { rs = LC_ERR_CAPACITY; break; }
        }
        if (r->cb) r->cb(r->user, r->id, rs, ids + q0 * k, ds + q0 * k, r->nq, (int32_t)k);
        q0 += (size_t)r->nq;
        delete r;
    }
    arena_free(s, b->off, b->need);
    sl.b = nullptr;
    delete b;
}

lc_status launch(lc_server *s, lc_server::Slot &sl, Batch *b)
{
    lc::DeviceIndex *dv = s->dv;
    const size_t k = (size_t)b->plan.k, nq = (size_t)b->nq, d = (size_t)dv->d;
    unsigned char *base = s->arena + b->off;
    float *dq = reinterpret_cast<float *>(base + b->o_q);
    int32_t *def = reinterpret_cast<int32_t *>(base + b->o_ef);
    int32_t *dids = reinterpret_cast<int32_t *>(base + b->o_ids);
    float *dd = reinterpret_cast<float *>(base + b->o_d);
    int32_t *dst = reinterpret_cast<int32_t *>(base + b->o_st);
    lc::SearchScratch sc;
    sc.yq = reinterpret_cast<float *>(base + b->o_yq);
    sc.shortlist = reinterpret_cast<int32_t *>(base + b->o_sl);
    sc.spill = reinterpret_cast<int32_t *>(base + b->o_sp);
    sc.ord = reinterpret_cast<int32_t *>(base + b->o_ord);
    sc.tab = reinterpret_cast<uint16_t *>(base + b->o_tab);
    sc.status = reinterpret_cast<int32_t *>(base + b->o_hdr);
    sc.counter = reinterpret_cast<unsigned long long *>(base + b->o_hdr + 8);
    float *hq = reinterpret_cast<float *>(sl.host + s->h_q);
    int32_t *hef = reinterpret_cast<int32_t *>(sl.host + s->h_ef);
    size_t q0 = 0;
    for (const Req *r : b->reqs) {
        std::memcpy(hq + q0 * d, r->q.data(), (size_t)r->nq * d * 4);
        std::fill(hef + q0, hef + q0 + r->nq, r->sp.ef);
        q0 += (size_t)r->nq;
    }
    if (cudaMemcpyAsync(dq, hq, nq * d * 4, cudaMemcpyHostToDevice, sl.st) != cudaSuccess ||
        cudaMemcpyAsync(def, hef, nq * 4, cudaMemcpyHostToDevice, sl.st) != cudaSuccess) {
        lc::set_error("query upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    lc_status rs = lc::run_search(dv, b->plan, dq, b->nq, dids, dd, dst, sc, sl.st, false, nullptr, def);
    if (rs != LC_OK) return rs;
    if (cudaMemcpyAsync(sl.host + s->h_ids, dids, nq * k * 4, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess ||
        cudaMemcpyAsync(sl.host + s->h_d, dd, nq * k * 4, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess ||
        cudaMemcpyAsync(sl.host + s->h_st, dst, nq * 3 * 4, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess ||
        cudaMemcpyAsync(sl.host + s->h_word, sc.status, 4, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess ||
        cudaEventRecord(sl.done, sl.st) != cudaSuccess) {
        lc::set_error("result download failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    return LC_OK;
}

// Starts waiting requests while a slot is free: the oldest one, merged with every later one of
// its group that fits the launch limits and the arena.
void admit(lc_server *s)
{
    while (!s->queue.empty()) {
        lc_server::Slot *free_slot = nullptr;
        for (auto &sl : s->slots)
            if (!sl.b) { free_slot = &sl; break; }
        if (!free_slot) return;
        Batch *b = new (std::nothrow) Batch();
        if (!b) return;
        Req *r0 = s->queue.front();
        const size_t k = (size_t)r0->sp.k;
        int nq = 0;
        for (Req *r : s->queue) {
            if (r != r0 && !same_group(*r0, *r)) continue;
            if (r != r0 && (nq + r->nq > s->max_merge || (size_t)(nq + r->nq) * k > s->out_cap)) continue;
            b->reqs.push_back(r);
            nq += r->nq;
        }
        // the largest prefix of the candidates whose state fits the arena
        const size_t room = arena_largest(s);
        lc_status rs = LC_OK;
        while (!b->reqs.empty()) {
            rs = plan_batch(s, *b);
            if (rs != LC_OK || b->need <= room) break;
            b->reqs.pop_back();
        }
        if (b->reqs.empty() || (rs == LC_OK && !arena_alloc(s, b->need, &b->off))) {
            delete b;                   // the oldest request waits for room
            return;
        }
        for (Req *r : b->reqs) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
        if (rs != LC_OK) {
            // planning failed (each request was planned alone at submission, so a merged plan
            // should not): the batch's requests report it
            for (Req *r : b->reqs) {
                if (r->cb) r->cb(r->user, r->id, rs, nullptr, nullptr, r->nq, r->sp.k);
                delete r;
            }
            delete b;
            continue;
        }
        free_slot->b = b;
        rs = launch(s, *free_slot, b);
        if (rs != LC_OK) {
            // a launch that failed part-way may have queued copies and kernels on the slot's
            // stream that still write the batch's arena range: wait for them before the
            // range is freed and handed to the next batch
            cudaStreamSynchronize(free_slot->st);
            cudaGetLastError();
            deliver(s, *free_slot, rs);
        }
    }
}

}  // namespace

extern "C" {

lc_status lc_serve_open(lc_index *ix, size_t device_budget_bytes, int max_inflight, int max_request,
                        lc_server **out)
{
    lc::set_error("");
    if (!ix || !out) { lc::set_error("null argument"); return LC_ERR_ARG; }
    *out = nullptr;
    if (max_inflight < 1 || max_inflight > 256) { lc::set_error("max_inflight outside 1..256"); return LC_ERR_ARG; }
    if (max_request < 1 || max_request > (1 << 20)) { lc::set_error("max_request outside 1..2^20"); return LC_ERR_ARG; }
    if (device_budget_bytes < 4096) { lc::set_error("device budget below 4 KiB"); return LC_ERR_ARG; }
    if (!ix->trained || (ix->n > 0 && !ix->has_codebook)) { lc::set_error("index is not searchable"); return LC_ERR_STATE; }
    if (ix->n == 0) { lc::set_error("cannot serve an empty index"); return LC_ERR_STATE; }
    lc_status rs = lc::upload(ix);
    if (rs != LC_OK) return rs;
    lc_server *s = new (std::nothrow) lc_server();
    if (!s) { lc::set_error("out of host memory"); return LC_ERR_OOM; }
    s->ix = ix;
    s->dv = ix->dev;
    s->device = ix->dev->device;
    s->budget = device_budget_bytes;
    s->max_request = max_request;
    s->max_merge = std::max(max_request, MERGE_QUERIES);
    s->out_cap = std::max((size_t)max_request * lc::MAX_K, (size_t)s->max_merge * 10);
    const size_t mq = (size_t)s->max_merge, d = (size_t)s->dv->d;
    size_t o = 0;
    s->h_q = o;    o += al(mq * d * 4);
    s->h_ef = o;   o += al(mq * 4);
    s->h_ids = o;  o += al(s->out_cap * 4);
    s->h_d = o;    o += al(s->out_cap * 4);
    s->h_st = o;   o += al(mq * 3 * 4);
    s->h_word = o; o += 256;
    s->h_total = o;
    if (cudaMalloc(&s->arena, device_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        lc::set_error("cudaMalloc of the %zu-byte serving budget failed", device_budget_bytes);
        return LC_ERR_OOM;
    }
    s->free_blocks[0] = device_budget_bytes;
    s->slots.resize(max_inflight);
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&sl.host), s->h_total, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            lc_serve_close(s);
            lc::set_error("could not create the serving streams, events or pinned staging");
            return LC_ERR_OOM;
        }
    }
    *out = s;
    return LC_OK;
}

lc_status lc_serve_submit(lc_server *s, const float *q, int32_t nq, const lc_search_params *sp,
                          lc_request_cb cb, void *user, uint64_t *req_id)
{
    lc::set_error("");
    if (!s || !q || !sp || nq < 1) { lc::set_error("null argument or empty request"); return LC_ERR_ARG; }
    lc_status rs = lc::check_search_params(sp);
    if (rs != LC_OK) return rs;
    if (nq > s->max_request) {
        lc::set_error("request of %d queries exceeds the server's %d", nq, s->max_request);
        return LC_ERR_BUDGET;
    }
    Req *r = new (std::nothrow) Req();
    if (!r) { lc::set_error("out of host memory"); return LC_ERR_OOM; }
    r->nq = nq;
    r->sp = *sp;
    r->cb = cb;
    r->user = user;
    r->efp = std::max(sp->ef, sp->k);
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    // the request's state alone must fit the budget (merged launches are cut to fit)
    Batch alone;
    alone.reqs.push_back(r);
    rs = plan_batch(s, alone);
    if (cur != s->device) cudaSetDevice(cur);
    if (rs != LC_OK) { delete r; return rs; }
    if (alone.need > s->budget) {
        lc::set_error("request needs %zu bytes of device state, more than the %zu-byte budget", alone.need, s->budget);
        delete r;
        return LC_ERR_BUDGET;
    }
    try {
        r->q.assign(q, q + (size_t)nq * s->dv->d);
        r->id = s->next_id++;
        s->queue.push_back(r);
    } catch (const std::bad_alloc &) {
        delete r;
        lc::set_error("out of host memory");
        return LC_ERR_OOM;
    }
    if (req_id) *req_id = r->id;
    if (cur != s->device) cudaSetDevice(s->device);
    admit(s);
    if (cur != s->device) cudaSetDevice(cur);
    return LC_OK;
}

lc_status lc_serve_poll(lc_server *s, int timeout_ms, int *n_completed)
{
    lc::set_error("");
    if (!s) { lc::set_error("null server"); return LC_ERR_ARG; }
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    int done = 0;
    lc_status out = LC_OK;
    for (;;) {
        bool inflight = false;
        for (auto &sl : s->slots) {
            if (!sl.b) continue;
            cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaSuccess) {
                done += (int)sl.b->reqs.size();
                deliver(s, sl, LC_OK);
            } else if (e == cudaErrorNotReady) {
                inflight = true;
            } else {
                cudaGetLastError();
                done += (int)sl.b->reqs.size();
                deliver(s, sl, LC_ERR_CUDA);
                out = LC_ERR_CUDA;
            }
        }
        admit(s);
        for (auto &sl : s->slots) inflight |= sl.b != nullptr;
        if (done > 0 || !inflight || std::chrono::steady_clock::now() >= deadline) break;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (cur != s->device) cudaSetDevice(cur);
    if (n_completed) *n_completed = done;
    return out;
}

lc_status lc_serve_close(lc_server *s)
{
    lc::set_error("");
    if (!s) return LC_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(s->device);
    // requests not yet started are cancelled; those on the device complete normally
    while (!s->queue.empty()) {
        Req *r = s->queue.front();
        s->queue.pop_front();
        if (r->cb) r->cb(r->user, r->id, LC_ERR_STATE, nullptr, nullptr, r->nq, r->sp.k);
        delete r;
    }
    for (auto &sl : s->slots) {
        if (sl.b) {
            cudaError_t e = cudaEventSynchronize(sl.done);
            deliver(s, sl, e == cudaSuccess ? LC_OK : LC_ERR_CUDA);
        }
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.host) cudaFreeHost(sl.host);
    }
    if (s->arena) cudaFree(s->arena);
    cudaSetDevice(cur);
    delete s;
    return LC_OK;
}

}  // extern "C"
