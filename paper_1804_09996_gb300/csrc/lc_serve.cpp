// Request server (lc_serve_*): continuous batching of k-NN requests on one GPU.
//
// The index stays resident on the device.  Each request (a batch of queries with its own k,
// efSearch and mode) needs device state for its queries, results and search scratch; the
// server owns one device arena of the caller's budget and sub-allocates that state first-fit.
// Requests are admitted in arrival order as soon as a stream slot and enough of the budget are
// free, so requests that arrive while others run start alongside them and their kernels
// overlap on the device.  A request whose state can never fit the budget is rejected at
// submission.  Completion is observed by lc_serve_poll, which invokes the request's callback
// on the polling thread.  The paper has no serving component; this is the library's own.
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <thread>

#include "lc_device.h"

namespace {

struct Req {
    uint64_t id = 0;
    int nq = 0;
    lc_search_params sp{};
    lc_request_cb cb = nullptr;
    void *user = nullptr;
    std::vector<float> q;
    lc::SearchPlan plan;
    size_t need = 0, off = 0;
    // byte offsets of the request's arrays inside its block
    size_t o_q = 0, o_ids = 0, o_d = 0, o_st = 0, o_yq = 0, o_sl = 0, o_sp = 0, o_hdr = 0;
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

void layout(Req &r, int d)
{
    const size_t nq = (size_t)r.nq, k = (size_t)r.plan.k;
    size_t o = 0;
    r.o_q = o;   o += al(nq * d * 4);
    r.o_ids = o; o += al(nq * k * 4);
    r.o_d = o;   o += al(nq * k * 4);
    r.o_st = o;  o += al(nq * 3 * 4);
    r.o_yq = o;  o += al(r.plan.yq_elems * 4);
    r.o_sl = o;  o += al(r.plan.sl_elems * 4);
    r.o_sp = o;  o += al(r.plan.spill_elems * 4);
    r.o_hdr = o; o += 256;                    // status word and query counter
    r.need = o;
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
    size_t host_q = 0, host_out = 0;           // pinned staging per slot: queries, results
    struct Slot {
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
        unsigned char *host = nullptr;
        Req *req = nullptr;
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

void arena_free(lc_server *s, size_t off, size_t size)
{
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

void deliver(lc_server *s, lc_server::Slot &sl, lc_status status)
{
    Req *r = sl.req;
    const size_t k = (size_t)r->plan.k;
    const int32_t *ids = reinterpret_cast<const int32_t *>(sl.host + s->host_q);
    const float *ds = reinterpret_cast<const float *>(sl.host + s->host_q + (size_t)s->max_request * lc::MAX_K * 4);
    const int32_t *word = reinterpret_cast<const int32_t *>(sl.host + s->host_q + (size_t)s->max_request * lc::MAX_K * 8);
    if (status == LC_OK && *word) status = LC_ERR_CAPACITY;
    if (r->cb) r->cb(r->user, r->id, status, ids, ds, r->nq, (int32_t)k);
    arena_free(s, r->off, r->need);
    sl.req = nullptr;
    delete r;
}

lc_status launch(lc_server *s, lc_server::Slot &sl, Req *r)
{
    lc::DeviceIndex *dv = s->dv;
    const size_t k = (size_t)r->plan.k, nq = (size_t)r->nq;
    unsigned char *base = s->arena + r->off;
    float *dq = reinterpret_cast<float *>(base + r->o_q);
    int32_t *dids = reinterpret_cast<int32_t *>(base + r->o_ids);
    float *dd = reinterpret_cast<float *>(base + r->o_d);
    int32_t *dst = reinterpret_cast<int32_t *>(base + r->o_st);
    lc::SearchScratch sc;
    sc.yq = reinterpret_cast<float *>(base + r->o_yq);
    sc.shortlist = reinterpret_cast<int32_t *>(base + r->o_sl);
    sc.spill = reinterpret_cast<int32_t *>(base + r->o_sp);
    sc.status = reinterpret_cast<int32_t *>(base + r->o_hdr);
    sc.counter = reinterpret_cast<unsigned long long *>(base + r->o_hdr + 8);
    std::memcpy(sl.host, r->q.data(), nq * dv->d * 4);
    unsigned char *ho = sl.host + s->host_q;
    if (cudaMemcpyAsync(dq, sl.host, nq * dv->d * 4, cudaMemcpyHostToDevice, sl.st) != cudaSuccess) {
        lc::set_error("query upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    lc_status rs = lc::run_search(dv, r->plan, dq, r->nq, dids, dd, dst, sc, sl.st, false);
    if (rs != LC_OK) return rs;
    cudaMemcpyAsync(ho, dids, nq * k * 4, cudaMemcpyDeviceToHost, sl.st);
    cudaMemcpyAsync(ho + (size_t)s->max_request * lc::MAX_K * 4, dd, nq * k * 4, cudaMemcpyDeviceToHost, sl.st);
    cudaMemcpyAsync(ho + (size_t)s->max_request * lc::MAX_K * 8, sc.status, 4, cudaMemcpyDeviceToHost, sl.st);
    if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) {
        lc::set_error("event record failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    sl.req = r;
    return LC_OK;
}

// Starts queued requests, in arrival order, while a slot and room in the arena are free.
void admit(lc_server *s)
{
    while (!s->queue.empty()) {
        lc_server::Slot *free_slot = nullptr;
        for (auto &sl : s->slots)
            if (!sl.req) { free_slot = &sl; break; }
        if (!free_slot) return;
        Req *r = s->queue.front();
        if (!arena_alloc(s, r->need, &r->off)) return;
        s->queue.pop_front();
        lc_status rs = launch(s, *free_slot, r);
        if (rs != LC_OK) {
            // a launch that failed part-way may have queued copies and kernels on the slot's
            // stream that still write the request's arena range: wait for them before the
            // range is freed and handed to the next request
            cudaStreamSynchronize(free_slot->st);
            cudaGetLastError();
            free_slot->req = r;
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
    s->host_q = al((size_t)max_request * s->dv->d * 4);
    s->host_out = (size_t)max_request * lc::MAX_K * 8 + 256;
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
            cudaHostAlloc(reinterpret_cast<void **>(&sl.host), s->host_q + s->host_out, cudaHostAllocDefault) != cudaSuccess) {
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
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    rs = lc::plan_search(s->dv, nq, sp, &r->plan);
    if (cur != s->device) cudaSetDevice(cur);
    if (rs != LC_OK) { delete r; return rs; }
    layout(*r, s->dv->d);
    if (r->need > s->budget) {
        lc::set_error("request needs %zu bytes of device state, more than the %zu-byte budget", r->need, s->budget);
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
            if (!sl.req) continue;
            cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaSuccess) {
                deliver(s, sl, LC_OK);
                done++;
            } else if (e == cudaErrorNotReady) {
                inflight = true;
            } else {
                cudaGetLastError();
                deliver(s, sl, LC_ERR_CUDA);
                done++;
                out = LC_ERR_CUDA;
            }
        }
        admit(s);
        for (auto &sl : s->slots) inflight |= sl.req != nullptr;
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
        if (r->cb) r->cb(r->user, r->id, LC_ERR_STATE, nullptr, nullptr, r->nq, r->plan.k);
        delete r;
    }
    for (auto &sl : s->slots) {
        if (sl.req) {
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
