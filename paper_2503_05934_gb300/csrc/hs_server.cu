// Serving loop: continuous batching of sort requests under a device-memory
// budget.
//
// Clients submit requests (a device array to sort in place) at any time.  A
// worker thread admits them in arrival order while the budget (the request's
// keys plus the workspace the server reserves for it) fits, and launches
// everything admitted as soon as a stream slot is free:
//   * requests of at most kBatchMaxKeys keys go into one persistent batched
//     launch over descriptors (one CTA per request, network leaves and merge
//     levels, scratch from the server's pool);
//   * longer requests run the multi-CTA merge path (hs_sort_i32) in the same
//     slot.
// Several slots (streams) are in flight at once, so requests that arrive while
// others run are admitted as memory frees up and their work overlaps on the
// GPU.  Completion is reported by a host function enqueued behind each
// slot's work (no polling); latency runs from submit to that report.
//
// The arithmetic is the same as hs_sort_i32 / hs_segsort_i32: a request's
// result does not depend on what it was batched with.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "hs_segsort.h"

struct hs_server;

namespace hs {

using Clock = std::chrono::steady_clock;

constexpr int64_t kBatchMaxKeys = 65536;
constexpr int kSlots = 4;
constexpr int kMaxBatch = 8192;  // requests per batched launch
constexpr size_t kPoolAlign = 256;

struct Req {
    uint64_t ticket;
    int32_t *keys;
    size_t n;
    hs_netset netset;
    Clock::time_point t_submit, t_done;
    size_t budget_bytes;  // keys + reserved workspace
    size_t ws_off = 0, ws_bytes = 0;
    bool done = false;
    hs_status result = HS_OK;
};

// First-fit allocator over the server's workspace pool (host-side metadata).
class Pool {
  public:
    void init(size_t bytes) {
        size_ = bytes;
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = align_up(std::max<size_t>(bytes, 1), kPoolAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(std::max<size_t>(bytes, 1), kPoolAlign);
        auto it = free_.emplace(off, bytes).first;
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

  private:
    size_t size_ = 0;
    std::map<size_t, size_t> free_;
};

struct Slot {
    cudaStream_t stream = nullptr;
    SegDesc *h_desc = nullptr;  // pinned staging
    SegDesc *d_desc = nullptr;
    unsigned long long *d_head = nullptr;
    std::vector<Req *> reqs;
    bool busy = false;
    hs_server *srv = nullptr;
};

}  // namespace hs

struct hs_server {
    int device = 0;
    size_t budget = 0, used = 0;
    char *d_pool = nullptr;
    hs::Pool pool;
    hs::Slot slots[hs::kSlots];
    std::mutex mu;
    std::condition_variable cv_worker, cv_client;
    std::deque<hs::Req *> pending;
    std::vector<hs::Req *> admitted;  // admitted, not yet launched
    std::map<uint64_t, hs::Req *> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::atomic<uint64_t> batches{0}, batched_reqs{0};
};

namespace hs {

static size_t request_ws_bytes(size_t n) {
    // Batched requests need n words of scratch once they exceed one tile;
    // longer requests need the merge path's workspace.
    return (int64_t)n <= kBatchMaxKeys ? align_up(n * sizeof(int32_t), kPoolAlign)
                                       : merge_workspace_bytes(n, 0);
}

static void CUDART_CB on_slot_done(void *arg) {
    Slot *slot = static_cast<Slot *>(arg);
    hs_server *srv = slot->srv;
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    for (Req *r : slot->reqs) {
        r->t_done = now;
        r->done = true;
        srv->pool.release(r->ws_off, r->ws_bytes);
        srv->used -= r->budget_bytes;
    }
    slot->reqs.clear();
    slot->busy = false;
    srv->cv_worker.notify_one();
    srv->cv_client.notify_all();
}

// Issues one slot's work.  Called WITHOUT the server lock: the completion
// callback takes that lock, and a CUDA call blocked behind a full queue must
// never wait for a callback that waits for us.  slot.reqs was set under the
// lock before this call, and the callback is queued last, so it cannot run
// before everything else is issued.
static void issue_slot(hs_server *srv, Slot &slot) {
    const std::vector<Req *> &batch = slot.reqs;
    int nb = 0;
    for (Req *r : batch)
        if ((int64_t)r->n <= kBatchMaxKeys) {
            SegDesc d{};
            d.keys = r->keys;
            d.scratch = reinterpret_cast<int32_t *>(srv->d_pool + r->ws_off);
            d.n = (int64_t)r->n;
            slot.h_desc[nb++] = d;
        }
    hs_status st = HS_OK;
    if (nb > 0) {
        cudaError_t e = cudaMemcpyAsync(slot.d_desc, slot.h_desc, nb * sizeof(SegDesc),
                                        cudaMemcpyHostToDevice, slot.stream);
        if (e != cudaSuccess) st = fail_cuda(e, "server: descriptor copy");
        if (st == HS_OK)
            st = seg_launch_descs(slot.d_desc, nb, slot.d_desc + kMaxBatch, slot.d_head,
                                  default_seg_plan(batch[0]->netset), slot.stream);
        srv->batches.fetch_add(1);
        srv->batched_reqs.fetch_add(nb);
    }
    for (Req *r : batch) {
        if ((int64_t)r->n > kBatchMaxKeys && st == HS_OK)
            st = merge_sort(r->keys, nullptr, r->n, r->netset, srv->d_pool + r->ws_off, r->ws_bytes,
                            slot.stream);
        r->result = st;
    }
    cudaError_t e = cudaLaunchHostFunc(slot.stream, on_slot_done, &slot);
    if (e != cudaSuccess) {
        // The completion report could not be queued: finish synchronously.
        cudaStreamSynchronize(slot.stream);
        for (Req *r : batch) r->result = HS_ERR_CUDA;
        on_slot_done(&slot);
    }
}

static void worker_loop(hs_server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        // Admission in arrival order while the budget and the pool allow.
        while (!srv->pending.empty()) {
            Req *r = srv->pending.front();
            if (srv->used + r->budget_bytes > srv->budget) break;
            size_t off = 0;
            if (!srv->pool.alloc(r->ws_bytes, &off)) break;
            r->ws_off = off;
            srv->used += r->budget_bytes;
            srv->pending.pop_front();
            srv->admitted.push_back(r);
        }
        // Everything admitted goes to one free slot (one network set and at
        // most kMaxBatch batched requests per launch).
        Slot *chosen = nullptr;
        if (!srv->admitted.empty()) {
            for (Slot &slot : srv->slots)
                if (!slot.busy) {
                    chosen = &slot;
                    break;
                }
        }
        if (chosen) {
            std::vector<Req *> batch, rest;
            const hs_netset s0 = srv->admitted.front()->netset;
            int nsmall = 0;
            for (Req *r : srv->admitted) {
                const bool small = (int64_t)r->n <= kBatchMaxKeys;
                if (r->netset == s0 && (!small || nsmall < kMaxBatch)) {
                    batch.push_back(r);
                    nsmall += small;
                } else {
                    rest.push_back(r);
                }
            }
            srv->admitted.swap(rest);
            chosen->reqs = batch;
            chosen->busy = true;
            lk.unlock();
            issue_slot(srv, *chosen);
            lk.lock();
            continue;
        }
        if (srv->stop && srv->pending.empty() && srv->admitted.empty()) {
            bool idle = true;
            for (Slot &slot : srv->slots) idle = idle && !slot.busy;
            if (idle) break;
        }
        srv->cv_worker.wait_for(lk, std::chrono::milliseconds(5));
    }
}

static void destroy_resources(hs_server *srv) {
    for (Slot &slot : srv->slots) {
        if (slot.stream) cudaStreamDestroy(slot.stream);
        if (slot.h_desc) cudaFreeHost(slot.h_desc);
        if (slot.d_desc) cudaFree(slot.d_desc);
        if (slot.d_head) cudaFree(slot.d_head);
    }
    if (srv->d_pool) cudaFree(srv->d_pool);
}

}  // namespace hs

using namespace hs;

extern "C" {

hs_status hs_server_create(size_t budget_bytes, hs_server **out) {
    clear_error();
    if (!out) return fail(HS_ERR_INVALID_ARG, "hs_server_create: NULL result");
    if (budget_bytes < (1u << 20)) return fail(HS_ERR_INVALID_ARG, "hs_server_create: budget below 1 MiB");
    hs_server *srv = new (std::nothrow) hs_server();
    if (!srv) return fail(HS_ERR_NO_MEMORY, "hs_server_create: host allocation");
    srv->budget = budget_bytes;
    cudaError_t e = cudaGetDevice(&srv->device);
    // The pool holds the workspace of admitted requests; it never exceeds the
    // budget, which also counts their keys.
    if (e == cudaSuccess) e = cudaMalloc(&srv->d_pool, budget_bytes);
    for (Slot &slot : srv->slots) {
        if (e != cudaSuccess) break;
        slot.srv = srv;
        e = cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost(&slot.h_desc, kMaxBatch * sizeof(SegDesc));
        // The batch's descriptors, then their classified copy.
        if (e == cudaSuccess) e = cudaMalloc(&slot.d_desc, 2 * kMaxBatch * sizeof(SegDesc));
        if (e == cudaSuccess) e = cudaMalloc(&slot.d_head, 256);
    }
    if (e != cudaSuccess) {
        destroy_resources(srv);
        delete srv;
        return fail_cuda(e, "hs_server_create");
    }
    srv->pool.init(budget_bytes);
    srv->worker = std::thread(worker_loop, srv);
    *out = srv;
    return HS_OK;
}

hs_status hs_server_submit(hs_server *srv, int32_t *d_keys, size_t n, hs_algo a, hs_netset s,
                           uint64_t *ticket) {
    clear_error();
    if (!srv || !ticket) return fail(HS_ERR_INVALID_ARG, "hs_server_submit: NULL argument");
    if (a != HS_ALGO_MERGE)
        return fail(a == HS_ALGO_QUICK ? HS_ERR_UNSUPPORTED : HS_ERR_INVALID_ARG,
                    "hs_server_submit: the server runs the merge path (HS_ALGO_MERGE) only");
    if (!netset_ok(s)) return fail(HS_ERR_INVALID_ARG, "hs_server_submit: netset is neither a set of sizes 3..8 nor a VarSort configuration");
    if (n > 0 && (!d_keys || !aligned(d_keys, 4)))
        return fail(HS_ERR_INVALID_ARG, "hs_server_submit: NULL or unaligned keys");
    Req *r = new (std::nothrow) Req();
    if (!r) return fail(HS_ERR_NO_MEMORY, "hs_server_submit: host allocation");
    r->keys = d_keys;
    r->n = n;
    r->netset = s;
    r->ws_bytes = request_ws_bytes(n);
    r->budget_bytes = align_up(n * sizeof(int32_t), kPoolAlign) + align_up(r->ws_bytes, kPoolAlign);
    if (r->budget_bytes > srv->budget) {
        delete r;
        return fail(HS_ERR_OVER_BUDGET, "hs_server_submit: request needs more than the server budget");
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) {
            delete r;
            return fail(HS_ERR_INVALID_ARG, "hs_server_submit: server is shutting down");
        }
        r->ticket = srv->next_ticket++;
        srv->reqs[r->ticket] = r;
        if (n <= 1) {
            r->done = true;
            r->t_done = r->t_submit;
        } else {
            srv->pending.push_back(r);
        }
        *ticket = r->ticket;
    }
    srv->cv_worker.notify_one();
    return HS_OK;
}

hs_status hs_server_wait(hs_server *srv, uint64_t ticket, hs_status *result, double *latency_s) {
    clear_error();
    if (!srv) return fail(HS_ERR_INVALID_ARG, "hs_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(HS_ERR_INVALID_ARG, "hs_server_wait: unknown ticket");
    Req *r = it->second;
    srv->cv_client.wait(lk, [r] { return r->done; });
    if (result) *result = r->result;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    srv->reqs.erase(it);
    delete r;
    return HS_OK;
}

hs_status hs_server_stats(hs_server *srv, uint64_t *batches, uint64_t *batched_requests,
                          size_t *bytes_in_use) {
    clear_error();
    if (!srv) return fail(HS_ERR_INVALID_ARG, "hs_server_stats: NULL server");
    if (batches) *batches = srv->batches.load();
    if (batched_requests) *batched_requests = srv->batched_reqs.load();
    if (bytes_in_use) {
        std::lock_guard<std::mutex> lk(srv->mu);
        *bytes_in_use = srv->used;
    }
    return HS_OK;
}

hs_status hs_server_replay(hs_server *srv, const double *arrival_s, int32_t *const *d_keys,
                           const size_t *n, size_t count, hs_netset s, double *latency_s,
                           double *makespan_s) {
    clear_error();
    if (!srv || (count && (!arrival_s || !d_keys || !n || !latency_s)))
        return fail(HS_ERR_INVALID_ARG, "hs_server_replay: NULL argument");
    std::vector<uint64_t> tickets(count);
    const Clock::time_point t0 = Clock::now();
    for (size_t i = 0; i < count; ++i) {
        const Clock::time_point due =
            t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
        }
        hs_status st = hs_server_submit(srv, d_keys[i], n[i], HS_ALGO_MERGE, s, &tickets[i]);
        if (st != HS_OK) return st;
    }
    hs_status first = HS_OK;
    for (size_t i = 0; i < count; ++i) {
        hs_status res = HS_OK;
        hs_status st = hs_server_wait(srv, tickets[i], &res, &latency_s[i]);
        if (st != HS_OK) return st;
        if (res != HS_OK && first == HS_OK) first = res;
    }
    if (makespan_s) *makespan_s = std::chrono::duration<double>(Clock::now() - t0).count();
    if (first != HS_OK) return fail(first, "hs_server_replay: a request failed");
    return HS_OK;
}

void hs_server_destroy(hs_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_worker.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    for (Slot &slot : srv->slots)
        if (slot.stream) cudaStreamSynchronize(slot.stream);
    for (auto &kv : srv->reqs) delete kv.second;
    destroy_resources(srv);
    delete srv;
}

}  // extern "C"
