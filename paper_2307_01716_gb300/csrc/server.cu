// Serving loop for the APRIL filter: continuous batching of join requests
// over sets that stay resident in device memory.
//
// A request is a list of candidate pairs in host memory.  april_submit queues
// it; a runtime thread admits queued requests in arrival order whenever a
// stream slot is free and the request's device buffers fit in the memory
// budget (a caller-provided device arena), and enqueues on that slot's stream:
// the copy of the pairs to the device, the batched filter (binning and the
// persistent kernel, with at most one CTA per 256 pairs so that small
// requests leave SMs to the others), and the copy of the verdicts back to the
// caller's host buffer.  Requests on different slots run concurrently on the
// device, so a request that arrives while others are being filtered starts
// as soon as a slot and memory are free instead of waiting for the device to
// drain.  The thread retires finished requests (CUDA event queries; no
// device-side waiting at all), releases their memory and stamps completion
// times.  With one slot the server degenerates to one request per launch.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "april_internal.h"

using april::fail;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

inline uint64_t r256(uint64_t b) { return (b + 255) / 256 * 256; }

struct Request {
    uint64_t ticket = 0;
    const uint32_t *h_r = nullptr, *h_s = nullptr;
    uint8_t *h_out = nullptr;
    uint64_t n = 0;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    april_status status = APRIL_PENDING;
    int slot = -1;
    uint64_t off = 0, bytes = 0;  // arena region
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Request *req = nullptr;
};

// Bytes a request of n pairs needs in the arena: pairs, verdicts, the batched
// mode's scratch and a status word.
uint64_t request_bytes(uint64_t n) {
    size_t sb = 0;
    april_filter_scratch_bytes(APRIL_MODE_BATCHED, n, &sb);
    return 2 * r256(4 * n) + r256(n) + r256(sb) + 256;
}

}  // namespace

struct april_server {
    april_ctx *ctx = nullptr;
    april_dev_sets R{}, S{};
    char *arena = nullptr;
    uint64_t arena_bytes = 0;
    std::vector<Slot> slots;
    uint32_t *h_status = nullptr;  // pinned, one word per slot
    std::map<uint64_t, uint64_t> free_blocks;  // arena offset -> length (first fit, coalesced)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> requests;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    // counters
    uint64_t admitted = 0, completed = 0, max_concurrent = 0, arena_used = 0, arena_peak = 0;

    bool alloc(uint64_t need, uint64_t &off) {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= need) {
                off = it->first;
                const uint64_t rest = it->second - need;
                free_blocks.erase(it);
                if (rest) free_blocks[off + need] = rest;
                arena_used += need;
                arena_peak = std::max(arena_peak, arena_used);
                return true;
            }
        }
        return false;
    }

    void release(uint64_t off, uint64_t len) {
        arena_used -= len;
        auto it = free_blocks.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }

    // Enqueues request q on slot k (lock held).
    april_status launch(Request *q, int k) {
        Slot &sl = slots[k];
        char *base = arena + q->off;
        uint32_t *d_r = (uint32_t *)base;
        uint32_t *d_s = (uint32_t *)(base + r256(4 * q->n));
        uint8_t *d_v = (uint8_t *)(base + 2 * r256(4 * q->n));
        size_t sb = 0;
        april_filter_scratch_bytes(APRIL_MODE_BATCHED, q->n, &sb);
        void *d_scr = base + 2 * r256(4 * q->n) + r256(q->n);
        uint32_t *d_status = (uint32_t *)(base + 2 * r256(4 * q->n) + r256(q->n) + r256(sb));
        cudaStream_t st = sl.stream;
        cudaError_t e = cudaMemcpyAsync(d_r, q->h_r, 4 * q->n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, q->h_s, 4 * q->n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, 4, st);
        if (e != cudaSuccess) return fail(APRIL_ERR_CUDA, std::string("serving copy-in: ") + cudaGetErrorString(e));
        const unsigned max_ctas = (unsigned)std::max<uint64_t>(1, (q->n + 255) / 256);
        april_status rc = april_enqueue_request(ctx, &R, &S, d_r, d_s, q->n, d_v, d_scr, d_status, max_ctas, st);
        if (rc) return rc;
        e = cudaMemcpyAsync(q->h_out, d_v, q->n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status[k], d_status, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
        if (e != cudaSuccess) return fail(APRIL_ERR_CUDA, std::string("serving copy-out: ") + cudaGetErrorString(e));
        return APRIL_OK;
    }

    void run() {
        cudaSetDevice(april_ctx_device(ctx));
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            bool changed = false;
            // retire finished requests
            size_t inflight = 0;
            for (size_t k = 0; k < slots.size(); ++k) {
                Slot &sl = slots[k];
                if (!sl.req) continue;
                const cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaErrorNotReady) {
                    ++inflight;
                    continue;
                }
                Request *r = sl.req;
                r->t_done = now_ns();
                if (q != cudaSuccess) r->status = APRIL_ERR_CUDA;
                else if (h_status[k] & 1u) r->status = APRIL_ERR_OUT_OF_RANGE_ID;
                else r->status = APRIL_OK;
                release(r->off, r->bytes);
                sl.req = nullptr;
                ++completed;
                changed = true;
            }
            // admit in arrival order while a slot and memory are free
            while (!pending.empty()) {
                int k = -1;
                for (size_t s = 0; s < slots.size(); ++s)
                    if (!slots[s].req) {
                        k = (int)s;
                        break;
                    }
                if (k < 0) break;
                Request *q = pending.front();
                uint64_t off = 0;
                if (!alloc(q->bytes, off)) break;  // waits for memory to free up
                pending.pop_front();
                q->off = off;
                q->slot = k;
                q->t_admit = now_ns();
                const april_status rc = launch(q, k);
                if (rc) {
                    q->status = rc;
                    q->t_done = now_ns();
                    release(q->off, q->bytes);
                } else {
                    slots[k].req = q;
                    ++admitted;
                    ++inflight;
                }
                changed = true;
            }
            max_concurrent = std::max<uint64_t>(max_concurrent, inflight);
            if (changed) cv.notify_all();
            if (stop && pending.empty() && inflight == 0) break;
            if (inflight) {
                // device work in flight: check again shortly
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                cv.wait_for(lk, std::chrono::milliseconds(2));
            }
        }
    }
};

extern "C" april_status april_server_create(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                            void *d_arena, size_t arena_bytes, uint32_t max_inflight,
                                            april_server **out) {
    if (!out) return fail(APRIL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx || !R || !S || !d_arena) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (((uintptr_t)d_arena) & 255u) return fail(APRIL_ERR_INVALID_ARG, "arena must be 256-byte aligned");
    if (max_inflight < 1 || max_inflight > 64) return fail(APRIL_ERR_INVALID_ARG, "max_inflight must be 1..64");
    if (R->order != S->order || R->parts != S->parts) return fail(APRIL_ERR_INVALID_ARG, "R and S use different grids");
    if (!R->posts || !S->posts || (((uintptr_t)R->iv | (uintptr_t)S->iv) & 255u))
        return fail(APRIL_ERR_INVALID_ARG, "device sets not laid out by april_upload or april_build_sets_device");
    auto *sv = new april_server();
    sv->ctx = ctx;
    sv->R = *R;
    sv->S = *S;
    sv->arena = (char *)d_arena;
    sv->arena_bytes = arena_bytes & ~255ull;
    sv->free_blocks[0] = sv->arena_bytes;
    cudaError_t e = cudaSetDevice(april_ctx_device(ctx));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sv->h_status, 4 * max_inflight, cudaHostAllocDefault);
    sv->slots.resize(max_inflight);
    for (auto &sl : sv->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        for (auto &sl : sv->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
        }
        if (sv->h_status) cudaFreeHost(sv->h_status);
        delete sv;
        return fail(APRIL_ERR_CUDA, std::string("april_server_create: ") + cudaGetErrorString(e));
    }
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return APRIL_OK;
}

extern "C" april_status april_submit(april_server *sv, const uint32_t *h_r, const uint32_t *h_s, uint64_t n,
                                     uint8_t *h_verdict, uint64_t *ticket) {
    if (!sv || !ticket) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (n && (!h_r || !h_s || !h_verdict)) return fail(APRIL_ERR_INVALID_ARG, "NULL host buffer");
    const uint64_t need = request_bytes(n);
    if (need > sv->arena_bytes)
        return fail(APRIL_ERR_OVER_BUDGET, "request needs more device memory than the server's whole budget");
    auto *q = new Request();
    q->h_r = h_r;
    q->h_s = h_s;
    q->h_out = h_verdict;
    q->n = n;
    q->bytes = need;
    q->t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete q;
            return fail(APRIL_ERR_CANCELLED, "server is shutting down");
        }
        q->ticket = sv->next_ticket++;
        *ticket = q->ticket;
        sv->requests[q->ticket] = q;
        if (n == 0) {
            q->status = APRIL_OK;
            q->t_admit = q->t_done = q->t_submit;
        } else {
            sv->pending.push_back(q);
        }
    }
    sv->cv.notify_all();
    return APRIL_OK;
}

static void fill_stats(const Request *q, april_req_stats *st) {
    if (!st) return;
    st->n_pairs = q->n;
    st->submit_ns = q->t_submit;
    st->admit_ns = q->t_admit;
    st->done_ns = q->t_done;
    st->slot = (uint32_t)q->slot;
    st->status = q->status;
}

extern "C" april_status april_poll(april_server *sv, uint64_t ticket, april_req_stats *stats) {
    if (!sv) return fail(APRIL_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->requests.find(ticket);
    if (it == sv->requests.end()) return fail(APRIL_ERR_INVALID_ARG, "unknown ticket");
    Request *q = it->second;
    if (q->status == APRIL_PENDING) return APRIL_PENDING;
    fill_stats(q, stats);
    const april_status st = q->status;
    sv->requests.erase(it);
    delete q;
    if (st < 0) {
        switch (st) {
            case APRIL_ERR_OUT_OF_RANGE_ID: return fail(st, "the request named an out-of-range object id");
            case APRIL_ERR_CANCELLED: return fail(st, "the request was cancelled");
            default: return fail(st, "the request failed");
        }
    }
    return st;
}

extern "C" april_status april_wait(april_server *sv, uint64_t ticket, uint32_t timeout_ms, april_req_stats *stats) {
    if (!sv) return fail(APRIL_ERR_INVALID_ARG, "server is NULL");
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->requests.find(ticket);
        if (it == sv->requests.end()) return fail(APRIL_ERR_INVALID_ARG, "unknown ticket");
        Request *q = it->second;
        const bool done = sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                          [q] { return q->status != APRIL_PENDING; });
        if (!done) return APRIL_PENDING;
    }
    return april_poll(sv, ticket, stats);
}

extern "C" april_status april_cancel(april_server *sv, uint64_t ticket) {
    if (!sv) return fail(APRIL_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->requests.find(ticket);
    if (it == sv->requests.end()) return fail(APRIL_ERR_INVALID_ARG, "unknown ticket");
    Request *q = it->second;
    auto pit = std::find(sv->pending.begin(), sv->pending.end(), q);
    if (pit == sv->pending.end()) return APRIL_PENDING;  // already on the device (or done): runs to completion
    sv->pending.erase(pit);
    q->status = APRIL_ERR_CANCELLED;
    q->t_done = now_ns();
    sv->cv.notify_all();
    return APRIL_OK;
}

extern "C" april_status april_server_get_info(april_server *sv, april_server_info *info) {
    if (!sv || !info) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    info->admitted = sv->admitted;
    info->completed = sv->completed;
    info->pending = sv->pending.size();
    size_t inflight = 0;
    for (auto &sl : sv->slots) inflight += sl.req != nullptr;
    info->in_flight = inflight;
    info->max_concurrent = sv->max_concurrent;
    info->arena_bytes = sv->arena_bytes;
    info->arena_peak_bytes = sv->arena_peak;
    return APRIL_OK;
}

extern "C" void april_server_destroy(april_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (Request *q : sv->pending) {
            q->status = APRIL_ERR_CANCELLED;
            q->t_done = now_ns();
        }
        sv->pending.clear();
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();  // in-flight requests finish first
    for (auto &sl : sv->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (sv->h_status) cudaFreeHost(sv->h_status);
    for (auto &kv : sv->requests) delete kv.second;
    delete sv;
}
