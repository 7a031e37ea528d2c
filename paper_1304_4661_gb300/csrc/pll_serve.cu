// pll_serve.cu -- a request loop serving distance queries from a resident index.
//
// The paper motivates exact distance queries by their use inside interactive,
// latency-sensitive services (Sec. 1); this loop serves Query(s, t) (Sec. 3.3
// with the bit-parallel part of Sec. 5.3) for many clients at once.
//
// Requests (pairs in host memory) are queued by pll_server_submit. One
// dispatcher thread runs continuous batching:
//   * admission by memory: a batch needs 9 bytes per pair on the device
//     (source, target, result, each block 256-byte aligned); it is admitted
//     when that fits in the free part of a FIFO ring over a fixed device
//     pool, so at most pool_bytes of query data are ever in flight;
//   * as soon as one of `streams` stream slots is free, the waiting requests
//     (in arrival order, up to max_batch_pairs and what the ring holds) are
//     packed into that slot's pinned staging, copied to the device, answered
//     by one query launch (k_query, one warp per pair) and copied back, all on
//     the slot's stream; requests that arrive while earlier batches run on the
//     GPU join the next batch, and batches on different slots overlap;
//   * completion is detected with CUDA events, in launch order; results go to
//     each request's output buffer and its latency (submit to completion on
//     the host's steady clock) is recorded.
// A result does not depend on what it was batched with: each pair is answered
// by its own warp from the immutable index.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pll_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const uint32_t *src = nullptr, *dst = nullptr;
    uint64_t q = 0;
    uint8_t *out = nullptr;
    Clock::time_point t_submit;
    double latency_us = 0;
    bool done = false;
    int status = PLL_OK;
};

struct Batch {
    std::vector<Request *> reqs;
    uint64_t pairs = 0;
    uint64_t ring_off = 0, ring_bytes = 0;
    int slot = -1;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint32_t *h_src = nullptr, *h_dst = nullptr;  // pinned staging
    uint8_t *h_out = nullptr;
    bool busy = false;
};

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }
uint64_t batch_bytes(uint64_t q) { return 2 * align256(4 * q) + align256(q); }

}  // namespace

struct pll_server {
    const pll_index *ix = nullptr;
    int device = 0;
    pll_server_opts opts{};
    unsigned char *pool = nullptr;  // device ring of opts.pool_bytes
    std::vector<Slot> slots;
    std::deque<Batch> inflight;     // dispatcher thread only; launch order == ring order
    uint64_t inflight_bytes = 0;
    std::mutex mu;                  // guards everything below
    std::condition_variable cv_submit, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> table;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    pll_server_stats st{};
    int fatal = PLL_OK;
};

namespace {

// First-fit allocation in a FIFO ring over the device pool. Batches hold
// [off, off + bytes) until they retire, oldest first, so the live blocks are
// the in-flight batches in order: one run [front.off, back end), or two once
// the ring has wrapped (back.off < front.off).
bool ring_alloc(const std::deque<Batch> &live, uint64_t cap, uint64_t bytes, uint64_t *off) {
    if (bytes > cap) return false;
    if (live.empty()) { *off = 0; return true; }
    const uint64_t first = live.front().ring_off;
    const uint64_t end = live.back().ring_off + live.back().ring_bytes;
    if (live.back().ring_off >= first) {  // not wrapped: free [end, cap) and [0, first)
        if (cap - end >= bytes) { *off = end; return true; }
        if (first >= bytes) { *off = 0; return true; }
        return false;
    }
    if (first - end >= bytes) { *off = end; return true; }  // wrapped: free [end, first)
    return false;
}

int launch_batch(pll_server *sv, const Batch &b) {
    Slot &sl = sv->slots[b.slot];
    uint64_t p = 0;
    for (const Request *r : b.reqs) {
        std::memcpy(sl.h_src + p, r->src, r->q * 4);
        std::memcpy(sl.h_dst + p, r->dst, r->q * 4);
        p += r->q;
    }
    unsigned char *base = sv->pool + b.ring_off;
    uint32_t *d_src = reinterpret_cast<uint32_t *>(base);
    uint32_t *d_dst = reinterpret_cast<uint32_t *>(base + align256(4 * b.pairs));
    uint8_t *d_out = base + 2 * align256(4 * b.pairs);
    PLL_TRY(cudaMemcpyAsync(d_src, sl.h_src, b.pairs * 4, cudaMemcpyHostToDevice, sl.stream));
    PLL_TRY(cudaMemcpyAsync(d_dst, sl.h_dst, b.pairs * 4, cudaMemcpyHostToDevice, sl.stream));
    PLL_CHECK(pll::query_launch(sv->ix, d_src, d_dst, b.pairs, d_out, sl.stream));
    PLL_TRY(cudaMemcpyAsync(sl.h_out, d_out, b.pairs, cudaMemcpyDeviceToHost, sl.stream));
    PLL_TRY(cudaEventRecord(sl.done, sl.stream));
    return PLL_OK;
}

void finish_batch(pll_server *sv, const Batch &b, int status) {
    Slot &sl = sv->slots[b.slot];
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lock(sv->mu);
    uint64_t p = 0;
    for (Request *r : b.reqs) {
        if (status == PLL_OK) std::memcpy(r->out, sl.h_out + p, r->q);
        p += r->q;
        r->latency_us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
        r->status = status;
        r->done = true;
    }
    sl.busy = false;
    sv->cv_done.notify_all();
}

void worker_loop(pll_server *sv) {
    cudaSetDevice(sv->device);
    const uint64_t cap = sv->opts.pool_bytes;
    for (;;) {
        // 1. retire finished batches, oldest first
        while (!sv->inflight.empty()) {
            const Batch &b = sv->inflight.front();
            const cudaError_t e = cudaEventQuery(sv->slots[b.slot].done);
            if (e == cudaErrorNotReady) break;
            if (e != cudaSuccess) sv->fatal = PLL_E_CUDA;
            finish_batch(sv, b, e == cudaSuccess ? PLL_OK : PLL_E_CUDA);
            sv->inflight_bytes -= b.ring_bytes;
            sv->inflight.pop_front();
        }
        // 2. with a free stream slot, admit waiting requests into one batch
        int slot = -1;
        for (size_t i = 0; i < sv->slots.size(); ++i)
            if (!sv->slots[i].busy) { slot = (int)i; break; }
        Batch b;
        bool quit = false;
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            if (sv->pending.empty() && sv->inflight.empty()) {
                if (sv->stop) quit = true;
                else sv->cv_submit.wait_for(lock, std::chrono::milliseconds(2),
                                            [&] { return sv->stop || !sv->pending.empty(); });
            }
            if (!quit && slot >= 0 && !sv->pending.empty()) {
                uint64_t pairs = 0;
                size_t take = 0;
                for (const Request *r : sv->pending) {
                    if (take > 0 && pairs + r->q > sv->opts.max_batch_pairs) break;
                    pairs += r->q;
                    ++take;
                }
                uint64_t off = 0;
                while (take > 0 && !ring_alloc(sv->inflight, cap, batch_bytes(pairs), &off))
                    pairs -= sv->pending[--take]->q;  // shrink until the block fits
                if (take > 0) {
                    b.reqs.assign(sv->pending.begin(), sv->pending.begin() + take);
                    sv->pending.erase(sv->pending.begin(), sv->pending.begin() + take);
                    b.pairs = pairs;
                    b.ring_off = off;
                    b.ring_bytes = batch_bytes(pairs);
                    b.slot = slot;
                    sv->slots[slot].busy = true;
                    sv->st.batches++;
                    sv->st.max_batch_pairs = std::max(sv->st.max_batch_pairs, pairs);
                    sv->st.max_inflight_bytes =
                        std::max(sv->st.max_inflight_bytes, sv->inflight_bytes + b.ring_bytes);
                }
            }
        }
        if (quit) return;
        if (b.slot >= 0) {
            const int s = launch_batch(sv, b);
            if (s != PLL_OK) {  // nothing of the batch is in flight once the stream drains
                cudaStreamSynchronize(sv->slots[b.slot].stream);
                sv->fatal = s;
                finish_batch(sv, b, s);
                continue;
            }
            sv->inflight_bytes += b.ring_bytes;
            sv->inflight.push_back(std::move(b));
        } else if (!sv->inflight.empty()) {
            std::this_thread::yield();
        }
    }
}

void destroy(pll_server *sv) {
    for (Slot &sl : sv->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.h_src) cudaFreeHost(sl.h_src);
        if (sl.h_dst) cudaFreeHost(sl.h_dst);
        if (sl.h_out) cudaFreeHost(sl.h_out);
    }
    if (sv->pool) cudaFree(sv->pool);
    for (auto &kv : sv->table) delete kv.second;
    delete sv;
}

int check_ids(const uint32_t *v, uint64_t q, uint32_t n) {
    for (uint64_t i = 0; i < q; ++i)
        if (v[i] >= n) return PLL_E_INVAL;
    return PLL_OK;
}

}  // namespace

extern "C" {

PLL_API int pll_server_start(const pll_index *idx, const pll_server_opts *opts, pll_server **out) {
    if (!idx || !out) return PLL_E_INVAL;
    *out = nullptr;
    pll_server_opts o{};
    if (opts) o = *opts;
    if (o.reserved != 0) return PLL_E_INVAL;
    if (o.pool_bytes == 0) o.pool_bytes = 256ull << 20;
    if (o.max_batch_pairs == 0) o.max_batch_pairs = 1u << 20;
    if (o.streams == 0) o.streams = 4;
    if (o.streams > 64 || o.pool_bytes < batch_bytes(1)) return PLL_E_INVAL;
    // a batch never holds more pairs than the pool has room for
    uint64_t fit = o.pool_bytes / 9;
    while (fit > 0 && batch_bytes(fit) > o.pool_bytes) --fit;
    o.max_batch_pairs = std::min<uint64_t>(o.max_batch_pairs, fit);
    pll_server *sv = new (std::nothrow) pll_server();
    if (!sv) return PLL_E_NOMEM;
    sv->ix = idx;
    sv->opts = o;
    sv->device = idx->device;
    sv->st.pool_bytes = o.pool_bytes;
    sv->st.max_request_pairs = o.max_batch_pairs;
    cudaError_t e = cudaSetDevice(sv->device);
    if (e == cudaSuccess) e = cudaMalloc(&sv->pool, o.pool_bytes);
    if (e == cudaSuccess) {
        sv->slots.resize(o.streams);
        for (Slot &sl : sv->slots) {
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMallocHost(&sl.h_src, o.max_batch_pairs * 4);
            if (e == cudaSuccess) e = cudaMallocHost(&sl.h_dst, o.max_batch_pairs * 4);
            if (e == cudaSuccess) e = cudaMallocHost(&sl.h_out, o.max_batch_pairs);
        }
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        destroy(sv);
        return e == cudaErrorMemoryAllocation ? PLL_E_NOMEM : pll::cuda_status(e);
    }
    try {
        sv->worker = std::thread(worker_loop, sv);
    } catch (...) {
        destroy(sv);
        return PLL_E_NOMEM;
    }
    *out = sv;
    return PLL_OK;
}

PLL_API int pll_server_submit(pll_server *sv, const uint32_t *src, const uint32_t *dst, uint64_t q,
                              uint8_t *out, uint64_t *ticket) {
    if (!sv || !ticket || q == 0 || !src || !dst || !out) return PLL_E_INVAL;
    *ticket = 0;
    if (q > sv->opts.max_batch_pairs) return PLL_E_RANGE;
    PLL_CHECK(check_ids(src, q, sv->ix->n));
    PLL_CHECK(check_ids(dst, q, sv->ix->n));
    Request *r = new (std::nothrow) Request();
    if (!r) return PLL_E_NOMEM;
    r->src = src;
    r->dst = dst;
    r->q = q;
    r->out = out;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (sv->stop) { delete r; return PLL_E_INVAL; }
        r->ticket = sv->next_ticket++;
        r->t_submit = Clock::now();
        sv->table[r->ticket] = r;
        sv->pending.push_back(r);
        sv->st.requests++;
        sv->st.pairs += q;
    }
    sv->cv_submit.notify_one();
    *ticket = r->ticket;
    return PLL_OK;
}

PLL_API int pll_server_wait(pll_server *sv, uint64_t ticket, int64_t timeout_us, double *latency_us) {
    if (!sv) return PLL_E_INVAL;
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->table.find(ticket);
    if (it == sv->table.end()) return PLL_E_INVAL;
    Request *r = it->second;
    auto ready = [r] { return r->done; };
    if (timeout_us < 0) sv->cv_done.wait(lock, ready);
    else if (!sv->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready))
        return PLL_E_TIMEOUT;
    if (latency_us) *latency_us = r->latency_us;
    const int s = r->status;
    sv->table.erase(it);
    delete r;
    return s;
}

PLL_API int pll_server_replay(pll_server *sv, const uint32_t *src, const uint32_t *dst,
                              const uint64_t *req_off, const double *arrival_us, uint64_t count,
                              uint8_t *out, double *latency_us, double *elapsed_us) {
    if (!sv || !req_off || (count > 0 && (!src || !dst || !out || !arrival_us || !latency_us)))
        return PLL_E_INVAL;
    for (uint64_t i = 0; i < count; ++i)
        if (req_off[i + 1] <= req_off[i] || (i > 0 && arrival_us[i] < arrival_us[i - 1]))
            return PLL_E_INVAL;
    std::vector<uint64_t> tickets(count, 0);
    std::atomic<uint64_t> submitted{0};
    std::atomic<int> first_err{PLL_OK};
    auto note = [&first_err](int s) {
        int ok = PLL_OK;
        if (s != PLL_OK) first_err.compare_exchange_strong(ok, s);
    };
    for (uint64_t i = 0; i < count; ++i) latency_us[i] = -1;
    std::thread collector;
    try {
        collector = std::thread([&] {
            for (uint64_t i = 0; i < count; ++i) {
                while (submitted.load(std::memory_order_acquire) <= i) std::this_thread::yield();
                if (tickets[i] != 0) note(pll_server_wait(sv, tickets[i], -1, &latency_us[i]));
            }
        });
    } catch (...) {
        return PLL_E_NOMEM;
    }
    const Clock::time_point t0 = Clock::now();
    for (uint64_t i = 0; i < count; ++i) {
        const Clock::time_point due = t0 + std::chrono::duration_cast<Clock::duration>(
                                               std::chrono::duration<double, std::micro>(arrival_us[i]));
        for (Clock::time_point now = Clock::now(); now < due; now = Clock::now())
            if (due - now > std::chrono::microseconds(200))
                std::this_thread::sleep_for(due - now - std::chrono::microseconds(100));
        if (first_err.load() == PLL_OK) {
            const uint64_t a = req_off[i], q = req_off[i + 1] - a;
            note(pll_server_submit(sv, src + a, dst + a, q, out + a, &tickets[i]));
        }
        submitted.store(i + 1, std::memory_order_release);
    }
    collector.join();
    if (elapsed_us) *elapsed_us = std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    return first_err.load();
}

PLL_API int pll_server_get_stats(pll_server *sv, pll_server_stats *out) {
    if (!sv || !out) return PLL_E_INVAL;
    std::lock_guard<std::mutex> lock(sv->mu);
    *out = sv->st;
    return PLL_OK;
}

PLL_API int pll_server_stop(pll_server *sv) {
    if (!sv) return PLL_OK;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
    }
    sv->cv_submit.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    const int s = sv->fatal;
    destroy(sv);
    return s;
}

}  // extern "C"
