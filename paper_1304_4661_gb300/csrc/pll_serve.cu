// pll_serve.cu -- a request loop serving distance queries from a resident index.
//
// The paper motivates exact distance queries by their use inside interactive,
// latency-sensitive services (Sec. 1); this loop serves Query(s, t) (Sec. 3.3
// with the bit-parallel part of Sec. 5.3) for many clients at once.
//
// Memory. The server owns one ring of P pair slots in pinned, mapped host
// memory that the GPU reads and writes directly (over NVLink-C2C on a GB300;
// no copies): pairs (s, t) as 8 bytes each, results as 1 byte each, 9 P bytes
// in all (pool_bytes). A large ring is cut into up to four parts, each with
// its own lock and FIFO, and a client thread always uses the same part, so
// that clients admitting requests at once rarely meet on one lock. A request
// of q pairs is ADMITTED when q contiguous slots of its part are free:
// pll_server_submit blocks until then, so at most P pairs are ever queued or
// in flight. The client's own thread copies its pairs into its slots
// (checking every id on the way); the slots stay held until the request's
// results are back.
//
// Continuous batching. One dispatcher thread takes, whenever one of `streams`
// stream slots is free, the longest run of staged requests that are waiting
// in a part (arrival order, contiguous in the ring, at most max_batch_pairs
// pairs; the parts in turn) and
// launches it as one unit on that slot's stream: one query launch (k_query,
// reading the run's interleaved pairs in place from the ring and writing its
// results into the ring) between two events.
// Requests that arrive while earlier runs are on the GPU form the next run,
// and runs on different stream slots overlap on the device. Runs retire in
// launch order: their results go to the requests' buffers, each request's
// latency (submit to results delivered, host steady clock) is recorded, and
// their slots return to the ring.
//
// A result does not depend on what it was batched with: each pair is answered
// by its own warp from the immutable index.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pll_internal.cuh"
#include "serve_ring.h"
#include "serve_sync.h"

// Locking. Every request passes through three hands (its client, the
// dispatcher, its waiter), so no lock is held across a sleep and none is
// shared by all of them:
//   * each part of the ring (admission, its FIFO of live requests, its
//     statistics) is guarded by a spin lock held for a few dozen
//     instructions: a contended hand-off is a cache-line transfer, not a
//     futex sleep and wake-up, which would cap the whole server at one
//     request per wake-up latency;
//   * tickets live in 64 shards, each with its own mutex;
//   * completion is a per-request flag; a waiter polls it for a while and
//     only then sleeps on its shard's SleepSlot, which the dispatcher
//     signals only when someone sleeps there.
// A full ring and an idle dispatcher sleep on SleepSlots too; serve_sync.h
// states why no wake-up is lost.

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;      // 0: a rejected request that still holds its slots
    uint64_t off = 0, q = 0;  // its ring slots [off, off + q)
    uint8_t *out = nullptr;
    Clock::time_point t_submit;
    double latency_us = 0;
    int status = PLL_OK;
    bool waiting = false;               // a pll_server_wait holds it (shard lock)
    std::atomic<bool> staged{false};    // set by the client once its pairs are in place
    std::atomic<bool> done{false};      // set by the dispatcher once its results are delivered
};

struct Run {
    std::vector<Request *> reqs;  // consecutive in the ring
    uint64_t off = 0, pairs = 0;
    int slot = -1, part = 0;
    int fail = PLL_OK;  // a launch that failed: retired with this status, in order
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    bool busy = false;  // dispatcher thread only
};

using pll::SleepSlot;
using pll::SpinLock;

struct alignas(64) Shard {
    SleepSlot slot;  // its mutex also guards the map
    std::unordered_map<uint64_t, Request *> map;
};

// One part of the pair ring: slots [base, base + cap).
struct alignas(64) RingPart {
    SpinLock lock;                    // guards the fields up to `dispatch`
    uint64_t base = 0, cap = 0;
    std::deque<Request *> live;       // hold slots of this part, ring order
    size_t nlaunched = 0;             // live[0, nlaunched) belong to launched runs
    uint64_t next_seq = 0;            // tickets issued here: part + 1 + seq * parts
    uint64_t requests = 0, pairs = 0, max_inflight_bytes = 0;
    SleepSlot space;                  // clients waiting for free slots here
    alignas(64) std::atomic<uint64_t> staged_seq{0};  // bumped by every staged request
    // dispatcher thread only
    uint64_t seen_seq = ~0ull;
    bool leftover = false;            // staged requests a run did not take (size, wrap)
};

constexpr int SHARDS = 64;
constexpr uint32_t MAX_PARTS = 4;

double us_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

std::atomic<uint32_t> g_client_threads{0};

// the part a client thread uses: threads are dealt out in turn
uint32_t client_part(uint32_t parts) {
    thread_local const uint32_t id = g_client_threads.fetch_add(1, std::memory_order_relaxed);
    return id % parts;
}

}  // namespace

struct pll_server {
    const pll_index *ix = nullptr;
    int device = 0;
    pll_server_opts opts{};
    uint64_t P = 0;                   // ring slots (pairs)
    uint64_t max_request = 0;         // largest request accepted
    uint32_t *h_pairs = nullptr;      // pinned, mapped [P][2]
    uint8_t *h_out = nullptr;         // pinned, mapped [P]
    uint32_t *g_pairs = nullptr;      // the same memory as the GPU addresses it
    uint8_t *g_out = nullptr;
    std::vector<Slot> slots;
    std::deque<Run> inflight;         // dispatcher thread only, launch order
    double device_us = 0;             // dispatcher thread only
    uint32_t nparts = 1, next_part = 0;  // next_part: dispatcher only
    std::unique_ptr<RingPart[]> parts;
    // ---- the dispatcher's statistics (batches, sizes, times)
    SpinLock stats_lock;
    pll_server_stats st{};
    // ---- tickets
    Shard shards[SHARDS];
    // ---- an idle dispatcher sleeps here
    SleepSlot work;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::atomic<unsigned long long> pack_ns{0};  // client staging time (no lock)
    int fatal = PLL_OK;

    Shard &shard(uint64_t ticket) { return shards[ticket % SHARDS]; }
    uint64_t staged_sum() const {
        uint64_t x = 0;
        for (uint32_t p = 0; p < nparts; ++p) x += parts[p].staged_seq.load(std::memory_order_seq_cst);
        return x;
    }
};

namespace {

// Slots for q pairs in a part's FIFO ring of live requests (serve_ring.h);
// offsets are the ring's own.
bool ring_alloc(const RingPart &rp, uint64_t q, uint64_t *off) {
    uint64_t rel = 0;
    bool ok;
    if (rp.live.empty()) {
        ok = pll::ring_place(true, 0, 0, 0, rp.cap, q, &rel);
    } else {
        const Request *f = rp.live.front(), *b = rp.live.back();
        ok = pll::ring_place(false, f->off - rp.base, b->off - rp.base, b->off + b->q - rp.base, rp.cap, q, &rel);
    }
    *off = rp.base + rel;
    return ok;
}

uint64_t ring_used(const RingPart &rp) {
    if (rp.live.empty()) return 0;
    const uint64_t first = rp.live.front()->off;
    const uint64_t end = rp.live.back()->off + rp.live.back()->q;
    return rp.live.back()->off >= first ? end - first : rp.cap - (first - end);
}

int launch_run(pll_server *sv, const Run &r) {
    const Slot &sl = sv->slots[r.slot];
    const uint32_t *gp = sv->g_pairs + 2 * r.off;
    PLL_TRY(cudaEventRecord(sl.start, sl.stream));
    PLL_CHECK(pll::query_launch_strided(sv->ix, gp, gp + 1, 2, r.pairs, sv->g_out + r.off, sl.stream));
    PLL_TRY(cudaEventRecord(sl.done, sl.stream));
    return PLL_OK;
}

// Deliver a run's results, return its slots to the ring, then mark its
// requests done (a waiter may free a request the moment it sees the flag, so
// the ring lets go of them first).
void retire_run(pll_server *sv, const Run &r, int status) {
    const Clock::time_point t0 = Clock::now();
    if (status == PLL_OK)
        for (const Request *q : r.reqs)  // the caller's buffer is ours until done is set
            if (q->ticket) std::memcpy(q->out, sv->h_out + q->off, q->q);
    const Clock::time_point now = Clock::now();
    sv->slots[r.slot].busy = false;
    RingPart &rp = sv->parts[r.part];
    rp.lock.lock();
    for (size_t i = 0; i < r.reqs.size(); ++i) rp.live.pop_front();
    rp.nlaunched -= r.reqs.size();
    rp.lock.unlock();
    sv->stats_lock.lock();
    sv->st.unpack_us += us_between(t0, now);
    sv->st.device_us = sv->device_us;
    sv->stats_lock.unlock();
    rp.space.wake();
    for (Request *q : r.reqs) {
        if (q->ticket == 0) { delete q; continue; }
        Shard &sh = sv->shard(q->ticket);
        q->latency_us = us_between(q->t_submit, now);
        q->status = status;
        q->done.store(true, std::memory_order_seq_cst);  // q may be gone after this
        sh.slot.wake();
    }
}

// The longest run of staged requests waiting at the head of a part (taken
// out of the part's unlaunched requests); empty if the first is not staged.
Run take_run(pll_server *sv, RingPart &rp) {
    Run run;
    rp.lock.lock();
    if (rp.nlaunched < rp.live.size() && rp.live[rp.nlaunched]->staged.load(std::memory_order_acquire)) {
        run.off = rp.live[rp.nlaunched]->off;
        for (size_t i = rp.nlaunched; i < rp.live.size(); ++i) {
            Request *q = rp.live[i];
            if (!q->staged.load(std::memory_order_acquire) || q->off != run.off + run.pairs)
                break;  // not staged, or wrapped
            if (!run.reqs.empty() && run.pairs + q->q > sv->opts.max_batch_pairs) break;
            run.reqs.push_back(q);
            run.pairs += q->q;
        }
        rp.nlaunched += run.reqs.size();
    }
    rp.leftover = rp.nlaunched < rp.live.size() && rp.live[rp.nlaunched]->staged.load(std::memory_order_acquire);
    rp.lock.unlock();
    return run;
}

void worker_loop(pll_server *sv) {
    cudaSetDevice(sv->device);
    // after work the dispatcher polls for SPIN_US before it sleeps: a thread
    // woken from sleep adds tens of microseconds
    constexpr int SPIN_US = 1000;
    Clock::time_point last_work = Clock::now();
    for (;;) {
        // 1. retire finished runs, oldest first
        while (!sv->inflight.empty()) {
            const Run &r = sv->inflight.front();
            if (r.fail != PLL_OK) {  // its event was never recorded
                retire_run(sv, r, r.fail);
                sv->inflight.pop_front();
                continue;
            }
            const Slot &sl = sv->slots[r.slot];
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady) break;
            float ms = 0;
            if (e == cudaSuccess && cudaEventElapsedTime(&ms, sl.start, sl.done) == cudaSuccess)
                sv->device_us += 1e3 * ms;
            if (e != cudaSuccess) sv->fatal = PLL_E_CUDA;
            retire_run(sv, r, e == cudaSuccess ? PLL_OK : PLL_E_CUDA);
            sv->inflight.pop_front();
            last_work = Clock::now();
        }
        // 2. while a stream slot is free, launch the staged requests of the
        // parts in turn, one run each; a part is looked at only when requests
        // were staged there since the last look, or some were left over
        bool launched = false;
        for (uint32_t k = 0; k < sv->nparts; ++k) {
            int slot = -1;
            for (size_t i = 0; i < sv->slots.size(); ++i)
                if (!sv->slots[i].busy) { slot = (int)i; break; }
            if (slot < 0) break;
            const uint32_t p = sv->next_part;
            sv->next_part = (p + 1) % sv->nparts;
            RingPart &rp = sv->parts[p];
            const uint64_t seq = rp.staged_seq.load(std::memory_order_seq_cst);
            if (seq == rp.seen_seq && !rp.leftover) continue;
            rp.seen_seq = seq;
            Run run = take_run(sv, rp);
            if (run.reqs.empty()) continue;
            run.slot = slot;
            run.part = (int)p;
            sv->stats_lock.lock();
            sv->st.batches++;
            sv->st.max_batch_pairs = std::max(sv->st.max_batch_pairs, run.pairs);
            sv->stats_lock.unlock();
            sv->slots[slot].busy = true;
            const int s = launch_run(sv, run);
            if (s != PLL_OK) {
                // nothing of the run is in flight once the stream drains; it
                // retires behind the runs launched before it (requests leave
                // the ring in order)
                cudaStreamSynchronize(sv->slots[slot].stream);
                sv->fatal = s;
                run.fail = s;
            }
            sv->inflight.push_back(std::move(run));
            last_work = Clock::now();
            launched = true;
        }
        if (launched || !sv->inflight.empty()) {
            if (!launched) std::this_thread::yield();
            continue;
        }
        // 3. nothing in flight and nothing launched: stop, or sleep a while.
        // The staged count is read before the parts are looked at, so a
        // request staged after the look changes it and ends the sleep.
        const uint64_t seen = sv->staged_sum();
        bool empty = true, ready = false;
        for (uint32_t p = 0; p < sv->nparts; ++p) {
            RingPart &rp = sv->parts[p];
            rp.lock.lock();
            empty = empty && rp.live.empty();
            ready = ready || rp.leftover ||
                    (rp.nlaunched < rp.live.size() && rp.live[rp.nlaunched]->staged.load(std::memory_order_acquire));
            rp.lock.unlock();
        }
        if (ready) {
            for (uint32_t p = 0; p < sv->nparts; ++p) sv->parts[p].leftover = true;  // look again
            continue;
        }
        if (sv->stop.load(std::memory_order_seq_cst) && empty) return;
        if (Clock::now() - last_work > std::chrono::microseconds(SPIN_US)) {
            sv->work.wait_until(
                [&] { return sv->stop.load(std::memory_order_seq_cst) || sv->staged_sum() != seen; },
                Clock::now() + std::chrono::milliseconds(2));
        } else {
            std::this_thread::yield();
        }
    }
}

void destroy(pll_server *sv) {
    for (Slot &sl : sv->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.start) cudaEventDestroy(sl.start);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (sv->h_pairs) cudaFreeHost(sv->h_pairs);
    // a request is in its part's `live` until its run retires, and in its
    // shard from staging until it is waited for: completed ones are only in a
    // shard
    for (Shard &sh : sv->shards)
        for (auto &kv : sh.map)
            if (kv.second->done.load()) delete kv.second;
    if (sv->parts)
        for (uint32_t p = 0; p < sv->nparts; ++p)
            for (Request *r : sv->parts[p].live) delete r;
    delete sv;
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
    const uint64_t P = o.pool_bytes / 9;
    if (o.streams > 64 || P == 0) return PLL_E_INVAL;
    pll_server *sv = new (std::nothrow) pll_server();
    if (!sv) return PLL_E_NOMEM;
    sv->ix = idx;
    sv->opts = o;
    sv->device = idx->device;
    sv->P = P;
    // parts only where each still holds two of the largest runs
    sv->nparts = (uint32_t)std::min<uint64_t>(MAX_PARTS, std::max<uint64_t>(1, P / (2 * o.max_batch_pairs)));
    sv->parts.reset(new (std::nothrow) RingPart[sv->nparts]);
    if (!sv->parts) { delete sv; return PLL_E_NOMEM; }
    for (uint32_t p = 0; p < sv->nparts; ++p) {
        sv->parts[p].base = P / sv->nparts * p;
        sv->parts[p].cap = p + 1 < sv->nparts ? P / sv->nparts : P - P / sv->nparts * p;
    }
    sv->max_request = std::min<uint64_t>(o.max_batch_pairs, P / sv->nparts);
    sv->st.pool_bytes = 9 * P;
    sv->st.max_request_pairs = sv->max_request;
    cudaError_t e = cudaSetDevice(sv->device);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&sv->h_pairs), 9 * P, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&sv->g_pairs), sv->h_pairs, 0);
    if (e == cudaSuccess) {
        sv->h_out = reinterpret_cast<uint8_t *>(sv->h_pairs + 2 * P);
        sv->g_out = reinterpret_cast<uint8_t *>(sv->g_pairs + 2 * P);
        sv->slots.resize(o.streams);
        for (Slot &sl : sv->slots) {
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreate(&sl.start);
            if (e == cudaSuccess) e = cudaEventCreate(&sl.done);
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
    if (q > sv->max_request) return PLL_E_RANGE;
    Request *r = new (std::nothrow) Request();
    if (!r) return PLL_E_NOMEM;
    r->q = q;
    r->out = out;
    r->t_submit = Clock::now();
    const uint32_t part = client_part(sv->nparts);
    RingPart &rp = sv->parts[part];
    // admission: q contiguous slots of this thread's part, else sleep until a
    // run of the part retires
    auto try_admit = [&] {
        uint64_t off = 0;
        rp.lock.lock();
        const bool ok = ring_alloc(rp, q, &off);
        if (ok) {
            r->off = off;
            r->ticket = part + 1 + rp.next_seq++ * sv->nparts;
            rp.live.push_back(r);
            rp.max_inflight_bytes = std::max(rp.max_inflight_bytes, 9 * ring_used(rp));
            rp.requests++;
            rp.pairs += q;
        }
        rp.lock.unlock();
        return ok;
    };
    for (bool admitted = false; !admitted;) {
        if (sv->stop.load(std::memory_order_seq_cst)) { delete r; return PLL_E_INVAL; }
        if (try_admit()) break;
        rp.space.wait_until(
            [&] { return sv->stop.load(std::memory_order_seq_cst) || (admitted = try_admit()); },
            Clock::now() + std::chrono::milliseconds(10));
    }
    const uint64_t tk = r->ticket;
    Shard &sh = sv->shard(tk);
    {
        std::lock_guard<std::mutex> lock(sh.slot.mu);
        sh.map[tk] = r;
    }
    // stage the pairs into the request's own slots, checking the ids on the way
    const Clock::time_point t0 = Clock::now();
    const uint32_t n = sv->ix->n;
    uint32_t *h = sv->h_pairs + 2 * r->off;
    uint32_t bad = 0;
    for (uint64_t i = 0; i < q; ++i) {
        const uint32_t a = src[i], b = dst[i];
        bad |= (uint32_t)(a >= n) | (uint32_t)(b >= n);
        h[2 * i] = a < n ? a : 0;
        h[2 * i + 1] = b < n ? b : 0;
    }
    if (bad) {  // keeps its slots until its run retires, answers nobody
        std::lock_guard<std::mutex> lock(sh.slot.mu);
        sh.map.erase(tk);
        r->ticket = 0;
    }
    sv->pack_ns.fetch_add((unsigned long long)(us_between(t0, Clock::now()) * 1e3), std::memory_order_relaxed);
    r->staged.store(true, std::memory_order_release);  // pairs and ticket before the flag
    rp.staged_seq.fetch_add(1, std::memory_order_seq_cst);
    sv->work.wake();
    if (bad) return PLL_E_INVAL;
    *ticket = tk;
    return PLL_OK;
}

PLL_API int pll_server_wait(pll_server *sv, uint64_t ticket, int64_t timeout_us, double *latency_us) {
    if (!sv) return PLL_E_INVAL;
    Shard &sh = sv->shard(ticket);
    Request *r = nullptr;
    bool finished = false;
    {
        std::lock_guard<std::mutex> lock(sh.slot.mu);
        auto it = sh.map.find(ticket);
        if (it == sh.map.end() || it->second->waiting) return PLL_E_INVAL;
        r = it->second;
        finished = r->done.load(std::memory_order_seq_cst);
        if (finished) sh.map.erase(it);  // done already: released in the same visit
        else r->waiting = true;          // no other wait may release it meanwhile
    }
    auto done = [r] { return r->done.load(std::memory_order_seq_cst); };
    if (finished) {
        if (latency_us) *latency_us = r->latency_us;
        const int s = r->status;
        delete r;
        return s;
    }
    {
        // poll for up to SPIN_US (a run is usually tens of microseconds from
        // retiring), then sleep until the dispatcher signals the shard
        constexpr int64_t SPIN_US = 50;
        const Clock::time_point t0 = Clock::now();
        const int64_t spin = timeout_us < 0 ? SPIN_US : std::min<int64_t>(SPIN_US, timeout_us);
        while (!done() && Clock::now() - t0 < std::chrono::microseconds(spin)) std::this_thread::yield();
        if (!done()) {
            bool ok = true;
            if (timeout_us < 0) sh.slot.wait(done);
            else ok = sh.slot.wait_until(done, t0 + std::chrono::microseconds(timeout_us));
            if (!ok) {
                std::lock_guard<std::mutex> lock(sh.slot.mu);
                r->waiting = false;
                return PLL_E_TIMEOUT;
            }
        }
    }
    if (latency_us) *latency_us = r->latency_us;
    const int s = r->status;
    {
        std::lock_guard<std::mutex> lock(sh.slot.mu);
        sh.map.erase(ticket);
    }
    delete r;
    return s;
}

PLL_API int pll_server_replay(pll_server *sv, const uint32_t *src, const uint32_t *dst,
                              const uint64_t *req_off, const double *arrival_us, uint64_t count,
                              uint32_t threads, uint8_t *out, double *latency_us,
                              double *elapsed_us) {
    if (!sv || !req_off || threads > 64 ||
        (count > 0 && (!src || !dst || !out || !arrival_us || !latency_us)))
        return PLL_E_INVAL;
    for (uint64_t i = 0; i < count; ++i)
        if (req_off[i + 1] <= req_off[i] || (i > 0 && arrival_us[i] < arrival_us[i - 1]))
            return PLL_E_INVAL;
    if (threads == 0) threads = 1;
    // client thread k submits requests k, k + threads, ... at their arrival
    // times; collector c of C waits for requests c, c + C, ... in order
    std::vector<uint64_t> tickets(count, 0);
    std::unique_ptr<std::atomic<uint8_t>[]> posted(new (std::nothrow) std::atomic<uint8_t>[count ? count : 1]);
    if (!posted) return PLL_E_NOMEM;
    for (uint64_t i = 0; i < count; ++i) posted[i].store(0, std::memory_order_relaxed);
    std::atomic<int> first_err{PLL_OK};
    auto note = [&first_err](int s) {
        int ok = PLL_OK;
        if (s != PLL_OK) first_err.compare_exchange_strong(ok, s);
    };
    for (uint64_t i = 0; i < count; ++i) latency_us[i] = -1;
    const Clock::time_point t0 = Clock::now();
    auto client = [&](uint32_t k) {
        for (uint64_t i = k; i < count; i += threads) {
            const Clock::time_point due = t0 + std::chrono::duration_cast<Clock::duration>(
                                                   std::chrono::duration<double, std::micro>(arrival_us[i]));
            for (Clock::time_point now = Clock::now(); now < due; now = Clock::now())
                if (due - now > std::chrono::microseconds(200))
                    std::this_thread::sleep_for(due - now - std::chrono::microseconds(100));
            if (first_err.load() == PLL_OK) {
                const uint64_t a = req_off[i], q = req_off[i + 1] - a;
                note(pll_server_submit(sv, src + a, dst + a, q, out + a, &tickets[i]));
            }
            posted[i].store(1, std::memory_order_release);
        }
    };
    // one collector per four clients: releasing a ticket costs about as much
    // host time as submitting a small request
    const uint32_t C = std::max<uint32_t>(1, threads / 4);
    auto collector = [&](uint32_t c) {
        for (uint64_t i = c; i < count; i += C) {
            while (!posted[i].load(std::memory_order_acquire)) std::this_thread::yield();
            if (tickets[i] != 0) note(pll_server_wait(sv, tickets[i], -1, &latency_us[i]));
        }
    };
    std::vector<std::thread> pool;
    uint32_t started = 1, collectors = 0;  // client 0 runs on this thread
    try {
        for (; started < threads; ++started) pool.emplace_back(client, started);
        for (; collectors < C; ++collectors) pool.emplace_back(collector, collectors);
    } catch (...) {
        note(PLL_E_NOMEM);
    }
    // clients or collectors that could not be started run here, after client
    // 0 (with the error noted, those clients only mark their requests posted),
    // so nothing is left waiting on `posted`
    client(0);
    for (uint32_t k = started; k < threads; ++k) client(k);
    for (uint32_t c = collectors; c < C; ++c) collector(c);
    for (std::thread &th : pool) th.join();
    if (elapsed_us) *elapsed_us = us_between(t0, Clock::now());
    return first_err.load();
}

PLL_API int pll_server_get_stats(pll_server *sv, pll_server_stats *out) {
    if (!sv || !out) return PLL_E_INVAL;
    sv->stats_lock.lock();
    *out = sv->st;
    sv->stats_lock.unlock();
    out->requests = out->pairs = out->max_inflight_bytes = 0;
    for (uint32_t p = 0; p < sv->nparts; ++p) {  // the parts' peaks, summed
        RingPart &rp = sv->parts[p];
        rp.lock.lock();
        out->requests += rp.requests;
        out->pairs += rp.pairs;
        out->max_inflight_bytes += rp.max_inflight_bytes;
        rp.lock.unlock();
    }
    out->pack_us = sv->pack_ns.load(std::memory_order_relaxed) / 1e3;
    return PLL_OK;
}

PLL_API int pll_server_stop(pll_server *sv) {
    if (!sv) return PLL_OK;
    sv->stop.store(true, std::memory_order_seq_cst);
    sv->work.wake();
    for (uint32_t p = 0; p < sv->nparts; ++p) sv->parts[p].space.wake();
    if (sv->worker.joinable()) sv->worker.join();
    const int s = sv->fatal;
    destroy(sv);
    return s;
}

}  // extern "C"
