// Stress check of the serving loop's synchronisation primitives
// (paper_1304_4661_gb300/csrc/serve_sync.h), host only. Built by
// tests/test_serve_sync.py, with ThreadSanitizer where the compiler has it.
//
// 1. SpinLock: threads add to a plain counter under the lock; the total must
//    be exact (and ThreadSanitizer must see no race on it).
// 2. SleepSlot, as the server uses it for completions: completer threads
//    write a request's result into plain fields, set its flag (sequentially
//    consistent) and wake the request's slot; waiter threads poll a flag for
//    a few rounds, then sleep on the slot. A lost wake-up would leave a waiter
//    asleep until its deadline (5 s): every wait must end well before it, and
//    every result must be the one written.
// 3. SleepSlot as the ring's free-space wait: producers take tokens from a
//    bounded pool (sleeping when it is empty), a consumer returns them; the
//    run must finish with every token back.
//
// Prints "ok <operations>" or a reason and exits non-zero.
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <memory>
#include <thread>
#include <vector>

#include "serve_sync.h"

using Clock = std::chrono::steady_clock;

namespace {

struct Req {
    uint64_t value = 0;  // written by the completer before `done`
    std::atomic<bool> done{false};
};

uint64_t mix(uint64_t x) {  // splitmix64's finaliser: a result to compare
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

bool check_spinlock(uint64_t *ops) {
    pll::SpinLock lock;
    uint64_t counter = 0;
    constexpr int T = 6, N = 20000;
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t)
        th.emplace_back([&] {
            for (int i = 0; i < N; ++i) {
                lock.lock();
                ++counter;
                lock.unlock();
            }
        });
    for (auto &x : th) x.join();
    *ops += (uint64_t)T * N;
    if (counter != (uint64_t)T * N) {
        std::printf("spinlock: counter %llu, expected %llu\n", (unsigned long long)counter,
                    (unsigned long long)T * N);
        return false;
    }
    return true;
}

bool check_completions(uint64_t *ops) {
    constexpr int R = 40000, SLOTS = 16, C = 3, W = 3;
    std::unique_ptr<Req[]> req(new Req[R]);
    std::unique_ptr<pll::SleepSlot[]> slot(new pll::SleepSlot[SLOTS]);
    std::atomic<int> slow{0}, wrong{0};
    std::vector<std::thread> th;
    for (int c = 0; c < C; ++c)
        th.emplace_back([&, c] {
            for (int i = c; i < R; i += C) {
                if ((mix(i) & 7) == 0) std::this_thread::yield();  // let waiters fall asleep
                req[i].value = mix(i);
                req[i].done.store(true, std::memory_order_seq_cst);
                slot[i % SLOTS].wake();
            }
        });
    for (int w = 0; w < W; ++w)
        th.emplace_back([&, w] {
            for (int i = w; i < R; i += W) {
                Req &r = req[i];
                auto done = [&r] { return r.done.load(std::memory_order_seq_cst); };
                for (int spin = 0; spin < (int)(mix(i + 1) & 3) && !done(); ++spin)
                    std::this_thread::yield();
                if (!done()) {
                    const Clock::time_point t0 = Clock::now();
                    slot[i % SLOTS].wait_until(done, t0 + std::chrono::seconds(5));
                    if (Clock::now() - t0 > std::chrono::seconds(1)) slow.fetch_add(1);
                }
                if (r.value != mix(i)) wrong.fetch_add(1);
            }
        });
    for (auto &x : th) x.join();
    *ops += R;
    if (slow.load() || wrong.load()) {
        std::printf("completions: %d waits reached their deadline, %d wrong results\n", slow.load(),
                    wrong.load());
        return false;
    }
    return true;
}

bool check_space(uint64_t *ops) {
    constexpr int P = 3, N = 20000, POOL = 4;
    pll::SleepSlot space;
    pll::SpinLock lock;
    int free_tokens = POOL;  // guarded by lock
    std::atomic<int> taken{0}, returned{0}, stalls{0};
    auto try_take = [&] {
        lock.lock();
        const bool ok = free_tokens > 0;
        if (ok) --free_tokens;
        lock.unlock();
        return ok;
    };
    std::vector<std::thread> th;
    for (int p = 0; p < P; ++p)
        th.emplace_back([&] {
            for (int i = 0; i < N; ++i) {
                for (bool got = try_take(); !got;) {
                    const Clock::time_point t0 = Clock::now();
                    space.wait_until([&] { return got = try_take(); }, t0 + std::chrono::seconds(5));
                    if (Clock::now() - t0 > std::chrono::seconds(1)) stalls.fetch_add(1);
                }
                taken.fetch_add(1);
            }
        });
    th.emplace_back([&] {  // the consumer: returns tokens as they are taken
        while (returned.load() < P * N) {
            if (returned.load() < taken.load()) {
                lock.lock();
                ++free_tokens;
                lock.unlock();
                returned.fetch_add(1);
                space.wake();
            } else {
                std::this_thread::yield();
            }
        }
    });
    for (auto &x : th) x.join();
    *ops += (uint64_t)P * N;
    if (stalls.load() || free_tokens != POOL) {
        std::printf("space: %d waits reached their deadline, %d tokens free of %d\n", stalls.load(),
                    free_tokens, POOL);
        return false;
    }
    return true;
}

}  // namespace

int main() {
    uint64_t ops = 0;
    if (!check_spinlock(&ops) || !check_completions(&ops) || !check_space(&ops)) return 1;
    std::printf("ok %llu\n", (unsigned long long)ops);
    return 0;
}
