// serve_sync.h -- the serving loop's synchronisation primitives (host only).
//
// SpinLock guards state held for a few dozen instructions (the ring): a
// contended hand-off costs a cache-line transfer, where a sleeping mutex
// would cost a futex wake-up.
//
// SleepSlot is a place to sleep until a condition holds that another thread
// makes true without taking a lock (a request's completion flag, a staged
// request, free ring slots). A sleeper increments `sleepers`, then checks its
// condition under `mu` before each sleep; a waker makes the condition true,
// then reads `sleepers` (both sequentially consistent) and, only when someone
// sleeps, passes through `mu` and notifies. Either the sleeper's check sees
// the condition, or the waker sees the sleeper and its notify finds it
// waiting on `cv` (it cannot slip in between: the sleeper holds `mu` from its
// check until the wait releases it), so no wake-up is lost, and a waker with
// nobody asleep pays one atomic load.
#pragma once

#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>

namespace pll {

class SpinLock {
    std::atomic<bool> held_{false};

  public:
    void lock() {
        for (unsigned spins = 0;;) {
            if (!held_.exchange(true, std::memory_order_acquire)) return;
            while (held_.load(std::memory_order_relaxed))
                if (++spins > 256) std::this_thread::yield();
        }
    }
    void unlock() { held_.store(false, std::memory_order_release); }
};

struct SleepSlot {
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<int> sleepers{0};

    // after making the condition true
    void wake() {
        if (sleepers.load(std::memory_order_seq_cst) == 0) return;
        { std::lock_guard<std::mutex> lock(mu); }
        cv.notify_all();
    }
    // sleep until pred() holds; pred runs under mu
    template <class Pred> void wait(Pred pred) {
        std::unique_lock<std::mutex> lock(mu);
        sleepers.fetch_add(1, std::memory_order_seq_cst);
        cv.wait(lock, pred);
        sleepers.fetch_sub(1, std::memory_order_seq_cst);
    }
    // the same, giving up at `deadline`; returns pred()'s last value
    template <class Pred, class TimePoint> bool wait_until(Pred pred, TimePoint deadline) {
        std::unique_lock<std::mutex> lock(mu);
        sleepers.fetch_add(1, std::memory_order_seq_cst);
        const bool ok = cv.wait_until(lock, deadline, pred);
        sleepers.fetch_sub(1, std::memory_order_seq_cst);
        return ok;
    }
};

}  // namespace pll
