// Random admit / retire sequences against the serving ring's slot placement
// (pll::ring_place), checked against a model of the live blocks:
//   - every placed block lies inside the ring and meets no live block;
//   - blocks leave in the order they entered (the live blocks keep the
//     one-or-two-run shape ring_place assumes);
//   - a refusal happens only when neither allowed region holds q slots;
//   - with nothing live, any q up to the ring's size is placed at 0.
// Prints "ok <placements>" and exits 0, or prints the first violation and
// exits 1.
#include <cstdint>
#include <cstdio>
#include <deque>
#include <random>
#include <utility>

#include "serve_ring.h"

struct Block {
    uint64_t off, q;
};

static bool overlaps(uint64_t a0, uint64_t a1, uint64_t b0, uint64_t b1) { return a0 < b1 && b0 < a1; }

int main() {
    std::mt19937_64 rng(12345);
    uint64_t placed = 0;
    for (int trial = 0; trial < 200; ++trial) {
        const uint64_t cap = 1 + rng() % 5000;
        std::deque<Block> live;
        for (int step = 0; step < 4000; ++step) {
            const bool admit = live.empty() || rng() % 3 != 0;
            if (!admit) {
                live.pop_front();
                continue;
            }
            const uint64_t q = 1 + rng() % (rng() % 4 == 0 ? cap : (cap / 8 + 1));
            uint64_t off = ~0ull;
            const bool ok = live.empty()
                                ? pll::ring_place(true, 0, 0, 0, cap, q, &off)
                                : pll::ring_place(false, live.front().off, live.back().off,
                                                  live.back().off + live.back().q, cap, q, &off);
            if (live.empty() && q <= cap && !(ok && off == 0)) {
                std::printf("empty ring refused q=%llu cap=%llu\n", (unsigned long long)q,
                            (unsigned long long)cap);
                return 1;
            }
            if (!ok) {
                // a refusal: neither allowed region holds q slots
                if (q <= cap && !live.empty()) {
                    const uint64_t first = live.front().off, bo = live.back().off,
                                   be = live.back().off + live.back().q;
                    const bool fits = bo >= first ? (cap - be >= q || first >= q) : (first - be >= q);
                    if (fits) {
                        std::printf("refused although a region fits\n");
                        return 1;
                    }
                }
                continue;
            }
            if (off + q > cap) {
                std::printf("block [%llu, %llu) outside the ring of %llu\n", (unsigned long long)off,
                            (unsigned long long)(off + q), (unsigned long long)cap);
                return 1;
            }
            for (const Block &b : live)
                if (overlaps(off, off + q, b.off, b.off + b.q)) {
                    std::printf("block [%llu, %llu) meets live [%llu, %llu)\n", (unsigned long long)off,
                                (unsigned long long)(off + q), (unsigned long long)b.off,
                                (unsigned long long)(b.off + b.q));
                    return 1;
                }
            live.push_back({off, q});
            ++placed;
            // the live blocks form one run, or two with the second starting at 0
            int wraps = 0;
            for (size_t i = 1; i < live.size(); ++i)
                if (live[i].off < live[i - 1].off) ++wraps;
            if (wraps > 1) {
                std::printf("live blocks wrapped twice\n");
                return 1;
            }
        }
    }
    std::printf("ok %llu\n", (unsigned long long)placed);
    return 0;
}
