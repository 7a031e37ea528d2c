// k_pruned.cu -- pruned BFSs (Alg. 1) for a batch of roots [k0, k0 + B).
//
// Alg. 2 runs Alg. 1 for k = 1..n one after another: the BFS from v_k is
// pruned at u when Query(v_k, u, L'_{k-1}) <= P[u]. Here a whole batch of
// roots runs at once and each root is pruned only with the labels of hubs
// < k0 (finished batches) plus the bit-parallel labels (Sec. 5.4). That
// emits a superset of the entries Alg. 1 would add; the cleanup pass in
// k_labels.cu removes exactly the surplus (an entry (u, k, d) is surplus iff
// an in-batch hub h < k lies on a shortest k-u path, and then both (h, .) in
// L(v_k) and (h, .) in L(u) were emitted by this batch). The result is the
// label set of the sequential algorithm for any batch size.
//
// The BFSs of all roots of the batch advance level by level together, as
// bulk-synchronous sweeps over one flat frontier of (root slot, vertex)
// pairs, so the work of a level is spread over the whole GPU whatever the
// mix of large and small BFSs:
//
//   init    per root: the level-0 entry (v_k, k, 0) (the root is never
//           pruned: Query(v_k, v_k) >= 2 for v_k outside X), its visited bit,
//           a hash table of its label L(v_k) -- the root array T of Sec.
//           4.5.1 ("Querying"), so a prune test costs O(|L(u)|) probes -- and
//           two 64-bit feasibility masks over the bit-parallel roots.
//   expand  one warp per entry (u, k, d) of the level: read u's neighbours 32
//           per step and look each one up in the root's visited row (a bitmap
//           [B][ceil(n / 32)], one row per root of the batch: the per-root
//           visited set of Alg. 1, one bit per vertex, so the 32 lanes of a
//           warp, which share the root, read neighbouring words). For a
//           neighbour w not yet visited, the lane first runs the cheap part of
//           the prune test (it decides ~90% of them on power-law graphs) and
//           claims w with an atomicOr only if w survives it. A vertex the
//           bit-parallel labels prune stays unmarked: the bit-parallel bound
//           of a pair does not depend on the level, so if it prunes w at level
//           d + 1 it prunes w again at any later level where w is reached, and
//           leaving the bit clear changes no label. The test: bit-parallel
//           distances only -- with
//           d~_i = d(v_k,r_i) + d(r_i,w), some d~_i <= d + 1 prunes (Sec. 5.3:
//           the distance through {r_i} U S_{r_i} is at most d~_i). Rows of t
//           bytes (padded to 16) arrive in 16-byte loads, four roots per
//           instruction (saturating byte add, byte compare). The lane also
//           records which roots could still reach the bound with their masks:
//           d~_i = d + 2 needs a reduction of 1 (possible only if S^{-1}(v_k)
//           or S^0(v_k) is non-empty), d~_i = d + 3 needs the S^{-1}
//           intersection (S^{-1}(v_k) non-empty). The lane then checks the
//           masks of the first QUICK roots itself: roots come in rank order,
//           so these are the largest hubs and they decide most mask tests.
//           Survivors are claimed; freshly claimed (slot, w) pairs and the
//           remaining feasible roots are the next level's candidates.
//   test    the rest of the test, one WARP per candidate so that lanes work
//           in parallel instead of a few lanes looping alone: each lane first
//           loads its own candidate's label offsets (32 candidates' loads in
//           flight at once), then for each candidate in turn the lanes take
//           the feasible bit-parallel roots (two each) and compare mask pairs;
//           if none prunes, they take L(w)'s entries 32 at a time and probe
//           the root's hash table. Survivors are appended as (w, k, d + 1).
//   clear   after the batch, the lazy reset of Sec. 4.5.1 ("Initialization"):
//           the only bits set are those of the roots and of the recorded
//           candidates, so their words are zeroed and nothing else is touched
//           (instead of clearing B * n / 8 bytes per batch).
//
// Level boundaries live in a device descriptor advanced by a one-thread
// kernel, so the host enqueues several levels ahead and reads back only to
// learn that the frontier is empty; sweeps over an empty range return at once.
#include <cub/cub.cuh>

#include "pll_internal.cuh"

namespace pll {
namespace {

#ifndef LABEL_ROUNDS
#define LABEL_ROUNDS 4
#endif
#ifndef LABEL_ROUNDS_LOOP
#define LABEL_ROUNDS_LOOP 2
#endif
#ifndef LONG_LABEL_ENTRIES
#define LONG_LABEL_ENTRIES 64
#endif

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t HT_EMPTY = 0xffffffffu;

// Slot of hub rank h in a table of mask + 1 = 2^lg slots (lg >= 5): the top lg
// bits of a two-multiply mix of h. Hub ranks of one graph in a batch share
// their low bits (ranks interleave the graphs), so an unmixed product would
// crowd them into few slots.
__device__ __forceinline__ uint32_t ht_slot(uint32_t h, uint32_t mask) {
    uint32_t x = h * 0x9E3779B1u;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    const uint32_t lg = 31 - __clz(mask + 1);
    return x >> (32 - lg);
}

// warp-aggregated append: returns this lane's slot (valid where want is true)
__device__ __forceinline__ unsigned long long warp_append(unsigned long long *counter, bool want,
                                                          int lane) {
    const unsigned m = __ballot_sync(FULL, want);
    unsigned long long base = 0;
    const int leader = m ? __ffs(m) - 1 : 0;
    if (m && lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
    base = __shfl_sync(FULL, base, leader);
    return base + __popc(m & ((1u << lane) - 1u));
}

// Bit of hub rank h in a root's 1024-bit filter: the top 10 bits of the same
// kind of mix as ht_slot (hub ranks of a batch build share their low bits).
__device__ __forceinline__ uint32_t filt_bit(uint32_t h) {
    uint32_t x = h * 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    return x >> 22;
}

__global__ void k_batch_init(BatchArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < a.B; slot += warps) {
        const uint32_t k = a.k0 + slot;
        if (a.inX[k]) continue;  // bit-parallel vertices get no pruned BFS
        if (lane == 0) {
            const unsigned long long pos = atomicAdd(&a.ctr->out_n, 1ull);
            if (pos < a.out_cap) a.out[pos] = pack_tuple(k, k, 0);
            else atomicOr(&a.ctr->err, ERR_BUF);
            atomicOr(&a.visited[(size_t)slot * a.NW + (k >> 5)], 1u << (k & 31));
        }
        // feasibility masks over the bit-parallel roots
        uint64_t h1 = 0, h01 = 0;
        for (uint32_t i0 = 0; i0 < a.t; i0 += 32) {
            const uint32_t i = i0 + lane;
            uint64_t k1 = 0, kz = 0;
            if (i < a.t) {
                const ulonglong2 m = reinterpret_cast<const ulonglong2 *>(a.bp_m)[(size_t)k * a.t + i];
                k1 = m.x;
                kz = m.y;
            }
            h1 |= (uint64_t)__ballot_sync(FULL, k1 != 0) << i0;
            h01 |= (uint64_t)__ballot_sync(FULL, (k1 | kz) != 0) << i0;
        }
        if (lane == 0) {
            a.rootbits[2 * slot] = h1;
            a.rootbits[2 * slot + 1] = h01;
        }
        // a 1024-bit filter of L(v_k)'s hubs: most hubs of a candidate's label
        // are not in the root's, and the filter tells so with one load (for
        // labels of up to FILT_MAX_LEN entries, where at most 12 % of its bits
        // are set; longer labels go to the table directly)
        const uint32_t len = a.lab_len[k];
        uint32_t *filt = a.filt + (size_t)slot * FILT_WORDS;
        if (len <= FILT_MAX_LEN) {
            filt[lane] = 0;
            __syncwarp();
            const uint32_t *lab = a.pool + a.lab_off[k];
            for (uint32_t j = lane; j < len; j += 32) {
                const uint32_t fb = filt_bit(entry_hub(lab[j]));
                atomicOr(&filt[fb >> 5], 1u << (fb & 31));
            }
        }
        // root array T as a hash table of 2 x |L(v_k)| slots (very long labels,
        // and tables past the pool's end, are binary-searched instead; the host
        // grows the pool for the next batches)
        const unsigned long long tb = a.ht_off[slot], te = a.ht_off[slot + 1];
        if (te > a.ht_cap) {
            if (lane == 0) atomicOr(&a.ctr->err, ERR_TABLE);
        } else if (te > tb) {
            uint32_t *ht = a.ht + tb;
            const uint32_t mask = (uint32_t)(te - tb) - 1;
            for (uint32_t s = lane; s <= mask; s += 32) ht[s] = HT_EMPTY;
            __syncwarp();
            const uint32_t *lab = a.pool + a.lab_off[k];
            for (uint32_t j = lane; j < len; j += 32) {
                const uint32_t e = lab[j];
                uint32_t s = ht_slot(entry_hub(e), mask);
                while (atomicCAS(&ht[s], HT_EMPTY, e) != HT_EMPTY) s = (s + 1) & mask;
            }
        }
    }
}

// table sizes of the batch's roots (0 for bit-parallel vertices)
__global__ void k_ht_sizes(BatchArgs a, unsigned long long *sizes) {
    for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot <= a.B; slot += gridDim.x * blockDim.x) {
        uint32_t sz = 0;
        if (slot < a.B) {
            const uint32_t k = a.k0 + slot;
            if (!a.inX[k]) sz = ht_size(a.lab_len[k]);
        }
        sizes[slot] = sz;
    }
}

// Cheap part of the prune test, one thread: bit-parallel distances only. With
// d~_i = d(v_k, r_i) + d(r_i, w), some d~_i <= level prunes (Sec. 5.3: the
// distance through {r_i} U S_{r_i} is at most d~_i); roots with d~_i = level + 1
// or level + 2 may still prune through their masks. kr and wq are the rows of
// v_k and w (nq 16-byte chunks, four roots per 32-bit word); the byte sums
// saturate at 255, so this form needs level + 2 < 255.

// Phase 1: is some d~_i <= level? Two byte instructions per four roots, with
// an exit at the first word that prunes: roots come in rank order (Sec. 5.4),
// so the first words, the largest hubs, prune most vertices, and the exit saves
// a fifth of the sweep's time against testing all t roots first.
__device__ __forceinline__ bool bp_prunes(const uint4 *kr, const uint4 (&wq)[PLL_MAX_T / 16], uint32_t nq,
                                          uint32_t lv) {
#pragma unroll
    for (uint32_t c = 0; c < PLL_MAX_T / 16; ++c) {
        if (c < nq) {
            const uint4 r = kr[c], q = wq[c];
            if (__vcmpleu4(__vaddus4(q.x, r.x), lv)) return true;
            if (__vcmpleu4(__vaddus4(q.y, r.y), lv)) return true;
            if (__vcmpleu4(__vaddus4(q.z, r.z), lv)) return true;
            if (__vcmpleu4(__vaddus4(q.w, r.w), lv)) return true;
        }
    }
    return false;
}

// bytes 0x00 / 0xff of x -> bits 0..3 (the four 0/1 bits gathered by one multiply)
__device__ __forceinline__ uint32_t byte_lanes(uint32_t x) { return ((x & 0x01010101u) * 0x01020408u) >> 24; }

// Phase 2, after phase 1 found no prune: c1 = roots with d~_i = level + 1,
// c2 = roots with d~_i = level + 2.
__device__ __forceinline__ void bp_feasible(const uint4 *kr, const uint4 (&wq)[PLL_MAX_T / 16], uint32_t nq,
                                            uint32_t level, uint64_t &c1, uint64_t &c2) {
    const uint32_t l1 = (level + 1) * 0x01010101u, l2 = (level + 2) * 0x01010101u;
    c1 = c2 = 0;
#pragma unroll
    for (uint32_t c = 0; c < PLL_MAX_T / 16; ++c) {
        if (c < nq) {
            const uint4 r = kr[c], q = wq[c];
            const uint32_t sx = __vaddus4(q.x, r.x), sy = __vaddus4(q.y, r.y);
            const uint32_t sz = __vaddus4(q.z, r.z), sw = __vaddus4(q.w, r.w);
            const uint32_t a1 = byte_lanes(__vcmpeq4(sx, l1)) | byte_lanes(__vcmpeq4(sy, l1)) << 4 |
                                byte_lanes(__vcmpeq4(sz, l1)) << 8 | byte_lanes(__vcmpeq4(sw, l1)) << 12;
            const uint32_t a2 = byte_lanes(__vcmpeq4(sx, l2)) | byte_lanes(__vcmpeq4(sy, l2)) << 4 |
                                byte_lanes(__vcmpeq4(sz, l2)) << 8 | byte_lanes(__vcmpeq4(sw, l2)) << 12;
            c1 |= (uint64_t)a1 << (16 * c);
            c2 |= (uint64_t)a2 << (16 * c);
        }
    }
}

// The clamped rows: bp_c holds min(d(r_i, v), 63) for every byte of bp_d
// (unreachable, 255, also becomes 63). Two clamped bytes add up to at most
// 126 with no carry between bytes, so plain 32-bit arithmetic tests four roots
// at once (the byte-SIMD intrinsics above take several instructions each).
// For a candidate level L <= FAST_LEVEL the test is exact: a clamped byte
// stands for a distance >= 63 > L + 2, so its sum can neither reach L nor
// equal L + 1 or L + 2, clamped or not.
constexpr uint32_t CLAMP = 63;
constexpr uint32_t FAST_LEVEL = CLAMP - 3;

// Phase 1 on clamped rows: with lb = (0x80 + L) in every byte, the byte of
// lb - (q + r) keeps its top bit iff q + r <= L (no borrow crosses a byte:
// every byte of lb is above every byte sum).
__device__ __forceinline__ bool bp_prunes_c(const uint4 *kr, const uint4 (&wq)[PLL_MAX_T / 16], uint32_t nq,
                                            uint32_t lb) {
#pragma unroll
    for (uint32_t c = 0; c < PLL_MAX_T / 16; ++c) {
        if (c < nq) {
            const uint4 r = kr[c], q = wq[c];
            if ((lb - (q.x + r.x)) & 0x80808080u) return true;
            if ((lb - (q.y + r.y)) & 0x80808080u) return true;
            if ((lb - (q.z + r.z)) & 0x80808080u) return true;
            if ((lb - (q.w + r.w)) & 0x80808080u) return true;
        }
    }
    return false;
}

// bits 0..3: which bytes of s equal those of cb (every byte of s ^ cb is
// below 0x80, so (x | 0x80) - 1 keeps its top bit iff the byte x is not 0)
__device__ __forceinline__ uint32_t eq_lanes(uint32_t s, uint32_t cb) {
    const uint32_t x = s ^ cb;
    const uint32_t z = ~((x | 0x80808080u) - 0x01010101u) & 0x80808080u;
    return ((z >> 7) * 0x01020408u) >> 24;
}

// Phase 2 on clamped rows: c1 = roots with d~_i = L + 1, c2 = roots with L + 2.
__device__ __forceinline__ void bp_feasible_c(const uint4 *kr, const uint4 (&wq)[PLL_MAX_T / 16], uint32_t nq,
                                              uint32_t level, uint64_t &c1, uint64_t &c2) {
    const uint32_t l1 = (level + 1) * 0x01010101u, l2 = (level + 2) * 0x01010101u;
    c1 = c2 = 0;
#pragma unroll
    for (uint32_t c = 0; c < PLL_MAX_T / 16; ++c) {
        if (c < nq) {
            const uint4 r = kr[c], q = wq[c];
            const uint32_t sx = q.x + r.x, sy = q.y + r.y, sz = q.z + r.z, sw = q.w + r.w;
            const uint32_t a1 = eq_lanes(sx, l1) | eq_lanes(sy, l1) << 4 | eq_lanes(sz, l1) << 8 |
                                eq_lanes(sw, l1) << 12;
            const uint32_t a2 = eq_lanes(sx, l2) | eq_lanes(sy, l2) << 4 | eq_lanes(sz, l2) << 8 |
                                eq_lanes(sw, l2) << 12;
            c1 |= (uint64_t)a1 << (16 * c);
            c2 |= (uint64_t)a2 << (16 * c);
        }
    }
}

// The same test for depths near 255, where byte sums would overflow: a plain
// loop over the roots. Returns true if some d~_i <= level.
__device__ __noinline__ bool bp_test_plain(const BatchArgs &a, uint32_t k, uint32_t w, uint32_t level,
                                           uint64_t &c1, uint64_t &c2) {
    const uint8_t *dw = a.bp_d + (size_t)w * a.tp, *dk = a.bp_d + (size_t)k * a.tp;
    c1 = c2 = 0;
    for (uint32_t i = 0; i < a.t; ++i) {
        const uint32_t x = dw[i], y = dk[i];
        if (x == INF8 || y == INF8) continue;
        const uint32_t td = x + y;
        if (td <= level) return true;
        if (td == level + 1) c1 |= 1ull << i;
        if (td == level + 2) c2 |= 1ull << i;
    }
    return false;
}

// Masks of the first QUICK bit-parallel roots, one thread. The roots are
// chosen in rank order (Sec. 5.4), so the first ones are the largest hubs and
// settle most mask tests; checking them here keeps most candidates out of
// the test sweep and away from the rest of their 1 KiB mask rows. Clears
// those roots from c1 / c2.
constexpr uint32_t QUICK = 4;
__device__ __forceinline__ bool quick_masks(const BatchArgs &a, uint32_t k, uint32_t w, uint64_t &c1,
                                            uint64_t &c2) {
    const uint32_t q1 = (uint32_t)c1 & ((1u << QUICK) - 1u), q2 = (uint32_t)c2 & ((1u << QUICK) - 1u);
    c1 &= ~(uint64_t)((1u << QUICK) - 1u);
    c2 &= ~(uint64_t)((1u << QUICK) - 1u);
    if (!(q1 | q2)) return false;
    const ulonglong2 *wm = reinterpret_cast<const ulonglong2 *>(a.bp_m) + (size_t)w * a.t;
    const ulonglong2 *km = reinterpret_cast<const ulonglong2 *>(a.bp_m) + (size_t)k * a.t;
    bool p = false;
#pragma unroll
    for (uint32_t i = 0; i < QUICK; ++i) {
        if (((q1 | q2) >> i) & 1u) {
            const ulonglong2 m = wm[i], r = km[i];
            if (((q1 >> i) & 1u) && ((((r.x | r.y) & m.x) | (r.x & m.y)) != 0)) p = true;
            if (((q2 >> i) & 1u) && ((r.x & m.x) != 0)) p = true;
        }
    }
    return p;
}


// One arc (u, w) of an entry of root ki (batch slot `slot`; kr = its row in
// shared memory, from `rows`): look w up in the root's visited row; if
// unvisited, the bit-parallel test and the first masks; claim w if it
// survives. Returns true for a fresh claim (w becomes a candidate with
// feasible roots c1 / c2). fast: the rows are the clamped ones.
__device__ __forceinline__ bool expand_arc(const BatchArgs &a, const uint8_t *rows, uint32_t ki, uint32_t slot,
                                           uint32_t w, const uint4 *kr, uint32_t nq, uint32_t nlevel,
                                           bool fast, bool near, uint32_t lv, uint64_t &c1, uint64_t &c2,
                                           uint32_t &nreach) {
    uint32_t *word = a.visited + (size_t)slot * a.NW + (w >> 5);
    const uint32_t wbit = 1u << (w & 31);
    uint4 wq[PLL_MAX_T / 16];
#pragma unroll
    for (uint32_t c = 0; c < PLL_MAX_T / 16; ++c)
        wq[c] = (c < nq) ? __ldg(reinterpret_cast<const uint4 *>(rows + (size_t)w * a.tp) + c)
                         : make_uint4(0, 0, 0, 0);
    if (*word & wbit) return false;
    ++nreach;
    bool pruned;
    if (nlevel >= INF8) {
        atomicOr(&a.ctr->err, ERR_DEPTH);
        return false;
    } else if (fast) {
        pruned = bp_prunes_c(kr, wq, nq, lv);
        if (!pruned) bp_feasible_c(kr, wq, nq, nlevel, c1, c2);
    } else if (!near) {
        pruned = bp_prunes(kr, wq, nq, lv);
        if (!pruned) bp_feasible(kr, wq, nq, nlevel, c1, c2);
    } else {
        pruned = bp_test_plain(a, ki, w, nlevel, c1, c2);
    }
    if (pruned) return false;
    c1 &= a.rootbits[2 * slot + 1];
    c2 &= a.rootbits[2 * slot];
    if (quick_masks(a, ki, w, c1, c2)) return false;
    return !(atomicOr(word, wbit) & wbit);
}

__device__ __forceinline__ void append_cand(const BatchArgs &a, bool keep, int lane, uint32_t slot, uint32_t w,
                                            uint64_t c1, uint64_t c2) {
    if (__any_sync(FULL, keep)) {
        const unsigned long long pos = warp_append(&a.ctr->cand_n, keep, lane);
        if (keep) {
            if (pos < a.cand_cap) {
                a.cand[pos] = ((uint64_t)slot << 32) | w;
                reinterpret_cast<ulonglong2 *>(a.candc)[pos] = make_ulonglong2(c1, c2);
            } else {
                atomicOr(&a.ctr->err, ERR_BUF);
            }
        }
    }
}
// entries [lvl_b, lvl_e) of the current level -> candidates of the next, one
// warp per entry, 32 consecutive arcs per step (coalesced column loads; the
// root's row, the same for every lane, sits once per warp in shared memory).
// 1280 threads per SM (48 registers a thread): the sweep hides the latency of
// its row and visited-word loads with resident warps.
// The sweep over entries [b, e) of level `level` by the warps of a grid;
// kr: this warp's row in shared memory. Adds the arcs it scans and the
// vertices it tests to nexp / nreach.
__device__ __forceinline__ void expand_body(const BatchArgs &a, unsigned long long b, unsigned long long e,
                                            uint32_t level, uint4 *kr, uint32_t &nexp, uint32_t &nreach) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long gw = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nq = a.tp >> 4;
    const uint32_t nlevel = level + 1;                // level of the candidates
    const bool fast = nlevel <= FAST_LEVEL;           // clamped rows, plain arithmetic
    const bool near = nlevel + 2 >= INF8;             // byte sums could overflow
    const uint32_t lv = fast ? (0x80u + nlevel) * 0x01010101u : nlevel * 0x01010101u;
    const uint8_t *rows = fast ? a.bp_c : a.bp_d;
    for (unsigned long long j = b + gw; j < e; j += nwarps) {
        // entries and candidates are written by other SMs between the phases of
        // one launch (k_batch_levels): read them from L2, never from a line the
        // L1 kept from an earlier level
        const uint64_t key = __ldcg(a.out + j);
        const uint32_t u = (uint32_t)(key >> 32);
        const uint32_t k = entry_hub((uint32_t)key);
        const uint32_t slot = k - a.k0;
        __syncwarp();
        if ((uint32_t)lane < nq) kr[lane] = __ldg(reinterpret_cast<const uint4 *>(rows + (size_t)k * a.tp) + lane);
        __syncwarp();
        const uint32_t eb = a.roff[u], ee = a.roff[u + 1];
        if (lane == 0) nexp += ee - eb;
        for (uint32_t x = eb; x < ee; x += 32) {
            bool keep = false;
            uint32_t w = 0;
            uint64_t c1 = 0, c2 = 0;
            if (x + lane < ee) {
                w = a.rcol[x + lane];
                keep = expand_arc(a, rows, k, slot, w, kr, nq, nlevel, fast, near, lv, c1, c2, nreach);
            }
            append_cand(a, keep, lane, slot, w, c1, c2);
        }
    }
}

// warp sums of the work counters into ctr->work[w0], ctr->work[w0 + 1]
__device__ __forceinline__ void flush_work(const BatchArgs &a, int w0, uint32_t x, uint32_t y) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(FULL, x, o);
        y += __shfl_xor_sync(FULL, y, o);
    }
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&a.ctr->work[w0], (unsigned long long)x);
    if ((threadIdx.x & 31) == 0 && y) atomicAdd(&a.ctr->work[w0 + 1], (unsigned long long)y);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_batch_expand(BatchArgs a) {
    extern __shared__ uint4 s_rows[];
    uint32_t nexp = 0, nreach = 0;
    expand_body(a, a.desc->lvl_b, a.desc->lvl_e, a.desc->level,
                s_rows + (size_t)(threadIdx.x >> 5) * (PLL_MAX_T / 16), nexp, nreach);
    flush_work(a, 2, nexp, nreach);
}

template <int BLOCK>
constexpr size_t expand_smem() { return (size_t)(BLOCK / 32) * (PLL_MAX_T / 16) * sizeof(uint4); }

// bp_c = min(bp_d, CLAMP) bytewise, 16 bytes per thread and step
__global__ void k_clamp_rows(const uint4 *bp_d, uint4 *bp_c, size_t n16) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x) {
        uint4 v = bp_d[i];
        uint32_t *x = reinterpret_cast<uint32_t *>(&v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            // bytes >= 64 have one of their two top bits set: they become 63
            const uint32_t hi = x[j] & 0xC0C0C0C0u;
            const uint32_t big = ((hi >> 6) | (hi >> 7)) & 0x01010101u;
            x[j] = (x[j] & 0x3F3F3F3Fu) | (big * CLAMP);
        }
        bp_c[i] = v;
    }
}

// Lazy reset: zero the visited words of the batch's roots and candidates (the
// only bits the batch set; several candidates may share a word). A batch whose
// candidates overflowed their buffer did not record them all: its rows are
// zeroed whole (it runs again with a larger buffer).
__global__ void k_batch_clear(BatchArgs a) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a.ctr->err & ERR_BUF) {
        const unsigned long long words = (unsigned long long)a.B * a.NW;
        uint4 *v4 = reinterpret_cast<uint4 *>(a.visited);  // the bitmap is 256-byte aligned
        for (unsigned long long i = i0; i < words / 4; i += stride) v4[i] = make_uint4(0, 0, 0, 0);
        for (unsigned long long i = (words & ~3ull) + i0; i < words; i += stride) a.visited[i] = 0;
        return;
    }
    const unsigned long long cn = a.ctr->cand_n < a.cand_cap ? a.ctr->cand_n : a.cand_cap;
    for (unsigned long long i = i0; i < a.B; i += stride)
        a.visited[i * a.NW + ((a.k0 + (uint32_t)i) >> 5)] = 0;
    for (unsigned long long i = i0; i < cn; i += stride) {
        const uint64_t c = a.cand[i];
        a.visited[(c >> 32) * a.NW + ((uint32_t)c >> 5)] = 0;
    }
}

// The rest of the prune test for 32 candidates per warp (lane j holds
// candidate j), in two parts:
//   masks   one candidate with feasible roots at a time: the lanes take the
//           roots (two each) and compare mask pairs (Sec. 5.3);
//   labels  of the candidates the masks did not prune: a long label (at
//           least LONG_LABEL entries) is scanned by the whole warp, LU rounds
//           of 32 entries per step; the shorter labels L(w) are laid end to end
//           and the lanes take LU x 32 consecutive entries per step (lane x's
//           candidate found by a binary search over a warp scan of the
//           lengths), so short labels do not leave lanes idle and the chunks
//           of different candidates are in flight together. Each entry
//           (h, d) is looked up in the root's filter (roots with labels of at
//           most FILT_MAX_LEN entries), and only if its bit is set in the
//           root's hash table T (or, without a table, by a binary search of
//           L(v_k)); d + T[h] <= level prunes the candidate. A candidate found
//           pruned takes no further entries.
// Per-candidate data sits in shared memory for the lanes that work on it.
constexpr int LU = LABEL_ROUNDS;  // label rounds per step of the test sweep
constexpr int LU_LOOP = LABEL_ROUNDS_LOOP;  // the same inside the level loop (fewer
                                            // registers: the loop's own state is live)
// candidates whose labels have at least this many entries are scanned one by
// one by the whole warp (no owner search per entry, and an exit at the first
// step that prunes); shorter labels are laid end to end over the lanes
constexpr uint32_t LONG_LABEL = LONG_LABEL_ENTRIES;

struct TestCand {
    unsigned long long lab_base;  // pool offset of L(w) minus the candidate's first flattened index
    unsigned long long tb;        // its root's table in the table pool
    unsigned long long koff;      // L(v_k) in the label pool (binary-search fallback)
    uint32_t slot, tmask, klen, pad;  // tmask = table slots - 1, NONE without a table
};

// The label test of LU label entries per lane (ent[u], of candidate own[u],
// where act[u]): in three stages so that the loads of all of them are in
// flight together -- the filter words, then the first table slot of each hub
// (collision chains and the binary-search fallback follow one by one). Returns
// the lane's candidates that an entry prunes (d + T[h] <= level), as bits.
template <int U>
__device__ __forceinline__ uint32_t lookup_entries(const BatchArgs &a, const TestCand *tc,
                                                   const uint32_t (&ent)[U], const uint32_t (&own)[U],
                                                   const bool (&act)[U], uint32_t level, uint32_t &n_scan) {
    uint32_t fw[U], y0[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        fw[u] = ~0u;  // no filter: every hub goes to the table
        if (act[u]) {
            const TestCand &c = tc[own[u]];
            if (c.klen <= FILT_MAX_LEN) {
                const uint32_t fb = filt_bit(entry_hub(ent[u]));
                fw[u] = a.filt[(size_t)c.slot * FILT_WORDS + (fb >> 5)] >> (fb & 31);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        y0[u] = HT_EMPTY;
        if (act[u] && (fw[u] & 1u)) {
            const TestCand &c = tc[own[u]];
            if (c.tmask != NONE) y0[u] = a.ht[c.tb + ht_slot(entry_hub(ent[u]), c.tmask)];
        }
    }
    uint32_t pm = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (!act[u]) continue;
        ++n_scan;
        if (!(fw[u] & 1u)) continue;
        const TestCand &c = tc[own[u]];
        const uint32_t h = entry_hub(ent[u]);
        uint32_t tk = INF8;
        if (c.tmask != NONE) {
            const uint32_t *ht = a.ht + c.tb;
            uint32_t sl = ht_slot(h, c.tmask), y = y0[u];
            for (;;) {
                if (y == HT_EMPTY) break;
                if (entry_hub(y) == h) { tk = entry_dist(y); break; }
                sl = (sl + 1) & c.tmask;
                y = ht[sl];
            }
        } else {
            const uint32_t *rlab = a.pool + c.koff;
            uint32_t lo = 0, hi = c.klen;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (entry_hub(rlab[mid]) < h) lo = mid + 1; else hi = mid;
            }
            if (lo < c.klen && entry_hub(rlab[lo]) == h) tk = entry_dist(rlab[lo]);
        }
        if (tk != INF8 && tk + entry_dist(ent[u]) <= level) pm |= 1u << own[u];
    }
    return pm;
}

// The sweep over candidates [b, e) of level `level` by the warps of a grid;
// tc: this warp's 32 records in shared memory. Adds the label entries it scans
// and the mask pairs it reads to n_scan / n_mask.
template <int U>
__device__ __forceinline__ void test_body(const BatchArgs &a, unsigned long long b, unsigned long long e,
                                          uint32_t level, TestCand *tc, uint32_t &n_scan, uint32_t &n_mask) {
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // warp-uniform trip count: each warp takes 32 consecutive candidates
    const unsigned long long span = ((e - b + 31) / 32) * 32;
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         i0 < span; i0 += stride) {
        const uint32_t cnt = (uint32_t)((e - b - i0) < 32 ? (e - b - i0) : 32);
        const bool valid = (uint32_t)lane < cnt;
        uint64_t mine = 0;
        ulonglong2 mc = make_ulonglong2(0, 0);
        uint32_t wlen = 0, klen = 0, slot = 0, w = 0;
        unsigned long long woff = 0, koff = 0, tb = 0, te = 0;
        if (valid) {  // per-candidate metadata, loaded in parallel
            mine = __ldcg(a.cand + b + i0 + lane);
            mc = __ldcg(reinterpret_cast<const ulonglong2 *>(a.candc) + b + i0 + lane);
            w = (uint32_t)mine;
            slot = (uint32_t)(mine >> 32);
            const uint32_t k = a.k0 + slot;
            wlen = a.lab_len[w];
            woff = a.lab_off[w];
            klen = a.lab_len[k];
            koff = a.lab_off[k];
            tb = a.ht_off[slot];
            te = a.ht_off[slot + 1];
        }
        // ---- masks
        uint32_t pruned = 0;
        for (uint32_t m = __ballot_sync(FULL, (mc.x | mc.y) != 0); m; m &= m - 1) {
            const uint32_t j = __ffs(m) - 1;
            const uint64_t c1 = __shfl_sync(FULL, mc.x, j), c2 = __shfl_sync(FULL, mc.y, j);
            const uint32_t wj = __shfl_sync(FULL, w, j), kj = a.k0 + __shfl_sync(FULL, slot, j);
            const ulonglong2 *wm = reinterpret_cast<const ulonglong2 *>(a.bp_m) + (size_t)wj * a.t;
            const ulonglong2 *km = reinterpret_cast<const ulonglong2 *>(a.bp_m) + (size_t)kj * a.t;
            bool p = false;
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
                const uint32_t i = lane + 32 * h;
                const bool b1 = (c1 >> i) & 1, b2 = (c2 >> i) & 1;
                if (b1 | b2) {
                    ++n_mask;
                    const ulonglong2 mw = wm[i], r = km[i];
                    if (b1 && (((r.x | r.y) & mw.x) | (r.x & mw.y))) p = true;  // reduction >= 1
                    if (b2 && (r.x & mw.x)) p = true;                           // reduction 2
                }
            }
            if (__any_sync(FULL, p)) pruned |= 1u << j;
        }
        // ---- labels: candidates with long labels get the whole warp in turn;
        // the labels of the others are laid end to end over the lanes
        const bool open = valid && !((pruned >> lane) & 1);
        const uint32_t len = (open && wlen < LONG_LABEL) ? wlen : 0;
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        const uint32_t excl = incl - len;
        __syncwarp();  // the previous group is done with tc
        if (valid) {
            TestCand c;
            c.lab_base = woff - excl;
            c.tb = tb;
            c.koff = koff;
            c.slot = slot;
            c.tmask = (te > tb && te <= a.ht_cap) ? (uint32_t)(te - tb) - 1 : NONE;
            c.klen = klen;
            c.pad = 0;
            tc[lane] = c;
        }
        __syncwarp();
        uint32_t ent[U], own[U];
        bool act[U];
        // long labels: LU rounds of 32 entries per step, leaving at the first
        // step that prunes
        for (uint32_t m = __ballot_sync(FULL, open && wlen >= LONG_LABEL); m; m &= m - 1) {
            const uint32_t j = __ffs(m) - 1;
            const uint32_t lj = __shfl_sync(FULL, wlen, j);
            const unsigned long long base = tc[j].lab_base + __shfl_sync(FULL, excl, j);
            // without bit-parallel labels (t = 0) the labels prune most
            // candidates, mostly with their first hubs (the highest-ranked):
            // the first 32 entries alone, then U rounds per step. With them,
            // most candidates that reach this test survive it and need every
            // entry, so U rounds from the start.
            if (a.t == 0) {
                uint32_t e1[1], o1[1] = {j};
                bool a1[1] = {true};
                e1[0] = a.pool[base + lane];
                if (__any_sync(FULL, lookup_entries(a, tc, e1, o1, a1, level, n_scan) != 0)) {
                    pruned |= 1u << j;
                    continue;
                }
            }
            for (uint32_t x0 = a.t == 0 ? 32u : 0u; x0 < lj; x0 += 32 * U) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t x = x0 + 32 * u + lane;
                    own[u] = j;
                    act[u] = x < lj;
                    ent[u] = act[u] ? a.pool[base + x] : 0u;
                }
                if (__any_sync(FULL, lookup_entries(a, tc, ent, own, act, level, n_scan) != 0)) {
                    pruned |= 1u << j;
                    break;
                }
            }
        }
        // short labels laid end to end (lane x's candidate found by a binary
        // search over the warp scan of their lengths)
        for (uint32_t x0 = 0; x0 < total; x0 += 32 * U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t x = x0 + 32 * u + lane;
                uint32_t j = 0;  // owner: the last candidate whose first entry is <= x
#pragma unroll
                for (uint32_t step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(FULL, excl, j + step) <= x) j += step;
                own[u] = j;
                act[u] = x < total && !((pruned >> j) & 1);
                ent[u] = act[u] ? a.pool[tc[j].lab_base + x] : 0u;
            }
            pruned |= __reduce_or_sync(FULL, lookup_entries(a, tc, ent, own, act, level, n_scan));
        }
        const bool keep = valid && !((pruned >> lane) & 1);
        if (__any_sync(FULL, keep)) {
            const unsigned long long pos = warp_append(&a.ctr->out_n, keep, lane);
            if (keep) {
                if (pos < a.out_cap) a.out[pos] = pack_tuple(w, a.k0 + slot, level);
                else atomicOr(&a.ctr->err, ERR_BUF);
            }
        }
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_batch_test(BatchArgs a) {
    __shared__ TestCand s_cand[BLOCK / 32][32];
    uint32_t n_scan = 0, n_mask = 0;
    test_body<LU>(a, a.desc->cand_b, a.desc->cand_e, a.desc->level + 1, s_cand[threadIdx.x >> 5], n_scan, n_mask);
    flush_work(a, 0, n_scan, n_mask);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (every CTA resident). The last
// CTA to arrive takes a snapshot of the counters (error word, candidate and
// entry counts) before it releases the others, so every CTA decides the next
// step from the same values. A wait longer than the state's timeout_ns sets
// ERR_TIMEOUT and returns false: the CTA leaves the level loop, and the
// others leave it at their next barrier, each wait bounded the same way.
__device__ __forceinline__ bool grid_barrier(const BatchArgs &a, LoopState *ls) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned int gen = *(volatile unsigned int *)&ls->gen;
        if (atomicAdd(&ls->count, 1u) == gridDim.x - 1) {
            ls->count = 0;
            ls->err = atomicOr(&a.ctr->err, 0u);
            ls->cand_n = atomicAdd(&a.ctr->cand_n, 0ull);
            ls->out_n = atomicAdd(&a.ctr->out_n, 0ull);
            __threadfence();
            atomicAdd(&ls->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns(), lim = ls->timeout_ns;
            while (*(volatile unsigned int *)&ls->gen == gen) {
                if (global_ns() - t0 > lim) {
                    atomicOr(&a.ctr->err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Every level of a root batch in one cooperative launch: expand, barrier,
// test, barrier, until the frontier is empty (or a buffer overflows, a depth
// reaches 255, or a barrier times out). Level bounds live in registers, the
// same in every CTA (they come from the barrier's snapshots), so no level
// needs the host. Block 0 adds the phases' wall times to the loop state.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_batch_levels(BatchArgs a) {
    extern __shared__ uint4 s_rows[];
    __shared__ TestCand s_cand[BLOCK / 32][32];
    LoopState *ls = a.loop;
    uint4 *kr = s_rows + (size_t)(threadIdx.x >> 5) * (PLL_MAX_T / 16);
    TestCand *tc = s_cand[threadIdx.x >> 5];
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long lvl_b = a.desc->lvl_b, lvl_e = a.desc->lvl_e, cand_e = 0;
    uint32_t level = 0, nexp = 0, nreach = 0, n_scan = 0, n_mask = 0;
    unsigned long long ns_e = 0, ns_t = 0;
    constexpr uint32_t STOP = ERR_DEPTH | ERR_BUF | ERR_TIMEOUT;
    while (lvl_b < lvl_e) {
        const unsigned long long t0 = timer ? global_ns() : 0;
        expand_body(a, lvl_b, lvl_e, level, kr, nexp, nreach);
        if (!grid_barrier(a, ls)) break;
        const unsigned long long t1 = timer ? global_ns() : 0;
        if (*(volatile uint32_t *)&ls->err & STOP) break;
        const unsigned long long cand_b = cand_e;
        const unsigned long long cn = *(volatile unsigned long long *)&ls->cand_n;
        cand_e = cn < a.cand_cap ? cn : a.cand_cap;
        test_body<LU_LOOP>(a, cand_b, cand_e, level + 1, tc, n_scan, n_mask);
        if (!grid_barrier(a, ls)) break;
        if (timer) {
            const unsigned long long t2 = global_ns();
            ns_e += t1 - t0;
            ns_t += t2 - t1;
        }
        if (*(volatile uint32_t *)&ls->err & STOP) break;
        const unsigned long long on = *(volatile unsigned long long *)&ls->out_n;
        lvl_b = lvl_e;
        lvl_e = on < a.out_cap ? on : a.out_cap;
        ++level;
    }
    flush_work(a, 2, nexp, nreach);
    flush_work(a, 0, n_scan, n_mask);
    if (timer) {
        ls->ns_expand += ns_e;
        ls->ns_test += ns_t;
        ls->levels += level;
    }
}

// descriptor steps between sweeps (one thread)
__device__ __forceinline__ void advance_desc(const BatchArgs &a, int phase) {
    LevelDesc *d = a.desc;
    const unsigned long long cn = a.ctr->cand_n, on = a.ctr->out_n;
    if (phase == 0) {          // after init: level 0 = the roots
        d->lvl_b = 0;
        d->lvl_e = on < a.out_cap ? on : a.out_cap;
        d->roots_n = d->lvl_e;
        d->level = 0;
        d->cand_b = 0;
        d->cand_e = 0;
        if (a.loop) a.loop->t_mark = global_ns();
    } else if (phase == 1) {   // after expand: candidates of level + 1
        d->cand_b = d->cand_e;
        d->cand_e = cn < a.cand_cap ? cn : a.cand_cap;
    } else {                   // after test: survivors become the level
        d->lvl_b = d->lvl_e;
        d->lvl_e = on < a.out_cap ? on : a.out_cap;
        d->level += 1;
    }
}

__global__ void k_batch_advance(BatchArgs a, int phase) { advance_desc(a, phase); }

// ---- the level loop as a CUDA graph: a while node whose body is expand,
// advance(1), test, advance(2); the second advance sets the loop condition.
// The kernels read the batch's arguments from device memory (the host writes
// them before each launch of the graph), so one instantiated graph serves
// every batch of a build.
// the batch's arguments, copied once per CTA from device memory into shared
// memory (read there as cheaply as kernel parameters)
__device__ __forceinline__ const BatchArgs &args_to_shared(const BatchArgs *ap, BatchArgs *sa) {
    static_assert(sizeof(BatchArgs) % 8 == 0, "BatchArgs is copied in 8-byte words");
    constexpr unsigned W = sizeof(BatchArgs) / 8;
    for (unsigned i = threadIdx.x; i < W; i += blockDim.x)
        reinterpret_cast<uint64_t *>(sa)[i] = reinterpret_cast<const uint64_t *>(ap)[i];
    __syncthreads();
    return *sa;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_batch_expand_g(const BatchArgs *__restrict__ ap) {
    extern __shared__ uint4 s_rows[];
    __shared__ BatchArgs s_args;
    const BatchArgs &a = args_to_shared(ap, &s_args);
    uint32_t nexp = 0, nreach = 0;
    expand_body(a, a.desc->lvl_b, a.desc->lvl_e, a.desc->level,
                s_rows + (size_t)(threadIdx.x >> 5) * (PLL_MAX_T / 16), nexp, nreach);
    flush_work(a, 2, nexp, nreach);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_batch_test_g(const BatchArgs *__restrict__ ap) {
    __shared__ TestCand s_cand[BLOCK / 32][32];
    __shared__ BatchArgs s_args;
    const BatchArgs &a = args_to_shared(ap, &s_args);
    uint32_t n_scan = 0, n_mask = 0;
    test_body<LU>(a, a.desc->cand_b, a.desc->cand_e, a.desc->level + 1, s_cand[threadIdx.x >> 5], n_scan, n_mask);
    flush_work(a, 0, n_scan, n_mask);
}

// phase 1 / 2 of advance_desc, plus the phases' wall times; phase 2 sets the
// loop's condition: another level while the frontier is not empty and no
// buffer overflowed and no depth reached 255
__global__ void k_batch_advance_g(const BatchArgs *__restrict__ ap, int phase, cudaGraphConditionalHandle h) {
    const BatchArgs &a = *ap;
    advance_desc(a, phase);
    LoopState *ls = a.loop;
    const unsigned long long now = global_ns();
    if (phase == 1) {
        ls->ns_expand += now - ls->t_mark;
    } else {
        ls->ns_test += now - ls->t_mark;
        ls->levels += 1;
        const bool more = a.desc->lvl_b < a.desc->lvl_e && !(a.ctr->err & (ERR_DEPTH | ERR_BUF));
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
    ls->t_mark = now;
}

}  // namespace

template <int BLOCK>
static cudaError_t occupancy(int *pe, int *pt) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_expand<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)expand_smem<BLOCK>());
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(pe, k_batch_expand<BLOCK>, BLOCK, expand_smem<BLOCK>());
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(pt, k_batch_test<BLOCK>, BLOCK, 0);
    return e;
}

// grid[0]: expand sweep, grid[1]: test sweep (resident CTAs of each)
int batch_grid(uint32_t block, int *grid) {
    int dev = 0, sms = 0, pe = 0, pt = 0;
    PLL_TRY(cudaGetDevice(&dev));
    PLL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaError_t e;
    switch (block) {
        case 128: e = occupancy<128>(&pe, &pt); break;
        case 512: e = occupancy<512>(&pe, &pt); break;
        case 1024: e = occupancy<1024>(&pe, &pt); break;
        default: e = occupancy<256>(&pe, &pt); break;
    }
    PLL_TRY(e);
    grid[0] = sms * (pe > 0 ? pe : 1);
    grid[1] = sms * (pt > 0 ? pt : 1);
    return PLL_OK;
}

size_t batch_init_temp_bytes(uint32_t bmax) {
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, (unsigned long long *)nullptr,
                                  (unsigned long long *)nullptr, (int)bmax + 1);
    return tb;
}

// temp: CUB scratch of batch_init_temp_bytes(B) bytes followed by B + 1
// 64-bit sizes
int batch_init(const BatchArgs &a, void *temp, size_t temp_bytes, cudaStream_t s) {
    unsigned long long *sizes = reinterpret_cast<unsigned long long *>(
        static_cast<unsigned char *>(temp) + ((temp_bytes - ((size_t)a.B + 1) * 8) & ~(size_t)255));
    const size_t cub_bytes = (size_t)((unsigned char *)sizes - (unsigned char *)temp);
    k_ht_sizes<<<(int)((a.B + 256) / 256), 256, 0, s>>>(a, sizes);
    size_t tb = cub_bytes;
    PLL_TRY(cub::DeviceScan::ExclusiveSum(temp, tb, sizes, a.ht_off, (int)a.B + 1, s));
    const int g = (int)((a.B * 32ull + 255) / 256);
    k_batch_init<<<g > 0 ? g : 1, 256, 0, s>>>(a);
    k_batch_advance<<<1, 1, 0, s>>>(a, 0);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

template <int BLOCK>
static void level_sweeps(const BatchArgs &a, const int *grid, cudaStream_t s, cudaEvent_t *ev) {
    if (ev) cudaEventRecord(ev[0], s);
    k_batch_expand<BLOCK><<<grid[0], BLOCK, expand_smem<BLOCK>(), s>>>(a);
    if (ev) cudaEventRecord(ev[1], s);
    k_batch_advance<<<1, 1, 0, s>>>(a, 1);
    if (ev) cudaEventRecord(ev[2], s);
    k_batch_test<BLOCK><<<grid[1], BLOCK, 0, s>>>(a);
    if (ev) cudaEventRecord(ev[3], s);
    k_batch_advance<<<1, 1, 0, s>>>(a, 2);
}

int batch_clamp_rows(const uint8_t *bp_d, uint8_t *bp_c, size_t bytes, int grid, cudaStream_t s) {
    if (bytes == 0) return PLL_OK;
    k_clamp_rows<<<grid > 0 ? grid : 1, 256, 0, s>>>(reinterpret_cast<const uint4 *>(bp_d),
                                                     reinterpret_cast<uint4 *>(bp_c), bytes / 16);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

int batch_clear(const BatchArgs &a, int grid, cudaStream_t s) {
    k_batch_clear<<<grid > 0 ? grid : 1, 256, 0, s>>>(a);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

template <int BLOCK>
static cudaError_t levels_grid(int *grid) {
    int dev = 0, sms = 0, coop = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_levels<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)expand_smem<BLOCK>());
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_levels<BLOCK>, BLOCK, expand_smem<BLOCK>());
    *grid = (e == cudaSuccess && coop && per > 0) ? sms * per : 0;
    return e;
}

int batch_levels_grid(uint32_t block, int *grid) {
    cudaError_t e;
    switch (block) {
        case 128: e = levels_grid<128>(grid); break;
        case 512: e = levels_grid<512>(grid); break;
        case 1024: e = levels_grid<1024>(grid); break;
        default: e = levels_grid<256>(grid); break;
    }
    PLL_TRY(e);
    return PLL_OK;
}

template <int BLOCK>
static cudaError_t launch_levels(const BatchArgs &a, int grid, cudaStream_t s) {
    BatchArgs arg = a;
    void *args[] = {&arg};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_batch_levels<BLOCK>), dim3(grid),
                                       dim3(BLOCK), args, expand_smem<BLOCK>(), s);
}

int batch_levels(const BatchArgs &a, uint32_t block, int grid, cudaStream_t s) {
    cudaError_t e;
    switch (block) {
        case 128: e = launch_levels<128>(a, grid, s); break;
        case 512: e = launch_levels<512>(a, grid, s); break;
        case 1024: e = launch_levels<1024>(a, grid, s); break;
        default: e = launch_levels<256>(a, grid, s); break;
    }
    PLL_TRY(e);
    return PLL_OK;
}

template <int BLOCK>
static int graph_build(const int *grid, const BatchArgs *d_args, cudaGraph_t *pg, cudaGraphExec_t *pexec) {
    cudaGraph_t g = nullptr;
    PLL_TRY(cudaGraphCreate(&g, 0));
    struct Guard {
        cudaGraph_t g;
        ~Guard() { if (g) cudaGraphDestroy(g); }
    } guard{g};
    PLL_TRY(cudaFuncSetAttribute(k_batch_expand_g<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)expand_smem<BLOCK>()));
    cudaGraphConditionalHandle h;
    PLL_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    PLL_TRY(cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const BatchArgs *ap = d_args;
    int ph1 = 1, ph2 = 2;
    void *a_exp[] = {&ap};
    void *a_adv1[] = {&ap, &ph1, &h};
    void *a_tst[] = {&ap};
    void *a_adv2[] = {&ap, &ph2, &h};
    cudaKernelNodeParams kp{};
    cudaGraphNode_t n[4];
    kp.func = reinterpret_cast<void *>(k_batch_expand_g<BLOCK>);
    kp.gridDim = dim3(grid[0]);
    kp.blockDim = dim3(BLOCK);
    kp.sharedMemBytes = (unsigned)expand_smem<BLOCK>();
    kp.kernelParams = a_exp;
    PLL_TRY(cudaGraphAddKernelNode(&n[0], body, nullptr, 0, &kp));
    kp.func = reinterpret_cast<void *>(k_batch_advance_g);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = a_adv1;
    PLL_TRY(cudaGraphAddKernelNode(&n[1], body, &n[0], 1, &kp));
    kp.func = reinterpret_cast<void *>(k_batch_test_g<BLOCK>);
    kp.gridDim = dim3(grid[1]);
    kp.blockDim = dim3(BLOCK);
    kp.kernelParams = a_tst;
    PLL_TRY(cudaGraphAddKernelNode(&n[2], body, &n[1], 1, &kp));
    kp.func = reinterpret_cast<void *>(k_batch_advance_g);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = a_adv2;
    PLL_TRY(cudaGraphAddKernelNode(&n[3], body, &n[2], 1, &kp));
    PLL_TRY(cudaGraphInstantiate(pexec, g, 0));
    *pg = g;
    guard.g = nullptr;
    return PLL_OK;
}

int batch_graph_build(uint32_t block, const int *grid, const BatchArgs *d_args, cudaGraph_t *g,
                      cudaGraphExec_t *exec) {
    switch (block) {
        case 128: return graph_build<128>(grid, d_args, g, exec);
        case 512: return graph_build<512>(grid, d_args, g, exec);
        case 1024: return graph_build<1024>(grid, d_args, g, exec);
        default: return graph_build<256>(grid, d_args, g, exec);
    }
}

// ev: null, or four events recorded around the expand and test sweeps
int batch_level(const BatchArgs &a, const int *grid, uint32_t block, cudaStream_t s,
                cudaEvent_t *ev) {
    switch (block) {
        case 128: level_sweeps<128>(a, grid, s, ev); break;
        case 512: level_sweeps<512>(a, grid, s, ev); break;
        case 1024: level_sweeps<1024>(a, grid, s, ev); break;
        default: level_sweeps<256>(a, grid, s, ev); break;
    }
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

}  // namespace pll
