// k_pruned.cu -- pruned BFSs (Alg. 1) for a batch of roots [k0, k1).
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
// One CTA ("team") runs one root at a time and pulls the next root from an
// atomic counter. Per root:
//   * the root's label L(v_k) (hubs < k0) goes into a shared-memory hash
//     table: the root array T of Sec. 4.5.1 ("Querying"), so a prune test
//     costs O(|L(u)|) shared-memory probes instead of a merge;
//   * the root's bit-parallel row (t distances + t mask pairs) is staged in
//     shared memory;
//   * the BFS is level-synchronous over a per-team queue in global memory
//     (each vertex enters at most once, so capacity n suffices); one warp
//     tests and expands one frontier vertex: the prune test reads u's t
//     bit-parallel distances in one coalesced load and fetches a mask pair
//     only for roots whose distance sum could reach the bound (d~ <= d + 2,
//     Sec. 5.3), then scans L(u) 32 entries per step; expansion reads u's
//     neighbours 32 per step and claims unvisited ones with an atomicOr on a
//     vertex-major bitmap [n][W] that holds one bit per root of the batch.
//   * Visited bits live per batch root, so the bitmap is cleared once per
//     batch instead of the per-root lazy reset of Sec. 4.5.1.
#include "pll_internal.cuh"

namespace pll {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int HT_LOG = 12;
constexpr uint32_t HT = 1u << HT_LOG;   // hash slots (16 KiB)
constexpr uint32_t HT_EMPTY = 0xffffffffu;

__device__ __forceinline__ uint32_t ht_slot(uint32_t h) { return (h * 0x9E3779B1u) >> (32 - HT_LOG); }

struct TeamSmem {
    uint32_t ht[HT];
    uint64_t bpm[2 * PLL_MAX_T];
    uint8_t bpd[PLL_MAX_T];
    uint32_t k;
    uint32_t tail;
};

// Root-array lookup: distance from v_k to hub h via L(v_k), or 255.
__device__ __forceinline__ uint32_t root_lookup(const TeamSmem &sm, bool use_ht,
                                                const uint32_t *__restrict__ rlab, uint32_t rlen,
                                                uint32_t h) {
    if (use_ht) {
        uint32_t s = ht_slot(h);
        for (;;) {
            uint32_t x = sm.ht[s];
            if (x == HT_EMPTY) return INF8;
            if (entry_hub(x) == h) return entry_dist(x);
            s = (s + 1) & (HT - 1);
        }
    }
    // long root label: binary search the sorted label in global memory
    uint32_t lo = 0, hi = rlen;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (entry_hub(rlab[mid]) < h) lo = mid + 1; else hi = mid;
    }
    return (lo < rlen && entry_hub(rlab[lo]) == h) ? entry_dist(rlab[lo]) : INF8;
}

// Query(v_k, u) <= level ?  (bit-parallel part first, then the normal label)
__device__ __forceinline__ bool prune_test(const PrunedBatch &b, const TeamSmem &sm, bool use_ht,
                                           const uint32_t *__restrict__ rlab, uint32_t rlen,
                                           uint32_t u, uint32_t level, int lane,
                                           uint32_t &n_scan, uint32_t &n_mask) {
    if (b.t) {
        bool p = false;
        const size_t row = (size_t)u * b.t;
        for (uint32_t i = lane; i < b.t; i += 32) {
            uint32_t du = b.bp_d[row + i], dk = sm.bpd[i];
            if (du == INF8 || dk == INF8) continue;
            uint32_t td = du + dk;
            if (td <= level) { p = true; continue; }
            if (td > level + 2) continue;
            ++n_mask;
            ulonglong2 m = *reinterpret_cast<const ulonglong2 *>(b.bp_m + 2 * (row + i));
            uint64_t k1 = sm.bpm[2 * i], k0 = sm.bpm[2 * i + 1];
            uint32_t red = (k1 & m.x) ? 2u : (((k0 & m.x) | (k1 & m.y)) ? 1u : 0u);
            if (td - red <= level) p = true;
        }
        if (__any_sync(FULL, p)) return true;
    }
    const uint32_t len = b.lab_len[u];
    if (len == 0) return false;
    const uint32_t *__restrict__ lab = b.pool + b.lab_off[u];
    for (uint32_t j = 0; j < len; j += 32) {
        bool p = false;
        if (j + lane < len) {
            ++n_scan;
            uint32_t e = lab[j + lane];
            uint32_t tk = root_lookup(sm, use_ht, rlab, rlen, entry_hub(e));
            p = (tk != INF8) && (tk + entry_dist(e) <= level);
        }
        if (__any_sync(FULL, p)) return true;
    }
    return false;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_pruned_batch(PrunedBatch b) {
    __shared__ TeamSmem sm;
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *__restrict__ Q = b.queues + (size_t)blockIdx.x * b.n;

    for (;;) {
        if (threadIdx.x == 0) sm.k = atomicAdd(b.next_root, 1u);
        __syncthreads();
        const uint32_t k = sm.k;
        if (k >= b.k1) break;
        if (b.inX[k]) {  // bit-parallel vertices get no pruned BFS
            __syncthreads();
            continue;
        }
        const uint32_t slot = k - b.k0;
        const uint32_t sw = slot >> 5, sbit = 1u << (slot & 31);

        // stage the root: bit-parallel row and the root array T
        for (uint32_t i = threadIdx.x; i < b.t; i += BLOCK) {
            const size_t ri = (size_t)k * b.t + i;
            sm.bpd[i] = b.bp_d[ri];
            sm.bpm[2 * i] = b.bp_m[2 * ri];
            sm.bpm[2 * i + 1] = b.bp_m[2 * ri + 1];
        }
        const uint32_t rlen = b.lab_len[k];
        const uint32_t *__restrict__ rlab = b.pool + b.lab_off[k];
        const bool use_ht = rlen <= HT / 2;
        if (use_ht) {
            for (uint32_t s = threadIdx.x; s < HT; s += BLOCK) sm.ht[s] = HT_EMPTY;
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < rlen; j += BLOCK) {
                uint32_t e = rlab[j];
                uint32_t s = ht_slot(entry_hub(e));
                while (atomicCAS(&sm.ht[s], HT_EMPTY, e) != HT_EMPTY) s = (s + 1) & (HT - 1);
            }
        }
        if (threadIdx.x == 0) {
            Q[0] = k;
            atomicOr(&b.visited[(size_t)k * b.W + sw], sbit);
            sm.tail = 1;
        }
        __syncthreads();

        uint32_t head = 0, level = 0;
        uint32_t n_scan = 0, n_mask = 0, n_exp = 0;  // per-thread work counters
        for (;;) {
            const uint32_t lvl_end = sm.tail;
            __syncthreads();  // everyone has read tail before it grows
            if (head >= lvl_end) break;
            if (threadIdx.x == 0) atomicAdd(b.visit_cnt, (unsigned long long)(lvl_end - head));
            for (uint32_t idx = head + warp; idx < lvl_end; idx += NW) {
                const uint32_t u = Q[idx];
                // the root is never pruned: Query(v_k, v_k) >= 2 for v_k outside X
                if (level > 0 && prune_test(b, sm, use_ht, rlab, rlen, u, level, lane, n_scan, n_mask))
                    continue;
                if (lane == 0) {
                    unsigned long long pos = atomicAdd(b.out_cnt, 1ull);
                    if (pos < b.out_cap) b.out[pos] = pack_tuple(u, k, level);
                    else atomicOr(b.err, ERR_BUF);
                }
                const uint32_t eb = b.roff[u], ee = b.roff[u + 1];
                if (lane == 0) n_exp += ee - eb;
                for (uint32_t x = eb; x < ee; x += 32) {
                    bool fresh = false;
                    uint32_t w = 0;
                    if (x + lane < ee) {
                        w = b.rcol[x + lane];
                        uint32_t *word = &b.visited[(size_t)w * b.W + sw];
                        if (!(*(volatile uint32_t *)word & sbit)) fresh = !(atomicOr(word, sbit) & sbit);
                    }
                    if (fresh && level + 1 >= INF8) {
                        atomicOr(b.err, ERR_DEPTH);
                        fresh = false;
                    }
                    const unsigned m = __ballot_sync(FULL, fresh);
                    if (m) {
                        uint32_t base = 0;
                        if (lane == 0) base = atomicAdd(&sm.tail, (uint32_t)__popc(m));
                        base = __shfl_sync(FULL, base, 0);
                        if (fresh) Q[base + __popc(m & ((1u << lane) - 1u))] = w;
                    }
                }
            }
            __syncthreads();
            head = lvl_end;
            ++level;
        }
        // fold the work counters (warp sums, one atomic per warp and root)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_scan += __shfl_xor_sync(FULL, n_scan, o);
            n_mask += __shfl_xor_sync(FULL, n_mask, o);
        }
        if (lane == 0 && (n_scan | n_mask | n_exp)) {
            atomicAdd(&b.work[0], (unsigned long long)n_scan);
            atomicAdd(&b.work[1], (unsigned long long)n_mask);
            atomicAdd(&b.work[2], (unsigned long long)n_exp);
        }
        __syncthreads();
    }
}

}  // namespace

int pruned_max_grid(uint32_t block, int *grid) {
    int dev = 0, sms = 0, per = 0;
    PLL_TRY(cudaGetDevice(&dev));
    PLL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaError_t e;
    switch (block) {
        case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pruned_batch<128>, 128, 0); break;
        case 512: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pruned_batch<512>, 512, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pruned_batch<256>, 256, 0); break;
    }
    PLL_TRY(e);
    if (per < 1) per = 1;
    *grid = sms * per;
    return PLL_OK;
}

int pruned_launch(const PrunedBatch &b, int grid, uint32_t block, cudaStream_t s) {
    switch (block) {
        case 128: k_pruned_batch<128><<<grid, 128, 0, s>>>(b); break;
        case 512: k_pruned_batch<512><<<grid, 512, 0, s>>>(b); break;
        default: k_pruned_batch<256><<<grid, 256, 0, s>>>(b); break;
    }
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

}  // namespace pll
