// k_query.cu -- batched distance queries over a built index.
//
// d(s, t) = min( bit-parallel query (Sec. 5.3), Query(s, t, L) (Sec. 3.3) ).
//
// A persistent grid (a few CTAs per SM) walks the pairs; one warp answers one
// pair. A launch too small to fill the GPU that way (up to 4 pairs per
// resident block) gives each pair 2, 4 or 8 warps instead, which split the
// label scan and meet in shared memory. Lanes own bit-parallel roots (lane, lane + 32): the t distance bytes
// of s and of t arrive in one coalesced load each, and d~_i = d(s,r_i) +
// d(r_i,t). Since the answer through {r_i} U S_{r_i} lies in [d~_i - 2, d~_i],
// only roots with d~_i <= min_i d~_i + 1 can decide the minimum, and only
// those whose d~_i - 2 beats the normal-label answer fetch their 16-byte mask
// pairs. The normal labels are hub-sorted (hub ranks, Sec. 4.5.1): a warp
// merges them 32 entries at a time (the merge join of Sec. 3.3, with the
// comparisons of a window done by shuffles), or, when one label is much
// longer, each lane takes entries of the shorter label and binary-searches the
// longer one; both find the same common hubs. No sentinel is needed
// (Sec. 4.5.2): bounds are explicit.
#include <atomic>

#include "pll_internal.cuh"

namespace pll {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t BIG = 1u << 20;

struct QueryArgs {
    uint32_t n, t, tp;
    const uint32_t *inv;
    const uint32_t *graph;  // graph of each rank (batch indices), or null
    const uint8_t *bp_d;
    const uint64_t *bp_m;
    const uint64_t *lab_off;
    const uint32_t *lab;
    const uint32_t *src, *dst;
    uint32_t stride;  // pair qi is (src[qi * stride], dst[qi * stride])
    uint64_t q;
    uint8_t *out;
    unsigned long long *err;  // [0] finite distance >= 255, [1] id >= n
};

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ uint32_t bp_reduce(uint32_t td, const uint64_t *__restrict__ ms,
                                              const uint64_t *__restrict__ mt) {
    ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(ms);
    ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(mt);
    if (a.x & b.x) return td - 2;
    if ((a.y & b.x) | (a.x & b.y)) return td - 1;
    return td;
}

// Resolves the cases that need no labels. Returns true with *ans set when
// the pair is decided (bad id, s == t, different graphs of a batch index).
__device__ __forceinline__ bool trivial_pair(const QueryArgs &a, uint32_t sid, uint32_t tid,
                                             uint32_t *s, uint32_t *t, uint32_t *ans, bool *bad) {
    *bad = false;
    if (sid >= a.n || tid >= a.n) { *ans = INF8; *bad = true; return true; }
    *s = a.inv[sid];
    *t = a.inv[tid];
    if (*s == *t) { *ans = 0; return true; }
    // graphs of a batch share slot numbers but not roots: no distance across
    if (a.graph && a.graph[*s] != a.graph[*t]) { *ans = INF8; return true; }
    return false;
}

// Bit-parallel distances d~ of the lane's roots (lane, lane + 32) and their
// warp-wide minimum d*.
__device__ __forceinline__ void bp_tilde(const QueryArgs &a, uint32_t s, uint32_t t, int lane,
                                         uint32_t *td0, uint32_t *td1, uint32_t *dstar) {
    *td0 = BIG;
    *td1 = BIG;
    const size_t ds = (size_t)s * a.tp, dt = (size_t)t * a.tp;
    if (lane < a.t) {
        uint32_t x = a.bp_d[ds + lane], y = a.bp_d[dt + lane];
        if (x != INF8 && y != INF8) *td0 = x + y;
    }
    if (lane + 32 < a.t) {
        uint32_t x = a.bp_d[ds + lane + 32], y = a.bp_d[dt + lane + 32];
        if (x != INF8 && y != INF8) *td1 = x + y;
    }
    *dstar = warp_min(min(*td0, *td1));
}

// min over common hubs of the two normal labels, over the entries
// first, first + step, ... of the shorter label taken by this lane's warp.
__device__ __forceinline__ uint32_t label_min(const QueryArgs &a, uint32_t s, uint32_t t, int lane,
                                              uint32_t first, uint32_t step) {
    const uint64_t os = a.lab_off[s], ot = a.lab_off[t];
    const uint32_t ls = (uint32_t)(a.lab_off[s + 1] - os), lt = (uint32_t)(a.lab_off[t + 1] - ot);
    const uint32_t *A = a.lab + (ls <= lt ? os : ot);
    const uint32_t *B = a.lab + (ls <= lt ? ot : os);
    const uint32_t la = ls <= lt ? ls : lt, lb = ls <= lt ? lt : ls;
    uint32_t best = BIG;
    for (uint32_t j = first; j < la; j += step) {
        if (j + lane < la) {
            const uint32_t e = A[j + lane], h = entry_hub(e);
            uint32_t lo = 0, hi = lb;
            while (lo < hi) {
                uint32_t mid = (lo + hi) >> 1;
                if (entry_hub(B[mid]) < h) lo = mid + 1; else hi = mid;
            }
            if (lo < lb && entry_hub(B[lo]) == h) best = min(best, entry_dist(e) + entry_dist(B[lo]));
        }
    }
    return warp_min(best);
}

#ifndef PLL_MERGE_RATIO
#define PLL_MERGE_RATIO 4
#endif

// min over common hubs of the two normal labels for one warp: a merge of the
// hub-sorted labels 32 entries at a time (the merge join of Sec. 3.3 done by
// a warp). Each lane holds one entry of the shorter label's window and finds
// its hub in the other window by a 5-step search over the lanes (shuffles);
// then the window whose last hub is smaller is passed whole and the other is
// advanced past the hubs not above it, which can meet nothing that is left.
// Labels read once, in coalesced 128-byte rows. When one label is more than
// PLL_MERGE_RATIO times longer, binary searches of its entries (label_min)
// touch less of it and are used instead. os / ls, ot / lt: the offsets and
// lengths of L(s) and L(t), already loaded by the caller.
__device__ __forceinline__ uint32_t label_min_merge_at(const QueryArgs &a, uint32_t s, uint32_t t,
                                                      uint64_t os, uint32_t ls, uint64_t ot, uint32_t lt,
                                                      int lane) {
    const uint32_t la = ls <= lt ? ls : lt, lb = ls <= lt ? lt : ls;
    if (la == 0) return BIG;
    if (lb > PLL_MERGE_RATIO * la) return label_min(a, s, t, lane, 0, 32);
    const uint32_t *A = a.lab + (ls <= lt ? os : ot);
    const uint32_t *B = a.lab + (ls <= lt ? ot : os);
    uint32_t best = BIG, ia = 0, ib = 0;
    while (ia < la && ib < lb) {
        const uint32_t na = min(32u, la - ia), nb = min(32u, lb - ib);
        const bool va = (uint32_t)lane < na, vb = (uint32_t)lane < nb;
        const uint32_t ea = va ? A[ia + lane] : NONE;  // padding sorts after every hub
        const uint32_t eb = vb ? B[ib + lane] : NONE;
        const uint32_t ha = entry_hub(ea), hb = entry_hub(eb);
        // lower bound of ha in the window of B held across the lanes
        uint32_t pos = 0;
#pragma unroll
        for (uint32_t stp = 16; stp > 0; stp >>= 1)
            if (entry_hub(__shfl_sync(FULL, eb, pos + stp - 1)) < ha) pos += stp;
        const uint32_t ep = __shfl_sync(FULL, eb, pos);
        if (va && pos < nb && entry_hub(ep) == ha) best = min(best, entry_dist(ea) + entry_dist(ep));
        const uint32_t lastA = entry_hub(__shfl_sync(FULL, ea, na - 1));
        const uint32_t lastB = entry_hub(__shfl_sync(FULL, eb, nb - 1));
        if (lastA <= lastB) {
            ia += na;
            ib += __popc(__ballot_sync(FULL, vb && hb <= lastA));
        } else {
            ib += nb;
            ia += __popc(__ballot_sync(FULL, va && ha <= lastB));
        }
    }
    return warp_min(best);
}

// The bit-parallel answer, fetching masks only where they can beat `best`
// (the normal-label answer), then the final byte.
__device__ __forceinline__ uint32_t finish_pair(const QueryArgs &a, uint32_t s, uint32_t t, int lane,
                                                uint32_t td0, uint32_t td1, uint32_t dstar,
                                                uint32_t best) {
    const size_t rs = (size_t)s * a.t, rt = (size_t)t * a.t;
    uint32_t bpb = BIG;
    if (dstar < BIG) {
        bpb = dstar;
        if (td0 <= dstar + 1 && td0 - 2 < best && td0 - 2 < bpb)
            bpb = min(bpb, bp_reduce(td0, a.bp_m + 2 * (rs + lane), a.bp_m + 2 * (rt + lane)));
        if (td1 <= dstar + 1 && td1 - 2 < best && td1 - 2 < bpb)
            bpb = min(bpb, bp_reduce(td1, a.bp_m + 2 * (rs + lane + 32), a.bp_m + 2 * (rt + lane + 32)));
        bpb = warp_min(bpb);
    }
    return min(best, bpb);
}

// the answer byte of a pair's minimum (255 for none or for a finite distance
// of 255 or more; the latter is counted as an error)
__device__ __forceinline__ uint32_t answer_byte(const QueryArgs &a, uint32_t best) {
    if (best >= BIG) return INF8;
    if (best >= INF8) {
        atomicAdd(a.err, 1ull);
        return INF8;
    }
    return best;
}

__device__ __forceinline__ void store_answer(const QueryArgs &a, uint64_t qi, uint32_t best) {
    a.out[qi] = (uint8_t)answer_byte(a, best);
}

// One warp per pair, PG pairs at a time: lane j < PG first fetches pair j's
// ids, ranks and label offsets (three dependent loads, in flight for PG pairs
// at once instead of one after another), and answers the trivial pairs; the
// warp then answers the others one by one from the lanes' registers. PG is
// 32 for launches that fill the GPU that way and smaller for launches that
// would otherwise leave warps idle. Eight CTAs per SM (32 registers a
// thread): the kernel is bound by the latency of its loads, so it wants every
// resident warp it can get.
template <int PG>
__global__ void __launch_bounds__(256, 8) k_query(QueryArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t q0 = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * PG; q0 < a.q;
         q0 += warps * PG) {
        const uint64_t qi = q0 + lane;
        const bool mine = lane < PG && qi < a.q;
        uint32_t s = 0, t = 0, ans = 0;
        bool bad = false, open = false;
        uint64_t os = 0, ot = 0;
        uint32_t ls = 0, lt = 0;
        if (mine) {
            open = !trivial_pair(a, a.src[qi * a.stride], a.dst[qi * a.stride], &s, &t, &ans, &bad);
            if (open) {
                os = a.lab_off[s];
                ot = a.lab_off[t];
                ls = (uint32_t)(a.lab_off[s + 1] - os);
                lt = (uint32_t)(a.lab_off[t + 1] - ot);
            } else if (bad) {
                atomicAdd(a.err + 1, 1ull);
            }
        }
        for (uint32_t m = __ballot_sync(FULL, open); m; m &= m - 1) {
            const int j = __ffs(m) - 1;
            const uint32_t sj = __shfl_sync(FULL, s, j), tj = __shfl_sync(FULL, t, j);
            const uint64_t osj = __shfl_sync(FULL, os, j), otj = __shfl_sync(FULL, ot, j);
            const uint32_t lsj = __shfl_sync(FULL, ls, j), ltj = __shfl_sync(FULL, lt, j);
            uint32_t td0, td1, dstar;
            bp_tilde(a, sj, tj, lane, &td0, &td1, &dstar);
            const uint32_t best = finish_pair(a, sj, tj, lane, td0, td1, dstar,
                                              label_min_merge_at(a, sj, tj, osj, lsj, otj, ltj, lane));
            if (lane == j) ans = answer_byte(a, best);  // best is the same on every lane
        }
        // the group's answers in one coalesced store (the output may be host
        // memory that the GPU writes directly)
        if (mine) a.out[qi] = (uint8_t)ans;
    }
}

// G warps of a block per pair, for launches too small to fill the GPU with
// one warp per pair: the label scan is split G ways (warp g takes entries
// 32 g, 32 (g + G), ...), which shortens the chain of dependent loads each
// pair waits on; the partial minima meet in shared memory.
template <int G>
__global__ void __launch_bounds__(256) k_query_wide(QueryArgs a) {
    __shared__ uint32_t part[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int member = warp % G;
    const uint64_t qi = (uint64_t)blockIdx.x * (8 / G) + warp / G;
    uint32_t s = 0, t = 0, ans = 0, td0 = BIG, td1 = BIG, dstar = BIG;
    bool bad = false, decided = true;
    if (qi < a.q) decided = trivial_pair(a, a.src[qi * a.stride], a.dst[qi * a.stride], &s, &t, &ans, &bad);
    if (!decided) {
        if (member == 0) bp_tilde(a, s, t, lane, &td0, &td1, &dstar);
        const uint32_t m = label_min(a, s, t, lane, 32u * member, 32u * G);
        if (lane == 0) part[warp] = m;
    }
    __syncthreads();  // every warp of the block arrives: no early exit above
    if (member != 0 || qi >= a.q) return;
    if (decided) {
        if (lane == 0) {
            a.out[qi] = (uint8_t)ans;
            if (bad) atomicAdd(a.err + 1, 1ull);
        }
        return;
    }
    uint32_t best = BIG;
#pragma unroll
    for (int g = 0; g < G; ++g) best = min(best, part[warp + g]);
    best = finish_pair(a, s, t, lane, td0, td1, dstar, best);
    if (lane == 0) store_answer(a, qi, best);
}

}  // namespace

int query_launch(const pll_index *ix, const uint32_t *d_src, const uint32_t *d_dst, uint64_t q,
                 uint8_t *d_out, cudaStream_t s) {
    return query_launch_strided(ix, d_src, d_dst, 1, q, d_out, s);
}

int query_launch_strided(const pll_index *ix, const uint32_t *d_src, const uint32_t *d_dst,
                         uint32_t stride, uint64_t q, uint8_t *d_out, cudaStream_t s) {
    if (q == 0) return PLL_OK;
    // resident blocks of k_query on this device (SMs x blocks per SM), looked
    // up once per device: the serving loop launches it thousands of times
    static std::atomic<int> resident[64];
    int dev = 0;
    PLL_TRY(cudaGetDevice(&dev));
    int res = dev < 64 ? resident[dev].load(std::memory_order_relaxed) : 0;
    if (res == 0) {
        int sms = 0, per = 0;
        PLL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        PLL_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_query<32>, 256, 0));
        res = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
        if (dev < 64) resident[dev].store(res, std::memory_order_relaxed);
    }
    QueryArgs a{ix->n, ix->t, ix->tp, ix->d_inv, ix->d_graph, ix->d_bp_d, ix->d_bp_m, ix->d_lab_off, ix->d_lab,
                d_src, d_dst, stride, q, d_out, ix->d_qerr};
    // Pairs one warp each would leave most of the GPU idle: give each pair G
    // warps (8, 4 or 2; 8 / G pairs per block) while the ceil(q G / 8)
    // blocks still fit in one resident wave.
    const uint64_t R = (uint64_t)res;
    if (q <= R) {
        k_query_wide<8><<<(unsigned)q, 256, 0, s>>>(a);
    } else if (q <= 2 * R) {
        k_query_wide<4><<<(unsigned)((q + 1) / 2), 256, 0, s>>>(a);
    } else if (q <= 4 * R) {
        k_query_wide<2><<<(unsigned)((q + 3) / 4), 256, 0, s>>>(a);
    } else {
        // pairs per warp group: as many as keep every resident warp busy (R
        // blocks of 8 warps), up to 32
        const uint64_t per = q / (R * 8);
        if (per >= 32) k_query<32><<<(unsigned)R, 256, 0, s>>>(a);
        else if (per >= 8) k_query<8><<<(unsigned)R, 256, 0, s>>>(a);
        else if (per >= 2) k_query<2><<<(unsigned)R, 256, 0, s>>>(a);
        else k_query<1><<<(unsigned)R, 256, 0, s>>>(a);
    }
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

}  // namespace pll
