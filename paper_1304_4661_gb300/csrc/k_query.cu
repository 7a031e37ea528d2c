// k_query.cu -- batched distance queries over a built index.
//
// d(s, t) = min( bit-parallel query (Sec. 5.3), Query(s, t, L) (Sec. 3.3) ).
//
// A persistent grid (a few CTAs per SM) walks the pairs; one warp answers one
// pair. Lanes own bit-parallel roots (lane, lane + 32): the t distance bytes
// of s and of t arrive in one coalesced load each, and d~_i = d(s,r_i) +
// d(r_i,t). Since the answer through {r_i} U S_{r_i} lies in [d~_i - 2, d~_i],
// only roots with d~_i <= min_i d~_i + 1 can decide the minimum, and only
// those whose d~_i - 2 beats the normal-label answer fetch their 16-byte mask
// pairs. The normal labels are hub-sorted (hub ranks, Sec. 4.5.1); instead of
// the sequential merge join of Sec. 3.3 each lane takes entries of the
// shorter label and binary-searches the longer one, which finds the same
// common hubs. No sentinel is needed (Sec. 4.5.2): bounds are explicit.
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

__global__ void __launch_bounds__(256) k_query(QueryArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t qi = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < a.q; qi += warps) {
        const uint32_t sid = a.src[qi], tid = a.dst[qi];
        if (sid >= a.n || tid >= a.n) {
            if (lane == 0) { a.out[qi] = INF8; atomicAdd(a.err + 1, 1ull); }
            continue;
        }
        const uint32_t s = a.inv[sid], t = a.inv[tid];
        if (s == t) {
            if (lane == 0) a.out[qi] = 0;
            continue;
        }
        // graphs of a batch share slot numbers but not roots: no distance across
        if (a.graph && a.graph[s] != a.graph[t]) {
            if (lane == 0) a.out[qi] = INF8;
            continue;
        }
        // bit-parallel distances: d~ per lane root
        uint32_t td0 = BIG, td1 = BIG;
        const size_t rs = (size_t)s * a.t, rt = (size_t)t * a.t;
        const size_t ds = (size_t)s * a.tp, dt = (size_t)t * a.tp;
        if (lane < a.t) {
            uint32_t x = a.bp_d[ds + lane], y = a.bp_d[dt + lane];
            if (x != INF8 && y != INF8) td0 = x + y;
        }
        if (lane + 32 < a.t) {
            uint32_t x = a.bp_d[ds + lane + 32], y = a.bp_d[dt + lane + 32];
            if (x != INF8 && y != INF8) td1 = x + y;
        }
        const uint32_t dstar = warp_min(min(td0, td1));

        // normal labels: lanes take entries of the shorter label
        const uint64_t os = a.lab_off[s], ot = a.lab_off[t];
        const uint32_t ls = (uint32_t)(a.lab_off[s + 1] - os), lt = (uint32_t)(a.lab_off[t + 1] - ot);
        const uint32_t *A = a.lab + (ls <= lt ? os : ot);
        const uint32_t *B = a.lab + (ls <= lt ? ot : os);
        const uint32_t la = ls <= lt ? ls : lt, lb = ls <= lt ? lt : ls;
        uint32_t best = BIG;
        for (uint32_t j = 0; j < la; j += 32) {
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
        best = warp_min(best);

        // masks only where they can lower the answer
        uint32_t bpb = BIG;
        if (dstar < BIG) {
            bpb = dstar;
            if (td0 <= dstar + 1 && td0 - 2 < best && td0 - 2 < bpb)
                bpb = min(bpb, bp_reduce(td0, a.bp_m + 2 * (rs + lane), a.bp_m + 2 * (rt + lane)));
            if (td1 <= dstar + 1 && td1 - 2 < best && td1 - 2 < bpb)
                bpb = min(bpb, bp_reduce(td1, a.bp_m + 2 * (rs + lane + 32), a.bp_m + 2 * (rt + lane + 32)));
            bpb = warp_min(bpb);
        }
        best = min(best, bpb);
        if (lane == 0) {
            if (best >= BIG) {
                a.out[qi] = INF8;
            } else if (best >= INF8) {
                a.out[qi] = INF8;
                atomicAdd(a.err, 1ull);
            } else {
                a.out[qi] = (uint8_t)best;
            }
        }
    }
}

}  // namespace

int query_launch(const pll_index *ix, const uint32_t *d_src, const uint32_t *d_dst, uint64_t q,
                 uint8_t *d_out, cudaStream_t s) {
    if (q == 0) return PLL_OK;
    int dev = 0, sms = 148, per = 0;
    PLL_TRY(cudaGetDevice(&dev));
    PLL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PLL_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_query, 256, 0));
    if (per < 1) per = 1;
    uint64_t want = (q * 32 + 255) / 256;
    uint64_t cap = (uint64_t)sms * per;
    int grid = (int)(want < cap ? want : cap);
    QueryArgs a{ix->n, ix->t, ix->tp, ix->d_inv, ix->d_graph, ix->d_bp_d, ix->d_bp_m, ix->d_lab_off, ix->d_lab,
                d_src, d_dst, q, d_out, ix->d_qerr};
    k_query<<<grid, 256, 0, s>>>(a);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

}  // namespace pll
