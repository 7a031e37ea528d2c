// k_bp.cu -- bit-parallel BFSs (Alg. 3, Sec. 5.2) for all t roots at once.
//
// Alg. 3 walks one root's BFS with two queues and two edge lists per level:
// E0 (edges inside level L) updates S^0 of level L, then E1 (edges from level
// L to L+1) carries S^{-1} and S^0 down one level. Sec. 5.2 writes the same
// recurrence per vertex:
//   S^{-1}(v) = OR of S^{-1}(w) over neighbours w one level closer to r,
//   S^0(v)    = OR of S^0(w) over those w  OR  S^{-1}(w) over same-level w.
// Here that per-vertex form is evaluated as a pull: every vertex reads its
// neighbours' rows instead of being pushed to, and all t roots advance level
// by level together. State is vertex-major ([n][tp] distances, [n][t] mask
// pairs); one warp works on one (vertex, chunk of <= CHUNK arcs) item, each
// lane owning roots lane and lane + 32, so a neighbour's distance bytes
// arrive in one coalesced load and its 16-byte mask pair is read only for the
// roots where it is a parent (or a same-level neighbour). Vertices of degree
// above CHUNK are split over several items whose partial ORs meet in 64-bit
// atomicOr, so a hub of any degree costs no more latency than CHUNK arcs.
//
// Per level L, two launches:
//   same-level pass (E0 of level L): S^0(u) |= S^{-1}(w) for u, w at level L;
//   next-level pass (E1 of level L): every u still at distance 255 for root i
//     with some neighbour at level L joins level L+1 with the OR of those
//     neighbours' S^{-1} and S^0.
// The host loops until a next-level pass discovers nothing (from level 1 on:
// level 1 can hold only seeded members of S_r). A last pass stores S^0 minus
// S^{-1}: Sec. 5.1 defines S^0 as the members at difference exactly 0, and the
// recurrence can leave S^{-1} members in it (they never change a query).
#include <algorithm>

#include <cub/cub.cuh>

#include "pll_internal.cuh"

namespace pll {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t CHUNK = 256;

// one block per (graph, slot): root slot q = g * t + i seeds slot i; the
// graphs of a batch are disjoint, so their slot-i BFSs run as one sweep
__global__ void k_bp_seed(uint32_t t, uint32_t tp, const uint32_t *__restrict__ root,
                          const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ S,
                          uint8_t *bp_d, uint64_t *bp_m) {
    const uint32_t q = blockIdx.x, i = q % t, j = threadIdx.x;
    const uint32_t r = root[q];
    if (r == NONE) return;
    if (j == 0) bp_d[(size_t)r * tp + i] = 0;
    if (j < cnt[q]) {
        uint32_t v = S[(size_t)q * BPW + j];
        bp_d[(size_t)v * tp + i] = 1;
        bp_m[2 * ((size_t)v * t + i)] = 1ull << j;  // S^{-1}(v) = {v}
    }
}

__global__ void k_chunk_counts(uint32_t n, const uint32_t *__restrict__ roff, uint32_t *cnt) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        cnt[u] = (roff[u + 1] - roff[u] + CHUNK - 1) / CHUNK;
}

__global__ void k_chunk_fill(uint32_t n, const uint32_t *__restrict__ coff, uint32_t *items) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        for (uint32_t j = coff[u]; j < coff[u + 1]; ++j) items[j] = u;
}

struct BpArgs {
    uint32_t n, t, tp, L;
    const uint32_t *roff, *rcol, *items, *coff;
    uint32_t nitems;
    uint8_t *bp_d;
    uint64_t *bp_m;
    uint32_t *changed, *err;
};

// Loads neighbour ids 32 at a time and hands them to the whole warp.
template <class F>
__device__ __forceinline__ void for_each_neighbour(const uint32_t *__restrict__ rcol, uint32_t b,
                                                   uint32_t e, int lane, F &&f) {
    for (uint32_t x = b; x < e; x += 32) {
        const uint32_t mine = (x + lane < e) ? rcol[x + lane] : 0;
        const uint32_t cnt = (e - x) < 32 ? (e - x) : 32;
        for (uint32_t j = 0; j < cnt; ++j) f(__shfl_sync(FULL, mine, j));
    }
}

__device__ __forceinline__ void item_range(const BpArgs &a, uint32_t j, uint32_t &u, uint32_t &b,
                                           uint32_t &e, bool &multi) {
    u = a.items[j];
    const uint32_t c = j - a.coff[u];
    const uint32_t lo = a.roff[u], hi = a.roff[u + 1];
    b = lo + c * CHUNK;
    e = min(b + CHUNK, hi);
    multi = hi - lo > CHUNK;
}

__global__ void k_bp_same_level(BpArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t i0 = lane, i1 = lane + 32;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t L = a.L;
    for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < a.nitems; j += warps) {
        uint32_t u, b, e;
        bool multi;
        item_range(a, j, u, b, e, multi);
        const size_t row = (size_t)u * a.t, drow = (size_t)u * a.tp;
        const bool a0 = i0 < a.t && a.bp_d[drow + i0] == L;
        const bool a1 = i1 < a.t && a.bp_d[drow + i1] == L;
        if (!__any_sync(FULL, a0 || a1)) continue;
        uint64_t acc0 = 0, acc1 = 0;
        for_each_neighbour(a.rcol, b, e, lane, [&](uint32_t w) {
            const size_t wr = (size_t)w * a.t, wd = (size_t)w * a.tp;
            if (a0 && a.bp_d[wd + i0] == L) acc0 |= a.bp_m[2 * (wr + i0)];
            if (a1 && a.bp_d[wd + i1] == L) acc1 |= a.bp_m[2 * (wr + i1)];
        });
        unsigned long long *m = reinterpret_cast<unsigned long long *>(a.bp_m);
        if (a0 && acc0) {
            if (multi) atomicOr(&m[2 * (row + i0) + 1], (unsigned long long)acc0);
            else m[2 * (row + i0) + 1] |= acc0;
        }
        if (a1 && acc1) {
            if (multi) atomicOr(&m[2 * (row + i1) + 1], (unsigned long long)acc1);
            else m[2 * (row + i1) + 1] |= acc1;
        }
    }
}

__global__ void k_bp_next_level(BpArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t i0 = lane, i1 = lane + 32;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t L = a.L;
    bool any = false;
    for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < a.nitems; j += warps) {
        uint32_t u, b, e;
        bool multi;
        item_range(a, j, u, b, e, multi);
        const size_t row = (size_t)u * a.t, drow = (size_t)u * a.tp;
        // several chunks of one vertex: a sibling chunk may already have set
        // L + 1 in this pass; its masks are merged by atomicOr either way
        const uint32_t d0 = i0 < a.t ? a.bp_d[drow + i0] : 0;
        const uint32_t d1 = i1 < a.t ? a.bp_d[drow + i1] : 0;
        const bool a0 = i0 < a.t && (d0 == INF8 || (multi && d0 == L + 1));
        const bool a1 = i1 < a.t && (d1 == INF8 || (multi && d1 == L + 1));
        if (!__any_sync(FULL, a0 || a1)) continue;
        bool f0 = false, f1 = false;
        uint64_t m10 = 0, m00 = 0, m11 = 0, m01 = 0;
        for_each_neighbour(a.rcol, b, e, lane, [&](uint32_t w) {
            const size_t wr = (size_t)w * a.t, wd = (size_t)w * a.tp;
            if (a0 && a.bp_d[wd + i0] == L) {
                f0 = true;
                m10 |= a.bp_m[2 * (wr + i0)];
                m00 |= a.bp_m[2 * (wr + i0) + 1];
            }
            if (a1 && a.bp_d[wd + i1] == L) {
                f1 = true;
                m11 |= a.bp_m[2 * (wr + i1)];
                m01 |= a.bp_m[2 * (wr + i1) + 1];
            }
        });
        if (f0 || f1) {
            if (L + 1 >= INF8) {
                atomicOr(a.err, ERR_DEPTH);
                continue;
            }
            any = true;
        }
        unsigned long long *m = reinterpret_cast<unsigned long long *>(a.bp_m);
        if (f0) {
            a.bp_d[drow + i0] = (uint8_t)(L + 1);
            if (multi) {
                atomicOr(&m[2 * (row + i0)], (unsigned long long)m10);
                atomicOr(&m[2 * (row + i0) + 1], (unsigned long long)m00);
            } else {
                m[2 * (row + i0)] = m10;
                m[2 * (row + i0) + 1] = m00;
            }
        }
        if (f1) {
            a.bp_d[drow + i1] = (uint8_t)(L + 1);
            if (multi) {
                atomicOr(&m[2 * (row + i1)], (unsigned long long)m11);
                atomicOr(&m[2 * (row + i1) + 1], (unsigned long long)m01);
            } else {
                m[2 * (row + i1)] = m11;
                m[2 * (row + i1) + 1] = m01;
            }
        }
    }
    if (__any_sync(FULL, any) && lane == 0) atomicOr(a.changed, 1u);
}

// S^0 := S^0 minus S^{-1} for every (v, i)
__global__ void k_bp_finish(size_t nt, ulonglong2 *m) {
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < nt;
         x += (size_t)gridDim.x * blockDim.x) {
        ulonglong2 p = m[x];
        p.y &= ~p.x;
        m[x] = p;
    }
}

}  // namespace

int bp_run(uint32_t n, uint32_t t, uint32_t graphs, const uint32_t *d_roff, const uint32_t *d_rcol,
           const uint32_t *d_root, const uint32_t *d_cnt, const uint32_t *d_S, uint8_t *d_bp_d,
           uint64_t *d_bp_m, uint32_t *d_err, cudaStream_t s, uint32_t *levels) {
    *levels = 0;
    if (t == 0 || n == 0) return PLL_OK;
    if (t > PLL_MAX_T) return PLL_E_RANGE;
    const size_t nt = (size_t)n * t;
    const uint32_t tp = bp_stride(t);
    PLL_TRY(cudaMemsetAsync(d_bp_d, 0xff, (size_t)n * tp, s));
    PLL_TRY(cudaMemsetAsync(d_bp_m, 0, nt * 16, s));
    k_bp_seed<<<t * graphs, BPW, 0, s>>>(t, tp, d_root, d_cnt, d_S, d_bp_d, d_bp_m);
    PLL_TRY(cudaGetLastError());

    // work items: (vertex, chunk of <= CHUNK arcs)
    PoolMem cnt(s), coff(s), items(s), temp(s), flag(s);
    PLL_CHECK(cnt.alloc(((size_t)n + 1) * 4));
    PLL_CHECK(coff.alloc(((size_t)n + 1) * 4));
    PLL_TRY(cudaMemsetAsync(cnt.p, 0, ((size_t)n + 1) * 4, s));
    const int g1 = (int)std::min<uint64_t>((n + 255) / 256, 65535);
    k_chunk_counts<<<g1, 256, 0, s>>>(n, d_roff, cnt.as<uint32_t>());
    size_t tb = 0;
    PLL_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt.as<uint32_t>(), coff.as<uint32_t>(),
                                          (int)n + 1, s));
    PLL_CHECK(temp.alloc(tb));
    PLL_TRY(cub::DeviceScan::ExclusiveSum(temp.p, tb, cnt.as<uint32_t>(), coff.as<uint32_t>(),
                                          (int)n + 1, s));
    uint32_t nitems = 0;
    PLL_TRY(cudaMemcpyAsync(&nitems, coff.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    PLL_CHECK(items.alloc(std::max<size_t>((size_t)nitems * 4, 4)));
    k_chunk_fill<<<g1, 256, 0, s>>>(n, coff.as<uint32_t>(), items.as<uint32_t>());
    PLL_TRY(cudaGetLastError());

    PLL_CHECK(flag.alloc(4));
    uint32_t *h_flag = nullptr;
    PLL_TRY(host_malloc(&h_flag, 4));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = ((uint64_t)nitems * 32 + 255) / 256;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 16));
    BpArgs a{n, t, tp, 0, d_roff, d_rcol, items.as<uint32_t>(), coff.as<uint32_t>(), nitems,
             d_bp_d, d_bp_m, flag.as<uint32_t>(), d_err};
    int st = PLL_OK;
    for (uint32_t L = 0; L < INF8; ++L) {
        a.L = L;
        cudaError_t e = cudaMemsetAsync(flag.p, 0, 4, s);
        if (e == cudaSuccess) {
            k_bp_same_level<<<grid, 256, 0, s>>>(a);
            k_bp_next_level<<<grid, 256, 0, s>>>(a);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_flag, flag.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = cuda_status(e); break; }
        *levels = L + 1;
        // level 1 may consist of the seeded members of S_r alone (nothing is
        // "discovered" from the root then), so it is always processed
        if (*h_flag == 0 && L >= 1) break;
    }
    host_free(h_flag);
    if (st == PLL_OK) {
        k_bp_finish<<<(int)std::min<size_t>((nt + 255) / 256, (size_t)sms * 32), 256, 0, s>>>(
            nt, reinterpret_cast<ulonglong2 *>(d_bp_m));
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // before the temporaries are freed
        if (e != cudaSuccess) st = cuda_status(e);
    }
    return st;
}

}  // namespace pll

namespace pll {

// The same bit-parallel stage as bp_run, for callers that provide all device
// scratch: nothing is allocated (the level flag is read into a host stack
// variable). scratch must be 256-byte aligned and at least
// bp_scratch_bytes(n, nnz) long; S-members / roots must already be chosen.
size_t bp_scratch_bytes(uint32_t n, uint64_t nnz, size_t *cub_bytes) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, (uint32_t *)nullptr, (uint32_t *)nullptr, (int)n + 1);
    if (cub_bytes) *cub_bytes = tb;
    const size_t items = (size_t)n + (nnz + CHUNK - 1) / CHUNK;
    return up(((size_t)n + 1) * 4) * 2 + up(items * 4) + up(8) + up(tb);
}

int bp_run_in(uint32_t n, uint32_t t, const uint32_t *d_roff, const uint32_t *d_rcol,
              uint64_t nnz, const uint32_t *d_root, const uint32_t *d_cnt, const uint32_t *d_S,
              uint8_t *d_bp_d, uint64_t *d_bp_m, uint32_t *d_err, void *scratch,
              size_t scratch_bytes, cudaStream_t s) {
    if (t == 0 || n == 0) return PLL_OK;
    if (t > PLL_MAX_T) return PLL_E_RANGE;
    size_t tb = 0;
    if (bp_scratch_bytes(n, nnz, &tb) > scratch_bytes) return PLL_E_RANGE;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    unsigned char *p = static_cast<unsigned char *>(scratch);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(p);
    p += up(((size_t)n + 1) * 4);
    uint32_t *coff = reinterpret_cast<uint32_t *>(p);
    p += up(((size_t)n + 1) * 4);
    uint32_t *items = reinterpret_cast<uint32_t *>(p);
    p += up(((size_t)n + (nnz + CHUNK - 1) / CHUNK) * 4);
    uint32_t *flag = reinterpret_cast<uint32_t *>(p);
    p += up(8);
    void *cub_temp = p;

    const size_t nt = (size_t)n * t;
    const uint32_t tp = bp_stride(t);
    PLL_TRY(cudaMemsetAsync(d_bp_d, 0xff, (size_t)n * tp, s));
    PLL_TRY(cudaMemsetAsync(d_bp_m, 0, nt * 16, s));
    k_bp_seed<<<t, BPW, 0, s>>>(t, tp, d_root, d_cnt, d_S, d_bp_d, d_bp_m);
    PLL_TRY(cudaMemsetAsync(cnt, 0, ((size_t)n + 1) * 4, s));
    const int g1 = (int)std::min<uint64_t>((n + 255) / 256, 65535);
    k_chunk_counts<<<g1, 256, 0, s>>>(n, d_roff, cnt);
    PLL_TRY(cub::DeviceScan::ExclusiveSum(cub_temp, tb, cnt, coff, (int)n + 1, s));
    uint32_t nitems = 0;
    PLL_TRY(cudaMemcpyAsync(&nitems, coff + n, 4, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    k_chunk_fill<<<g1, 256, 0, s>>>(n, coff, items);
    PLL_TRY(cudaGetLastError());
    int dev = 0, sms = 148;
    PLL_TRY(cudaGetDevice(&dev));
    PLL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t want = ((uint64_t)nitems * 32 + 255) / 256;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 16));
    BpArgs a{n, t, tp, 0, d_roff, d_rcol, items, coff, nitems, d_bp_d, d_bp_m, flag, d_err};
    for (uint32_t L = 0; L < INF8; ++L) {
        a.L = L;
        PLL_TRY(cudaMemsetAsync(flag, 0, 4, s));
        k_bp_same_level<<<grid, 256, 0, s>>>(a);
        k_bp_next_level<<<grid, 256, 0, s>>>(a);
        PLL_TRY(cudaGetLastError());
        uint32_t h_flag = 0;
        PLL_TRY(cudaMemcpyAsync(&h_flag, flag, 4, cudaMemcpyDeviceToHost, s));
        PLL_TRY(cudaStreamSynchronize(s));
        if (h_flag == 0 && L >= 1) break;
    }
    k_bp_finish<<<(int)std::min<size_t>((nt + 255) / 256, (size_t)sms * 32), 256, 0, s>>>(
        nt, reinterpret_cast<ulonglong2 *>(d_bp_m));
    PLL_TRY(cudaGetLastError());
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

}  // namespace pll
