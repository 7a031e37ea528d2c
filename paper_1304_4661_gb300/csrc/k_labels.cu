// k_labels.cu -- the label store and the redundancy cleanup of a root batch.
//
// Cleanup. A batch emits tuples (u, k, d) for roots k in [k0, k1), each
// pruned only with hubs < k0. Alg. 1 run sequentially would also prune with
// the batch's own hubs h < k. Sorted by (u, k), the tuples of vertex u and of
// vertex v_k (= rank k) are contiguous. (u, k, d) is dropped iff some hub
// h < k has tuples (v_k, h, a) and (u, h, b) in the batch with a + b <= d.
// Every emitted distance is exact, so a + b <= d means h lies on a shortest
// v_k-u path, which the sequential run would have pruned at (Sec. 4.2:
// Query(v_k, u, L'_{k-1}) <= d). Conversely, if an in-batch hub lies on such
// a path, the one of least rank does, and its tuples for v_k and u were
// emitted (nothing of rank < k0, no bit-parallel vertex lies on those
// subpaths), so the test catches every surplus entry. The batch therefore
// yields exactly the entries of L'_{k1-1} minus L'_{k0-1} (Thm 4.1 argument).
//
// Store. Labels only ever grow by hubs larger than every hub already present
// (Sec. 4.5.1 "Sorting Labels"), so each vertex owns a growable array in one
// pool: (offset, length, capacity), reallocated by doubling from an atomic
// bump pointer. Entries are packed (hub rank << 8 | distance) so one 32-bit
// load serves the prune test (the paper keeps hubs and distances in separate
// arrays, Sec. 4.5.2, because its merge touches distances only on a match;
// the root-array probe here needs both for every entry).
#include <cub/cub.cuh>

#include "pll_internal.cuh"

namespace pll {
namespace {

__device__ __forceinline__ uint64_t lower_bound_u64(const uint64_t *__restrict__ a, uint64_t lo,
                                                    uint64_t hi, uint64_t key) {
    while (lo < hi) {
        uint64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Tuples of vertex v_k with hub < k, for every root k of the batch: their
// range [seg[2 (k - k0)], seg[2 (k - k0) + 1]) in the sorted tuples, found once
// per root instead of once per tuple.
__global__ void k_root_segments(const uint64_t *__restrict__ T, uint64_t P, uint32_t k0, uint32_t B,
                                uint64_t *seg) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint32_t k = k0 + i;
    const uint64_t lo = lower_bound_u64(T, 0, P, (uint64_t)k << 32);
    seg[2 * i] = lo;
    seg[2 * i + 1] = lower_bound_u64(T, lo, P, pack_tuple(k, k, 0));
}

// Tuple x = (u, k, d) is surplus iff some in-batch hub h < k has (u, h, a)
// and (v_k, h, b) with a + b <= d (the lowest such h lies on a shortest
// v_k-u path). u's tuples with hub < k are [lo_u, x): the run of u ends at x,
// and its start is found by galloping back from x (runs are short). v_k's
// come from seg (or, without it, a binary search).
__global__ void k_cleanup(const uint64_t *__restrict__ T, uint64_t P, const uint64_t *__restrict__ seg,
                          uint32_t k0, uint8_t *keep) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < P;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = T[x];
        const uint32_t u = (uint32_t)(key >> 32);
        const uint32_t e = (uint32_t)key;
        const uint32_t k = entry_hub(e), d = entry_dist(e);
        // start of u's run: gallop back while the entry is still u's, then
        // search the last step
        uint64_t b = x, stp = 1;
        while (b >= stp && (uint32_t)(T[b - stp] >> 32) == u) {
            b -= stp;
            stp <<= 1;
        }
        const uint64_t lo_u = lower_bound_u64(T, b >= stp ? b - stp : 0, b, (uint64_t)u << 32);
        uint64_t lo_k, hi_k;
        if (seg) {
            lo_k = seg[2 * (k - k0)];
            hi_k = seg[2 * (k - k0) + 1];
        } else {
            lo_k = lower_bound_u64(T, 0, P, (uint64_t)k << 32);
            hi_k = lower_bound_u64(T, lo_k, P, pack_tuple(k, k, 0));
        }
        uint64_t i = lo_u, j = lo_k;
        bool drop = false;
        while (i < x && j < hi_k) {
            const uint32_t ei = (uint32_t)T[i], ej = (uint32_t)T[j];
            const uint32_t hi = entry_hub(ei), hj = entry_hub(ej);
            if (hi == hj) {
                if (entry_dist(ei) + entry_dist(ej) <= d) { drop = true; break; }
                ++i; ++j;
            } else if (hi < hj) {
                ++i;
            } else {
                ++j;
            }
        }
        keep[x] = drop ? 0 : 1;
    }
}

// One thread per run of equal vertex in the sorted kept tuples.
__global__ void k_append(LabelStore st, const uint64_t *__restrict__ K,
                         const unsigned long long *__restrict__ nkept, uint32_t *err) {
    const uint64_t cnt = *nkept;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < cnt;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)(K[x] >> 32);
        if (x > 0 && (uint32_t)(K[x - 1] >> 32) == u) continue;
        uint64_t y = x + 1;
        while (y < cnt && (uint32_t)(K[y] >> 32) == u) ++y;
        const uint32_t c = (uint32_t)(y - x);
        const uint32_t len = st.len[u], cap = st.cap[u];
        uint64_t off = st.off[u];
        if (len + c > cap) {
            uint32_t nc = cap * 2;
            if (nc < len + c) nc = len + c;
            if (nc < 8) nc = 8;
            nc = (nc + 3u) & ~3u;  // every array starts on 16 bytes (vector loads)
            const unsigned long long base = atomicAdd(st.pool_top, (unsigned long long)nc);
            if (base + nc > st.pool_cap) {
                atomicOr(err, ERR_POOL);
                continue;
            }
            for (uint32_t j = 0; j < len; ++j) st.pool[base + j] = st.pool[off + j];
            off = base;
            st.off[u] = off;
            st.cap[u] = nc;
        }
        for (uint32_t j = 0; j < c; ++j) st.pool[off + len + j] = (uint32_t)K[x + j];
        st.len[u] = len + c;
    }
}

// One warp per vertex: dst[doff[v] + j] = src[soff[v] + j], j < len[v].
__global__ void k_gather_labels(uint32_t n, const uint64_t *__restrict__ soff,
                                const uint32_t *__restrict__ len, const uint32_t *__restrict__ src,
                                const uint64_t *__restrict__ doff, uint32_t *dst) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint32_t l = len[v];
        const uint32_t *s = src + soff[v];
        uint32_t *d = dst + doff[v];
        for (uint32_t j = lane; j < l; j += 32) d[j] = s[j];
    }
}

__global__ void k_set_u64(uint64_t *a, uint64_t idx, uint64_t val) { a[idx] = val; }

__global__ void k_widen(const uint32_t *__restrict__ in, uint64_t *out, uint32_t n, uint32_t round) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (in[i] + round - 1) / round * round;
}

__global__ void k_round_caps(const uint32_t *__restrict__ len, uint32_t *cap, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        cap[i] = (len[i] + 3u) & ~3u;
}

inline int grid_for(uint64_t items, int block) {
    uint64_t g = (items + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 16384) g = 16384;
    return (int)g;
}

}  // namespace

int labels_sort_tuples(uint64_t *d_in, uint64_t *d_out, uint64_t count, int begin_bit, int end_bit,
                       void *d_temp, size_t *temp_bytes, cudaStream_t s) {
    PLL_TRY(cub::DeviceRadixSort::SortKeys(d_temp, *temp_bytes, d_in, d_out, (int64_t)count, begin_bit,
                                           end_bit, s));
    return PLL_OK;
}

int labels_cleanup(const uint64_t *d_sorted, uint64_t count, uint8_t *d_keep, uint32_t k0, uint32_t B,
                   void *scratch, size_t scratch_bytes, cudaStream_t s) {
    if (count == 0) return PLL_OK;
    uint64_t *seg = nullptr;
    if (scratch && scratch_bytes >= (size_t)B * 16) {
        seg = static_cast<uint64_t *>(scratch);
        k_root_segments<<<(B + 255) / 256, 256, 0, s>>>(d_sorted, count, k0, B, seg);
        PLL_TRY(cudaGetLastError());
    }
    k_cleanup<<<grid_for(count, 256), 256, 0, s>>>(d_sorted, count, seg, k0, d_keep);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

int labels_compact(const uint64_t *d_in, const uint8_t *d_keep, uint64_t count, uint64_t *d_out,
                   unsigned long long *d_nout, void *d_temp, size_t *temp_bytes, cudaStream_t s) {
    PLL_TRY(cub::DeviceSelect::Flagged(d_temp, *temp_bytes, d_in, d_keep, d_out, d_nout,
                                       (int64_t)count, s));
    return PLL_OK;
}

int labels_append(const LabelStore &st, const uint64_t *d_kept,
                  const unsigned long long *d_nkept, uint64_t max_count, uint32_t *d_err,
                  cudaStream_t s) {
    if (max_count == 0) return PLL_OK;
    // d_kept holds *d_nkept <= max_count tuples; the exact count is read on device
    k_append<<<grid_for(max_count, 256), 256, 0, s>>>(st, d_kept, d_nkept, d_err);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

// d_out[v] = sum of round_up(d_in[u], round) for u < v (v < n); widened in
// place, then scanned.
int scan_u32_to_u64(const uint32_t *d_in, uint64_t *d_out, uint32_t n, void *d_temp,
                    size_t *temp_bytes, cudaStream_t s, uint32_t round) {
    if (d_temp == nullptr) {
        PLL_TRY(cub::DeviceScan::ExclusiveSum(nullptr, *temp_bytes, d_out, (int64_t)n, s));
        return PLL_OK;
    }
    k_widen<<<grid_for(n, 256), 256, 0, s>>>(d_in, d_out, n, round);
    PLL_TRY(cudaGetLastError());
    PLL_TRY(cub::DeviceScan::ExclusiveSum(d_temp, *temp_bytes, d_out, (int64_t)n, s));
    return PLL_OK;
}

// Rewrites the pool (capacity = length rounded up to 4 entries, so arrays
// stay 16-byte aligned) into a new buffer of new_cap entries. Used when the
// bump pointer would run past the pool.
int labels_regrow(LabelStore &st, uint64_t new_cap, cudaStream_t s) {
    const uint32_t n = st.n;
    DevMem dpool;
    PoolMem ppool(s), noff(s), temp(s);
    uint32_t *np = nullptr;
    if (st.pooled) {
        PLL_CHECK(ppool.alloc(new_cap * 4));
        np = ppool.as<uint32_t>();
    } else {
        PLL_CHECK(dpool.alloc(new_cap * 4));
        np = dpool.as<uint32_t>();
    }
    PLL_CHECK(noff.alloc(((size_t)n + 1) * 8));
    size_t tb = 0;
    PLL_CHECK(scan_u32_to_u64(st.len, noff.as<uint64_t>(), n, nullptr, &tb, s, 4));
    PLL_CHECK(temp.alloc(tb));
    PLL_CHECK(scan_u32_to_u64(st.len, noff.as<uint64_t>(), n, temp.p, &tb, s, 4));
    k_gather_labels<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(n, st.off, st.len, st.pool,
                                                                    noff.as<uint64_t>(), np);
    PLL_TRY(cudaGetLastError());
    PLL_TRY(cudaMemcpyAsync(st.off, noff.p, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    k_round_caps<<<grid_for(n, 256), 256, 0, s>>>(st.len, st.cap, n);
    PLL_TRY(cudaGetLastError());
    // new bump pointer = total entries = noff[n-1] + len[n-1]
    uint64_t last_off = 0;
    uint32_t last_len = 0;
    if (n) {
        PLL_TRY(cudaMemcpyAsync(&last_off, noff.as<uint64_t>() + (n - 1), 8, cudaMemcpyDeviceToHost, s));
        PLL_TRY(cudaMemcpyAsync(&last_len, st.len + (n - 1), 4, cudaMemcpyDeviceToHost, s));
    }
    PLL_TRY(cudaStreamSynchronize(s));
    unsigned long long top = last_off + ((last_len + 3u) & ~3u);
    PLL_TRY(cudaMemcpyAsync(st.pool_top, &top, 8, cudaMemcpyHostToDevice, s));
    PLL_TRY(cudaStreamSynchronize(s));
    if (st.pooled) pool_free(st.pool, s);
    else dev_free(st.pool);
    st.pool = np;
    ppool.release();
    dpool.release();
    st.pool_cap = new_cap;
    return PLL_OK;
}

int labels_finalize(const LabelStore &st, uint64_t total, uint64_t *d_off, uint32_t *d_lab,
                    void *d_temp, size_t *temp_bytes, cudaStream_t s) {
    const uint32_t n = st.n;
    if (n == 0) {
        PLL_TRY(cudaMemsetAsync(d_off, 0, 8, s));
        return PLL_OK;
    }
    if (d_temp == nullptr) return scan_u32_to_u64(st.len, d_off, n, nullptr, temp_bytes, s, 1);
    PLL_CHECK(scan_u32_to_u64(st.len, d_off, n, d_temp, temp_bytes, s, 1));
    k_set_u64<<<1, 1, 0, s>>>(d_off, n, total);
    k_gather_labels<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(n, st.off, st.len, st.pool,
                                                                    d_off, d_lab);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

}  // namespace pll
