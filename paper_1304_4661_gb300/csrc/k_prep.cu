// k_prep.cu -- graph checks, vertex order and rank-space relabelling, and the
// greedy choice of bit-parallel roots.
//
//   validate     symmetric simple CSR with ascending neighbour lists (the
//                undirected, unweighted graphs of Sec. 3.1)
//   degree order Sec. 4.4.2 Degree strategy: descending degree, ties broken by
//                ascending vertex id; one 64-bit radix sort
//   relabel      CSR in rank space (vertex id := rank), neighbour lists
//                ascending, so "lowest rank" == "highest priority"
//   BP roots     Sec. 5.4: r = highest-priority unused vertex, S_r = up to 64
//                highest-priority unused neighbours of r, bit j = j-th chosen
#include <algorithm>

#include <cub/cub.cuh>

#include "pll_internal.cuh"

namespace pll {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// Offsets: offsets[0] = 0, non-decreasing, offsets[n] = nnz.
__global__ void k_validate_offsets(uint32_t n, uint64_t nnz, const uint32_t *__restrict__ off,
                                   uint32_t *err) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint32_t b = off[v], e = off[v + 1];
        if (b > e || e > nnz || (v == 0 && b != 0) || (v + 1 == n && e != nnz)) atomicOr(err, ERR_CSR);
    }
}

constexpr uint32_t ARCS_PER_THREAD = 8;

// Arcs (valid offsets assumed): ids < n, no self-loop, strict ascent within a
// list, and the reverse arc present (binary search of v in N(w)). Each thread
// takes ARCS_PER_THREAD consecutive arcs, so hubs of any degree spread over
// many threads; the source vertex is found once by binary search on offsets.
__global__ void k_validate_arcs(uint32_t n, uint64_t nnz, const uint32_t *__restrict__ off,
                                const uint32_t *__restrict__ col, uint32_t *err) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * ARCS_PER_THREAD;
    for (uint64_t x0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * ARCS_PER_THREAD; x0 < nnz;
         x0 += stride) {
        // v = last vertex with off[v] <= x0
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid] <= x0) lo = mid; else hi = mid;
        }
        uint32_t v = lo;
        const uint64_t x1 = x0 + ARCS_PER_THREAD < nnz ? x0 + ARCS_PER_THREAD : nnz;
        bool bad = false;
        for (uint64_t x = x0; x < x1; ++x) {
            while (off[v + 1] <= x) ++v;  // skip empty lists
            const uint32_t w = col[x];
            if (w >= n || w == v || (x > off[v] && col[x - 1] >= w)) { bad = true; break; }
            uint32_t a = off[w], c = off[w + 1];
            while (a < c) {  // lower bound of v in N(w)
                const uint32_t mid = a + ((c - a) >> 1);
                if (col[mid] < v) a = mid + 1; else c = mid;
            }
            if (!(a < off[w + 1] && col[a] == v)) { bad = true; break; }
        }
        if (bad) atomicOr(err, ERR_CSR);
    }
}

// key = (~degree << 32) | id: ascending keys give descending degree, then
// ascending id.
__global__ void k_degree_keys(uint32_t n, const uint32_t *__restrict__ off, uint64_t *keys) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t deg = off[v + 1] - off[v];
        keys[v] = ((uint64_t)(0xffffffffu - deg) << 32) | v;
    }
}

__global__ void k_keys_to_order(uint32_t n, const uint64_t *__restrict__ keys, uint32_t *order) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        order[r] = (uint32_t)keys[r];
}

__global__ void k_count_order(uint32_t n, const uint32_t *__restrict__ order, uint32_t *cnt,
                              uint32_t *err) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        uint32_t v = order[r];
        if (v >= n) atomicOr(err, ERR_ORDER);
        else atomicAdd(&cnt[v], 1u);
    }
}

__global__ void k_check_counts(uint32_t n, const uint32_t *__restrict__ cnt, uint32_t *err) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (cnt[v] != 1) atomicOr(err, ERR_ORDER);
}

__global__ void k_inverse_and_degree(uint32_t n, const uint32_t *__restrict__ order,
                                     const uint32_t *__restrict__ off, uint32_t *inv,
                                     uint32_t *rdeg) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        uint32_t v = order[r];
        inv[v] = r;
        rdeg[r] = off[v + 1] - off[v];
    }
}

// One warp per rank r: rcol[roff[r] + j] = inv[col[off[v] + j]], v = order[r].
__global__ void k_relabel(uint32_t n, const uint32_t *__restrict__ order,
                          const uint32_t *__restrict__ off, const uint32_t *__restrict__ col,
                          const uint32_t *__restrict__ inv, const uint32_t *__restrict__ roff,
                          uint32_t *rcol) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        uint32_t v = order[r];
        uint32_t b = off[v], e = off[v + 1], o = roff[r];
        for (uint32_t x = b + lane; x < e; x += 32) rcol[o + (x - b)] = inv[col[x]];
    }
}

__global__ void k_set_last(uint32_t *a, uint32_t idx, uint32_t val) { a[idx] = val; }

// Sec. 5.4 greedy choice, one warp. inX doubles as the "used" mark.
__global__ void k_select_bp(uint32_t n, uint32_t t, const uint32_t *__restrict__ roff,
                            const uint32_t *__restrict__ rcol, uint8_t *inX, uint32_t *root,
                            uint32_t *cnt, uint32_t *S) {
    const int lane = threadIdx.x;
    uint32_t next = 0;
    for (uint32_t i = 0; i < t; ++i) {
        // lowest unused rank >= next
        uint32_t r = NONE;
        while (next < n) {
            uint32_t c = next + lane;
            bool ok = c < n && !inX[c];
            unsigned m = __ballot_sync(FULL, ok);
            if (m) { r = next + __ffs(m) - 1; break; }
            next += 32;
        }
        if (r == NONE) {
            if (lane == 0) { root[i] = NONE; cnt[i] = 0; }
            continue;
        }
        if (lane == 0) { inX[r] = 1; root[i] = r; }
        next = r + 1;
        __syncwarp();
        uint32_t c = 0;
        const uint32_t b = roff[r], e = roff[r + 1];
        for (uint32_t x = b; x < e && c < BPW; x += 32) {
            uint32_t w = (x + lane < e) ? rcol[x + lane] : NONE;
            bool ok = (w != NONE) && !inX[w];
            unsigned m = __ballot_sync(FULL, ok);
            uint32_t pos = c + __popc(m & ((1u << lane) - 1u));
            __syncwarp();
            if (ok && pos < BPW) {
                S[(size_t)i * BPW + pos] = w;
                inX[w] = 1;
            }
            c += __popc(m);
            __syncwarp();
        }
        if (lane == 0) cnt[i] = c < BPW ? c : BPW;
        __syncwarp();
    }
}

// ---- several graphs built as one disjoint union (pll_build_batch)

// graph id of every vertex; graph g owns vertices [gs[g], gs[g+1])
__global__ void k_graph_of(uint32_t G, const uint32_t *__restrict__ gs, uint32_t *gof) {
    for (uint32_t g = blockIdx.x; g < G; g += gridDim.x)
        for (uint32_t v = gs[g] + threadIdx.x; v < gs[g + 1]; v += blockDim.x) gof[v] = g;
}

// every arc stays inside its graph
__global__ void k_check_graph_arcs(uint32_t n, const uint32_t *__restrict__ off,
                                   const uint32_t *__restrict__ col,
                                   const uint32_t *__restrict__ gof, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint32_t g = gof[v];
        for (uint32_t x = off[v] + lane; x < off[v + 1]; x += 32)
            if (gof[col[x]] != g) atomicOr(err, ERR_CSR);
    }
}

// first key: (graph, descending degree); a stable sort keeps ascending ids
__global__ void k_batch_keys1(uint32_t n, const uint32_t *__restrict__ off,
                              const uint32_t *__restrict__ gof, uint64_t *keys, uint32_t *vals) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        keys[v] = ((uint64_t)gof[v] << 32) | (0xffffffffu - (off[v + 1] - off[v]));
        vals[v] = v;
    }
}

// second key: (rank inside the graph, graph): graphs interleave by local rank
__global__ void k_batch_keys2(uint32_t n, const uint32_t *__restrict__ gs,
                              const uint32_t *__restrict__ gof, const uint32_t *__restrict__ local_order,
                              uint64_t *keys, uint32_t *vals) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t v = local_order[p], g = gof[v];
        keys[p] = ((uint64_t)(p - gs[g]) << 24) | g;
        vals[p] = v;
    }
}

// Sec. 5.4 greedy choice inside each graph, one warp per graph. local_order
// lists each graph's vertices by its own rank; rcol is in global rank space,
// which orders every neighbour list by the graph's own rank too.
__global__ void k_select_bp_graphs(uint32_t G, uint32_t t, const uint32_t *__restrict__ gs,
                                   const uint32_t *__restrict__ local_order,
                                   const uint32_t *__restrict__ inv,
                                   const uint32_t *__restrict__ roff,
                                   const uint32_t *__restrict__ rcol, uint8_t *inX, uint32_t *root,
                                   uint32_t *cnt, uint32_t *S) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += warps) {
        const uint32_t e = gs[g + 1];
        uint32_t next = gs[g];
        for (uint32_t i = 0; i < t; ++i) {
            const size_t slot = (size_t)g * t + i;
            uint32_t r = NONE;
            while (next < e) {
                const uint32_t p = next + lane;
                const uint32_t rp = p < e ? inv[local_order[p]] : NONE;
                const bool ok = p < e && !inX[rp];
                const unsigned m = __ballot_sync(FULL, ok);
                if (m) {
                    const int l = __ffs(m) - 1;
                    r = __shfl_sync(FULL, rp, l);
                    next = next + l + 1;
                    break;
                }
                next += 32;
            }
            if (r == NONE) {
                if (lane == 0) { root[slot] = NONE; cnt[slot] = 0; }
                continue;
            }
            if (lane == 0) { inX[r] = 1; root[slot] = r; }
            __syncwarp();
            uint32_t c = 0;
            const uint32_t b = roff[r], ee = roff[r + 1];
            for (uint32_t x = b; x < ee && c < BPW; x += 32) {
                const uint32_t w = (x + lane < ee) ? rcol[x + lane] : NONE;
                const bool ok = (w != NONE) && !inX[w];
                const unsigned m = __ballot_sync(FULL, ok);
                const uint32_t pos = c + __popc(m & ((1u << lane) - 1u));
                __syncwarp();
                if (ok && pos < BPW) {
                    S[slot * BPW + pos] = w;
                    inX[w] = 1;
                }
                c += __popc(m);
                __syncwarp();
            }
            if (lane == 0) cnt[slot] = c < BPW ? c : BPW;
            __syncwarp();
        }
    }
}

inline int grid_for(uint64_t items, int block, int per_thread = 1) {
    uint64_t g = (items + (uint64_t)block * per_thread - 1) / ((uint64_t)block * per_thread);
    if (g < 1) g = 1;
    if (g > 65535) g = 65535;
    return (int)g;
}

}  // namespace

int prep_validate_csr(const Graph &g, uint32_t *d_err, cudaStream_t s) {
    if (g.n == 0) return PLL_OK;
    k_validate_offsets<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, g.nnz, g.off, d_err);
    PLL_TRY(cudaGetLastError());
    uint32_t h = 0;
    PLL_TRY(cudaMemcpyAsync(&h, d_err, 4, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    if (h || g.nnz == 0) return PLL_OK;  // arcs are read only behind valid offsets
    k_validate_arcs<<<grid_for(g.nnz, 256, ARCS_PER_THREAD), 256, 0, s>>>(g.n, g.nnz, g.off, g.col, d_err);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

int prep_degree_order(const Graph &g, uint32_t *d_order, cudaStream_t s) {
    if (g.n == 0) return PLL_OK;
    PoolMem keys(s), sorted(s), temp(s);
    PLL_CHECK(keys.alloc((size_t)g.n * 8));
    PLL_CHECK(sorted.alloc((size_t)g.n * 8));
    k_degree_keys<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, g.off, keys.as<uint64_t>());
    PLL_TRY(cudaGetLastError());
    size_t tb = 0;
    PLL_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, keys.as<uint64_t>(), sorted.as<uint64_t>(),
                                           (int)g.n, 0, 64, s));
    PLL_CHECK(temp.alloc(tb));
    PLL_TRY(cub::DeviceRadixSort::SortKeys(temp.p, tb, keys.as<uint64_t>(), sorted.as<uint64_t>(),
                                           (int)g.n, 0, 64, s));
    k_keys_to_order<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, sorted.as<uint64_t>(), d_order);
    PLL_TRY(cudaGetLastError());
    PLL_TRY(cudaStreamSynchronize(s));  // before the temporaries are freed
    return PLL_OK;
}

int prep_check_order(const Graph &g, const uint32_t *d_order, uint32_t *d_err, cudaStream_t s) {
    if (g.n == 0) return PLL_OK;
    PoolMem cnt(s);
    PLL_CHECK(cnt.alloc((size_t)g.n * 4));
    PLL_TRY(cudaMemsetAsync(cnt.p, 0, (size_t)g.n * 4, s));
    k_count_order<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, d_order, cnt.as<uint32_t>(), d_err);
    k_check_counts<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, cnt.as<uint32_t>(), d_err);
    PLL_TRY(cudaGetLastError());
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

int prep_relabel(const Graph &g, const uint32_t *d_order, uint32_t *d_inv, uint32_t *d_roff,
                 uint32_t *d_rcol, cudaStream_t s) {
    if (g.n == 0) {
        PLL_TRY(cudaMemsetAsync(d_roff, 0, 4, s));
        return PLL_OK;
    }
    PoolMem rdeg(s), tmpcol(s), temp(s);
    PLL_CHECK(rdeg.alloc((size_t)g.n * 4));
    k_inverse_and_degree<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, d_order, g.off, d_inv,
                                                            rdeg.as<uint32_t>());
    PLL_TRY(cudaGetLastError());
    size_t tb = 0;
    PLL_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, rdeg.as<uint32_t>(), d_roff, (int)g.n, s));
    PLL_CHECK(temp.alloc(tb));
    PLL_TRY(cub::DeviceScan::ExclusiveSum(temp.p, tb, rdeg.as<uint32_t>(), d_roff, (int)g.n, s));
    k_set_last<<<1, 1, 0, s>>>(d_roff, g.n, (uint32_t)g.nnz);
    PLL_TRY(cudaGetLastError());
    if (g.nnz == 0) {
        PLL_TRY(cudaStreamSynchronize(s));
        return PLL_OK;
    }
    PLL_CHECK(tmpcol.alloc(g.nnz * 4));
    k_relabel<<<grid_for((uint64_t)g.n * 32, 256), 256, 0, s>>>(g.n, d_order, g.off, g.col, d_inv,
                                                                d_roff, tmpcol.as<uint32_t>());
    PLL_TRY(cudaGetLastError());
    size_t tb2 = 0;
    PLL_TRY(cub::DeviceSegmentedSort::SortKeys(nullptr, tb2, tmpcol.as<uint32_t>(), d_rcol,
                                               (int64_t)g.nnz, (int64_t)g.n, d_roff, d_roff + 1, s));
    if (tb2 > temp.bytes) PLL_CHECK(temp.alloc(tb2));
    PLL_TRY(cub::DeviceSegmentedSort::SortKeys(temp.p, tb2, tmpcol.as<uint32_t>(), d_rcol,
                                               (int64_t)g.nnz, (int64_t)g.n, d_roff, d_roff + 1, s));
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

int prep_select_bp_roots(uint32_t n, uint32_t t, const uint32_t *d_roff, const uint32_t *d_rcol,
                         uint8_t *d_inX, uint32_t *d_root, uint32_t *d_cnt, uint32_t *d_S,
                         cudaStream_t s) {
    if (t == 0) return PLL_OK;
    k_select_bp<<<1, 32, 0, s>>>(n, t, d_roff, d_rcol, d_inX, d_root, d_cnt, d_S);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

}  // namespace pll

namespace pll {
namespace {
__global__ void k_graph_by_rank(uint32_t n, const uint32_t *__restrict__ order,
                                const uint32_t *__restrict__ gof, uint32_t *out) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        out[r] = gof[order[r]];
}
}  // namespace

int prep_graph_by_rank(uint32_t n, const uint32_t *d_order, const uint32_t *d_gof, uint32_t *d_out,
                       cudaStream_t s) {
    if (n == 0) return PLL_OK;
    k_graph_by_rank<<<grid_for(n, 256), 256, 0, s>>>(n, d_order, d_gof, d_out);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

int prep_batch_order(const Graph &g, const uint32_t *d_gs, uint32_t G, uint32_t *d_gof,
                     uint32_t *d_local_order, uint32_t *d_order, uint32_t *d_err, cudaStream_t s) {
    if (g.n == 0) return PLL_OK;
    k_graph_of<<<(int)std::min<uint32_t>(G, 65535), 256, 0, s>>>(G, d_gs, d_gof);
    k_check_graph_arcs<<<grid_for((uint64_t)g.n * 32, 256), 256, 0, s>>>(g.n, g.off, g.col, d_gof, d_err);
    PoolMem k1(s), k1s(s), v1(s), k2(s), temp(s);
    PLL_CHECK(k1.alloc((size_t)g.n * 8));
    PLL_CHECK(k1s.alloc((size_t)g.n * 8));
    PLL_CHECK(v1.alloc((size_t)g.n * 4));
    k_batch_keys1<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, g.off, d_gof, k1.as<uint64_t>(), v1.as<uint32_t>());
    PLL_TRY(cudaGetLastError());
    size_t tb = 0;
    PLL_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, k1.as<uint64_t>(), k1s.as<uint64_t>(),
                                            v1.as<uint32_t>(), d_local_order, (int)g.n, 0, 64, s));
    PLL_CHECK(temp.alloc(tb));
    PLL_TRY(cub::DeviceRadixSort::SortPairs(temp.p, tb, k1.as<uint64_t>(), k1s.as<uint64_t>(),
                                            v1.as<uint32_t>(), d_local_order, (int)g.n, 0, 64, s));
    k_batch_keys2<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, d_gs, d_gof, d_local_order,
                                                     k1.as<uint64_t>(), v1.as<uint32_t>());
    PLL_TRY(cudaGetLastError());
    size_t tb2 = 0;
    PLL_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb2, k1.as<uint64_t>(), k1s.as<uint64_t>(),
                                            v1.as<uint32_t>(), d_order, (int)g.n, 0, 48, s));
    if (tb2 > temp.bytes) PLL_CHECK(temp.alloc(tb2));
    PLL_TRY(cub::DeviceRadixSort::SortPairs(temp.p, tb2, k1.as<uint64_t>(), k1s.as<uint64_t>(),
                                            v1.as<uint32_t>(), d_order, (int)g.n, 0, 48, s));
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

int prep_select_bp_graphs(uint32_t G, uint32_t t, const uint32_t *d_gs, const uint32_t *d_local_order,
                          const uint32_t *d_inv, const uint32_t *d_roff, const uint32_t *d_rcol,
                          uint8_t *d_inX, uint32_t *d_root, uint32_t *d_cnt, uint32_t *d_S,
                          cudaStream_t s) {
    if (t == 0 || G == 0) return PLL_OK;
    const int grid = (int)std::min<uint64_t>(((uint64_t)G * 32 + 255) / 256, 65535);
    k_select_bp_graphs<<<grid, 256, 0, s>>>(G, t, d_gs, d_local_order, d_inv, d_roff, d_rcol, d_inX,
                                            d_root, d_cnt, d_S);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

}  // namespace pll
