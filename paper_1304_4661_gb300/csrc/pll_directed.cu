// pll_directed.cu -- directed graphs (Sec. 6, "Directed Graphs").
//
// Two label sets per vertex: L_IN(v) holds (u, d(u, v)) and L_OUT(v) holds
// (u, d(v, u)); d(s, t) = min over common hubs of L_OUT(s) and L_IN(t). Each
// root v_k, in rank order, runs a pruned BFS along arcs that fills L_IN
// (u is pruned when L_OUT(v_k) and L_IN(u) already give d(v_k, u)) and one
// against arcs that fills L_OUT (pruned when L_OUT(u) and L_IN(v_k) give
// d(u, v_k)). There are no bit-parallel labels: the masks of Sec. 5 rest on
// |d(s, v) - d(r, v)| <= 1 for neighbours s of r, which one-way arcs do not
// give.
//
// Root batches, as in the undirected build: the BFSs of roots [k0, k1) run
// together, pruned only with hubs < k0, then a cleanup removes the entries an
// in-batch hub h < k covers. A forward tuple (u, k, d) is surplus iff some
// in-batch h < k has a reverse tuple (v_k, h, a) (a = d(v_k, h)) and a forward
// tuple (u, h, b) (b = d(h, u)) with a + b <= d; a reverse tuple (u, k, d)
// iff some h < k has (u, h, a) reverse and (v_k, h, b) forward with
// a + b <= d. Every emitted distance is exact (a vertex reached late would
// have been pruned), and the least such h has tuples at both ends (nothing
// of rank < k0 lies on the subpaths), so the cleanup leaves exactly the
// sequential labels.
//
// Kernels: k_dvalidate (CSR checks), k_dindeg / k_ddeg (in- plus out-degree
// for the Degree order), k_dcount_in / k_dfill_in (the reverse CSR),
// k_dinit, k_dtest (thread per frontier entry: merge of the two labels),
// k_dexpand (warp per surviving entry, lanes over arcs, one visited bit per
// (vertex, root) claimed by atomicOr), k_dcleanup (thread per tuple) and
// k_dquery (warp per pair). Sorting, compaction and the label store are the
// undirected build's (k_labels.cu).
#include <algorithm>
#include <new>
#include <vector>

#include <cub/cub.cuh>

#include "pll_internal.cuh"

using namespace pll;

// The directed index: labels in rank space, [0] = L_IN, [1] = L_OUT.
struct pll_dindex {
    int device = 0;
    uint32_t n = 0;
    uint64_t nnz = 0;
    uint32_t *d_order = nullptr;  // rank -> caller vertex id
    uint32_t *d_inv = nullptr;    // caller vertex id -> rank
    uint64_t *d_off[2] = {nullptr, nullptr};
    uint32_t *d_lab[2] = {nullptr, nullptr};
    uint64_t entries[2] = {0, 0};
    unsigned long long *d_qerr = nullptr;  // [0] finite distance >= 255, [1] id >= n
    uint64_t batches = 0;
    uint64_t pre_cleanup = 0;
};

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t BIG = 1u << 20;

struct DCounters {
    unsigned long long out_n;     // tuples emitted by the current direction of the batch
    unsigned long long alive_n;   // frontier entries that passed the prune test
    unsigned long long deg_sum;   // arcs leaving them
    unsigned long long next_n;    // entries of the next frontier
    unsigned long long nkept;     // tuples kept by the cleanup
    unsigned long long pool_top[2];
    uint32_t err;
    uint32_t pad;
};

inline int blocks_for(uint64_t items, int per_block) {
    uint64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > 16384) g = 16384;
    return (int)g;
}

// ---------------------------------------------------------------- checks
// Offsets start at 0, never decrease and end at nnz; each row is strictly
// ascending, without self-loops or ids >= n. A row is read only behind
// offsets that passed.
__global__ void k_dvalidate(uint32_t n, uint64_t nnz, const uint32_t *__restrict__ off,
                            const uint32_t *__restrict__ col, uint32_t *err) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (v == 0 && off[0] != 0) atomicOr(err, ERR_CSR);
        if (v == n - 1 && off[n] != nnz) atomicOr(err, ERR_CSR);
        const uint32_t b = off[v], e = off[v + 1];
        if (b > e || e > nnz) {
            atomicOr(err, ERR_CSR);
            continue;
        }
        for (uint32_t x = b; x < e; ++x) {
            const uint32_t c = col[x];
            if (c >= n || c == v || (x > b && col[x - 1] >= c)) {
                atomicOr(err, ERR_CSR);
                break;
            }
        }
    }
}

__global__ void k_dindeg(uint32_t n, const uint32_t *__restrict__ off, const uint32_t *__restrict__ col,
                         uint32_t *indeg) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        for (uint32_t x = off[v]; x < off[v + 1]; ++x) atomicAdd(&indeg[col[x]], 1u);
}

// deg[v] = out-degree + in-degree (deg[n] is left 0 for the scan)
__global__ void k_ddeg(uint32_t n, const uint32_t *__restrict__ off, uint32_t *deg) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        deg[v] += off[v + 1] - off[v];
}

// ------------------------------------------------------- reverse CSR
__global__ void k_dcount_in(uint32_t n, const uint32_t *__restrict__ off,
                            const uint32_t *__restrict__ col, uint32_t *cnt) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        for (uint32_t x = off[u]; x < off[u + 1]; ++x) atomicAdd(&cnt[col[x]], 1u);
}

__global__ void k_dfill_in(uint32_t n, const uint32_t *__restrict__ off, const uint32_t *__restrict__ col,
                           uint32_t *cursor, uint32_t *icol) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        for (uint32_t x = off[u]; x < off[u + 1]; ++x) icol[atomicAdd(&cursor[col[x]], 1u)] = u;
}

// ------------------------------------------------------- batch BFS
// Level 0: each root of the batch, its own visited bit set.
__global__ void k_dinit(uint32_t k0, uint32_t B, uint32_t W, uint32_t *vis, uint64_t *F) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
        F[i] = ((uint64_t)(k0 + i) << 32) | i;
        vis[(size_t)(k0 + i) * W + (i >> 5)] = 1u << (i & 31);
    }
}

// Prune test of Alg. 1 for each frontier entry (u, root slot) at distance
// `level`: a common hub of the root's label on the `from` side and u's label
// on the `to` side (both hold hubs < k0 only) with a + b <= level prunes u.
// Otherwise (u, k, level) is emitted and u goes on to be expanded.
__global__ void k_dtest(const uint64_t *__restrict__ F, uint64_t fn, uint32_t level, uint32_t k0,
                        LabelStore from, LabelStore to, const uint32_t *__restrict__ adj_off,
                        uint64_t *T, uint64_t *A, DCounters *c) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < fn;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t f = F[x];
        const uint32_t u = (uint32_t)(f >> 32), k = k0 + (uint32_t)f;
        const uint32_t *R = from.pool + from.off[k];
        const uint32_t *U = to.pool + to.off[u];
        const uint32_t lr = from.len[k], lu = to.len[u];
        uint32_t i = 0, j = 0;
        bool pruned = false;
        while (i < lr && j < lu) {
            const uint32_t hr = entry_hub(R[i]), hu = entry_hub(U[j]);
            if (hr == hu) {
                if (entry_dist(R[i]) + entry_dist(U[j]) <= level) { pruned = true; break; }
                ++i; ++j;
            } else if (hr < hu) {
                ++i;
            } else {
                ++j;
            }
        }
        if (pruned) continue;
        T[atomicAdd(&c->out_n, 1ull)] = pack_tuple(u, k, level);
        A[atomicAdd(&c->alive_n, 1ull)] = f;
        atomicAdd(&c->deg_sum, (unsigned long long)(adj_off[u + 1] - adj_off[u]));
    }
}

// One warp per surviving entry: lanes claim the root's bit at each
// neighbour; a first claim puts (neighbour, slot) on the next frontier.
__global__ void k_dexpand(const uint64_t *__restrict__ A, uint64_t an, const uint32_t *__restrict__ adj_off,
                          const uint32_t *__restrict__ adj_col, uint32_t *vis, uint32_t W, uint64_t *NF,
                          DCounters *c) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < an; i += warps) {
        const uint64_t f = A[i];
        const uint32_t u = (uint32_t)(f >> 32), slot = (uint32_t)f;
        const uint32_t word = slot >> 5, bit = 1u << (slot & 31);
        const uint32_t b = adj_off[u], e = adj_off[u + 1];
        for (uint32_t x = b + lane; x < e; x += 32) {
            const uint32_t w = adj_col[x];
            const uint32_t old = atomicOr(&vis[(size_t)w * W + word], bit);
            if (!(old & bit)) NF[atomicAdd(&c->next_n, 1ull)] = ((uint64_t)w << 32) | slot;
        }
    }
}

__device__ __forceinline__ uint64_t lower_bound64(const uint64_t *__restrict__ a, uint64_t lo, uint64_t hi,
                                                  uint64_t key) {
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Cleanup of one direction's sorted tuples S against the other direction's
// sorted tuples O (both pre-cleanup): x = (u, k, d) in S is dropped iff some
// hub h < k has (u, h, a) in S and (v_k, h, b) in O with a + b <= d.
__global__ void k_dcleanup(const uint64_t *__restrict__ S, uint64_t ps, const uint64_t *__restrict__ O,
                           uint64_t po, uint8_t *keep) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < ps;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = S[x];
        const uint32_t u = (uint32_t)(key >> 32), e = (uint32_t)key;
        const uint32_t k = entry_hub(e), d = entry_dist(e);
        const uint64_t lo_u = lower_bound64(S, 0, x, (uint64_t)u << 32);  // u's hubs < k: [lo_u, x)
        const uint64_t lo_k = lower_bound64(O, 0, po, (uint64_t)k << 32);
        const uint64_t hi_k = lower_bound64(O, lo_k, po, pack_tuple(k, k, 0));
        uint64_t i = lo_u, j = lo_k;
        bool drop = false;
        while (i < x && j < hi_k) {
            const uint32_t ei = (uint32_t)S[i], ej = (uint32_t)O[j];
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

// ------------------------------------------------------------- query
struct DQueryArgs {
    uint32_t n;
    const uint32_t *inv;
    const uint64_t *off_in, *off_out;
    const uint32_t *lab_in, *lab_out;
    const uint32_t *src, *dst;
    uint64_t q;
    uint8_t *out;
    unsigned long long *err;
};

// One warp per pair: lanes take entries of the shorter of L_OUT(s), L_IN(t)
// and binary-search the other by hub.
__global__ void __launch_bounds__(256) k_dquery(DQueryArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t qi = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < a.q; qi += warps) {
        const uint32_t sid = a.src[qi], tid = a.dst[qi];
        if (sid >= a.n || tid >= a.n) {
            if (lane == 0) {
                a.out[qi] = INF8;
                atomicAdd(a.err + 1, 1ull);
            }
            continue;
        }
        const uint32_t s = a.inv[sid], t = a.inv[tid];
        if (s == t) {
            if (lane == 0) a.out[qi] = 0;
            continue;
        }
        const uint64_t os = a.off_out[s], ot = a.off_in[t];
        const uint32_t ls = (uint32_t)(a.off_out[s + 1] - os), lt = (uint32_t)(a.off_in[t + 1] - ot);
        const bool sa = ls <= lt;
        const uint32_t *A = sa ? a.lab_out + os : a.lab_in + ot;
        const uint32_t *B = sa ? a.lab_in + ot : a.lab_out + os;
        const uint32_t la = sa ? ls : lt, lb = sa ? lt : ls;
        uint32_t best = BIG;
        for (uint32_t j = lane; j < la; j += 32) {
            const uint32_t ea = A[j], h = entry_hub(ea);
            uint32_t lo = 0, hi = lb;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (entry_hub(B[mid]) < h) lo = mid + 1; else hi = mid;
            }
            if (lo < lb && entry_hub(B[lo]) == h) best = min(best, entry_dist(ea) + entry_dist(B[lo]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(FULL, best, o));
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

// ------------------------------------------------------------- host
int read_back(const void *d, void *h, size_t bytes, cudaStream_t s) {
    PLL_TRY(cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

// a device buffer that keeps its contents when it grows
int ensure(DevMem &m, size_t bytes, size_t keep, cudaStream_t s) {
    if (m.bytes >= bytes) return PLL_OK;
    DevMem nm;
    PLL_CHECK(nm.alloc(std::max(bytes, m.bytes + m.bytes / 2)));
    if (keep) PLL_TRY(cudaMemcpyAsync(nm.p, m.p, keep, cudaMemcpyDeviceToDevice, s));
    PLL_TRY(cudaStreamSynchronize(s));
    const size_t nb = nm.bytes;
    m.reset();
    m.p = nm.release();
    m.bytes = nb;
    return PLL_OK;
}

void dindex_release(pll_dindex *ix) {
    if (!ix) return;
    dev_free(ix->d_order);
    dev_free(ix->d_inv);
    for (int i = 0; i < 2; ++i) {
        dev_free(ix->d_off[i]);
        dev_free(ix->d_lab[i]);
    }
    dev_free(ix->d_qerr);
    delete ix;
}

// Step 1: checks, order, relabel, reverse CSR. adj_off/adj_col[0] = arcs
// (out-neighbours), [1] = reversed arcs (in-neighbours), both in rank space.
int directed_prep(pll_dindex *ix, const uint32_t *off, const uint32_t *col, const uint32_t *order,
                  DevMem *adj_off, DevMem *adj_col, uint32_t *d_err, cudaStream_t s) {
    const uint32_t n = ix->n;
    const uint64_t nnz = ix->nnz;
    uint32_t h_err = 0;
    k_dvalidate<<<blocks_for(n, 256), 256, 0, s>>>(n, nnz, off, col, d_err);
    PLL_TRY(cudaGetLastError());
    PLL_CHECK(read_back(d_err, &h_err, 4, s));
    if (h_err) return PLL_E_INVAL;
    Graph g;
    g.n = n; g.nnz = nnz; g.off = off; g.col = col;
    if (order) {
        PLL_TRY(cudaMemcpyAsync(ix->d_order, order, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        PLL_CHECK(prep_check_order(g, ix->d_order, d_err, s));
        PLL_CHECK(read_back(d_err, &h_err, 4, s));
        if (h_err) return PLL_E_ORDER;
    } else {
        // the Degree order by in- plus out-degree: a CSR-shaped array whose
        // row lengths are those degrees feeds the undirected order's sort
        // (differences of the wrapped 32-bit scan are exact)
        DevMem deg, doff, temp;
        PLL_CHECK(deg.alloc(((size_t)n + 1) * 4));
        PLL_CHECK(doff.alloc(((size_t)n + 1) * 4));
        PLL_TRY(cudaMemsetAsync(deg.p, 0, ((size_t)n + 1) * 4, s));
        k_dindeg<<<blocks_for(n, 256), 256, 0, s>>>(n, off, col, deg.as<uint32_t>());
        k_ddeg<<<blocks_for(n, 256), 256, 0, s>>>(n, off, deg.as<uint32_t>());
        PLL_TRY(cudaGetLastError());
        size_t tb = 0;
        PLL_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, deg.as<uint32_t>(), doff.as<uint32_t>(),
                                              (int64_t)n + 1, s));
        PLL_CHECK(temp.alloc(tb));
        PLL_TRY(cub::DeviceScan::ExclusiveSum(temp.p, tb, deg.as<uint32_t>(), doff.as<uint32_t>(),
                                              (int64_t)n + 1, s));
        Graph gd;
        gd.n = n; gd.nnz = nnz; gd.off = doff.as<uint32_t>(); gd.col = col;
        PLL_CHECK(prep_degree_order(gd, ix->d_order, s));
    }
    PLL_CHECK(adj_off[0].alloc(((size_t)n + 1) * 4));
    PLL_CHECK(adj_col[0].alloc(std::max<uint64_t>(nnz, 1) * 4));
    PLL_CHECK(prep_relabel(g, ix->d_order, ix->d_inv, adj_off[0].as<uint32_t>(), adj_col[0].as<uint32_t>(), s));
    // reverse CSR: count, scan, scatter, then sort each row
    PLL_CHECK(adj_off[1].alloc(((size_t)n + 1) * 4));
    PLL_CHECK(adj_col[1].alloc(std::max<uint64_t>(nnz, 1) * 4));
    DevMem cnt, cursor, unsorted, temp;
    PLL_CHECK(cnt.alloc(((size_t)n + 1) * 4));
    PLL_CHECK(cursor.alloc(((size_t)n + 1) * 4));
    PLL_CHECK(unsorted.alloc(std::max<uint64_t>(nnz, 1) * 4));
    PLL_TRY(cudaMemsetAsync(cnt.p, 0, ((size_t)n + 1) * 4, s));
    const uint32_t *ro = adj_off[0].as<uint32_t>(), *rc = adj_col[0].as<uint32_t>();
    k_dcount_in<<<blocks_for(n, 256), 256, 0, s>>>(n, ro, rc, cnt.as<uint32_t>());
    PLL_TRY(cudaGetLastError());
    size_t tb = 0;
    PLL_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt.as<uint32_t>(), adj_off[1].as<uint32_t>(),
                                          (int64_t)n + 1, s));
    PLL_CHECK(temp.alloc(tb));
    PLL_TRY(cub::DeviceScan::ExclusiveSum(temp.p, tb, cnt.as<uint32_t>(), adj_off[1].as<uint32_t>(),
                                          (int64_t)n + 1, s));
    PLL_TRY(cudaMemcpyAsync(cursor.p, adj_off[1].p, ((size_t)n + 1) * 4, cudaMemcpyDeviceToDevice, s));
    k_dfill_in<<<blocks_for(n, 256), 256, 0, s>>>(n, ro, rc, cursor.as<uint32_t>(), unsorted.as<uint32_t>());
    PLL_TRY(cudaGetLastError());
    if (nnz) {
        size_t tb2 = 0;
        PLL_TRY(cub::DeviceSegmentedSort::SortKeys(nullptr, tb2, unsorted.as<uint32_t>(), adj_col[1].as<uint32_t>(),
                                                   (int64_t)nnz, (int64_t)n, adj_off[1].as<uint32_t>(),
                                                   adj_off[1].as<uint32_t>() + 1, s));
        if (tb2 > temp.bytes) PLL_CHECK(temp.alloc(tb2));
        PLL_TRY(cub::DeviceSegmentedSort::SortKeys(temp.p, tb2, unsorted.as<uint32_t>(), adj_col[1].as<uint32_t>(),
                                                   (int64_t)nnz, (int64_t)n, adj_off[1].as<uint32_t>(),
                                                   adj_off[1].as<uint32_t>() + 1, s));
    }
    PLL_TRY(cudaStreamSynchronize(s));  // before the temporaries go
    return PLL_OK;
}

struct Store {
    LabelStore st;
    DevMem off, len, cap;
    ~Store() { dev_free(st.pool); }
    int init(uint32_t n, unsigned long long *top, cudaStream_t s) {
        st.n = n;
        PLL_CHECK(off.alloc((size_t)n * 8));
        PLL_CHECK(len.alloc((size_t)n * 4));
        PLL_CHECK(cap.alloc((size_t)n * 4));
        PLL_TRY(cudaMemsetAsync(off.p, 0, (size_t)n * 8, s));
        PLL_TRY(cudaMemsetAsync(len.p, 0, (size_t)n * 4, s));
        PLL_TRY(cudaMemsetAsync(cap.p, 0, (size_t)n * 4, s));
        st.off = off.as<uint64_t>();
        st.len = len.as<uint32_t>();
        st.cap = cap.as<uint32_t>();
        st.pool_cap = std::max<uint64_t>((uint64_t)n * 8, 1ull << 20);
        PLL_TRY(dev_malloc(&st.pool, st.pool_cap * 4));
        st.pool_top = top;
        return PLL_OK;
    }
};

// Steps 2-4: root batches, both directions, cleanup, append; then the CSR.
int directed_labels(pll_dindex *ix, DevMem *adj_off, DevMem *adj_col, uint32_t bmax, cudaStream_t s) {
    const uint32_t n = ix->n;
    DevMem m_ctr;
    PLL_CHECK(m_ctr.alloc(sizeof(DCounters)));
    PLL_TRY(cudaMemsetAsync(m_ctr.p, 0, sizeof(DCounters), s));
    DCounters *c = m_ctr.as<DCounters>();
    Store store[2];  // [0] L_IN, [1] L_OUT
    PLL_CHECK(store[0].init(n, &c->pool_top[0], s));
    PLL_CHECK(store[1].init(n, &c->pool_top[1], s));
    const uint32_t wmax = (bmax + 31) / 32;
    DevMem vis, F, A, NF, T[2], S[2], keep, temp;
    PLL_CHECK(vis.alloc((size_t)n * wmax * 4));
    DCounters h{};
    uint64_t total[2] = {0, 0};
    uint32_t B = std::min<uint32_t>(64, bmax);
    for (uint32_t k0 = 0; k0 < n;) {
        const uint32_t k1 = (uint32_t)std::min<uint64_t>((uint64_t)k0 + B, n), Bc = k1 - k0;
        const uint32_t W = (Bc + 31) / 32;
        uint64_t P[2] = {0, 0};
        for (int dir = 0; dir < 2; ++dir) {
            // forward: along arcs, root label L_OUT, visited labels L_IN;
            // reverse: against arcs, root label L_IN, visited labels L_OUT
            const LabelStore &from = store[1 - dir].st, &to = store[dir].st;
            const uint32_t *ao = adj_off[dir].as<uint32_t>(), *ac = adj_col[dir].as<uint32_t>();
            PLL_TRY(cudaMemsetAsync(vis.p, 0, (size_t)n * W * 4, s));
            PLL_CHECK(ensure(F, (size_t)Bc * 8, 0, s));
            k_dinit<<<blocks_for(Bc, 256), 256, 0, s>>>(k0, Bc, W, vis.as<uint32_t>(), F.as<uint64_t>());
            PLL_TRY(cudaGetLastError());
            PLL_TRY(cudaMemsetAsync(&c->out_n, 0, 8, s));
            uint64_t fn = Bc, out_n = 0;
            for (uint32_t level = 0; fn > 0; ++level) {
                if (level >= INF8) return PLL_E_RANGE;
                PLL_CHECK(ensure(T[dir], (size_t)(out_n + fn) * 8, (size_t)out_n * 8, s));
                PLL_CHECK(ensure(A, (size_t)fn * 8, 0, s));
                PLL_TRY(cudaMemsetAsync(&c->alive_n, 0, 16, s));  // alive_n, deg_sum
                k_dtest<<<blocks_for(fn, 256), 256, 0, s>>>(F.as<uint64_t>(), fn, level, k0, from, to, ao,
                                                            T[dir].as<uint64_t>(), A.as<uint64_t>(), c);
                PLL_TRY(cudaGetLastError());
                PLL_CHECK(read_back(c, &h, sizeof(DCounters), s));
                out_n = h.out_n;
                if (h.alive_n == 0) break;
                PLL_CHECK(ensure(NF, (size_t)std::max<unsigned long long>(h.deg_sum, 1) * 8, 0, s));
                PLL_TRY(cudaMemsetAsync(&c->next_n, 0, 8, s));
                k_dexpand<<<blocks_for(h.alive_n * 32, 256), 256, 0, s>>>(
                    A.as<uint64_t>(), h.alive_n, ao, ac, vis.as<uint32_t>(), W, NF.as<uint64_t>(), c);
                PLL_TRY(cudaGetLastError());
                PLL_CHECK(read_back(&c->next_n, &h.next_n, 8, s));
                std::swap(F.p, NF.p);
                std::swap(F.bytes, NF.bytes);
                fn = h.next_n;
            }
            P[dir] = out_n;
        }
        ix->pre_cleanup += P[0] + P[1];
        // sort both directions, then clean each against the pre-cleanup other
        for (int dir = 0; dir < 2; ++dir) {
            PLL_CHECK(ensure(S[dir], std::max<uint64_t>(P[dir], 1) * 8, 0, s));
            if (P[dir] == 0) continue;
            size_t tb = 0;
            PLL_CHECK(labels_sort_tuples(T[dir].as<uint64_t>(), S[dir].as<uint64_t>(), P[dir], 0, 64, nullptr, &tb, s));
            PLL_CHECK(ensure(temp, tb, 0, s));
            tb = temp.bytes;
            PLL_CHECK(labels_sort_tuples(T[dir].as<uint64_t>(), S[dir].as<uint64_t>(), P[dir], 0, 64, temp.p, &tb, s));
        }
        for (int dir = 0; dir < 2; ++dir) {
            if (P[dir] == 0) continue;
            PLL_CHECK(ensure(keep, P[dir], 0, s));
            k_dcleanup<<<blocks_for(P[dir], 256), 256, 0, s>>>(S[dir].as<uint64_t>(), P[dir],
                                                              S[1 - dir].as<uint64_t>(), P[1 - dir],
                                                              keep.as<uint8_t>());
            PLL_TRY(cudaGetLastError());
            size_t tb = 0;
            PLL_CHECK(labels_compact(S[dir].as<uint64_t>(), keep.as<uint8_t>(), P[dir], T[dir].as<uint64_t>(),
                                     &c->nkept, nullptr, &tb, s));
            PLL_CHECK(ensure(temp, tb, 0, s));
            tb = temp.bytes;
            PLL_CHECK(labels_compact(S[dir].as<uint64_t>(), keep.as<uint8_t>(), P[dir], T[dir].as<uint64_t>(),
                                     &c->nkept, temp.p, &tb, s));
            // worst-case pool growth of one append: 2 x (entries + new) + 8 per run
            PLL_CHECK(read_back(c, &h, sizeof(DCounters), s));
            const uint64_t need = h.pool_top[dir] + 2 * (total[dir] + P[dir]) + 12 * P[dir];
            if (need > store[dir].st.pool_cap)
                PLL_CHECK(labels_regrow(store[dir].st, std::max<uint64_t>(store[dir].st.pool_cap * 2,
                                                                          3 * (total[dir] + P[dir]) + 12 * P[dir]), s));
            PLL_CHECK(labels_append(store[dir].st, T[dir].as<uint64_t>(), &c->nkept, P[dir], &c->err, s));
            PLL_CHECK(read_back(c, &h, sizeof(DCounters), s));
            if (h.err & ERR_POOL) return PLL_E_NOMEM;
            total[dir] += h.nkept;
        }
        ++ix->batches;
        k0 = k1;
        B = std::min<uint32_t>(B * 2, bmax);
    }
    for (int dir = 0; dir < 2; ++dir) {
        PLL_TRY(dev_malloc(&ix->d_off[dir], ((size_t)n + 1) * 8));
        PLL_TRY(dev_malloc(&ix->d_lab[dir], std::max<uint64_t>(total[dir], 1) * 4));
        size_t ftb = 0;
        PLL_CHECK(labels_finalize(store[dir].st, total[dir], ix->d_off[dir], ix->d_lab[dir], nullptr, &ftb, s));
        PLL_CHECK(ensure(temp, std::max<size_t>(ftb, 16), 0, s));
        ftb = temp.bytes;
        PLL_CHECK(labels_finalize(store[dir].st, total[dir], ix->d_off[dir], ix->d_lab[dir], temp.p, &ftb, s));
        ix->entries[dir] = total[dir];
    }
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

}  // namespace

extern "C" {

PLL_API int pll_build_directed(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                               const uint32_t *order, const pll_build_opts *opts, void *stream,
                               pll_dindex **out) {
    if (!out) return PLL_E_INVAL;
    *out = nullptr;
    pll_build_opts o{};
    if (opts) o = *opts;
    if (o.t != 0 || o.flags != 0 || o.reserved != 0) return PLL_E_INVAL;
    if (n > MAX_N || nnz >= 0xffffffffull) return PLL_E_RANGE;
    if ((n > 0 && !offsets) || (nnz > 0 && !cols) || (n == 0 && nnz != 0)) return PLL_E_INVAL;
    uint32_t bmax = o.root_batch ? o.root_batch : 1024;
    if (bmax > (1u << 16)) bmax = 1u << 16;
    while (bmax > 64 && (uint64_t)n * bmax / 8 > (2ull << 30)) bmax >>= 1;
    cudaStream_t s = (cudaStream_t)stream;
    pll_dindex *ix = new (std::nothrow) pll_dindex();
    if (!ix) return PLL_E_NOMEM;
    struct Guard {
        pll_dindex *ix;
        ~Guard() { dindex_release(ix); }
    } guard{ix};
    PLL_TRY(cudaGetDevice(&ix->device));
    ix->n = n;
    ix->nnz = nnz;
    PLL_TRY(dev_malloc(&ix->d_order, std::max<size_t>((size_t)n * 4, 4)));
    PLL_TRY(dev_malloc(&ix->d_inv, std::max<size_t>((size_t)n * 4, 4)));
    PLL_TRY(dev_malloc(&ix->d_qerr, 16));
    PLL_TRY(cudaMemsetAsync(ix->d_qerr, 0, 16, s));
    if (n == 0) {
        for (int dir = 0; dir < 2; ++dir) {
            PLL_TRY(dev_malloc(&ix->d_off[dir], 8));
            PLL_TRY(dev_malloc(&ix->d_lab[dir], 4));
            PLL_TRY(cudaMemsetAsync(ix->d_off[dir], 0, 8, s));
        }
    } else {
        DevMem m_err, adj_off[2], adj_col[2];
        PLL_CHECK(m_err.alloc(4));
        PLL_TRY(cudaMemsetAsync(m_err.p, 0, 4, s));
        PLL_CHECK(directed_prep(ix, offsets, cols, order, adj_off, adj_col, m_err.as<uint32_t>(), s));
        PLL_CHECK(directed_labels(ix, adj_off, adj_col, bmax, s));
    }
    PLL_TRY(cudaStreamSynchronize(s));
    guard.ix = nullptr;
    *out = ix;
    return PLL_OK;
}

PLL_API int pll_dquery(const pll_dindex *idx, const uint32_t *src, const uint32_t *dst, uint64_t q,
                       uint8_t *out, void *stream) {
    if (!idx) return PLL_E_INVAL;
    if (q == 0) return PLL_OK;
    if (!src || !dst || !out) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    DQueryArgs a{idx->n, idx->d_inv, idx->d_off[0], idx->d_off[1], idx->d_lab[0], idx->d_lab[1],
                 src, dst, q, out, idx->d_qerr};
    int dev = 0, sms = 0;
    PLL_TRY(cudaGetDevice(&dev));
    PLL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t want = (q + 7) / 8, most = (uint64_t)(sms > 0 ? sms : 1) * 8;
    k_dquery<<<(unsigned)std::min(want, most), 256, 0, s>>>(a);
    PLL_TRY(cudaGetLastError());
    unsigned long long h[2] = {0, 0};
    PLL_TRY(cudaMemcpyAsync(h, idx->d_qerr, 16, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    if (h[0] == 0 && h[1] == 0) return PLL_OK;
    PLL_TRY(cudaMemsetAsync(idx->d_qerr, 0, 16, s));
    PLL_TRY(cudaStreamSynchronize(s));
    return h[1] ? PLL_E_INVAL : PLL_E_RANGE;
}

PLL_API int pll_dlabel_entries(const pll_dindex *idx, uint64_t *in_entries, uint64_t *out_entries) {
    if (!idx || !in_entries || !out_entries) return PLL_E_INVAL;
    *in_entries = idx->entries[0];
    *out_entries = idx->entries[1];
    return PLL_OK;
}

PLL_API int pll_dexport_labels(const pll_dindex *idx, int which, uint64_t *offsets, uint32_t *hubs,
                               uint8_t *dists) {
    if (!idx || (which != 0 && which != 1) || !offsets) return PLL_E_INVAL;
    const uint64_t E = idx->entries[which];
    if (E && (!hubs || !dists)) return PLL_E_INVAL;
    const uint32_t n = idx->n;
    std::vector<uint64_t> off((size_t)n + 1);
    std::vector<uint32_t> lab(E), inv(n);
    PLL_TRY(cudaMemcpy(off.data(), idx->d_off[which], ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost));
    if (E) PLL_TRY(cudaMemcpy(lab.data(), idx->d_lab[which], E * 4, cudaMemcpyDeviceToHost));
    if (n) PLL_TRY(cudaMemcpy(inv.data(), idx->d_inv, (size_t)n * 4, cudaMemcpyDeviceToHost));
    uint64_t p = 0;
    for (uint32_t v = 0; v < n; ++v) {
        offsets[v] = p;
        const uint32_t r = inv[v];
        for (uint64_t j = off[r]; j < off[(size_t)r + 1]; ++j, ++p) {
            hubs[p] = entry_hub(lab[j]);
            dists[p] = (uint8_t)entry_dist(lab[j]);
        }
    }
    offsets[n] = p;
    return PLL_OK;
}

PLL_API int pll_dexport_order(const pll_dindex *idx, uint32_t *order) {
    if (!idx || (idx->n && !order)) return PLL_E_INVAL;
    if (idx->n) PLL_TRY(cudaMemcpy(order, idx->d_order, (size_t)idx->n * 4, cudaMemcpyDeviceToHost));
    return PLL_OK;
}

PLL_API void pll_dfree(pll_dindex *idx) { dindex_release(idx); }

}  // extern "C"
