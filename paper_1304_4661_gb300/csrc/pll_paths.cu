// pll_paths.cu -- shortest-path queries (Sec. 6, "Shortest-Path Queries").
//
// The paper keeps with each label entry (h, d) of L(v) the parent of v in the
// pruned BFS tree of h and restores an s-t path by climbing that tree from
// both ends. Here the parents are found once, after the build, from the
// finished labels: for (h, d) in L(v) with d > 0, the first neighbour w of v
// (in rank order) whose label holds (h, d - 1). Such a w is one hop nearer to
// h, and it holds h one hop lower in turn, so the climb reaches h in d steps.
// The BFS-tree parent itself is one such neighbour (the pruned BFS of h
// labels every vertex it expands); which one is kept does not change the
// path's length.
//
// When the bit-parallel label alone reaches d(s, t), the path runs through
// r_i or a member of S_{r_i}. The label gives that vertex's exact distance to
// every v: d(r_i, v) - 1, d(r_i, v) or d(r_i, v) + 1 as the member is in
// S^{-1}_{r_i}(v), S^0_{r_i}(v) or neither (Sec. 5.1). So each end walks to it
// one hop at a time, always to the first neighbour one hop nearer. The
// paper leaves paths through bit-parallel labels open; this is the reading
// taken here.
//
// Kernels: k_parents (a warp per vertex, lanes per label entry, each lane
// binary-searching the labels of the vertex's neighbours), k_path_lengths and
// k_paths (a warp per pair: lanes split the label join and the bit-parallel
// slots; the two climbs run on lanes 0 and 1; bit-parallel walks scan 32
// neighbours per step and take the first by ballot).
#include <algorithm>
#include <new>
#include <vector>

#include <cub/device/device_scan.cuh>

#include "pll_internal.cuh"

using namespace pll;

// Shortest-path support over a built index (borrowed: it must outlive this).
struct pll_paths {
    const pll_index *ix = nullptr;
    uint32_t *d_roff = nullptr;  // the graph in rank space, neighbours by rank
    uint32_t *d_rcol = nullptr;
    uint32_t *d_par = nullptr;   // parent (rank) of each label entry
};

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t BIG = 1u << 20;
constexpr uint64_t NOPOS = ~0ull;

// error bits of the path kernels
enum : uint32_t {
    PERR_ID = 1u << 0,      // vertex id >= n
    PERR_SLOT = 1u << 1,    // path_off not non-decreasing, past cap, or a slot too short
    PERR_RANGE = 1u << 2,   // finite distance >= 255
    PERR_WALK = 1u << 3,    // a climb or a walk found no next vertex (graph is not the index's)
};

// position of the packed entry `key` in the hub-sorted label lab[lo, hi)
// (hubs are unique in a label, so packed entries are sorted too)
__device__ __forceinline__ uint64_t find_entry(const uint32_t *__restrict__ lab, uint64_t lo,
                                               uint64_t hi, uint32_t key) {
    const uint64_t end = hi;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (lab[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < end && lab[lo] == key) ? lo : NOPOS;
}

struct ParentArgs {
    uint32_t n;
    const uint32_t *roff, *rcol;
    const uint64_t *lab_off;
    const uint32_t *lab;
    uint32_t *par;
    uint32_t *err;
};

// One warp per vertex v; each lane takes label entries of v and tries v's
// neighbours in rank order until one holds (h, d - 1).
__global__ void __launch_bounds__(256) k_parents(ParentArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < a.n; v += warps) {
        const uint64_t b = a.lab_off[v], e = a.lab_off[v + 1];
        const uint32_t nb = a.roff[v], ne = a.roff[v + 1];
        for (uint64_t j = b + lane; j < e; j += 32) {
            const uint32_t ent = a.lab[j], h = entry_hub(ent), d = entry_dist(ent);
            uint32_t p = NONE;
            if (d == 0) {
                if (h == (uint32_t)v) p = (uint32_t)v;
            } else {
                const uint32_t key = pack_entry(h, d - 1);
                for (uint32_t x = nb; x < ne; ++x) {
                    const uint32_t w = a.rcol[x];
                    if (find_entry(a.lab, a.lab_off[w], a.lab_off[w + 1], key) != NOPOS) { p = w; break; }
                }
            }
            if (p == NONE) atomicOr(a.err, PERR_WALK);
            a.par[j] = p;
        }
    }
}

struct PathArgs {
    uint32_t n, t, tp;
    const uint32_t *inv, *order, *graph;
    const uint8_t *bp_d;
    const uint64_t *bp_m;
    const uint64_t *lab_off;
    const uint32_t *lab, *par;
    const uint32_t *roff, *rcol;
    const uint32_t *src, *dst;
    uint64_t q;
    uint64_t *len;             // k_path_lengths: vertices of each path
    const uint64_t *path_off;  // k_paths: slot of pair i is [path_off[i], path_off[i + 1])
    uint64_t cap;
    uint32_t *path;
    uint32_t *err;
};

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(FULL, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// The common hub of L(s) and L(t) with the least distance sum (lowest rank
// among equals), as (sum << 32) | (hub << 8) | d(hub, s); NOPOS if none.
// Lanes take entries of the shorter label and binary-search the longer.
__device__ __forceinline__ uint64_t best_hub(const PathArgs &a, uint32_t s, uint32_t t, int lane) {
    const uint64_t os = a.lab_off[s], ot = a.lab_off[t];
    const uint32_t ls = (uint32_t)(a.lab_off[s + 1] - os), lt = (uint32_t)(a.lab_off[t + 1] - ot);
    const bool sa = ls <= lt;
    const uint32_t *A = a.lab + (sa ? os : ot), *B = a.lab + (sa ? ot : os);
    const uint32_t la = sa ? ls : lt, lb = sa ? lt : ls;
    uint64_t best = NOPOS;
    for (uint32_t j = lane; j < la; j += 32) {
        const uint32_t ea = A[j], h = entry_hub(ea);
        uint32_t lo = 0, hi = lb;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (entry_hub(B[mid]) < h) lo = mid + 1; else hi = mid;
        }
        if (lo < lb && entry_hub(B[lo]) == h) {
            const uint32_t da = entry_dist(ea), db = entry_dist(B[lo]);
            const uint64_t key = ((uint64_t)(da + db) << 32) | ((uint64_t)h << 8) | (sa ? da : db);
            best = key < best ? key : best;
        }
    }
    return warp_min64(best);
}

// The bit-parallel slot with the least distance (lowest slot among equals) as
// (distance << 16) | (slot << 8) | (kind << 6) | bit: kind 0 meets in
// S^{-1} of both ends (d~ - 2), kind 1 in S^{-1} of one and S^0 of the other
// (d~ - 1), kind 2 at r_i (d~); bit = the lowest member where they meet.
// NONE if no slot reaches both.
__device__ __forceinline__ uint32_t best_bp(const PathArgs &a, uint32_t s, uint32_t t, int lane) {
    uint32_t best = NONE;
    for (uint32_t i = lane; i < a.t; i += 32) {
        const uint32_t x = a.bp_d[(size_t)s * a.tp + i], y = a.bp_d[(size_t)t * a.tp + i];
        if (x == INF8 || y == INF8) continue;
        const uint64_t *ms = a.bp_m + 2 * ((size_t)s * a.t + i);
        const uint64_t *mt = a.bp_m + 2 * ((size_t)t * a.t + i);
        const uint64_t s1 = ms[0], s0 = ms[1], t1 = mt[0], t0 = mt[1];
        uint32_t val = x + y, kind = 2, bit = 0;
        if (s1 & t1) {
            val -= 2; kind = 0; bit = __ffsll((long long)(s1 & t1)) - 1;
        } else if ((s1 & t0) | (s0 & t1)) {
            val -= 1; kind = 1; bit = __ffsll((long long)((s1 & t0) | (s0 & t1))) - 1;
        }
        best = min(best, (val << 16) | (i << 8) | (kind << 6) | bit);
    }
    return warp_min(best);
}

// d(s, t) of two distinct vertices of one graph (BIG if unreachable), with
// its witnesses: hk from best_hub, bk from best_bp.
struct Witness {
    uint64_t hk;
    uint32_t bk, d;
};
__device__ __forceinline__ Witness pair_witness(const PathArgs &a, uint32_t s, uint32_t t, int lane) {
    Witness w;
    w.hk = best_hub(a, s, t, lane);
    w.bk = best_bp(a, s, t, lane);
    const uint32_t dn = w.hk == NOPOS ? BIG : (uint32_t)(w.hk >> 32);
    const uint32_t db = w.bk == NONE ? BIG : (w.bk >> 16);
    w.d = min(dn, db);
    return w;
}

// Distance from the bit-parallel vertex of slot i (r_i for kind 2, else member
// `bit` of S_{r_i}) to v; BIG if unreachable.
__device__ __forceinline__ uint32_t bp_dist_to(const PathArgs &a, uint32_t i, uint32_t kind,
                                               uint32_t bit, uint32_t v) {
    const uint32_t d = a.bp_d[(size_t)v * a.tp + i];
    if (d == INF8) return BIG;
    if (kind == 2) return d;
    const uint64_t *m = a.bp_m + 2 * ((size_t)v * a.t + i);
    const uint64_t b = 1ull << bit;
    if (m[0] & b) return d - 1;
    if (m[1] & b) return d;
    return d + 1;
}

// Walks from v (at distance dv) down to the bit-parallel vertex, writing the
// dv + 1 vertices at path[pos], path[pos + step], ... (lane 0 writes). Every
// lane returns the same value: false if some vertex has no nearer neighbour.
__device__ bool bp_walk(const PathArgs &a, uint32_t i, uint32_t kind, uint32_t bit, uint32_t v,
                        uint32_t dv, int64_t pos, int step, int lane) {
    if (lane == 0) a.path[pos] = a.order[v];
    while (dv > 0) {
        const uint32_t b = a.roff[v], e = a.roff[v + 1];
        uint32_t next = NONE;
        for (uint32_t x = b; x < e; x += 32) {
            const bool ok = x + lane < e && bp_dist_to(a, i, kind, bit, a.rcol[x + lane]) == dv - 1;
            const unsigned m = __ballot_sync(FULL, ok);
            if (m) { next = a.rcol[x + __ffs(m) - 1]; break; }
        }
        if (next == NONE) return false;
        v = next;
        --dv;
        pos += step;
        if (lane == 0) a.path[pos] = a.order[v];
    }
    return true;
}

// Climbs the pruned BFS tree of hub h from v, which holds (h, d), writing the
// d + 1 vertices at path[pos], path[pos + step], ... (one thread).
__device__ bool climb(const PathArgs &a, uint32_t h, uint32_t v, uint32_t d, int64_t pos, int step) {
    for (uint32_t k = d;; --k) {
        a.path[pos] = a.order[v];
        if (k == 0) return v == h;
        const uint64_t j = find_entry(a.lab, a.lab_off[v], a.lab_off[v + 1], pack_entry(h, k));
        if (j == NOPOS) return false;
        v = a.par[j];
        if (v >= a.n) return false;
        pos += step;
    }
}

// Vertices on the path of each pair: d + 1, 0 if unreachable (and for a bad
// id or an out-of-range distance, which raise their error bits).
__global__ void __launch_bounds__(256) k_path_lengths(PathArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t qi = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < a.q; qi += warps) {
        const uint32_t sid = a.src[qi], tid = a.dst[qi];
        uint64_t len = 0;
        if (sid >= a.n || tid >= a.n) {
            if (lane == 0) atomicOr(a.err, PERR_ID);
        } else {
            const uint32_t s = a.inv[sid], t = a.inv[tid];
            if (s == t) {
                len = 1;
            } else if (!a.graph || a.graph[s] == a.graph[t]) {
                const uint32_t d = pair_witness(a, s, t, lane).d;
                if (d < INF8) len = d + 1;
                else if (d < BIG && lane == 0) atomicOr(a.err, PERR_RANGE);
            }
        }
        if (lane == 0) a.len[qi] = len;
    }
}

// One shortest path per pair into its slot; the rest of the slot (all of it
// for an unreachable pair) is filled with NONE.
__global__ void __launch_bounds__(256) k_paths(PathArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t qi = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < a.q; qi += warps) {
        const uint64_t o0 = a.path_off[qi], o1 = a.path_off[qi + 1];
        if (o1 < o0 || o1 > a.cap) {
            if (lane == 0) atomicOr(a.err, PERR_SLOT);
            continue;
        }
        const uint32_t sid = a.src[qi], tid = a.dst[qi];
        uint64_t len = 0;
        if (sid >= a.n || tid >= a.n) {
            if (lane == 0) atomicOr(a.err, PERR_ID);
        } else {
            const uint32_t s = a.inv[sid], t = a.inv[tid];
            if (s == t) {
                if (o1 > o0) {
                    if (lane == 0) a.path[o0] = sid;
                    len = 1;
                } else if (lane == 0) {
                    atomicOr(a.err, PERR_SLOT);
                }
            } else if (!a.graph || a.graph[s] == a.graph[t]) {
                const Witness w = pair_witness(a, s, t, lane);
                const uint64_t hk = w.hk;
                const uint32_t bk = w.bk, d = w.d;
                if (d >= BIG) {
                    // unreachable: an empty path
                } else if (d >= INF8) {
                    if (lane == 0) atomicOr(a.err, PERR_RANGE);
                } else if (o1 - o0 < (uint64_t)d + 1) {
                    if (lane == 0) atomicOr(a.err, PERR_SLOT);
                } else {
                    bool ok;
                    const uint32_t dn = hk == NOPOS ? BIG : (uint32_t)(hk >> 32);
                    if (dn == d) {  // a common hub: climb its tree from both ends
                        const uint32_t h = (uint32_t)(hk >> 8) & 0xffffffu, ds = (uint32_t)hk & 0xffu;
                        bool mine = true;
                        if (lane == 0) mine = climb(a, h, s, ds, (int64_t)o0, 1);
                        else if (lane == 1) mine = climb(a, h, t, d - ds, (int64_t)(o0 + d), -1);
                        ok = __all_sync(FULL, mine);
                    } else {        // through r_i or a member of S_{r_i}
                        const uint32_t i = (bk >> 8) & 0xffu, kind = (bk >> 6) & 3u, bit = bk & 63u;
                        const uint32_t ds = bp_dist_to(a, i, kind, bit, s), dt = bp_dist_to(a, i, kind, bit, t);
                        ok = ds + dt == d && bp_walk(a, i, kind, bit, s, ds, (int64_t)o0, 1, lane) &&
                             bp_walk(a, i, kind, bit, t, dt, (int64_t)(o0 + d), -1, lane);
                    }
                    if (ok) len = (uint64_t)d + 1;
                    else if (lane == 0) atomicOr(a.err, PERR_WALK);
                }
            }
        }
        __syncwarp();  // the walk's writes come before the fill that may cover them
        for (uint64_t x = o0 + len + lane; x < o1; x += 32) a.path[x] = NONE;
    }
}

int warp_grid(uint64_t items, int *blocks) {
    int dev = 0, sms = 0;
    PLL_TRY(cudaGetDevice(&dev));
    PLL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t want = (items + 7) / 8;  // 8 warps per block
    const uint64_t most = (uint64_t)(sms > 0 ? sms : 1) * 8;
    *blocks = (int)(want < most ? (want > 0 ? want : 1) : most);
    return PLL_OK;
}

// stream-ordered 4-byte error word, one per call
struct ErrWord {
    uint32_t *p = nullptr;
    cudaStream_t s;
    explicit ErrWord(cudaStream_t st) : s(st) {}
    ~ErrWord() { if (p) cudaFreeAsync(p, s); }
    int alloc() {
        if (cudaMallocAsync(reinterpret_cast<void **>(&p), 4, s) != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            return PLL_E_NOMEM;
        }
        PLL_TRY(cudaMemsetAsync(p, 0, 4, s));
        return PLL_OK;
    }
    int read(uint32_t *h) {
        PLL_TRY(cudaMemcpyAsync(h, p, 4, cudaMemcpyDeviceToHost, s));
        PLL_TRY(cudaStreamSynchronize(s));
        return PLL_OK;
    }
};

int path_status(uint32_t e) {
    if (e & (PERR_ID | PERR_SLOT | PERR_WALK)) return PLL_E_INVAL;
    if (e & PERR_RANGE) return PLL_E_RANGE;
    return PLL_OK;
}

void paths_release(pll_paths *p) {
    if (!p) return;
    dev_free(p->d_roff);
    dev_free(p->d_rcol);
    dev_free(p->d_par);
    delete p;
}

PathArgs path_args(const pll_paths *p, const uint32_t *src, const uint32_t *dst, uint64_t q,
                   uint32_t *err) {
    const pll_index *ix = p->ix;
    PathArgs a{};
    a.n = ix->n; a.t = ix->t; a.tp = ix->tp;
    a.inv = ix->d_inv; a.order = ix->d_order; a.graph = ix->d_graph;
    a.bp_d = ix->d_bp_d; a.bp_m = ix->d_bp_m;
    a.lab_off = ix->d_lab_off; a.lab = ix->d_lab; a.par = p->d_par;
    a.roff = p->d_roff; a.rcol = p->d_rcol;
    a.src = src; a.dst = dst; a.q = q;
    a.err = err;
    return a;
}

}  // namespace

extern "C" {

PLL_API int pll_paths_create(const pll_index *idx, const uint32_t *offsets, const uint32_t *cols,
                             uint32_t n, uint64_t nnz, void *stream, pll_paths **out) {
    if (!out) return PLL_E_INVAL;
    *out = nullptr;
    if (!idx || n != idx->n || nnz != idx->nnz) return PLL_E_INVAL;
    if ((n > 0 && !offsets) || (nnz > 0 && !cols)) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    pll_paths *p = new (std::nothrow) pll_paths();
    if (!p) return PLL_E_NOMEM;
    struct Guard {
        pll_paths *p;
        ~Guard() { paths_release(p); }
    } guard{p};
    p->ix = idx;
    ErrWord err(s);
    PLL_CHECK(err.alloc());
    uint32_t h = 0;
    Graph g;
    g.n = n; g.nnz = nnz; g.off = offsets; g.col = cols;
    PLL_CHECK(prep_validate_csr(g, err.p, s));
    PLL_CHECK(err.read(&h));
    if (h) return PLL_E_INVAL;
    PLL_TRY(dev_malloc(&p->d_roff, ((size_t)n + 1) * 4));
    PLL_TRY(dev_malloc(&p->d_rcol, std::max<uint64_t>(nnz, 1) * 4));
    PLL_TRY(dev_malloc(&p->d_par, std::max<uint64_t>(idx->entries, 1) * 4));
    {
        DevMem inv;  // relabel writes an inverse order; the index keeps its own
        PLL_CHECK(inv.alloc(std::max<size_t>((size_t)n * 4, 4)));
        PLL_CHECK(prep_relabel(g, idx->d_order, inv.as<uint32_t>(), p->d_roff, p->d_rcol, s));
    }
    if (n > 0 && idx->entries > 0) {
        ParentArgs a{n, p->d_roff, p->d_rcol, idx->d_lab_off, idx->d_lab, p->d_par, err.p};
        int blocks = 0;
        PLL_CHECK(warp_grid(n, &blocks));
        k_parents<<<blocks, 256, 0, s>>>(a);
        PLL_TRY(cudaGetLastError());
    }
    PLL_CHECK(err.read(&h));
    if (h) return PLL_E_INVAL;  // some entry has no parent: not the index's graph
    guard.p = nullptr;
    *out = p;
    return PLL_OK;
}

PLL_API int pll_paths_parents(const pll_paths *p, uint32_t *parents) {
    if (!p) return PLL_E_INVAL;
    const pll_index *ix = p->ix;
    if (ix->entries && !parents) return PLL_E_INVAL;
    const uint32_t n = ix->n;
    std::vector<uint64_t> off((size_t)n + 1);
    std::vector<uint32_t> par(ix->entries), inv(n), order(n);
    PLL_TRY(cudaMemcpy(off.data(), ix->d_lab_off, ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost));
    if (ix->entries)
        PLL_TRY(cudaMemcpy(par.data(), p->d_par, ix->entries * 4, cudaMemcpyDeviceToHost));
    if (n) {
        PLL_TRY(cudaMemcpy(inv.data(), ix->d_inv, (size_t)n * 4, cudaMemcpyDeviceToHost));
        PLL_TRY(cudaMemcpy(order.data(), ix->d_order, (size_t)n * 4, cudaMemcpyDeviceToHost));
    }
    uint64_t k = 0;
    for (uint32_t v = 0; v < n; ++v) {
        const uint32_t r = inv[v];
        for (uint64_t j = off[r]; j < off[(size_t)r + 1]; ++j, ++k)
            parents[k] = par[j] < n ? order[par[j]] : NONE;
    }
    return PLL_OK;
}

PLL_API int pll_path_offsets(const pll_paths *p, const uint32_t *src, const uint32_t *dst, uint64_t q,
                             uint64_t *path_off, uint64_t *total, void *stream) {
    if (!p || !path_off || !total) return PLL_E_INVAL;
    if (q > 0 && (!src || !dst)) return PLL_E_INVAL;
    if (q >= 0x7fffffffull) return PLL_E_RANGE;
    cudaStream_t s = (cudaStream_t)stream;
    ErrWord err(s);
    PLL_CHECK(err.alloc());
    DevMem len, temp;
    PLL_CHECK(len.alloc((q + 1) * 8));
    PLL_TRY(cudaMemsetAsync(len.p, 0, (q + 1) * 8, s));
    if (q > 0) {
        PathArgs a = path_args(p, src, dst, q, err.p);
        a.len = len.as<uint64_t>();
        int blocks = 0;
        PLL_CHECK(warp_grid(q, &blocks));
        k_path_lengths<<<blocks, 256, 0, s>>>(a);
        PLL_TRY(cudaGetLastError());
    }
    size_t tb = 0;
    PLL_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, len.as<uint64_t>(), path_off, (int)(q + 1), s));
    PLL_CHECK(temp.alloc(tb));
    PLL_TRY(cub::DeviceScan::ExclusiveSum(temp.p, tb, len.as<uint64_t>(), path_off, (int)(q + 1), s));
    PLL_TRY(cudaMemcpyAsync(total, path_off + q, 8, cudaMemcpyDeviceToHost, s));
    uint32_t h = 0;
    PLL_CHECK(err.read(&h));  // synchronises: the scan is done before temp and len go
    return path_status(h);
}

PLL_API int pll_path_query(const pll_paths *p, const uint32_t *src, const uint32_t *dst, uint64_t q,
                           const uint64_t *path_off, uint64_t cap, uint32_t *path, void *stream) {
    if (!p) return PLL_E_INVAL;
    if (q == 0) return PLL_OK;
    if (!src || !dst || !path_off || (cap > 0 && !path)) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ErrWord err(s);
    PLL_CHECK(err.alloc());
    PathArgs a = path_args(p, src, dst, q, err.p);
    a.path_off = path_off;
    a.cap = cap;
    a.path = path;
    int blocks = 0;
    PLL_CHECK(warp_grid(q, &blocks));
    k_paths<<<blocks, 256, 0, s>>>(a);
    PLL_TRY(cudaGetLastError());
    uint32_t h = 0;
    PLL_CHECK(err.read(&h));
    return path_status(h);
}

PLL_API void pll_paths_free(pll_paths *p) { paths_release(p); }

}  // extern "C"
