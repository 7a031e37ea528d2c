// pll_internal.cuh -- shared declarations of libpll.so (never installed).
//
// Everything inside the library works in RANK SPACE: vertex ids are replaced
// by their rank in the vertex order (the paper stores hub ranks instead of
// vertex ids so labels come out sorted, Sec. 4.5.1 "Sorting Labels"; here the
// whole graph is relabelled once so that hub rank == vertex id). The caller's
// ids are translated only at the ABI boundary (queries, exports).
//
// Device layouts (all in rank space, n vertices, t bit-parallel roots):
//   roff[n+1], rcol[nnz]      CSR, neighbour lists ascending by rank
//   bp_d[n*tp]                d_G(r_i, v), 255 = unreachable (Sec. 5.1); rows
//                             padded to tp = t rounded up to 16 bytes (pad 255)
//   bp_m[2*(n*t)]             interleaved (S^{-1}, S^0) 64-bit sets per (v, i)
//   label entry (uint32)      (hub rank << 8) | distance, hub rank < 2^24
//   labels during the build   per-vertex growable arrays in one pool, each
//                             starting on a 16-byte boundary
//   labels after the build    CSR: lab_off[n+1] (uint64), lab[...] (uint32)
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pll.h"

namespace pll {

constexpr uint8_t INF8 = 255;
constexpr uint32_t NONE = 0xffffffffu;
constexpr int BPW = 64;                  // bits per bit-parallel word (b, Sec. 5)
constexpr uint32_t MAX_N = (1u << 24) - 1;  // hub ranks are packed into 24 bits

// error bits raised by kernels into a device word
enum : uint32_t {
    ERR_CSR = 1u << 0,     // malformed CSR
    ERR_ORDER = 1u << 1,   // order is not a permutation
    ERR_DEPTH = 1u << 2,   // BFS depth reached 255
    ERR_BUF = 1u << 3,     // tuple buffer overflow (batch must be split)
    ERR_POOL = 1u << 4,    // label pool overflow
};

__host__ __device__ inline uint32_t pack_entry(uint32_t hub, uint32_t d) { return (hub << 8) | d; }
__host__ __device__ inline uint32_t entry_hub(uint32_t e) { return e >> 8; }
__host__ __device__ inline uint32_t entry_dist(uint32_t e) { return e & 0xffu; }

// A pre-cleanup tuple of a root batch: (vertex u, hub k, distance).
// Sorting the 64-bit key orders tuples by vertex, then hub.
__host__ __device__ inline uint64_t pack_tuple(uint32_t u, uint32_t k, uint32_t d) {
    return ((uint64_t)u << 32) | pack_entry(k, d);
}

}  // namespace pll

// The opaque index of the C ABI.
struct pll_index {
    int device = 0;
    uint32_t n = 0, t = 0;
    uint32_t tp = 0;               // bp_d row stride: t rounded up to 16
    uint32_t graphs = 1;           // graphs built together (disjoint union)
    uint64_t nnz = 0;
    uint32_t *d_order = nullptr;   // rank -> caller vertex id
    uint32_t *d_inv = nullptr;     // caller vertex id -> rank
    uint8_t *d_bp_d = nullptr;     // [n][tp]
    uint64_t *d_bp_m = nullptr;    // [n][t][2]
    uint32_t *d_bp_root = nullptr; // [graphs][t] ranks (NONE = empty slot)
    uint32_t *d_bp_cnt = nullptr;  // [graphs][t]
    uint32_t *d_bp_S = nullptr;    // [graphs][t][64] ranks
    uint32_t *d_graph = nullptr;   // [n] graph of each rank (batch indices only)
    uint64_t *d_lab_off = nullptr; // [n+1]
    uint32_t *d_lab = nullptr;     // packed entries
    uint64_t entries = 0;
    unsigned long long *d_qerr = nullptr;  // query error counter
    pll_stats stats{};
};

namespace pll {

// ---- host helpers (pll_abi.cu) ----
int cuda_status(cudaError_t e);  // maps a CUDA error to a pll_status
void index_release(pll_index *ix);  // frees every device array and the index

#define PLL_TRY(expr)                                   \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return ::pll::cuda_status(_e); \
    } while (0)

#define PLL_CHECK(st)              \
    do {                           \
        int _s = (st);             \
        if (_s != PLL_OK) return _s; \
    } while (0)

// Every device and pinned allocation of the build goes through these: they
// keep a count of live allocations and carry the allocation-failure test
// hook (pll_test_fail_alloc), both kept in pll_abi.cu.
bool alloc_should_fail();
void alloc_note(long long delta);
// initial capacities of the pruned stage's buffers set by pll_test_capacities
// (0 = the library's own sizing); entries of each buffer
struct TestCaps {
    uint64_t cand = 0, out = 0, pool = 0, ht = 0;
};
TestCaps test_caps();
// longest wait of a grid barrier of the level loop, ns (pll_test_barrier_timeout)
uint64_t test_barrier_timeout_ns();
template <class T> inline cudaError_t dev_malloc(T **p, size_t b) {
    *p = nullptr;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), b);
    if (e == cudaSuccess) alloc_note(1);
    return e;
}
inline void dev_free(void *p) {
    if (!p) return;
    cudaFree(p);
    alloc_note(-1);
}
template <class T> inline cudaError_t host_malloc(T **p, size_t b) {
    *p = nullptr;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(p), b);
    if (e == cudaSuccess) alloc_note(1);
    return e;
}
inline void host_free(void *p) {
    if (!p) return;
    cudaFreeHost(p);
    alloc_note(-1);
}

// The library's stream-ordered memory pool of the current CUDA context
// (pll_abi.cu), which keeps freed memory mapped for later calls; nullptr if
// the driver cannot name the context (the default pool is used then).
cudaMemPool_t scratch_pool();
// Stream-ordered scratch from that pool (counted and failed like dev_malloc).
template <class T> inline cudaError_t pool_malloc(T **p, size_t b, cudaStream_t s) {
    *p = nullptr;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    void *q = nullptr;
    const cudaMemPool_t pool = scratch_pool();
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, b ? b : 16, pool, s)
                               : cudaMallocAsync(&q, b ? b : 16, s);
    if (e == cudaSuccess) { *p = static_cast<T *>(q); alloc_note(1); }
    return e;
}
inline void pool_free(void *p, cudaStream_t s) {
    if (!p) return;
    cudaFreeAsync(p, s);
    alloc_note(-1);
}
// Scratch of one call: freed in stream order on its stream when it goes out
// of scope, so no host wait and no unmapping; release() hands ownership out
// (the new owner frees it with pool_free on the same stream).
struct PoolMem {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s;
    explicit PoolMem(cudaStream_t st) : s(st) {}
    PoolMem(const PoolMem &) = delete;
    PoolMem &operator=(const PoolMem &) = delete;
    ~PoolMem() { reset(); }
    int alloc(size_t b) {
        reset();
        if (b == 0) b = 16;
        const cudaError_t e = pool_malloc(&p, b, s);
        if (e != cudaSuccess) { p = nullptr; (void)cudaGetLastError(); return PLL_E_NOMEM; }
        bytes = b;
        return PLL_OK;
    }
    void reset() {
        pool_free(p, s);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
    void *release() { void *q = p; p = nullptr; bytes = 0; return q; }
};

// Device allocation that frees itself; release() hands ownership out (the
// new owner frees it with dev_free).
struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    ~DevMem() { reset(); }
    int alloc(size_t b) {
        reset();
        if (b == 0) b = 16;
        cudaError_t e = dev_malloc(&p, b);
        if (e != cudaSuccess) { p = nullptr; (void)cudaGetLastError(); return PLL_E_NOMEM; }
        bytes = b;
        return PLL_OK;
    }
    void reset() {
        dev_free(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
    void *release() { void *q = p; p = nullptr; bytes = 0; return q; }
};

// ---- launchers (one translation unit each) ----
struct Graph {
    uint32_t n = 0;
    uint64_t nnz = 0;
    const uint32_t *off = nullptr;  // caller space
    const uint32_t *col = nullptr;
};

// k_prep.cu
int prep_validate_csr(const Graph &g, uint32_t *d_err, cudaStream_t s);
int prep_degree_order(const Graph &g, uint32_t *d_order, cudaStream_t s);
int prep_check_order(const Graph &g, const uint32_t *d_order, uint32_t *d_err, cudaStream_t s);
int prep_relabel(const Graph &g, const uint32_t *d_order, uint32_t *d_inv, uint32_t *d_roff,
                 uint32_t *d_rcol, cudaStream_t s);
int prep_select_bp_roots(uint32_t n, uint32_t t, const uint32_t *d_roff, const uint32_t *d_rcol,
                         uint8_t *d_inX, uint32_t *d_root, uint32_t *d_cnt, uint32_t *d_S,
                         cudaStream_t s);
// several graphs as one disjoint union: d_gs[G+1] device vertex ranges
int prep_batch_order(const Graph &g, const uint32_t *d_gs, uint32_t G, uint32_t *d_gof,
                     uint32_t *d_local_order, uint32_t *d_order, uint32_t *d_err, cudaStream_t s);
int prep_graph_by_rank(uint32_t n, const uint32_t *d_order, const uint32_t *d_gof, uint32_t *d_out,
                       cudaStream_t s);
int prep_select_bp_graphs(uint32_t G, uint32_t t, const uint32_t *d_gs, const uint32_t *d_local_order,
                          const uint32_t *d_inv, const uint32_t *d_roff, const uint32_t *d_rcol,
                          uint8_t *d_inX, uint32_t *d_root, uint32_t *d_cnt, uint32_t *d_S,
                          cudaStream_t s);

// k_bp.cu
inline uint32_t bp_stride(uint32_t t) { return (t + 15u) & ~15u; }
int bp_run(uint32_t n, uint32_t t, uint32_t graphs, const uint32_t *d_roff, const uint32_t *d_rcol,
           const uint32_t *d_root, const uint32_t *d_cnt, const uint32_t *d_S, uint8_t *d_bp_d,
           uint64_t *d_bp_m, uint32_t *d_err, cudaStream_t s, uint32_t *levels);

// k_bp.cu, for pll_bp_labels_noalloc: the same stage on caller scratch
size_t bp_scratch_bytes(uint32_t n, uint64_t nnz, size_t *cub_bytes);
int bp_run_in(uint32_t n, uint32_t t, const uint32_t *d_roff, const uint32_t *d_rcol,
              uint64_t nnz, const uint32_t *d_root, const uint32_t *d_cnt, const uint32_t *d_S,
              uint8_t *d_bp_d, uint64_t *d_bp_m, uint32_t *d_err, void *scratch,
              size_t scratch_bytes, cudaStream_t s);

// k_pruned.cu -- batch-synchronous pruned BFS over roots [k0, k0 + B)
// root label hash tables: 2 x |L(v_k)| slots rounded up to a power of two,
// at least HT_MIN; labels longer than HT_MAX / 2 are binary-searched instead
constexpr uint32_t FILT_WORDS = 32;     // 1024-bit hub filter per root of a batch
constexpr uint32_t FILT_MAX_LEN = 128;  // roots with longer labels have no filter
constexpr uint32_t HT_MIN = 32;
constexpr uint32_t HT_MAX = 1u << 16;
__host__ __device__ inline uint32_t ht_size(uint32_t len) {
    if (len == 0 || 2 * len > HT_MAX) return 0;
    uint32_t s = HT_MIN;
    while (s < 2 * len) s <<= 1;
    return s;
}

struct BatchCounters {
    unsigned long long cand_n;    // candidates appended (all levels of the batch)
    unsigned long long out_n;     // entries (u, k, d) appended
    unsigned long long work[4];   // label entries scanned, mask pairs, arcs, vertices
                                  // claimed (cumulative)
    unsigned long long nkept;     // entries kept by the cleanup
    unsigned long long pool_top;  // label pool bump pointer
    uint32_t err;                 // errors of the batch's BFS (reset per batch)
    uint32_t err_post;            // errors of the appends (never reset)
};
constexpr uint32_t ERR_TABLE = 1u << 5;    // root hash-table pool too small
constexpr uint32_t ERR_TIMEOUT = 1u << 6;  // a grid barrier waited past its limit

// State of the device-side level loop (k_batch_levels): a grid barrier and
// the snapshots its last CTA takes; phase times summed over the build.
struct LoopState {
    unsigned int count, gen;            // barrier arrivals, generation
    unsigned int err, pad;              // snapshot of BatchCounters::err
    unsigned long long cand_n, out_n;   // snapshots of the counts
    unsigned long long timeout_ns;      // longest barrier wait
    unsigned long long ns_expand, ns_test;  // phase wall times (block 0)
    unsigned long long levels;          // levels run
    unsigned long long t_mark;          // graph loop: start of the current phase
};

struct LevelDesc {
    unsigned long long lvl_b, lvl_e;    // entries of the current level
    unsigned long long cand_b, cand_e;  // candidates of the next level
    unsigned long long roots_n;         // level-0 entries
    uint32_t level;
    uint32_t pad;
};

struct BatchArgs {
    uint32_t n, t, tp;
    const uint32_t *roff, *rcol;
    const uint8_t *bp_d;
    const uint8_t *bp_c;       // bp_d with every byte clamped to 63 (same stride)
    const uint64_t *bp_m;
    const uint8_t *inX;
    const uint64_t *lab_off;   // per-vertex start in pool
    const uint32_t *lab_len;   // per-vertex length (entries with hub < k0)
    const uint32_t *pool;
    uint32_t k0, B, NW;        // roots [k0, k0 + B), NW = ceil(n / 32)
    uint32_t *visited;         // [B][NW] bitmap: row of root slot s holds one bit
                               // per vertex (the per-root visited set of Alg. 1)
    uint32_t *ht;              // pool of root label hash tables
    unsigned long long *ht_off;  // [B + 1] table offsets in the pool (exclusive sums)
    unsigned long long ht_cap;   // pool capacity (entries)
    uint64_t *rootbits;        // [B][2] feasibility masks
    uint32_t *filt;            // [B][FILT_WORDS] per-root filter of its label's hubs
    uint64_t *cand;            // (slot << 32 | vertex), all levels
    uint64_t *candc;           // [cand_cap][2] roots whose masks may still prune
    unsigned long long cand_cap;
    uint64_t *out;             // entries (u << 32 | k << 8 | d), all levels
    unsigned long long out_cap;
    BatchCounters *ctr;
    LevelDesc *desc;
    LoopState *loop;           // device-side level loop (k_batch_levels)
};
int batch_grid(uint32_t block, int *grid);  // grid[2]: expand, test
int batch_init(const BatchArgs &a, void *temp, size_t temp_bytes, cudaStream_t s);
size_t batch_init_temp_bytes(uint32_t bmax);
int batch_level(const BatchArgs &a, const int *grid, uint32_t block, cudaStream_t s,
                cudaEvent_t *ev);
// all levels of a batch in one cooperative launch (grid from
// batch_levels_grid; 0 there means cooperative launches are unavailable)
int batch_levels_grid(uint32_t block, int *grid);
int batch_levels(const BatchArgs &a, uint32_t block, int grid, cudaStream_t s);
// the level loop as a CUDA graph (a while node over the two sweeps), reading
// the batch's arguments from d_args; one instantiation serves every batch
int batch_graph_build(uint32_t block, const int *grid, const BatchArgs *d_args, cudaGraph_t *g,
                      cudaGraphExec_t *exec);
// lazy reset of the visited bitmap after a batch: clears the words of the
// roots and of every recorded candidate (all bits the batch set)
int batch_clear(const BatchArgs &a, int grid, cudaStream_t s);
// bp_c = min(bp_d, 63) bytewise (bytes a multiple of 16)
int batch_clamp_rows(const uint8_t *bp_d, uint8_t *bp_c, size_t bytes, int grid, cudaStream_t s);

// k_labels.cu
struct LabelStore {
    uint32_t n = 0;
    uint64_t *off = nullptr;   // [n]
    uint32_t *len = nullptr;   // [n]
    uint32_t *cap = nullptr;   // [n]
    uint32_t *pool = nullptr;
    uint64_t pool_cap = 0;
    unsigned long long *pool_top = nullptr;
    bool pooled = false;  // `pool` comes from pool_malloc (else dev_malloc)
};
// radix sort of packed tuples by their bits [begin_bit, end_bit)
int labels_sort_tuples(uint64_t *d_in, uint64_t *d_out, uint64_t count, int begin_bit, int end_bit,
                       void *d_temp, size_t *temp_bytes, cudaStream_t s);
// scratch (>= 16 B bytes, may be NULL) holds each root's own tuple range
int labels_cleanup(const uint64_t *d_sorted, uint64_t count, uint8_t *d_keep, uint32_t k0, uint32_t B,
                   void *scratch, size_t scratch_bytes, cudaStream_t s);
int labels_compact(const uint64_t *d_in, const uint8_t *d_keep, uint64_t count, uint64_t *d_out,
                   unsigned long long *d_nout, void *d_temp, size_t *temp_bytes, cudaStream_t s);
int labels_append(const LabelStore &st, const uint64_t *d_kept,
                  const unsigned long long *d_nkept, uint64_t max_count, uint32_t *d_err,
                  cudaStream_t s);
int labels_regrow(LabelStore &st, uint64_t new_cap, cudaStream_t s);
int labels_finalize(const LabelStore &st, uint64_t total, uint64_t *d_off, uint32_t *d_lab,
                    void *d_temp, size_t *temp_bytes, cudaStream_t s);
int scan_u32_to_u64(const uint32_t *d_in, uint64_t *d_out, uint32_t n, void *d_temp,
                    size_t *temp_bytes, cudaStream_t s, uint32_t round);

// k_query.cu
int query_launch(const pll_index *ix, const uint32_t *d_src, const uint32_t *d_dst, uint64_t q,
                 uint8_t *d_out, cudaStream_t s);
// as query_launch with pair i at (d_src[i * stride], d_dst[i * stride])
int query_launch_strided(const pll_index *ix, const uint32_t *d_src, const uint32_t *d_dst,
                         uint32_t stride, uint64_t q, uint8_t *d_out, cudaStream_t s);

}  // namespace pll
