/*
 * pll.h -- C ABI of libpll.so: GB300 (sm_103a) index construction and
 * distance queries for Pruned Landmark Labeling (Akiba, Iwata, Yoshida,
 * "Fast Exact Shortest-Path Distance Queries on Large Networks by Pruned
 * Landmark Labeling", SIGMOD 2013).
 *
 * Problem (Sec. 3.2): given an undirected, unweighted graph G = (V, E), build
 * an index that answers the distance d_G(s, t) for any pair exactly. Sec. 6
 * variants: shortest paths over such an index (pll_paths_*, pll_path_*) and
 * directed graphs (pll_build_directed, pll_dquery, pll_d*).
 *
 * Conventions shared by every entry point
 *   - Graphs are symmetric CSR: offsets[n + 1] (uint32, offsets[0] = 0,
 *     non-decreasing, offsets[n] = nnz) and cols[nnz] (uint32 vertex ids).
 *     Every undirected edge appears as two arcs; neighbour lists are strictly
 *     ascending (so no duplicates); no self-loops. nnz < 2^32, n < 2^24.
 *   - Distances are 8-bit: 255 means unreachable (Sec. 4.5.1, "Arrays").
 *   - Vertex ids in and out of the library are the caller's ids. Inside a
 *     label, hubs are identified by their rank in the vertex order (Sec.
 *     4.5.1, "Sorting Labels"), so every exported label is sorted by hub.
 *   - "device" pointers are CUDA global-memory pointers of the current
 *     device; "host" pointers are ordinary (preferably pinned) host memory.
 *     The caller owns every buffer it passes in; the library owns the index.
 *   - A stream argument is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream). Functions marked "synchronous" wait for that stream
 *     before they return.
 *   - Every function returns a pll_status; no C++ exception crosses the ABI.
 *     On failure no output is valid and nothing is leaked. Apart from the
 *     scratch array of pll_bp_labels_noalloc and the scratch memory pool of
 *     each CUDA context (freed temporaries kept mapped for later calls; see
 *     pll_release_cached), the library holds no global mutable state between
 *     calls; an index is immutable after pll_build, so queries on one index
 *     may run concurrently on different streams.
 */
#ifndef PLL_H
#define PLL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PLL_API __attribute__((visibility("default")))
#else
#define PLL_API
#endif

typedef enum pll_status {
    PLL_OK = 0,
    PLL_E_INVAL = 1,   /* bad argument or malformed CSR (asymmetric, self-loop,
                          duplicate or unsorted neighbours, id >= n) */
    PLL_E_ORDER = 2,   /* order is not a permutation of 0..n-1 */
    PLL_E_RANGE = 3,   /* a size limit is exceeded (n >= 2^24, t > PLL_MAX_T),
                          a BFS depth reaches 255, or a finite query distance
                          is >= 255 */
    PLL_E_NOMEM = 4,   /* device or host allocation failed */
    PLL_E_TIMEOUT = 5, /* a bounded device-side wait ran out */
    PLL_E_CUDA = 6     /* any other CUDA runtime error */
} pll_status;

/* Largest number of bit-parallel roots (t in Sec. 5.4). */
#define PLL_MAX_T 64

/* Opaque index: bit-parallel labels L_BP and normal labels L, resident in
 * device memory of the device that was current at pll_build. */
typedef struct pll_index pll_index;

/* Build options. Zero-initialise and set what you need. */
/* pll_build_opts.flags: how the levels of each root batch run (the same
 * labels every way).
 *   PLL_BUILD_GRAPH_LEVELS (the default, also with flags 0): one CUDA graph
 *     launch per batch, a conditional while node over the expand and test
 *     sweeps (separate kernels); a device-side step after each level stops it
 *     when the frontier is empty. No host read-back within a batch.
 *   PLL_BUILD_COOP_LEVELS: one cooperative launch per batch that runs every
 *     level itself, with grid barriers whose waits are bounded (a wait that
 *     runs out is PLL_E_TIMEOUT); falls back to the graph where the device
 *     cannot launch cooperatively.
 *   PLL_BUILD_HOST_LEVELS: the host enqueues the sweeps of each level as
 *     separate launches and reads a counter block back every few levels; it
 *     takes precedence over the other two. */
#define PLL_BUILD_HOST_LEVELS 1u
#define PLL_BUILD_GRAPH_LEVELS 2u
#define PLL_BUILD_COOP_LEVELS 4u

typedef struct pll_build_opts {
    uint32_t t;          /* bit-parallel roots, 0..PLL_MAX_T (Sec. 5.4). */
    uint32_t root_batch; /* largest number of pruned-BFS roots processed in
                            one batch (batches double from 64 up to it); 0 =
                            16384, halved while n * root_batch / 8 bytes of
                            visited bitmap would exceed 8 GiB. Any value
                            gives the same labels. */
    uint32_t block;      /* threads per CTA of the pruned-BFS kernel: 128,
                            256, 512 or 1024; 0 = library default (256). */
    uint32_t flags;      /* 0 or one of PLL_BUILD_*_LEVELS (below). */
    uint64_t reserved;   /* must be 0. */
} pll_build_opts;

typedef struct pll_stats {
    uint32_t n;                  /* vertices */
    uint32_t t;                  /* bit-parallel roots (per graph) */
    uint64_t nnz;                /* arcs */
    uint64_t label_entries;      /* sum over v of |L(v)| (normal labels) */
    uint64_t pre_cleanup;        /* entries emitted by batched pruned BFSs
                                    before the redundancy cleanup */
    uint64_t visited;            /* vertices dequeued by pruned BFSs */
    uint64_t batches;            /* root batches */
    uint64_t index_bytes;        /* device bytes held by the index */
    double ms_prep;              /* order, relabel, root selection */
    double ms_bp;                /* bit-parallel BFSs */
    double ms_pruned;            /* pruned BFS + cleanup + append + compaction */
    double ms_finalize;          /* label compaction (part of ms_pruned) */
    /* work of the pruned-BFS kernel, summed over its launches */
    double ms_pruned_kernel;     /* CUDA-event time of the pruned-BFS launches */
    uint64_t pruned_launches;    /* its launches */
    uint64_t pruned_scanned;     /* label entries read by prune tests */
    uint64_t pruned_masks;       /* bit-parallel mask pairs read by prune tests */
    uint64_t pruned_expanded;    /* arcs scanned from unpruned vertices */
    uint64_t launches;           /* kernels of this library launched by the build
                                    (not counting CUB's; the kernels a CUDA
                                    graph runs are counted one by one) */
    uint64_t cub_calls;          /* CUB device-wide sorts, scans, selects */
    /* the two sweeps of the pruned stage, CUDA-event time summed over launches */
    double ms_expand;            /* expand sweeps (claim + distance check) */
    double ms_test;              /* test sweeps (masks + labels) */
    uint64_t expand_launches;
    uint64_t test_launches;
    uint64_t candidates;         /* candidates passed from expand to test */
    uint32_t graphs;             /* graphs in the index (1 unless pll_build_batch) */
    uint32_t reserved32;
    /* buffer growth of the pruned stage (none of it changes the labels) */
    uint64_t redone_batches;     /* batches run again after a buffer overflowed */
    uint64_t pool_regrows;       /* times the label pool was moved to a larger one */
    uint64_t table_fallbacks;    /* batches whose root tables did not all fit
                                    (those roots' labels were binary-searched) */
    /* the device-side level loop (one graph or cooperative launch per root
       batch; 0 under PLL_BUILD_HOST_LEVELS): its launches and their
       CUDA-event time. ms_expand / ms_test are then the wall times of its two
       phases. */
    uint64_t levels_launches;
    double ms_levels;
    /* CUDA-event time of each root batch's sort, cleanup, compaction and
       append, summed (ms_pruned less ms_pruned_kernel, ms_post and
       ms_finalize is the time the GPU waited on the host between batches) */
    double ms_post;
    /* most scratch memory the build held at once (its temporaries, from the
       library's scratch pool; the index's own arrays are index_bytes) */
    uint64_t scratch_peak_bytes;
} pll_stats;

/*
 * pll_build -- construct the index (Alg. 2 with the bit-parallel stage of
 * Sec. 5.4; Alg. 1 for each root; Alg. 3 for each bit-parallel root).
 *
 *   offsets, cols  device; the graph (see conventions). Read only.
 *   n, nnz         vertex and arc counts.
 *   order          device, or NULL. order[r] = vertex of rank r (v_{r+1} in
 *                  the paper's 1-based notation). NULL selects the Degree
 *                  strategy of Sec. 4.4.2: descending degree, ties by
 *                  ascending vertex id.
 *   opts           build options (t, batching); NULL = t 0, defaults.
 *   stream         cudaStream_t as void*.
 *   out            receives the new index; free it with pll_free.
 *
 * The CSR is always checked first (offsets, ids, self-loops, strict ascent,
 * symmetry); a malformed graph gives PLL_E_INVAL and no index.
 * The labels are the unique ones Alg. 1/2 produce for this order and t,
 * whatever root_batch and block are. Synchronous. Errors: PLL_E_INVAL,
 * PLL_E_ORDER, PLL_E_RANGE, PLL_E_NOMEM, PLL_E_CUDA.
 */
PLL_API int pll_build(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                      const uint32_t *order, const pll_build_opts *opts, void *stream,
                      pll_index **out);

/* pll_build_host -- as pll_build, but offsets, cols and order are HOST
 * pointers; the library copies them to the device inside the call. */
PLL_API int pll_build_host(const uint32_t *offsets, const uint32_t *cols, uint32_t n,
                           uint64_t nnz, const uint32_t *order, const pll_build_opts *opts,
                           void *stream, pll_index **out);

/*
 * pll_build_batch -- build the indices of several graphs in one call, as one
 * index over their disjoint union. Graph g owns the vertex ids
 * [graph_start[g], graph_start[g + 1]) of the union CSR (offsets, cols: device,
 * same rules as pll_build; no arc may join two graphs, else PLL_E_INVAL).
 * graph_start is a HOST uint32[graphs + 1] with graph_start[0] = 0 and
 * graph_start[graphs] = n.
 *
 * Each graph keeps its own Degree order (Sec. 4.4.2, ties by id) and its own
 * t bit-parallel roots chosen inside it (Sec. 5.4), so its labels and
 * bit-parallel labels are exactly those pll_build gives for that graph alone,
 * with hub ranks counted in the union's order (graphs interleaved by their
 * own ranks: all rank-0 vertices first, then all rank-1 vertices, ...);
 * pll_export_order gives that order. Bit-parallel slot i of a vertex refers to
 * its own graph's i-th root (pll_export_bp_roots then returns graphs * t
 * roots, graph-major). The small graphs' pruned BFSs share the GPU's sweeps.
 * Queries across graphs answer 255. Synchronous.
 */
PLL_API int pll_build_batch(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                            const uint32_t *graph_start, uint32_t graphs,
                            const pll_build_opts *opts, void *stream, pll_index **out);

/*
 * pll_autotune -- pick the pruned-stage batch size and block shape for a
 * graph (or, with graph_start, a batch of graphs as for pll_build_batch) by
 * timing trial builds: root_batch in {1024, 2048, 4096, 8192, 16384} at block
 * 256, then block in {128, 512} at the best root_batch (7 builds, CUDA-event
 * timed on the stream). Writes the fastest options (t included) to *best and
 * their build time to *best_ms (may be NULL). The labels are the same for
 * every choice; only the time differs. Synchronous.
 */
PLL_API int pll_autotune(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                         const uint32_t *graph_start, uint32_t graphs, uint32_t t, void *stream,
                         pll_build_opts *best, double *best_ms);

/*
 * pll_query -- out[i] = d_G(src[i], dst[i]) for i < q: the minimum of the
 * label query Query(s, t, L) (Sec. 3.3, merge join of hub-sorted labels) and
 * the bit-parallel query (Sec. 5.3); 255 if s and t are disconnected;
 * d(s, s) = 0.
 *
 *   src, dst   device uint32[q], caller's vertex ids (< n).
 *   out        device uint8[q].
 *
 * Synchronous: waits for the stream, then returns PLL_E_RANGE if some
 * distance is finite but >= 255 (those entries hold 255) or PLL_E_INVAL if
 * some id is >= n (those entries hold 255).
 */
PLL_API int pll_query(const pll_index *idx, const uint32_t *src, const uint32_t *dst, uint64_t q,
                      uint8_t *out, void *stream);

/* pll_query_async -- as pll_query but only enqueues the work on the stream.
 * Range or id errors are counted on the device; pll_query_errors reads and
 * clears that count (synchronising the stream). */
PLL_API int pll_query_async(const pll_index *idx, const uint32_t *src, const uint32_t *dst,
                            uint64_t q, uint8_t *out, void *stream);
PLL_API int pll_query_errors(const pll_index *idx, void *stream, uint64_t *count);

/* pll_query_host -- as pll_query with HOST src, dst and out; the copies to
 * and from the device happen inside the call.
 *
 * Staging (pll_build_host, pll_query_host): the device copies are
 * stream-ordered allocations from the library's scratch pool (see
 * pll_release_cached), so a repeated call does not map its ~100 MB of
 * staging afresh (that cost milliseconds per call). A staging allocation
 * that fails returns PLL_E_NOMEM. */
PLL_API int pll_query_host(const pll_index *idx, const uint32_t *src, const uint32_t *dst,
                           uint64_t q, uint8_t *out, void *stream);

/*
 * Exports (synchronous, HOST outputs, indexed by the caller's vertex ids).
 *
 * pll_label_entries: *total = sum over v of |L(v)|.
 * pll_export_labels: offsets[n + 1] (uint64), hubs[total] (hub RANKS,
 *   ascending within each vertex), dists[total]. Normal labels only
 *   (Sec. 3.3); the sentinel of Sec. 4.5.2 is not part of the export.
 * pll_export_bp: vertex-major [n][t] arrays of L_BP (Sec. 5.1): d[v*t + i] =
 *   d_G(r_i, v) (255 if unreachable), m1 = S^{-1}_{r_i}(v), m0 = S^0_{r_i}(v)
 *   as 64-bit sets over S_{r_i} (bit j = j-th member in rank order).
 * pll_export_bp_roots: roots[G * t] (vertex ids; 0xFFFFFFFF = empty slot),
 *   cnt[G * t] = |S_{r_i}|, S[G * t * 64] = members of S_{r_i} (vertex ids);
 *   G = 1 for pll_build, the number of graphs for pll_build_batch.
 * pll_export_order: order[n], order[r] = vertex of rank r.
 */
PLL_API int pll_label_entries(const pll_index *idx, uint64_t *total);
PLL_API int pll_export_labels(const pll_index *idx, uint64_t *offsets, uint32_t *hubs,
                              uint8_t *dists);
PLL_API int pll_export_bp(const pll_index *idx, uint8_t *d, uint64_t *m1, uint64_t *m0);
PLL_API int pll_export_bp_roots(const pll_index *idx, uint32_t *roots, uint32_t *cnt,
                                uint32_t *S);
PLL_API int pll_export_order(const pll_index *idx, uint32_t *order);

/* Scratch that pll_bp_labels_noalloc keeps in device memory (64 MiB). */
#define PLL_NOALLOC_SCRATCH_BYTES (64u << 20)

/*
 * pll_bp_labels_noalloc -- the bit-parallel labels that pll_build computes
 * (the greedy choice of roots r_i and neighbour sets S_{r_i}, then one
 * bit-parallel BFS per root), produced without allocating anything. The
 * paper has no counterpart: the entry point is for callers that cannot call
 * cudaMalloc -- their device memory belongs to another allocator (a
 * framework's caching allocator may hold nearly the whole GPU), or their
 * process forbids allocation once it runs. It allocates no device or host
 * memory and calls no allocating library routine.
 *
 *   rank_offsets, rank_cols  device; the graph with vertices relabelled so that
 *                  vertex id == rank in the vertex order (same CSR rules as
 *                  pll_build; it is checked, PLL_E_INVAL if malformed).
 *   n, nnz, t      n >= 1, 1 <= t <= PLL_MAX_T.
 *   d              device uint8[n * tp], tp = t rounded up to a multiple of 16:
 *                  d[v * tp + i] = d_G(r_i, v), 255 if unreachable; the bytes
 *                  t..tp-1 of each row are set to 255.
 *   masks          device uint64[n * t * 2]: masks[2 * (v * t + i)] = S^{-1},
 *                  masks[2 * (v * t + i) + 1] = S^0 of (r_i, v).
 *   roots, cnt, S  device uint32[t], uint32[t], uint32[t * 64]: as
 *                  pll_export_bp_roots, with ranks as vertex ids.
 *
 * The values equal those of pll_build for the same order and t. Scratch is
 * one file-scope device array of PLL_NOALLOC_SCRATCH_BYTES, held by every GPU
 * that loads the library until the process exits; a call needs about
 * 13 * n + nnz / 64 bytes of it plus a few KiB, and returns PLL_E_RANGE if the
 * graph does not fit. Every call looks the array's device address up in the
 * current context (nothing is cached, so a device reset between calls does no
 * harm). Under lazy module loading (the CUDA default) the 64 MiB are reserved
 * on a device by the first call there: make that call early, before the GPU
 * is filled (a reservation that fails is PLL_E_NOMEM) and before any stream
 * capture. All calls share the array, so calls that overlap on the GPU race.
 * Synchronous.
 */
PLL_API int pll_bp_labels_noalloc(const uint32_t *rank_offsets, const uint32_t *rank_cols,
                                  uint32_t n, uint64_t nnz, uint32_t t, uint8_t *d,
                                  uint64_t *masks, uint32_t *roots, uint32_t *cnt, uint32_t *S,
                                  void *stream);

/*
 * Serving loop: an index resident in device memory answers distance requests
 * from many clients with continuous batching. The paper has no counterpart
 * beyond its motivation (exact distances inside latency-sensitive services,
 * Sec. 1); every answer is Query(s, t) exactly as pll_query gives it.
 *
 * A request is q >= 1 pairs in HOST memory plus a HOST uint8[q] result
 * buffer, all owned by the caller; the pairs are read inside
 * pll_server_submit, the result buffer must stay valid until the request is
 * waited for. The server holds a ring of P = pool_bytes / 9 pair slots (8
 * bytes per pair, 1 per result) in pinned, mapped host memory that the GPU
 * reads and writes directly (over NVLink-C2C on a GB300; no copies):
 *   - admission by memory: a ring of at least 4 * max_batch_pairs slots is
 *     cut into up to four parts (each at least 2 * max_batch_pairs), each
 *     with its own lock; a client thread always uses the same part. A
 *     request is admitted when q contiguous slots of its part are free;
 *     until then pll_server_submit blocks. Its slots are held until its
 *     results are back, so at most P pairs are queued or in flight;
 *   - continuous batching: one dispatcher thread launches, whenever one of
 *     `streams` stream slots is free, the admitted requests not yet launched
 *     at the head of a part (arrival order, up to max_batch_pairs pairs; the
 *     parts in turn) as one query launch that
 *     reads the pairs from the ring and writes the results into it; requests
 *     that arrive while others are on the
 *     GPU form the next launch, and launches on different stream slots
 *     overlap on the device;
 *   - requests complete in launch order; each latency is measured from the
 *     start of pll_server_submit to the results being in the caller's buffer
 *     (host steady clock, microseconds), admission wait included.
 * A result never depends on which requests it was batched with.
 *
 * pll_server_start   starts a server on idx's device. opts may be NULL;
 *                    zero fields take the defaults (pool_bytes 256 MiB,
 *                    max_batch_pairs 2^20, streams 4). The index must outlive
 *                    the server. PLL_E_INVAL for streams > 64, pool_bytes < 9
 *                    or reserved != 0; PLL_E_NOMEM if the ring cannot be
 *                    allocated.
 * pll_server_submit  admits and stages a request and returns its ticket.
 *                    PLL_E_RANGE if q exceeds min(max_batch_pairs, P /
 *                    parts) (stats field max_request_pairs), PLL_E_INVAL if
 *                    an id is >= n
 *                    (nothing is queued for the caller then).
 * pll_server_wait    waits for a ticket (timeout_us < 0: no limit; on
 *                    PLL_E_TIMEOUT the ticket stays valid), writes its latency
 *                    and releases the ticket. Returns the request's status.
 * pll_server_replay  an open-loop load generator: `threads` client threads
 *                    (0 = 1, at most 64) submit request i (pairs
 *                    src/dst[req_off[i] .. req_off[i+1]), results to the same
 *                    range of out) at arrival_us[i] microseconds after the
 *                    call starts (non-decreasing), thread i % threads taking
 *                    request i; it waits for all, and writes
 *                    latency_us[i] (-1 for a request not submitted after an
 *                    error) and the wall time to *elapsed_us (may be NULL).
 * pll_server_stop    finishes every admitted request, stops the thread and
 *                    frees the server; tickets not yet waited for are
 *                    released. No other call on the server may run during or
 *                    after it. Returns the first launch error seen, if any.
 */
typedef struct pll_server pll_server;

typedef struct pll_server_opts {
    uint64_t pool_bytes;       /* bytes of the ring (pinned host memory) */
    uint64_t max_batch_pairs;  /* most pairs in one launch */
    uint32_t streams;          /* stream slots (batches in flight), <= 64 */
    uint32_t reserved;         /* must be 0 */
} pll_server_opts;

typedef struct pll_server_stats {
    uint64_t requests, pairs, batches;  /* submitted requests and pairs; launches */
    uint64_t max_batch_pairs;           /* largest batch launched */
    uint64_t max_inflight_bytes;        /* peak pool bytes held (the ring
                                           parts' peaks, summed) */
    uint64_t pool_bytes;                /* the pool's size */
    uint64_t max_request_pairs;         /* largest request accepted */
    double pack_us;                     /* client time staging pairs at submit */
    double unpack_us;                   /* dispatcher time delivering results */
    double device_us;                   /* sum over batches of copy-in..copy-out
                                           stream time (batches overlap) */
} pll_server_stats;

PLL_API int pll_server_start(const pll_index *idx, const pll_server_opts *opts, pll_server **out);
PLL_API int pll_server_submit(pll_server *sv, const uint32_t *src, const uint32_t *dst, uint64_t q,
                              uint8_t *out, uint64_t *ticket);
PLL_API int pll_server_wait(pll_server *sv, uint64_t ticket, int64_t timeout_us,
                            double *latency_us);
PLL_API int pll_server_replay(pll_server *sv, const uint32_t *src, const uint32_t *dst,
                              const uint64_t *req_off, const double *arrival_us, uint64_t count,
                              uint32_t threads, uint8_t *out, double *latency_us,
                              double *elapsed_us);
PLL_API int pll_server_get_stats(pll_server *sv, pll_server_stats *out);
PLL_API int pll_server_stop(pll_server *sv);

/*
 * Learned vertex order. The labels are exact and minimal for any order
 * (Thm 4.1, 4.2) but their size depends on it (Sec. 4.4, Table 4); besides
 * the Degree order of Sec. 4.4.2 the library can order vertices by the score
 * of a small network over per-vertex features. The paper has no such order.
 *
 * pll_features -- feat (device float[n][8], by caller id) receives, each
 *   column standardised over the vertices ((x - mean) / population std, 0
 *   where the std is 0): log(1 + deg), log(1 + sum of the neighbours'
 *   degrees), log(1 + core number), and, from the bit-parallel labels of the
 *   Degree order with t roots (t = 0: zeros) with d_i = min(d(r_i, v), 32):
 *   mean d_i, min d_i, the share of i with d_i <= 2, mean |S^-1_{r_i}(v)| / 64
 *   and mean |S^0_{r_i}(v)| / 64. core (device uint32[n]) and two_hop (device
 *   uint64[n]) receive the raw core numbers and neighbour-degree sums; either
 *   may be NULL. Same CSR rules and errors as pll_build. Synchronous.
 *
 * pll_hub_counts -- counts (device uint32[n], by caller id) = number of label
 *   entries of idx whose hub is the vertex (vertices with none: 0, among them
 *   every bit-parallel vertex); log1p_counts (device float[n] or NULL) =
 *   log(1 + counts), the training target. Synchronous.
 *
 * pll_order_from_scores -- order (device uint32[n]) = vertices by descending
 *   score (device float[n]), ties by ascending id; -0 equals +0, NaN last.
 *   Synchronous.
 *
 * pll_mlp -- the scoring network 8 -> 64 -> 64 -> 1 with ReLU: 4801
 *   parameters, float32 master copy and Adam moments on the device, a
 *   bfloat16 copy used by every forward and backward pass (float32
 *   arithmetic). Parameter layout: W1 [64][8], b1 [64], W2 [64][64], b2 [64],
 *   w3 [64], b3 [1] (row j = weights into unit j).
 *   pll_mlp_create      on the current device, for batches up to max_batch.
 *   pll_mlp_set_params  host float[4801] -> master and bf16 copy; zeroes the
 *                       Adam moments and step. Synchronous.
 *   pll_mlp_get_params  master (host float[4801]) and/or bf16 copy (host
 *                       uint16[4801] bit patterns). Synchronous.
 *   pll_mlp_forward     y[i] = score of row i of x (device float[n][8]).
 *   pll_mlp_grad        gradient of the mean squared error over the batch
 *                       (row g = x[idx[g]] with target[idx[g]], or row g if
 *                       idx is NULL; idx device uint32[batch], every entry
 *                       a row of x and target -- not checked, as x's length
 *                       is not passed) with respect to the bf16 parameters,
 *                       kept on the device with the loss; deterministic.
 *                       PLL_E_RANGE if batch > max_batch.
 *   pll_mlp_read_grad   gradient (host float[4801]) and/or loss (host float).
 *                       Synchronous.
 *   pll_mlp_adam        one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias
 *                       corrected) with the last gradient; refreshes the bf16
 *                       copy.
 *   pll_mlp_train_step  pll_mlp_grad then pll_mlp_adam.
 *
 * pll_learned_order -- pll_features, pll_mlp_forward and
 *   pll_order_from_scores in one call; order (device uint32[n]) can be passed
 *   to pll_build. Synchronous.
 */
typedef struct pll_mlp pll_mlp;

PLL_API int pll_features(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                         uint32_t t, void *stream, float *feat, uint32_t *core, uint64_t *two_hop);
PLL_API int pll_hub_counts(const pll_index *idx, uint32_t *counts, float *log1p_counts,
                           void *stream);
PLL_API int pll_order_from_scores(const float *scores, uint32_t n, uint32_t *order, void *stream);
PLL_API int pll_mlp_create(uint32_t max_batch, pll_mlp **out);
PLL_API void pll_mlp_free(pll_mlp *mlp);
PLL_API int pll_mlp_set_params(pll_mlp *mlp, const float *host_params, void *stream);
PLL_API int pll_mlp_get_params(const pll_mlp *mlp, float *host_master, uint16_t *host_bf16);
PLL_API int pll_mlp_forward(const pll_mlp *mlp, const float *x, uint64_t n, float *y, void *stream);
PLL_API int pll_mlp_grad(pll_mlp *mlp, const float *x, const float *target, const uint32_t *idx,
                         uint32_t batch, void *stream);
PLL_API int pll_mlp_read_grad(const pll_mlp *mlp, float *host_grad, float *host_loss, void *stream);
PLL_API int pll_mlp_adam(pll_mlp *mlp, float lr, void *stream);
PLL_API int pll_mlp_train_step(pll_mlp *mlp, const float *x, const float *target,
                               const uint32_t *idx, uint32_t batch, float lr, void *stream);
PLL_API int pll_learned_order(const uint32_t *offsets, const uint32_t *cols, uint32_t n,
                              uint64_t nnz, uint32_t t, const pll_mlp *mlp, uint32_t *order,
                              void *stream);

/*
 * Shortest-path queries (Sec. 6, "Shortest-Path Queries"): each label entry
 * (h, d) of L(v) gets a parent, a neighbour of v whose label holds (h, d - 1),
 * i.e. the next vertex towards h on a shortest path. A path is restored by
 * climbing from s and from t towards the best common hub. Where only the
 * bit-parallel label reaches d(s, t), the path runs through r_i or a member
 * of S_{r_i}. The label gives that vertex's exact distance to every vertex
 * (Sec. 5.1), so each end walks to it one hop at a time.
 *
 * pll_paths_create -- parents for every label entry of `idx`, plus a copy of
 *   the graph in the index's rank space (4 (n + 1) + 4 nnz + 4 entries bytes
 *   of device memory).
 *     offsets, cols  device; the graph the index was built from (as for
 *                    pll_build; the union CSR for pll_build_batch). Read only.
 *     n, nnz         must equal the index's.
 *     out            receives the object; free it with pll_paths_free.
 *   The index is borrowed, not copied: it must outlive the object. A
 *   malformed CSR, or a graph in which some label entry has no parent (not
 *   the index's graph), gives PLL_E_INVAL. Synchronous. Errors: PLL_E_INVAL,
 *   PLL_E_NOMEM, PLL_E_CUDA.
 */
typedef struct pll_paths pll_paths;
PLL_API int pll_paths_create(const pll_index *idx, const uint32_t *offsets, const uint32_t *cols,
                             uint32_t n, uint64_t nnz, void *stream, pll_paths **out);

/* pll_paths_parents -- host parents[total entries] in the layout of
 * pll_export_labels (vertices by caller id, hubs ascending): the caller id
 * of the parent of v for that hub; v itself for the entry (v, 0).
 * Synchronous. */
PLL_API int pll_paths_parents(const pll_paths *p, uint32_t *parents);

/* pll_path_offsets -- slot offsets for pll_path_query.
 *   src, dst   device uint32[q], caller ids.
 *   path_off   device uint64[q + 1]: path_off[i] = sum over j < i of the
 *              vertex count of pair j's path (d(s_j, t_j) + 1, 0 when
 *              unreachable); path_off[q] = the total.
 *   total      host; receives path_off[q].
 * q < 2^31 - 1 (else PLL_E_RANGE). Synchronous. Errors: PLL_E_INVAL (null
 * pointer, id >= n), PLL_E_RANGE (a finite distance >= 255), PLL_E_CUDA. */
PLL_API int pll_path_offsets(const pll_paths *p, const uint32_t *src, const uint32_t *dst,
                             uint64_t q, uint64_t *path_off, uint64_t *total, void *stream);

/* pll_path_query -- one shortest path per pair.
 *   src, dst   device uint32[q], caller ids.
 *   path_off   device uint64[q + 1]: pair i owns path[path_off[i],
 *              path_off[i + 1]); e.g. the output of pll_path_offsets.
 *   cap        elements of `path`; every path_off[i + 1] must be <= cap.
 *   path       device uint32[cap], caller-owned. Pair i gets s_i, ..., t_i
 *              (d + 1 caller ids; only s_i when s_i = t_i; none when t_i is
 *              unreachable). The rest of its slot is set to 0xffffffff.
 * Synchronous. Errors: PLL_E_INVAL (null pointer; offsets that decrease or
 * pass cap, whose pair is left unwritten; an id >= n or a slot shorter than
 * its path, whose slot is all 0xffffffff), PLL_E_RANGE (a finite distance
 * >= 255), PLL_E_CUDA. */
PLL_API int pll_path_query(const pll_paths *p, const uint32_t *src, const uint32_t *dst,
                           uint64_t q, const uint64_t *path_off, uint64_t cap, uint32_t *path,
                           void *stream);

PLL_API void pll_paths_free(pll_paths *p);

/*
 * Directed graphs (Sec. 6, "Directed Graphs"): two labels per vertex, L_IN(v)
 * = {(u, d(u, v))} and L_OUT(v) = {(u, d(v, u))}, from a pruned BFS along the
 * arcs and one against them for every vertex in rank order; d(s, t) is the
 * least d(s, u) + d(u, t) over hubs u of L_OUT(s) and L_IN(t). There are no
 * bit-parallel labels (their masks need edges both ways), so opts->t must be
 * 0.
 *
 * pll_build_directed -- builds a directed index.
 *   offsets, cols  device; out-neighbour CSR: the arcs u -> cols[e] for e in
 *                  [offsets[u], offsets[u + 1]), each row strictly ascending,
 *                  no self-loops, ids < n, offsets[0] = 0, offsets[n] = nnz.
 *                  A graph whose arcs all come in both directions gives the
 *                  undirected labels (t = 0) in both sets.
 *   order          device or NULL: rank -> vertex; NULL = descending in- plus
 *                  out-degree, ties by ascending id.
 *   opts           t = 0; root_batch as for pll_build (0 = 1024, halved while
 *                  n x root_batch / 8 bytes of visited bits pass 2 GiB); block,
 *                  flags, reserved: 0. NULL = defaults.
 *   out            receives the index; free it with pll_dfree.
 * The labels are the unique ones the sequential method gives for this order.
 * Synchronous. Errors: PLL_E_INVAL (malformed CSR, t != 0), PLL_E_ORDER,
 * PLL_E_RANGE (n >= 2^24, a BFS depth of 255), PLL_E_NOMEM, PLL_E_CUDA.
 */
typedef struct pll_dindex pll_dindex;
PLL_API int pll_build_directed(const uint32_t *offsets, const uint32_t *cols, uint32_t n,
                               uint64_t nnz, const uint32_t *order, const pll_build_opts *opts,
                               void *stream, pll_dindex **out);

/* pll_dquery -- d(src[i], dst[i]) along arcs into out[i] (device uint8, 255 =
 * unreachable). src, dst: device uint32[q], caller ids. Synchronous. Errors:
 * PLL_E_INVAL (id >= n; those answers are 255), PLL_E_RANGE (a finite
 * distance >= 255), PLL_E_CUDA. */
PLL_API int pll_dquery(const pll_dindex *idx, const uint32_t *src, const uint32_t *dst, uint64_t q,
                       uint8_t *out, void *stream);

/* Entry counts of L_IN and L_OUT. */
PLL_API int pll_dlabel_entries(const pll_dindex *idx, uint64_t *in_entries, uint64_t *out_entries);

/* pll_dexport_labels -- host copy of L_IN (which = 0) or L_OUT (which = 1)
 * in the layout of pll_export_labels: offsets[n + 1] by caller id, hub ranks
 * ascending, distances. Synchronous. */
PLL_API int pll_dexport_labels(const pll_dindex *idx, int which, uint64_t *offsets, uint32_t *hubs,
                               uint8_t *dists);

/* pll_dexport_order -- host order[n]: rank -> caller vertex id. */
PLL_API int pll_dexport_order(const pll_dindex *idx, uint32_t *order);

PLL_API void pll_dfree(pll_dindex *idx);

/*
 * The index as a file (the paper answers queries from a disk-resident index,
 * Sec. 6; here the file is an image to keep and load, not to query in place).
 *
 * pll_save -- writes the index to `path` (created or truncated): a 48-byte
 *   header (magic "PLLINDEX", version 1, n, t, row stride, graphs, a flag for
 *   the batch graph array, nnz, label entries) followed by the device arrays
 *   as they are (order, inverse order, bit-parallel distances and masks,
 *   roots, graph of each rank for batch indices, label offsets, labels),
 *   little-endian. PLL_E_INVAL if the file cannot be written. Synchronous.
 * pll_load -- reads such a file into a new index on the current device.
 *   Everything a query indexes with is checked first (the two orders are
 *   inverse permutations, label offsets start at 0, never decrease and end
 *   at the entry count); a file that fails, is truncated or has another
 *   magic or version gives PLL_E_INVAL and no index. Build statistics other
 *   than the sizes are zero. Synchronous.
 */
PLL_API int pll_save(const pll_index *idx, const char *path);
PLL_API int pll_load(const char *path, pll_index **out);

/* Build statistics (sizes, per-phase times in milliseconds). */
PLL_API int pll_get_stats(const pll_index *idx, pll_stats *out);

/* Release the index and its device memory. NULL is ignored. */
PLL_API void pll_free(pll_index *idx);

/*
 * Test hooks for the allocation-failure paths; the paper has no counterpart.
 * pll_test_fail_alloc(k): of the library's device and pinned host
 *   allocations made by index builds, the next k succeed and the one after
 *   fails as if the device were out of memory (the build then returns
 *   PLL_E_NOMEM); k < 0 turns the hook off (the default). Process-wide.
 * pll_test_live_allocs(): those allocations currently alive (an index holds
 *   its own), so a failed build can be checked for leaks.
 */
PLL_API void pll_test_fail_alloc(int64_t k);
PLL_API int64_t pll_test_live_allocs(void);

/*
 * Test hook for the buffer-growth paths of the pruned stage; the paper has no
 * counterpart. pll_test_capacities(cand, out, pool, tables) sets the initial
 * sizes, in entries, of the candidate buffer, the pre-cleanup tuple buffer,
 * the label pool and the root-table pool of every later build (0 keeps the
 * library's own sizing, which is the default). With cand or out set, buffers
 * are not grown ahead of demand, so a batch that overflows one is run again
 * with a larger one; with tables set, the root-table pool keeps that size for
 * the whole build, so the roots whose tables do not fit have their labels
 * binary-searched. None of this changes the labels. Process-wide; the
 * counts appear in pll_stats.
 */
PLL_API void pll_test_capacities(uint64_t cand, uint64_t out, uint64_t pool, uint64_t tables);

/*
 * Test hook for the bounded waits of the cooperative level loop
 * (PLL_BUILD_COOP_LEVELS); the paper has no counterpart.
 * pll_test_barrier_timeout(ns) sets the longest time a CTA waits at one grid
 * barrier of later builds (0 = the default of 10 s). A wait
 * that runs out makes the build return PLL_E_TIMEOUT, with every CTA gone from
 * the kernel and the context usable. Process-wide.
 */
PLL_API void pll_test_barrier_timeout(uint64_t ns);

/*
 * Scratch memory. Every temporary of a build (pll_build, pll_build_host,
 * pll_build_batch, pll_autotune's trials) and the staging copies of the
 * host-pointer entry points are stream-ordered allocations from one memory
 * pool of this library per CUDA context, which keeps freed scratch (up to an
 * eighth of the device's memory) mapped so that the next call does not map
 * and unmap pages again (about 3 ms per GiB). pll_release_cached synchronises the current device
 * and hands the current context's cached scratch back to the driver; later
 * calls work as before. PLL_E_CUDA if the device reports an error.
 */
PLL_API int pll_release_cached(void);

/* Static, human-readable text for a status code. */
PLL_API const char *pll_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* PLL_H */
