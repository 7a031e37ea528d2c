// pll_abi.cu -- the C ABI of include/pll.h and the host side of the build.
//
// pll_build runs, on the caller's stream:
//   1. CSR checks, vertex order (given, or the Degree strategy of Sec. 4.4.2),
//      relabelling into rank space;
//   2. the greedy bit-parallel root choice and t bit-parallel BFSs (Sec. 5.4,
//      Alg. 3);
//   3. Alg. 2 over batches of roots [k0, k1): the BFSs of all roots of a
//      batch advance level by level as bulk-synchronous sweeps (Alg. 1 per
//      root, pruned with hubs < k0 and the bit-parallel labels), then sort +
//      redundancy cleanup + append of the batch's entries; batch sizes double
//      from 64 up to root_batch;
//   4. compaction of the labels into one hub-sorted CSR for queries.
// Level boundaries stay on the device; the host reads a small counter block
// every few levels (to see an empty frontier) and once after the append.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <atomic>

#include "pll_internal.cuh"

namespace pll {

int cuda_status(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PLL_E_NOMEM : PLL_E_CUDA;
}

namespace {

int err_to_status(uint32_t err) {
    if (err & ERR_CSR) return PLL_E_INVAL;
    if (err & ERR_ORDER) return PLL_E_ORDER;
    if (err & ERR_DEPTH) return PLL_E_RANGE;
    if (err & ERR_POOL) return PLL_E_NOMEM;
    if (err & ERR_TIMEOUT) return PLL_E_TIMEOUT;
    return PLL_OK;
}

int read_err(uint32_t *d_err, cudaStream_t s, uint32_t *h) {
    PLL_TRY(cudaMemcpyAsync(h, d_err, 4, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

int bit_length(uint32_t x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

void free_index(pll_index *ix) {
    if (!ix) return;
    dev_free(ix->d_order);
    dev_free(ix->d_inv);
    dev_free(ix->d_bp_d);
    dev_free(ix->d_bp_m);
    dev_free(ix->d_bp_root);
    dev_free(ix->d_bp_cnt);
    dev_free(ix->d_bp_S);
    dev_free(ix->d_graph);
    dev_free(ix->d_lab_off);
    dev_free(ix->d_lab);
    dev_free(ix->d_qerr);
    delete ix;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    void start() { cudaEventRecord(a, s); }
    double stop_ms() {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
};

// Step 3: batched pruned BFS + cleanup + append, then step 4.
int pruned_stage(pll_index *ix, const uint32_t *roff, const uint32_t *rcol, const uint8_t *inX,
                 uint32_t bmax, uint32_t block, uint32_t flags, cudaStream_t s) {
    // how each batch's levels run: a CUDA graph whose while node loops over
    // the two sweeps (the default), one cooperative persistent launch, or
    // separate launches enqueued by the host
    const bool host_levels = (flags & PLL_BUILD_HOST_LEVELS) != 0;
    const bool coop_levels = !host_levels && (flags & PLL_BUILD_COOP_LEVELS) != 0;
    const uint32_t n = ix->n;
    LabelStore st;
    st.n = n;
    // every temporary of the stage is stream-ordered scratch from the pool
    PoolMem m_off(s), m_len(s), m_cap(s), m_pool(s), m_ctr(s), m_desc(s);
    PLL_CHECK(m_off.alloc((size_t)n * 8));
    PLL_CHECK(m_len.alloc((size_t)n * 4));
    PLL_CHECK(m_cap.alloc((size_t)n * 4));
    PLL_CHECK(m_ctr.alloc(sizeof(BatchCounters)));
    PLL_CHECK(m_desc.alloc(sizeof(LevelDesc)));
    PLL_TRY(cudaMemsetAsync(m_off.p, 0, (size_t)n * 8, s));
    PLL_TRY(cudaMemsetAsync(m_len.p, 0, (size_t)n * 4, s));
    PLL_TRY(cudaMemsetAsync(m_cap.p, 0, (size_t)n * 4, s));
    PLL_TRY(cudaMemsetAsync(m_ctr.p, 0, sizeof(BatchCounters), s));
    PLL_TRY(cudaMemsetAsync(m_desc.p, 0, sizeof(LevelDesc), s));
    BatchCounters *d_ctr = m_ctr.as<BatchCounters>();
    LevelDesc *d_desc = m_desc.as<LevelDesc>();
    st.off = m_off.as<uint64_t>();
    st.len = m_len.as<uint32_t>();
    st.cap = m_cap.as<uint32_t>();
    st.pool_cap = test_caps().pool ? test_caps().pool : std::max<uint64_t>((uint64_t)n * 64, 1ull << 22);
    PLL_CHECK(m_pool.alloc(st.pool_cap * 4));
    st.pool = m_pool.as<uint32_t>();
    st.pooled = true;
    m_pool.release();  // owned through st.pool from here on (regrow swaps it)
    st.pool_top = &d_ctr->pool_top;
    struct PoolGuard {
        LabelStore *st;
        cudaStream_t s;
        ~PoolGuard() { pool_free(st->pool, s); }
    } pool_guard{&st, s};

    int grid[2] = {0, 0};
    PLL_CHECK(batch_grid(block, grid));
    // the device-side level loop: one cooperative launch per batch (the host
    // enqueues the levels itself when asked to, or when the device cannot
    // launch cooperatively)
    int lgrid = 0;
    if (coop_levels) PLL_CHECK(batch_levels_grid(block, &lgrid));
    const bool device_levels = lgrid > 0;  // the cooperative launch is available
    const bool graph_levels = !host_levels && !device_levels;
    PoolMem m_loop(s);
    PLL_CHECK(m_loop.alloc(sizeof(LoopState)));
    LoopState *d_loop = m_loop.as<LoopState>();
    {
        LoopState init{};
        init.timeout_ns = test_barrier_timeout_ns();
        PLL_TRY(cudaMemcpyAsync(d_loop, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    }
    // clamped copy of the bit-parallel distance rows for the expand sweep
    PoolMem m_bpc(s);
    PLL_CHECK(m_bpc.alloc(std::max<size_t>((size_t)n * ix->tp, 16)));
    PLL_CHECK(batch_clamp_rows(ix->d_bp_d, m_bpc.as<uint8_t>(), (size_t)n * ix->tp, grid[0], s));
    ix->stats.launches += 1;
    // visited bitmap, one row of ceil(n / 32) words per root slot; cleared once
    // here, then lazily after each batch (only the words the batch set)
    const uint32_t NW = (n + 31) / 32;
    PoolMem m_vis(s), m_ht(s), m_htoff(s), m_itemp(s), m_bits(s), m_cand(s), m_candc(s), m_out(s),
        m_sorted(s), m_keep(s), m_temp(s);
    PLL_CHECK(m_vis.alloc((size_t)bmax * NW * 4));
    PLL_TRY(cudaMemsetAsync(m_vis.p, 0, (size_t)bmax * NW * 4, s));
    const TestCaps caps = test_caps();
    // Initial sizes generous enough that the first large root batches do not
    // overflow (a batch that overflows runs again; roots whose tables do not
    // fit are binary-searched): scratch comes from the pool, so a large buffer
    // costs memory but no mapping time. The candidate and tuple buffers, the
    // two largest, take at most a sixteenth of the free memory each.
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        (void)cudaGetLastError();
        free_b = 0;
    }
    uint64_t ht_cap = caps.ht ? caps.ht : std::max<uint64_t>((uint64_t)bmax * 2048, 1ull << 20);
    PLL_CHECK(m_ht.alloc(ht_cap * 4));
    PLL_CHECK(m_htoff.alloc(((size_t)bmax + 1) * 8));
    const size_t itemp_bytes = ((batch_init_temp_bytes(bmax) + 255) & ~(size_t)255) + ((size_t)bmax + 1) * 8 + 256;
    PLL_CHECK(m_itemp.alloc(itemp_bytes));
    PLL_CHECK(m_bits.alloc((size_t)bmax * 16));
    PoolMem m_filt(s);
    PLL_CHECK(m_filt.alloc((size_t)bmax * FILT_WORDS * 4));
    uint64_t cand_cap = caps.cand ? caps.cand
                                  : std::max<uint64_t>(std::min<uint64_t>((uint64_t)n * 256, free_b / 16 / 24),
                                                       1ull << 24);
    uint64_t out_cap = caps.out ? caps.out
                                : std::max<uint64_t>(std::min<uint64_t>((uint64_t)n * 64, free_b / 16 / 17),
                                                     1ull << 22);
    size_t temp_bytes = 0;
    const int end_bit = 32 + std::max(1, bit_length(n - 1));
    // the distance byte is no sort key: a root's BFS labels a vertex at most
    // once (one visited bit per root and vertex), so (u, k) is unique within
    // a batch and the order by (u, k) is the whole order
    constexpr int SORT_BEGIN_BIT = 8;
    auto alloc_out = [&]() -> int {
        PLL_CHECK(m_out.alloc(out_cap * 8));
        PLL_CHECK(m_sorted.alloc(out_cap * 8));
        PLL_CHECK(m_keep.alloc(out_cap));
        size_t a = 0, b = 0;
        PLL_CHECK(labels_sort_tuples(nullptr, nullptr, out_cap, SORT_BEGIN_BIT, end_bit, nullptr, &a, s));
        PLL_CHECK(labels_compact(nullptr, nullptr, out_cap, nullptr, nullptr, nullptr, &b, s));
        temp_bytes = std::max(a, b);
        PLL_CHECK(m_temp.alloc(temp_bytes));
        return PLL_OK;
    };
    PLL_CHECK(m_cand.alloc(cand_cap * 8));
    PLL_CHECK(m_candc.alloc(cand_cap * 16));
    PLL_CHECK(alloc_out());

    // pinned mirror of the counters and the level descriptor
    struct Mirror {
        BatchCounters c;
        LevelDesc d;
        BatchArgs args;  // staging of the graph loop's device-side arguments
    };
    Mirror *h = nullptr;
    PLL_TRY(host_malloc(&h, sizeof(Mirror)));
    struct HostGuard {
        Mirror *h;
        ~HostGuard() { host_free(h); }
    } host_guard{h};
    auto read_back = [&]() -> int {
        PLL_TRY(cudaMemcpyAsync(&h->c, d_ctr, sizeof(BatchCounters), cudaMemcpyDeviceToHost, s));
        PLL_TRY(cudaMemcpyAsync(&h->d, d_desc, sizeof(LevelDesc), cudaMemcpyDeviceToHost, s));
        PLL_TRY(cudaStreamSynchronize(s));
        return PLL_OK;
    };
    // ev[0..1]: a batch's BFS part (init, levels, reset); ev[2..3]: its
    // sort, cleanup, compaction and append; sweep_ev: the level sweeps
    cudaEvent_t ev[4] = {}, sweep_ev[16] = {};
    struct EvGuard {
        cudaEvent_t *a, *sw;
        ~EvGuard() {
            for (int i = 0; i < 4; ++i) if (a[i]) cudaEventDestroy(a[i]);
            for (int i = 0; i < 16; ++i) if (sw[i]) cudaEventDestroy(sw[i]);
        }
    } ev_guard{ev, sweep_ev};
    for (auto &e : ev) PLL_TRY(cudaEventCreate(&e));
    for (auto &e : sweep_ev) PLL_TRY(cudaEventCreate(&e));
    cudaEvent_t ev0 = ev[0], ev1 = ev[1];

    // the level loop as a CUDA graph: instantiated once, launched per batch
    // after the batch's arguments are copied in
    PoolMem m_args(s);
    cudaGraph_t lgraph = nullptr;
    cudaGraphExec_t lexec = nullptr;
    struct GraphGuard {
        cudaGraph_t *g;
        cudaGraphExec_t *e;
        ~GraphGuard() {
            if (*e) cudaGraphExecDestroy(*e);
            if (*g) cudaGraphDestroy(*g);
        }
    } graph_guard{&lgraph, &lexec};
    if (graph_levels) {
        PLL_CHECK(m_args.alloc(sizeof(BatchArgs)));
        PLL_CHECK(batch_graph_build(block, grid, m_args.as<BatchArgs>(), &lgraph, &lexec));
    }

    uint64_t total = 0, pre = 0, batches = 0;
    // A batch's sort, cleanup, compaction and append are not waited for: the
    // next batch is enqueued right behind them, and its first read-back
    // brings the kept count and the appends' error word (neither is touched
    // by a batch's BFS) along with its own counters.
    bool post_pending = false;
    auto settle_post = [&]() -> int {
        if (!post_pending) return PLL_OK;
        post_pending = false;
        if (h->c.err_post & ERR_POOL) return PLL_E_NOMEM;
        total += h->c.nkept;
        float ms = 0;
        PLL_TRY(cudaEventElapsedTime(&ms, ev[2], ev[3]));
        ix->stats.ms_post += ms;
        return PLL_OK;
    };
    uint32_t k0 = 0, B = std::min<uint32_t>(64, bmax);
    uint64_t last_cand = 0, last_out = 0, last_B = 1;
    unsigned long long work0[4] = {0, 0, 0, 0};
    while (k0 < n) {
        const uint32_t k1 = (uint32_t)std::min<uint64_t>(n, (uint64_t)k0 + B);
        // grow the buffers ahead of demand (the last batch scaled to this size;
        // not under the test capacities, which exist to make batches overflow)
        if (!caps.cand && !caps.out) {
            const double f = 1.5 * (double)(k1 - k0) / (double)last_B;
            if ((double)last_cand * f > (double)cand_cap) {
                cand_cap = (uint64_t)((double)last_cand * f);
                PLL_CHECK(m_cand.alloc(cand_cap * 8));
                PLL_CHECK(m_candc.alloc(cand_cap * 16));
            }
            if ((double)last_out * f > (double)out_cap) {
                out_cap = (uint64_t)((double)last_out * f);
                PLL_CHECK(alloc_out());
            }
        }
        BatchArgs a{};
        a.n = n; a.t = ix->t; a.tp = ix->tp;
        a.roff = roff; a.rcol = rcol;
        a.bp_d = ix->d_bp_d; a.bp_c = m_bpc.as<uint8_t>(); a.bp_m = ix->d_bp_m; a.inX = inX;
        a.lab_off = st.off; a.lab_len = st.len; a.pool = st.pool;
        a.k0 = k0; a.B = k1 - k0; a.NW = NW;
        a.visited = m_vis.as<uint32_t>();
        a.ht = m_ht.as<uint32_t>();
        a.ht_off = m_htoff.as<unsigned long long>();
        a.ht_cap = ht_cap;
        a.rootbits = m_bits.as<uint64_t>();
        a.filt = m_filt.as<uint32_t>();
        a.cand = m_cand.as<uint64_t>(); a.candc = m_candc.as<uint64_t>(); a.cand_cap = cand_cap;
        a.out = m_out.as<uint64_t>(); a.out_cap = out_cap;
        a.ctr = d_ctr; a.desc = d_desc; a.loop = d_loop;
        PLL_TRY(cudaEventRecord(ev0, s));
        PLL_TRY(cudaMemsetAsync(d_ctr, 0, 16, s));  // cand_n, out_n
        PLL_TRY(cudaMemsetAsync(&d_ctr->err, 0, 4, s));
        PLL_CHECK(batch_init(a, m_itemp.p, itemp_bytes, s));
        ix->stats.launches += 3;
        ix->stats.cub_calls += 1;
        if (device_levels) {
            // every level of the batch in one launch; events around it
            PLL_TRY(cudaMemsetAsync(&d_loop->count, 0, 4, s));
            PLL_TRY(cudaEventRecord(sweep_ev[0], s));
            PLL_CHECK(batch_levels(a, block, lgrid, s));
            PLL_TRY(cudaEventRecord(sweep_ev[1], s));
            ix->stats.launches += 1;
            ix->stats.levels_launches += 1;
        } else if (graph_levels) {
            // every level of the batch in one graph launch (a while node)
            h->args = a;
            PLL_TRY(cudaMemcpyAsync(m_args.p, &h->args, sizeof(BatchArgs), cudaMemcpyHostToDevice, s));
            PLL_TRY(cudaEventRecord(sweep_ev[0], s));
            PLL_TRY(cudaGraphLaunch(lexec, s));
            PLL_TRY(cudaEventRecord(sweep_ev[1], s));
            ix->stats.levels_launches += 1;
        }
        // or: enqueue levels ahead; read back only to find the empty frontier.
        // Events around every expand and test sweep give their device times.
        uint32_t ahead = 4;
        for (; !device_levels && !graph_levels;) {
            for (uint32_t l = 0; l < ahead; ++l)
                PLL_CHECK(batch_level(a, grid, block, s, sweep_ev + 4 * l));
            ix->stats.launches += 4ull * ahead;
            PLL_CHECK(read_back());
            for (uint32_t l = 0; l < ahead; ++l) {
                float me = 0, mt = 0;
                PLL_TRY(cudaEventElapsedTime(&me, sweep_ev[4 * l], sweep_ev[4 * l + 1]));
                PLL_TRY(cudaEventElapsedTime(&mt, sweep_ev[4 * l + 2], sweep_ev[4 * l + 3]));
                ix->stats.ms_expand += me;
                ix->stats.ms_test += mt;
            }
            ix->stats.expand_launches += ahead;
            ix->stats.test_launches += ahead;
            if ((h->c.err & (ERR_DEPTH | ERR_BUF)) || h->d.lvl_b == h->d.lvl_e) break;
            ahead = 2;
        }
        // lazy reset of the visited rows (the kernel reads the error word: an
        // overflowed batch, which did not record all of its candidates, has
        // its rows cleared whole before the redo)
        PLL_CHECK(batch_clear(a, grid[0], s));
        ix->stats.launches += 1;
        PLL_TRY(cudaEventRecord(ev1, s));
        PLL_CHECK(read_back());
        PLL_CHECK(settle_post());
        {
            float ms = 0;
            PLL_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
            ix->stats.ms_pruned_kernel += ms;
            ix->stats.pruned_launches += 1;
            if (device_levels || graph_levels) {
                PLL_TRY(cudaEventElapsedTime(&ms, sweep_ev[0], sweep_ev[1]));
                ix->stats.ms_levels += ms;
            }
        }
        if (h->c.err & ERR_TIMEOUT) return PLL_E_TIMEOUT;
        if (h->c.err & ERR_DEPTH) return PLL_E_RANGE;
        if (h->c.err & ERR_TABLE) {  // some root tables did not fit: those roots were
            // binary-searched (same answers); grow the pool for later batches
            unsigned long long need = 0;
            PLL_TRY(cudaMemcpyAsync(&need, m_htoff.as<unsigned long long>() + a.B, 8,
                                    cudaMemcpyDeviceToHost, s));
            PLL_TRY(cudaStreamSynchronize(s));
            ix->stats.table_fallbacks += 1;
            if (!caps.ht) {  // the test capacity keeps the pool small for the whole build
                ht_cap = std::max<uint64_t>(need + need / 4, ht_cap * 2);
                PLL_CHECK(m_ht.alloc(ht_cap * 4));
            }
            h->c.err &= ~ERR_TABLE;
        }
        if (h->c.err & ERR_BUF) {  // a buffer overflowed: grow and redo the batch
            ix->stats.redone_batches += 1;
            PLL_TRY(cudaMemcpyAsync(d_ctr->work, work0, sizeof(work0), cudaMemcpyHostToDevice, s));
            if (h->c.cand_n > cand_cap) {
                cand_cap = std::max<uint64_t>(cand_cap * 2, h->c.cand_n + h->c.cand_n / 4);
                PLL_CHECK(m_cand.alloc(cand_cap * 8));
                PLL_CHECK(m_candc.alloc(cand_cap * 16));
            }
            if (h->c.out_n > out_cap) {
                out_cap = std::max<uint64_t>(out_cap * 2, h->c.out_n + h->c.out_n / 4);
                PLL_CHECK(alloc_out());
            }
            continue;
        }
        ix->stats.candidates += h->c.cand_n;
        last_cand = h->c.cand_n;
        last_out = h->c.out_n;
        last_B = k1 - k0;
        const uint64_t P = h->c.out_n;
        pre += P;
        if (P > 0) {
            // worst-case pool growth of one append: 2 x (entries + new) + 8 per run
            const uint64_t need = h->c.pool_top + 2 * (total + P) + 12 * P;
            if (need > st.pool_cap) {
                uint64_t nc = std::max<uint64_t>(st.pool_cap * 2, 3 * (total + P) + 12 * P);
                PLL_CHECK(labels_regrow(st, nc, s));
                ix->stats.pool_regrows += 1;
                ix->stats.launches += 3;
                ix->stats.cub_calls += 1;
            }
            PLL_TRY(cudaEventRecord(ev[2], s));
            size_t tb = temp_bytes;
            PLL_CHECK(labels_sort_tuples(m_out.as<uint64_t>(), m_sorted.as<uint64_t>(), P, SORT_BEGIN_BIT, end_bit,
                                         m_temp.p, &tb, s));
            // the sort is done with the temporary space; the cleanup borrows it
            PLL_CHECK(labels_cleanup(m_sorted.as<uint64_t>(), P, m_keep.as<uint8_t>(), k0, k1 - k0,
                                     m_temp.p, temp_bytes, s));
            tb = temp_bytes;
            PLL_CHECK(labels_compact(m_sorted.as<uint64_t>(), m_keep.as<uint8_t>(), P,
                                     m_out.as<uint64_t>(), &d_ctr->nkept, m_temp.p, &tb, s));
            PLL_CHECK(labels_append(st, m_out.as<uint64_t>(), &d_ctr->nkept, P, &d_ctr->err_post, s));
            ix->stats.launches += 2;   // cleanup, append
            ix->stats.cub_calls += 2;  // sort, select
            PLL_TRY(cudaEventRecord(ev[3], s));
            post_pending = true;
        }
        for (int w = 0; w < 4; ++w) work0[w] = h->c.work[w];  // the sweeps' counts so far
        ++batches;
        k0 = k1;
        B = std::min<uint32_t>(B * 2, bmax);
    }
    if (post_pending) {
        PLL_CHECK(read_back());
        PLL_CHECK(settle_post());
    }
    if (device_levels || graph_levels) {  // phase times and level counts of the device-side loop
        LoopState ls{};
        PLL_TRY(cudaMemcpyAsync(&ls, d_loop, sizeof(ls), cudaMemcpyDeviceToHost, s));
        PLL_TRY(cudaStreamSynchronize(s));
        ix->stats.ms_expand = ls.ns_expand * 1e-6;
        ix->stats.ms_test = ls.ns_test * 1e-6;
        ix->stats.expand_launches = ls.levels;
        ix->stats.test_launches = ls.levels;
        // the graph's body runs four kernels a level (expand, step, test, step)
        if (graph_levels) ix->stats.launches += 4ull * ls.levels;
    }
    ix->stats.pruned_scanned = h->c.work[0];
    ix->stats.pruned_masks = h->c.work[1];
    ix->stats.pruned_expanded = h->c.work[2];
    ix->stats.label_entries = total;
    ix->stats.pre_cleanup = pre;
    ix->stats.visited = h->c.work[3];
    ix->stats.batches = batches;
    ix->entries = total;

    // step 4: compact CSR
    PLL_TRY(dev_malloc(&ix->d_lab_off, ((size_t)n + 1) * 8));
    PLL_TRY(dev_malloc(&ix->d_lab, std::max<uint64_t>(total, 1) * 4));
    size_t ftb = 0;
    PLL_CHECK(labels_finalize(st, total, ix->d_lab_off, ix->d_lab, nullptr, &ftb, s));
    PoolMem ftemp(s);
    PLL_CHECK(ftemp.alloc(ftb));
    Timer tf(s);
    tf.start();
    PLL_CHECK(labels_finalize(st, total, ix->d_lab_off, ix->d_lab, ftemp.p, &ftb, s));
    ix->stats.ms_finalize = tf.stop_ms();
    ix->stats.launches += 3;   // widen, set, gather
    ix->stats.cub_calls += 1;  // scan
    return PLL_OK;
}

// graph_start: null for one graph; else host uint32[graphs + 1] vertex ranges
// of graphs built together as one disjoint union.
int build_device(const uint32_t *off, const uint32_t *col, uint32_t n, uint64_t nnz,
                 const uint32_t *order, const uint32_t *graph_start, uint32_t graphs,
                 const pll_build_opts *opts, cudaStream_t s, pll_index **out) {
    pll_build_opts o{};
    if (opts) o = *opts;
    if (!out) return PLL_E_INVAL;
    *out = nullptr;
    if (o.reserved != 0 ||
        (o.flags & ~(PLL_BUILD_HOST_LEVELS | PLL_BUILD_GRAPH_LEVELS | PLL_BUILD_COOP_LEVELS)) != 0)
        return PLL_E_INVAL;
    if (o.t > PLL_MAX_T) return PLL_E_RANGE;
    if (n > MAX_N || nnz >= 0xffffffffull) return PLL_E_RANGE;
    if (n > 0 && !off) return PLL_E_INVAL;
    if (nnz > 0 && !col) return PLL_E_INVAL;
    if (n == 0 && nnz != 0) return PLL_E_INVAL;
    uint32_t block = o.block ? o.block : 256;
    if (block != 128 && block != 256 && block != 512 && block != 1024) return PLL_E_INVAL;
    // default: 16384 roots per batch (fewer, larger batches: one R-MAT-20 build
    // is ~10% faster than at 4096), halved while the batch's visited bitmap
    // (n x batch / 8 bytes) would pass 8 GiB
    uint32_t bmax = o.root_batch;
    if (!bmax) {
        bmax = 16384;
        while (bmax > 1024 && (uint64_t)n * bmax / 8 > (8ull << 30)) bmax >>= 1;
    }
    if (bmax > (1u << 16)) bmax = 1u << 16;
    const bool batch = graph_start != nullptr;
    if (!batch) graphs = 1;
    if (batch) {
        if (graphs == 0 || graphs > MAX_N || order) return PLL_E_INVAL;
        if (graph_start[0] != 0 || graph_start[graphs] != n) return PLL_E_INVAL;
        for (uint32_t gi = 0; gi < graphs; ++gi)
            if (graph_start[gi] > graph_start[gi + 1]) return PLL_E_INVAL;
    }

    pll_index *ix = new (std::nothrow) pll_index();
    if (!ix) return PLL_E_NOMEM;
    struct Guard {
        pll_index *ix;
        ~Guard() { free_index(ix); }
    } guard{ix};
    PLL_TRY(cudaGetDevice(&ix->device));
    ix->n = n;
    ix->t = o.t;
    ix->tp = bp_stride(o.t);
    ix->graphs = graphs;
    ix->nnz = nnz;
    ix->stats.n = n;
    ix->stats.t = o.t;
    ix->stats.nnz = nnz;
    Timer tm(s);
    const cudaMemPool_t spool = scratch_pool();
    if (spool) {  // the build's scratch peak, from here on
        uint64_t zero = 0;
        (void)cudaMemPoolSetAttribute(spool, cudaMemPoolAttrUsedMemHigh, &zero);
    }

    // ---- 1. checks, order, relabel
    tm.start();
    PoolMem m_err(s);
    PLL_CHECK(m_err.alloc(4));
    uint32_t *d_err = m_err.as<uint32_t>();
    uint32_t h_err = 0;
    PLL_TRY(cudaMemsetAsync(d_err, 0, 4, s));
    Graph g;
    g.n = n; g.nnz = nnz; g.off = off; g.col = col;
    PLL_CHECK(prep_validate_csr(g, d_err, s));
    PLL_CHECK(read_err(d_err, s, &h_err));
    if (h_err) return PLL_E_INVAL;
    PLL_TRY(dev_malloc(&ix->d_order, std::max<size_t>((size_t)n * 4, 4)));
    PLL_TRY(dev_malloc(&ix->d_inv, std::max<size_t>((size_t)n * 4, 4)));
    PoolMem m_gs(s), m_gof(s), m_local(s);
    if (batch) {  // each graph's own Degree order, graphs interleaved by local rank
        PLL_CHECK(m_gs.alloc(((size_t)graphs + 1) * 4));
        PLL_CHECK(m_gof.alloc(std::max<size_t>((size_t)n * 4, 4)));
        PLL_CHECK(m_local.alloc(std::max<size_t>((size_t)n * 4, 4)));
        PLL_TRY(cudaMemcpyAsync(m_gs.p, graph_start, ((size_t)graphs + 1) * 4, cudaMemcpyHostToDevice, s));
        PLL_CHECK(prep_batch_order(g, m_gs.as<uint32_t>(), graphs, m_gof.as<uint32_t>(),
                                   m_local.as<uint32_t>(), ix->d_order, d_err, s));
        PLL_CHECK(read_err(d_err, s, &h_err));
        if (h_err) return PLL_E_INVAL;  // an arc joins two graphs
    } else if (order) {
        if (n) PLL_TRY(cudaMemcpyAsync(ix->d_order, order, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        PLL_CHECK(prep_check_order(g, ix->d_order, d_err, s));
        PLL_CHECK(read_err(d_err, s, &h_err));
        if (h_err) return PLL_E_ORDER;
    } else {
        PLL_CHECK(prep_degree_order(g, ix->d_order, s));
    }
    PoolMem m_roff(s), m_rcol(s), m_inX(s);
    PLL_CHECK(m_roff.alloc(((size_t)n + 1) * 4));
    PLL_CHECK(m_rcol.alloc(std::max<uint64_t>(nnz, 1) * 4));
    PLL_CHECK(prep_relabel(g, ix->d_order, ix->d_inv, m_roff.as<uint32_t>(), m_rcol.as<uint32_t>(), s));
    PLL_CHECK(m_inX.alloc(std::max<size_t>(n, 1)));
    PLL_TRY(cudaMemsetAsync(m_inX.p, 0, std::max<size_t>(n, 1), s));
    const uint32_t t = o.t;
    const size_t gt = (size_t)graphs * t;
    PLL_TRY(dev_malloc(&ix->d_bp_root, std::max<size_t>(gt, 1) * 4));
    PLL_TRY(dev_malloc(&ix->d_bp_cnt, std::max<size_t>(gt, 1) * 4));
    PLL_TRY(dev_malloc(&ix->d_bp_S, std::max<size_t>(gt * BPW, 1) * 4));
    PLL_TRY(cudaMemsetAsync(ix->d_bp_S, 0xff, std::max<size_t>(gt * BPW, 1) * 4, s));
    if (batch) {
        PLL_TRY(dev_malloc(&ix->d_graph, std::max<size_t>((size_t)n * 4, 4)));
        PLL_CHECK(prep_graph_by_rank(n, ix->d_order, m_gof.as<uint32_t>(), ix->d_graph, s));
    }
    if (batch)
        PLL_CHECK(prep_select_bp_graphs(graphs, t, m_gs.as<uint32_t>(), m_local.as<uint32_t>(),
                                        ix->d_inv, m_roff.as<uint32_t>(), m_rcol.as<uint32_t>(),
                                        m_inX.as<uint8_t>(), ix->d_bp_root, ix->d_bp_cnt,
                                        ix->d_bp_S, s));
    else
        PLL_CHECK(prep_select_bp_roots(n, t, m_roff.as<uint32_t>(), m_rcol.as<uint32_t>(),
                                       m_inX.as<uint8_t>(), ix->d_bp_root, ix->d_bp_cnt, ix->d_bp_S, s));
    if (n) {
        ix->stats.launches += (nnz ? 2 : 1) + 2 + (nnz ? 3 : 2) + (t ? 1 : 0);
        ix->stats.cub_calls += (order ? 0 : 1) + 1 + (nnz ? 1 : 0);
    }
    ix->stats.ms_prep = tm.stop_ms();

    // ---- 2. bit-parallel labels
    tm.start();
    const size_t nt = (size_t)n * t;
    PLL_TRY(dev_malloc(&ix->d_bp_d, std::max<size_t>((size_t)n * ix->tp, 16)));
    PLL_TRY(dev_malloc(&ix->d_bp_m, std::max<size_t>(nt, 1) * 16));
    uint32_t bp_levels = 0;
    PLL_CHECK(bp_run(n, t, graphs, m_roff.as<uint32_t>(), m_rcol.as<uint32_t>(), ix->d_bp_root,
                     ix->d_bp_cnt, ix->d_bp_S, ix->d_bp_d, ix->d_bp_m, d_err, s, &bp_levels));
    if (t && n) {
        ix->stats.launches += 4 + 2ull * bp_levels;  // seed, chunk counts/fill, passes, finish
        ix->stats.cub_calls += 1;
    }
    PLL_CHECK(read_err(d_err, s, &h_err));
    if (h_err) return err_to_status(h_err);
    ix->stats.ms_bp = tm.stop_ms();

    // ---- 3 + 4. pruned labels
    tm.start();
    PLL_CHECK(pruned_stage(ix, m_roff.as<uint32_t>(), m_rcol.as<uint32_t>(), m_inX.as<uint8_t>(),
                           bmax, block, o.flags, s));
    ix->stats.ms_pruned = tm.stop_ms();
    if (spool) {
        uint64_t high = 0;
        if (cudaMemPoolGetAttribute(spool, cudaMemPoolAttrUsedMemHigh, &high) == cudaSuccess)
            ix->stats.scratch_peak_bytes = high;
        (void)cudaGetLastError();
    }

    PLL_TRY(dev_malloc(&ix->d_qerr, 16));
    PLL_TRY(cudaMemsetAsync(ix->d_qerr, 0, 16, s));
    PLL_TRY(cudaStreamSynchronize(s));
    ix->stats.index_bytes = (uint64_t)n * 8 + (uint64_t)n * ix->tp + nt * 16 + ((uint64_t)n + 1) * 8 +
                            ix->entries * 4 + gt * (BPW + 2) * 4;
    ix->stats.graphs = graphs;
    *out = ix;
    guard.ix = nullptr;
    return PLL_OK;
}

}  // namespace

// The scratch pool: every temporary of a build and the staging copies of the
// host-pointer entry points are allocated from it in stream order. The
// default pool hands freed memory back at every synchronisation, and a
// cudaMalloc / cudaFree pair maps and unmaps pages synchronously (about 3 ms
// per GiB, and a build needs a few GiB of scratch); this pool keeps up to
// an eighth of the device's memory mapped between calls (only what calls
// actually used), until pll_release_cached. One pool per CUDA context, found
// by the context's unique id (a context destroyed by a device reset takes its
// pool with it and is never asked for it again).

namespace {
std::mutex g_pool_mu;
struct PoolEntry { unsigned long long ctx_id; cudaMemPool_t pool; };
std::vector<PoolEntry> g_pools;

// unique id of the current context (false if there is none or the driver
// cannot say)
bool current_ctx_id(unsigned long long *id) {
    static PFN_cuCtxGetCurrent_v4000 get_ctx = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void **>(&get_ctx), 4000,
                                             cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void **>(&get_id), 12000,
                                             cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            get_ctx = nullptr;
            get_id = nullptr;
        }
    }
    CUcontext ctx = nullptr;
    return get_ctx && get_id && get_ctx(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, id) == CUDA_SUCCESS;
}
}  // namespace

cudaMemPool_t scratch_pool() {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    unsigned long long id = 0;
    if (!current_ctx_id(&id)) return nullptr;
    for (const PoolEntry &e : g_pools)
        if (e.ctx_id == id) return e.pool;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { (void)cudaGetLastError(); total_b = 8ull << 33; }
    uint64_t keep = total_b / 8;
    (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools.push_back({id, pool});
    return pool;
}

namespace {

// temporary device copy of a host array, stream ordered
using AsyncBuf = PoolMem;

int query_status(const pll_index *ix, cudaStream_t s) {
    // the two counters come back into pinned memory (a pageable target makes
    // the copy a staged one); one buffer per thread: pll_query is synchronous,
    // so a thread has one in flight at a time. It lives as long as the thread.
    static thread_local unsigned long long *pinned = nullptr;
    unsigned long long stack_h[2] = {0, 0};
    if (!pinned && cudaMallocHost(&pinned, 16) != cudaSuccess) {
        (void)cudaGetLastError();
        pinned = nullptr;
    }
    unsigned long long *h = pinned ? pinned : stack_h;
    PLL_TRY(cudaMemcpyAsync(h, ix->d_qerr, 16, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    if (h[0] == 0 && h[1] == 0) return PLL_OK;
    PLL_TRY(cudaMemsetAsync(ix->d_qerr, 0, 16, s));
    PLL_TRY(cudaStreamSynchronize(s));
    return h[1] ? PLL_E_INVAL : PLL_E_RANGE;
}

}  // namespace

void index_release(pll_index *ix) { free_index(ix); }

// allocation-failure test hook and live-allocation count
static std::atomic<long long> g_fail_after{-1};
static std::atomic<long long> g_live{0};

bool alloc_should_fail() {
    long long k = g_fail_after.load(std::memory_order_relaxed);
    while (k >= 0) {
        // k allocations still pass; the one that finds k == 0 fails and ends the countdown
        if (g_fail_after.compare_exchange_weak(k, k - 1, std::memory_order_relaxed)) return k == 0;
    }
    return false;
}

void alloc_note(long long delta) { g_live.fetch_add(delta, std::memory_order_relaxed); }

// longest wait of a grid barrier of the level loop (test hook; 0 = default)
static std::atomic<uint64_t> g_barrier_ns{0};
constexpr uint64_t BARRIER_TIMEOUT_NS = 10ull * 1000 * 1000 * 1000;  // 10 s

uint64_t test_barrier_timeout_ns() {
    const uint64_t v = g_barrier_ns.load(std::memory_order_relaxed);
    return v ? v : BARRIER_TIMEOUT_NS;
}

// test capacities of the pruned stage (0 = the library's own sizing)
static std::atomic<uint64_t> g_cap_cand{0}, g_cap_out{0}, g_cap_pool{0}, g_cap_ht{0};

TestCaps test_caps() {
    TestCaps c;
    c.cand = g_cap_cand.load(std::memory_order_relaxed);
    c.out = g_cap_out.load(std::memory_order_relaxed);
    c.pool = g_cap_pool.load(std::memory_order_relaxed);
    c.ht = g_cap_ht.load(std::memory_order_relaxed);
    return c;
}

}  // namespace pll

using namespace pll;

extern "C" {

PLL_API int pll_release_cached(void) {
    using namespace pll;
    cudaError_t e = cudaDeviceSynchronize();  // frees in flight complete first
    if (e != cudaSuccess) return cuda_status(e);
    std::lock_guard<std::mutex> lock(g_pool_mu);
    unsigned long long id = 0;
    if (!current_ctx_id(&id)) return PLL_OK;
    for (const PoolEntry &pe : g_pools)
        if (pe.ctx_id == id && (e = cudaMemPoolTrimTo(pe.pool, 0)) != cudaSuccess) return cuda_status(e);
    return PLL_OK;
}

PLL_API const char *pll_status_str(int status) {
    switch (status) {
        case PLL_OK: return "ok";
        case PLL_E_INVAL: return "invalid argument or malformed graph";
        case PLL_E_ORDER: return "order is not a permutation of 0..n-1";
        case PLL_E_RANGE: return "size or distance out of range";
        case PLL_E_NOMEM: return "out of memory";
        case PLL_E_TIMEOUT: return "bounded device wait expired";
        case PLL_E_CUDA: return "CUDA runtime error";
        default: return "unknown status";
    }
}

PLL_API int pll_build(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                      const uint32_t *order, const pll_build_opts *opts, void *stream,
                      pll_index **out) {
    return build_device(offsets, cols, n, nnz, order, nullptr, 1, opts, (cudaStream_t)stream, out);
}

PLL_API int pll_build_host(const uint32_t *offsets, const uint32_t *cols, uint32_t n,
                           uint64_t nnz, const uint32_t *order, const pll_build_opts *opts,
                           void *stream, pll_index **out) {
    if (!out) return PLL_E_INVAL;
    *out = nullptr;
    if (n > MAX_N || nnz >= 0xffffffffull) return PLL_E_RANGE;
    if ((n > 0 && !offsets) || (nnz > 0 && !cols)) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int st = PLL_OK;
    {
        AsyncBuf doff(s), dcol(s), dord(s);
        PLL_CHECK(doff.alloc(((size_t)n + 1) * 4));
        PLL_CHECK(dcol.alloc(std::max<uint64_t>(nnz, 1) * 4));
        if (offsets)
            PLL_TRY(cudaMemcpyAsync(doff.p, offsets, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, s));
        else
            PLL_TRY(cudaMemsetAsync(doff.p, 0, 4, s));
        if (nnz) PLL_TRY(cudaMemcpyAsync(dcol.p, cols, nnz * 4, cudaMemcpyHostToDevice, s));
        if (order) {
            PLL_CHECK(dord.alloc(std::max<size_t>((size_t)n * 4, 4)));
            if (n) PLL_TRY(cudaMemcpyAsync(dord.p, order, (size_t)n * 4, cudaMemcpyHostToDevice, s));
        }
        st = build_device((const uint32_t *)doff.p, (const uint32_t *)dcol.p, n, nnz,
                          order ? (const uint32_t *)dord.p : nullptr, nullptr, 1, opts, s, out);
    }
    if (st == PLL_OK) PLL_TRY(cudaStreamSynchronize(s));
    return st;
}

PLL_API int pll_build_batch(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                            const uint32_t *graph_start, uint32_t graphs,
                            const pll_build_opts *opts, void *stream, pll_index **out) {
    if (!graph_start) return PLL_E_INVAL;
    return build_device(offsets, cols, n, nnz, nullptr, graph_start, graphs, opts,
                        (cudaStream_t)stream, out);
}

PLL_API int pll_autotune(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                         const uint32_t *graph_start, uint32_t graphs, uint32_t t, void *stream,
                         pll_build_opts *best, double *best_ms) {
    if (!best) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PLL_TRY(cudaEventCreate(&e0));
    PLL_TRY(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    double best_t = 1e30;
    pll_build_opts bo{};
    auto trial = [&](uint32_t rb, uint32_t block) -> int {
        pll_build_opts o{};
        o.t = t;
        o.root_batch = rb;
        o.block = block;
        pll_index *ix = nullptr;
        PLL_TRY(cudaEventRecord(e0, s));
        const int st = build_device(offsets, cols, n, nnz, nullptr, graph_start, graphs, &o, s, &ix);
        if (st != PLL_OK) return st;
        PLL_TRY(cudaEventRecord(e1, s));
        PLL_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        PLL_TRY(cudaEventElapsedTime(&ms, e0, e1));
        free_index(ix);
        if (ms < best_t) { best_t = ms; bo = o; }
        return PLL_OK;
    };
    // root-batch sizes at the default block, then block shapes at the best size
    static const uint32_t batches[] = {1024, 2048, 4096, 8192, 16384};
    for (uint32_t rb : batches) PLL_CHECK(trial(rb, 256));
    const uint32_t rb = bo.root_batch;
    static const uint32_t blocks[] = {128, 512};
    for (uint32_t bl : blocks) PLL_CHECK(trial(rb, bl));
    *best = bo;
    if (best_ms) *best_ms = best_t;
    return PLL_OK;
}

PLL_API int pll_query_async(const pll_index *idx, const uint32_t *src, const uint32_t *dst,
                            uint64_t q, uint8_t *out, void *stream) {
    if (!idx) return PLL_E_INVAL;
    if (q == 0) return PLL_OK;
    if (!src || !dst || !out) return PLL_E_INVAL;
    return query_launch(idx, src, dst, q, out, (cudaStream_t)stream);
}

PLL_API int pll_query_errors(const pll_index *idx, void *stream, uint64_t *count) {
    if (!idx || !count) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long h[2] = {0, 0};
    PLL_TRY(cudaMemcpyAsync(h, idx->d_qerr, 16, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaMemsetAsync(idx->d_qerr, 0, 16, s));
    PLL_TRY(cudaStreamSynchronize(s));
    *count = h[0] + h[1];
    return PLL_OK;
}

PLL_API int pll_query(const pll_index *idx, const uint32_t *src, const uint32_t *dst, uint64_t q,
                      uint8_t *out, void *stream) {
    if (!idx) return PLL_E_INVAL;
    if (q == 0) return PLL_OK;
    if (!src || !dst || !out) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PLL_CHECK(query_launch(idx, src, dst, q, out, s));
    return query_status(idx, s);
}

PLL_API int pll_query_host(const pll_index *idx, const uint32_t *src, const uint32_t *dst,
                           uint64_t q, uint8_t *out, void *stream) {
    if (!idx) return PLL_E_INVAL;
    if (q == 0) return PLL_OK;
    if (!src || !dst || !out) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int st;
    {
        AsyncBuf ds(s), dd(s), dout(s);
        PLL_CHECK(ds.alloc(q * 4));
        PLL_CHECK(dd.alloc(q * 4));
        PLL_CHECK(dout.alloc(q));
        PLL_TRY(cudaMemcpyAsync(ds.p, src, q * 4, cudaMemcpyHostToDevice, s));
        PLL_TRY(cudaMemcpyAsync(dd.p, dst, q * 4, cudaMemcpyHostToDevice, s));
        PLL_CHECK(query_launch(idx, (const uint32_t *)ds.p, (const uint32_t *)dd.p, q,
                               (uint8_t *)dout.p, s));
        PLL_TRY(cudaMemcpyAsync(out, dout.p, q, cudaMemcpyDeviceToHost, s));
        st = query_status(idx, s);
    }
    PLL_TRY(cudaStreamSynchronize(s));
    return st;
}

PLL_API int pll_label_entries(const pll_index *idx, uint64_t *total) {
    if (!idx || !total) return PLL_E_INVAL;
    *total = idx->entries;
    return PLL_OK;
}

PLL_API int pll_export_labels(const pll_index *idx, uint64_t *offsets, uint32_t *hubs,
                              uint8_t *dists) {
    if (!idx || !offsets || (idx->entries && (!hubs || !dists))) return PLL_E_INVAL;
    const uint32_t n = idx->n;
    std::vector<uint64_t> off((size_t)n + 1);
    std::vector<uint32_t> lab(idx->entries), inv(n);
    PLL_TRY(cudaMemcpy(off.data(), idx->d_lab_off, ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost));
    if (idx->entries)
        PLL_TRY(cudaMemcpy(lab.data(), idx->d_lab, idx->entries * 4, cudaMemcpyDeviceToHost));
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

PLL_API int pll_export_bp(const pll_index *idx, uint8_t *d, uint64_t *m1, uint64_t *m0) {
    if (!idx) return PLL_E_INVAL;
    const uint32_t n = idx->n, t = idx->t;
    if (t == 0 || n == 0) return PLL_OK;
    if (!d || !m1 || !m0) return PLL_E_INVAL;
    const size_t nt = (size_t)n * t;
    const uint32_t tp = idx->tp;
    std::vector<uint8_t> hd((size_t)n * tp);
    std::vector<uint64_t> hm(2 * nt);
    std::vector<uint32_t> inv(n);
    PLL_TRY(cudaMemcpy(hd.data(), idx->d_bp_d, (size_t)n * tp, cudaMemcpyDeviceToHost));
    PLL_TRY(cudaMemcpy(hm.data(), idx->d_bp_m, nt * 16, cudaMemcpyDeviceToHost));
    PLL_TRY(cudaMemcpy(inv.data(), idx->d_inv, (size_t)n * 4, cudaMemcpyDeviceToHost));
    for (uint32_t v = 0; v < n; ++v) {
        const size_t r = (size_t)inv[v] * t, rd = (size_t)inv[v] * tp, o = (size_t)v * t;
        for (uint32_t i = 0; i < t; ++i) {
            d[o + i] = hd[rd + i];
            m1[o + i] = hm[2 * (r + i)];
            m0[o + i] = hm[2 * (r + i) + 1];
        }
    }
    return PLL_OK;
}

PLL_API int pll_export_bp_roots(const pll_index *idx, uint32_t *roots, uint32_t *cnt, uint32_t *S) {
    if (!idx) return PLL_E_INVAL;
    const uint32_t t = idx->t, n = idx->n;
    const size_t gt = (size_t)idx->graphs * t;
    if (t == 0) return PLL_OK;
    if (!roots || !cnt || !S) return PLL_E_INVAL;
    std::vector<uint32_t> order(n);
    std::vector<uint32_t> hr(gt), hc(gt), hs(gt * BPW);
    if (n) PLL_TRY(cudaMemcpy(order.data(), idx->d_order, (size_t)n * 4, cudaMemcpyDeviceToHost));
    PLL_TRY(cudaMemcpy(hr.data(), idx->d_bp_root, gt * 4, cudaMemcpyDeviceToHost));
    PLL_TRY(cudaMemcpy(hc.data(), idx->d_bp_cnt, gt * 4, cudaMemcpyDeviceToHost));
    PLL_TRY(cudaMemcpy(hs.data(), idx->d_bp_S, gt * BPW * 4, cudaMemcpyDeviceToHost));
    for (size_t q = 0; q < gt; ++q) {
        roots[q] = hr[q] == NONE ? NONE : order[hr[q]];
        cnt[q] = hc[q];
        for (uint32_t j = 0; j < BPW; ++j) {
            const uint32_t r = hs[q * BPW + j];
            S[q * BPW + j] = (j < hc[q] && r != NONE) ? order[r] : NONE;
        }
    }
    return PLL_OK;
}

PLL_API int pll_export_order(const pll_index *idx, uint32_t *order) {
    if (!idx || (idx->n && !order)) return PLL_E_INVAL;
    if (idx->n) PLL_TRY(cudaMemcpy(order, idx->d_order, (size_t)idx->n * 4, cudaMemcpyDeviceToHost));
    return PLL_OK;
}

PLL_API int pll_get_stats(const pll_index *idx, pll_stats *out) {
    if (!idx || !out) return PLL_E_INVAL;
    *out = idx->stats;
    return PLL_OK;
}

PLL_API void pll_free(pll_index *idx) { free_index(idx); }

PLL_API void pll_test_fail_alloc(int64_t k) { g_fail_after.store(k < 0 ? -1 : k); }

PLL_API int64_t pll_test_live_allocs(void) { return g_live.load(); }

PLL_API void pll_test_barrier_timeout(uint64_t ns) { g_barrier_ns.store(ns); }

PLL_API void pll_test_capacities(uint64_t cand, uint64_t out, uint64_t pool, uint64_t tables) {
    g_cap_cand.store(cand);
    g_cap_out.store(out);
    g_cap_pool.store(pool);
    g_cap_ht.store(tables);
}

}  // extern "C"
