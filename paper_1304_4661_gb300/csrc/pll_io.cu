// pll_io.cu -- the index as a file: pll_save / pll_load.
//
// The index is the artefact of the method: labels built once answer queries
// for as long as the graph stands (the paper's disk-based answering, Sec. 6,
// reads labels from a file). The file is a flat image of the device arrays:
//
//   header   magic "PLLINDEX", u32 version (1), u32 n, u32 t, u32 tp,
//            u32 graphs, u32 has_graph, u64 nnz, u64 entries   (48 bytes)
//   order    u32[n]        rank -> vertex id
//   inv      u32[n]        vertex id -> rank
//   bp_d     u8[n * tp]    bit-parallel distances, rows padded to tp
//   bp_m     u64[n * t * 2] (S^-1, S^0) per (rank, root)
//   bp_root  u32[graphs * t], bp_cnt u32[graphs * t], bp_S u32[graphs * t * 64]
//   graph    u32[n]        graph of each rank (only if has_graph)
//   lab_off  u64[n + 1]    label offsets by rank
//   lab      u32[entries]  (hub rank << 8) | distance
//
// all little-endian (the byte order of every machine the library builds for).
// pll_load checks what a query would use as an index before anything reaches
// the device: order and inv are inverse permutations of 0..n-1 and lab_off
// starts at 0, never decreases and ends at entries; a file that fails is
// PLL_E_INVAL and leaves nothing allocated.
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "pll_internal.cuh"

namespace {

constexpr char MAGIC[8] = {'P', 'L', 'L', 'I', 'N', 'D', 'E', 'X'};
constexpr uint32_t VERSION = 1;

struct Header {
    char magic[8];
    uint32_t version, n, t, tp, graphs, has_graph;
    uint64_t nnz, entries;
};
static_assert(sizeof(Header) == 48, "file header is 48 bytes");

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

// device -> file, through a bounded host buffer
int put(FILE *f, const void *d, size_t bytes) {
    if (bytes == 0) return PLL_OK;
    const size_t chunk = 64u << 20;
    std::unique_ptr<unsigned char[]> buf(new (std::nothrow) unsigned char[bytes < chunk ? bytes : chunk]);
    if (!buf) return PLL_E_NOMEM;
    for (size_t o = 0; o < bytes; o += chunk) {
        const size_t k = bytes - o < chunk ? bytes - o : chunk;
        PLL_TRY(cudaMemcpy(buf.get(), static_cast<const unsigned char *>(d) + o, k, cudaMemcpyDeviceToHost));
        if (fwrite(buf.get(), 1, k, f) != k) return PLL_E_INVAL;
    }
    return PLL_OK;
}

// file -> device (allocated here), through a bounded host buffer
template <class T>
int get(FILE *f, T **d, size_t count) {
    const size_t bytes = count * sizeof(T);
    PLL_TRY(pll::dev_malloc(d, bytes ? bytes : 16));
    const size_t chunk = 64u << 20;
    std::unique_ptr<unsigned char[]> buf(new (std::nothrow) unsigned char[bytes < chunk ? (bytes ? bytes : 1) : chunk]);
    if (!buf) return PLL_E_NOMEM;
    for (size_t o = 0; o < bytes; o += chunk) {
        const size_t k = bytes - o < chunk ? bytes - o : chunk;
        if (fread(buf.get(), 1, k, f) != k) return PLL_E_INVAL;
        PLL_TRY(cudaMemcpy(reinterpret_cast<unsigned char *>(*d) + o, buf.get(), k, cudaMemcpyHostToDevice));
    }
    return PLL_OK;
}

template <class T>
int get_host(FILE *f, std::vector<T> &v, size_t count) {
    v.resize(count);
    if (count && fread(v.data(), sizeof(T), count, f) != count) return PLL_E_INVAL;
    return PLL_OK;
}

}  // namespace

extern "C" {

PLL_API int pll_save(const pll_index *idx, const char *path) {
    if (!idx || !path) return PLL_E_INVAL;
    File file;
    file.f = fopen(path, "wb");
    if (!file.f) return PLL_E_INVAL;
    const uint64_t n = idx->n, t = idx->t, gt = (uint64_t)idx->graphs * t;
    Header h{};
    std::memcpy(h.magic, MAGIC, 8);
    h.version = VERSION;
    h.n = idx->n;
    h.t = idx->t;
    h.tp = idx->tp;
    h.graphs = idx->graphs;
    h.has_graph = idx->d_graph != nullptr;
    h.nnz = idx->nnz;
    h.entries = idx->entries;
    if (fwrite(&h, sizeof h, 1, file.f) != 1) return PLL_E_INVAL;
    PLL_CHECK(put(file.f, idx->d_order, n * 4));
    PLL_CHECK(put(file.f, idx->d_inv, n * 4));
    PLL_CHECK(put(file.f, idx->d_bp_d, n * idx->tp));
    PLL_CHECK(put(file.f, idx->d_bp_m, n * t * 16));
    PLL_CHECK(put(file.f, idx->d_bp_root, gt * 4));
    PLL_CHECK(put(file.f, idx->d_bp_cnt, gt * 4));
    PLL_CHECK(put(file.f, idx->d_bp_S, gt * pll::BPW * 4));
    if (h.has_graph) PLL_CHECK(put(file.f, idx->d_graph, n * 4));
    PLL_CHECK(put(file.f, idx->d_lab_off, (n + 1) * 8));
    PLL_CHECK(put(file.f, idx->d_lab, idx->entries * 4));
    if (fflush(file.f) != 0) return PLL_E_INVAL;
    return PLL_OK;
}

PLL_API int pll_load(const char *path, pll_index **out) {
    if (!path || !out) return PLL_E_INVAL;
    *out = nullptr;
    File file;
    file.f = fopen(path, "rb");
    if (!file.f) return PLL_E_INVAL;
    Header h{};
    if (fread(&h, sizeof h, 1, file.f) != 1) return PLL_E_INVAL;
    if (std::memcmp(h.magic, MAGIC, 8) != 0 || h.version != VERSION) return PLL_E_INVAL;
    if (h.n > pll::MAX_N || h.t > PLL_MAX_T || h.tp != pll::bp_stride(h.t) || h.graphs == 0 ||
        h.graphs > (h.n ? h.n : 1) || h.has_graph > 1 || h.entries > (1ull << 40))
        return PLL_E_INVAL;
    const uint64_t n = h.n, t = h.t, gt = (uint64_t)h.graphs * t;
    // what queries index with is checked on the host first
    std::vector<uint32_t> order, inv;
    PLL_CHECK(get_host(file.f, order, n));
    PLL_CHECK(get_host(file.f, inv, n));
    for (uint64_t v = 0; v < n; ++v)
        if (inv[v] >= n || order[inv[v]] != v) return PLL_E_INVAL;
    pll_index *ix = new (std::nothrow) pll_index();
    if (!ix) return PLL_E_NOMEM;
    struct Guard {
        pll_index *ix;
        ~Guard() {
            if (ix) pll::index_release(ix);
        }
    } guard{ix};
    PLL_TRY(cudaGetDevice(&ix->device));
    ix->n = h.n;
    ix->t = h.t;
    ix->tp = h.tp;
    ix->graphs = h.graphs;
    ix->nnz = h.nnz;
    ix->entries = h.entries;
    PLL_TRY(pll::dev_malloc(&ix->d_order, n ? n * 4 : 16));
    PLL_TRY(pll::dev_malloc(&ix->d_inv, n ? n * 4 : 16));
    if (n) {
        PLL_TRY(cudaMemcpy(ix->d_order, order.data(), n * 4, cudaMemcpyHostToDevice));
        PLL_TRY(cudaMemcpy(ix->d_inv, inv.data(), n * 4, cudaMemcpyHostToDevice));
    }
    PLL_CHECK(get(file.f, &ix->d_bp_d, n * h.tp));
    PLL_CHECK(get(file.f, &ix->d_bp_m, n * t * 2));
    PLL_CHECK(get(file.f, &ix->d_bp_root, gt));
    PLL_CHECK(get(file.f, &ix->d_bp_cnt, gt));
    PLL_CHECK(get(file.f, &ix->d_bp_S, gt * pll::BPW));
    if (h.has_graph) PLL_CHECK(get(file.f, &ix->d_graph, n));
    std::vector<uint64_t> off;
    PLL_CHECK(get_host(file.f, off, n + 1));
    if (off[0] != 0 || off[n] != h.entries) return PLL_E_INVAL;
    for (uint64_t v = 0; v < n; ++v)
        if (off[v + 1] < off[v]) return PLL_E_INVAL;
    PLL_TRY(pll::dev_malloc(&ix->d_lab_off, (n + 1) * 8));
    PLL_TRY(cudaMemcpy(ix->d_lab_off, off.data(), (n + 1) * 8, cudaMemcpyHostToDevice));
    PLL_CHECK(get(file.f, &ix->d_lab, h.entries));
    PLL_TRY(pll::dev_malloc(&ix->d_qerr, 16));
    PLL_TRY(cudaMemset(ix->d_qerr, 0, 16));
    ix->stats.n = h.n;
    ix->stats.t = h.t;
    ix->stats.nnz = h.nnz;
    ix->stats.graphs = h.graphs;
    ix->stats.label_entries = h.entries;
    ix->stats.index_bytes = n * 8 + n * h.tp + n * t * 16 + (n + 1) * 8 + h.entries * 4 + gt * (pll::BPW + 2) * 4;
    *out = ix;
    guard.ix = nullptr;
    return PLL_OK;
}

}  // extern "C"
