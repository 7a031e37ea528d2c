// pll_noalloc.cu -- pll_bp_labels_noalloc: the bit-parallel labelling stage
// (root choice of Sec. 5.4, Alg. 3 for every root) without any allocation.
//
// Some callers cannot call cudaMalloc: their device memory belongs to another
// allocator (a framework's caching allocator may hold nearly all of the GPU),
// or their process forbids allocating after start-up. This entry point takes
// the caller's input and output buffers and keeps all of its own scratch in
// one file-scope __device__ array of PLL_NOALLOC_SCRATCH_BYTES, which every
// GPU that loads this library holds until the process exits.
//
// In host code the array's name is a host-side stand-in, not a device address,
// so every call, with the caller's device current, asks the runtime for the
// array's device address with cudaGetSymbolAddress. The lookup is cheap and
// nothing is cached: after a reset of the device (or a release and re-creation
// of its primary context) the module is loaded again at a new address, which a
// cached pointer would miss. With lazy module loading (the CUDA default) the
// array itself is reserved on a device by the first call there, so make that
// first call early, before the GPU is filled and before any stream capture.
// Every call shares the one array: the parts that must start at zero are
// cleared on each call, and calls whose work overlaps on the GPU (other
// streams, other threads) race on it.
#include "pll_internal.cuh"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[PLL_NOALLOC_SCRATCH_BYTES];

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// bytes of scratch a call needs: error word, X flags, then the stage's own
size_t needed_bytes(uint32_t n, uint64_t nnz) {
    return 256 + up256((size_t)n) + pll::bp_scratch_bytes(n, nnz, nullptr);
}

// device address of g_noalloc_scratch in the current context; a reservation
// that fails at a lazy module load (no memory left) is PLL_E_NOMEM
int scratch_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return pll::cuda_status(e);
    if (p == nullptr) return PLL_E_CUDA;
    *out = p;
    return PLL_OK;
}

}  // namespace

extern "C" PLL_API int pll_bp_labels_noalloc(const uint32_t *rank_offsets, const uint32_t *rank_cols,
                                             uint32_t n, uint64_t nnz, uint32_t t, uint8_t *d,
                                             uint64_t *masks, uint32_t *roots, uint32_t *cnt,
                                             uint32_t *S, void *stream) {
    using namespace pll;
    if (t == 0 || t > PLL_MAX_T) return t == 0 ? PLL_E_INVAL : PLL_E_RANGE;
    if (n == 0 || n > MAX_N || nnz >= 0xffffffffull) return n == 0 ? PLL_E_INVAL : PLL_E_RANGE;
    if (!rank_offsets || (nnz && !rank_cols) || !d || !masks || !roots || !cnt || !S) return PLL_E_INVAL;
    if (needed_bytes(n, nnz) > PLL_NOALLOC_SCRATCH_BYTES) return PLL_E_RANGE;
    cudaStream_t s = (cudaStream_t)stream;
    void *base = nullptr;
    PLL_CHECK(scratch_address(&base));
    unsigned char *p = static_cast<unsigned char *>(base);
    uint32_t *err = reinterpret_cast<uint32_t *>(p);
    uint8_t *inX = p + 256;
    void *rest = p + 256 + up256((size_t)n);
    const size_t rest_bytes = PLL_NOALLOC_SCRATCH_BYTES - 256 - up256((size_t)n);

    PLL_TRY(cudaMemsetAsync(err, 0, 4, s));
    PLL_TRY(cudaMemsetAsync(inX, 0, n, s));
    Graph g;
    g.n = n;
    g.nnz = nnz;
    g.off = rank_offsets;
    g.col = rank_cols;
    PLL_CHECK(prep_validate_csr(g, err, s));
    uint32_t h_err = 0;
    PLL_TRY(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    if (h_err) return PLL_E_INVAL;
    PLL_TRY(cudaMemsetAsync(S, 0xff, (size_t)t * BPW * 4, s));
    PLL_CHECK(prep_select_bp_roots(n, t, rank_offsets, rank_cols, inX, roots, cnt, S, s));
    PLL_CHECK(bp_run_in(n, t, rank_offsets, rank_cols, nnz, roots, cnt, S, d, masks, err, rest,
                        rest_bytes, s));
    PLL_TRY(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    if (h_err & ERR_DEPTH) return PLL_E_RANGE;
    return h_err ? PLL_E_CUDA : PLL_OK;
}
