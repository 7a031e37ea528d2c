// k_learned.cu -- a learned vertex order for the labelling.
//
// The labels are exact and minimal for ANY order (Thm 4.1, 4.2), but their
// size depends on it (Sec. 4.4, Table 4). Besides the paper's Degree order,
// a small network scores every vertex from local features, and vertices are
// taken by descending score:
//
//   features   per vertex: log(1 + deg), log(1 + sum of neighbour degrees),
//              log(1 + core number), and five statistics of the bit-parallel
//              labels of the Degree order (Alg. 3, Sec. 5.4): mean and min of
//              min(d(r_i, v), 32), the share of roots within distance 2, and
//              the mean sizes of S^-1 and S^0 over 64; every column then
//              standardised over the graph's vertices.
//   network    8 -> 64 -> 64 -> 1 with ReLU, parameters held as bfloat16 for
//              the forward and backward passes (float32 master copy, Adam),
//              all arithmetic in float32 (a dense but tiny contraction: 4.7k
//              multiply-adds per vertex; CUDA cores, weights staged in shared
//              memory).
//   target     log(1 + number of label entries whose hub is v) from builds in
//              the Degree order; vertices that get no pruned BFS are left out.
//   order      descending score, ties by ascending vertex id (one radix sort
//              of 64-bit keys).
#include <cub/cub.cuh>
#include <cuda_bf16.h>

#include <cmath>
#include <new>

#include "pll_internal.cuh"

namespace pll {
namespace {

constexpr int NF = 8, HID = 64;
constexpr int O_W1 = 0, O_B1 = 512, O_W2 = 576, O_B2 = 4672, O_W3 = 4736, O_B3 = 4800;
constexpr int NP = 4801;
constexpr uint32_t D_CAP = 32;

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ features
// deg(v) and the walks of length two, sum over neighbours of their degree;
// one warp per vertex.
__global__ void k_deg_twohop(uint32_t n, const uint32_t *__restrict__ off,
                             const uint32_t *__restrict__ col, uint32_t *deg,
                             unsigned long long *two_hop) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint32_t b = off[v], e = off[v + 1];
        unsigned long long s = 0;
        for (uint32_t j = b + lane; j < e; j += 32) {
            const uint32_t u = col[j];
            s += off[u + 1] - off[u];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) {
            deg[v] = e - b;
            two_hop[v] = s;
        }
    }
}

struct CoreCtl {
    unsigned long long removed;  // vertices removed by the pass
    unsigned long long alive;    // vertices left after it
    uint32_t min_deg;            // least remaining degree among them
    uint32_t pad;
};

__global__ void k_core_init(uint32_t n, const uint32_t *__restrict__ deg, uint32_t *cur,
                            uint8_t *alive) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        cur[v] = deg[v];
        alive[v] = 1;
    }
}

// One peeling pass at level k: every remaining vertex with at most k
// remaining neighbours is removed with core number k and lowers its
// remaining neighbours' degrees. The vertices left at the start of level k
// form the k-core, so everything removed during level k has core number k; a
// degree lowered during the pass may hide a removal until the next pass, and
// the level ends with a pass that removes nothing.
__global__ void k_core_pass(uint32_t n, const uint32_t *__restrict__ off,
                            const uint32_t *__restrict__ col, uint32_t k, uint32_t *cur,
                            uint8_t *alive, uint32_t *core, CoreCtl *ctl) {
    const int lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n;
         base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = base + threadIdx.x;
        bool rm = false, keep = false;
        uint32_t d = 0xffffffffu;
        if (v < n && alive[v]) {
            d = *reinterpret_cast<volatile uint32_t *>(&cur[v]);  // neighbours lower it concurrently
            if (d <= k) {
                rm = true;
                alive[v] = 0;
                core[v] = k;
                for (uint32_t j = off[v]; j < off[v + 1]; ++j) {
                    const uint32_t u = col[j];
                    if (alive[u]) atomicSub(&cur[u], 1u);
                }
            } else {
                keep = true;
            }
        }
        const unsigned mr = __ballot_sync(FULL, rm), mk = __ballot_sync(FULL, keep);
        uint32_t dm = keep ? d : 0xffffffffu;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dm = min(dm, __shfl_xor_sync(FULL, dm, o));
        if (lane == 0) {
            if (mr) atomicAdd(&ctl->removed, (unsigned long long)__popc(mr));
            if (mk) {
                atomicAdd(&ctl->alive, (unsigned long long)__popc(mk));
                atomicMin(&ctl->min_deg, dm);
            }
        }
    }
}

// Raw features of vertex v (caller id), one warp per vertex; the bit-parallel
// rows are in rank space (row inv[v]), lanes own roots lane and lane + 32.
__global__ void k_features_raw(uint32_t n, uint32_t t, uint32_t tp, const uint32_t *__restrict__ inv,
                               const uint32_t *__restrict__ deg,
                               const unsigned long long *__restrict__ two_hop,
                               const uint32_t *__restrict__ core, const uint8_t *__restrict__ bp_d,
                               const uint64_t *__restrict__ bp_m, float *X) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        uint32_t sum = 0, mn = D_CAP, near = 0, p1 = 0, p0 = 0;
        if (t) {
            const size_t r = inv[v];
            for (uint32_t i = lane; i < t; i += 32) {
                const uint32_t dc = min((uint32_t)bp_d[r * tp + i], D_CAP);
                sum += dc;
                mn = min(mn, dc);
                near += dc <= 2;
                p1 += __popcll(bp_m[2 * (r * t + i)]);
                p0 += __popcll(bp_m[2 * (r * t + i) + 1]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sum += __shfl_xor_sync(FULL, sum, o);
                mn = min(mn, __shfl_xor_sync(FULL, mn, o));
                near += __shfl_xor_sync(FULL, near, o);
                p1 += __shfl_xor_sync(FULL, p1, o);
                p0 += __shfl_xor_sync(FULL, p0, o);
            }
        }
        if (lane < NF) {
            double f = 0;
            switch (lane) {
                case 0: f = log1p((double)deg[v]); break;
                case 1: f = log1p((double)two_hop[v]); break;
                case 2: f = log1p((double)core[v]); break;
                case 3: f = t ? (double)sum / t : 0; break;
                case 4: f = t ? (double)mn : 0; break;
                case 5: f = t ? (double)near / t : 0; break;
                case 6: f = t ? (double)p1 / (64.0 * t) : 0; break;
                default: f = t ? (double)p0 / (64.0 * t) : 0; break;
            }
            X[v * NF + lane] = (float)f;
        }
    }
}

// Column sums (pass 0) or sums of squared deviations from mean[] (pass 1),
// in double, one atomic per column per block.
__global__ void k_col_moments(uint32_t n, const float *__restrict__ X, const double *__restrict__ mean,
                              int pass, double *acc) {
    __shared__ double part[NF][33];
    double s[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) s[j] = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            const double x = X[v * NF + j];
            s[j] += pass == 0 ? x : (x - mean[j]) * (x - mean[j]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        double a = s[j];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
        if (lane == 0) part[j][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < NF) {
        double a = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += part[threadIdx.x][w];
        atomicAdd(&acc[threadIdx.x], a);
    }
}

__global__ void k_mean(uint32_t n, double *acc) {
    if (threadIdx.x < NF) acc[threadIdx.x] = n ? acc[threadIdx.x] / n : 0;
}

__global__ void k_standardise(uint32_t n, const double *__restrict__ mean, const double *__restrict__ ssd,
                              float *X) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (uint64_t)n * NF;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % NF);
        const double sd = sqrt(ssd[j] / n);
        X[i] = sd > 0 ? (float)(((double)X[i] - mean[j]) / sd) : 0.f;
    }
}

// ------------------------------------------------------------------ hubs
__global__ void k_hub_counts(uint64_t entries, const uint32_t *__restrict__ lab,
                             const uint32_t *__restrict__ order, uint32_t *counts) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < entries;
         e += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&counts[order[entry_hub(lab[e])]], 1u);
}

__global__ void k_log1p_counts(uint32_t n, const uint32_t *__restrict__ counts, float *target) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        target[v] = (float)log1p((double)counts[v]);
}

// ------------------------------------------------------------------ network
__device__ __forceinline__ void load_weights(const __nv_bfloat16 *__restrict__ w16, float *W) {
    for (int i = threadIdx.x; i < NP; i += blockDim.x) W[i] = __bfloat162float(w16[i]);
}

// y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, one thread per row.
__global__ void __launch_bounds__(256) k_mlp_fwd(uint64_t n, const float *__restrict__ X,
                                                 const __nv_bfloat16 *__restrict__ w16, float *y) {
    __shared__ float W[NP];
    load_weights(w16, W);
    __syncthreads();
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[NF], h1[HID];
#pragma unroll
    for (int k = 0; k < NF; ++k) x[k] = X[r * NF + k];
#pragma unroll
    for (int i = 0; i < HID; ++i) {
        float z = W[O_B1 + i];
#pragma unroll
        for (int k = 0; k < NF; ++k) z = fmaf(W[O_W1 + i * NF + k], x[k], z);
        h1[i] = fmaxf(z, 0.f);
    }
    float out = W[O_B3];
    for (int j = 0; j < HID; ++j) {
        float z = W[O_B2 + j];
#pragma unroll
        for (int i = 0; i < HID; ++i) z = fmaf(W[O_W2 + j * HID + i], h1[i], z);
        out = fmaf(W[O_W3 + j], fmaxf(z, 0.f), out);
    }
    y[r] = out;
}

constexpr int GT = 128;      // rows per block of the gradient kernel
constexpr int RS = HID + 1;  // padded row stride of the activation tiles
constexpr int XS = NF + 1;
constexpr size_t GRAD_SMEM =
    sizeof(float) * ((NP + 3) / 4 * 4 + GT * XS + 4 * GT * RS + 2 * GT);

// Gradient of the mean squared error over `batch` rows (row g of the batch
// is sample idx[g], or g without idx). Each block takes GT rows: one thread
// per row runs the forward pass and back-propagates to dZ2 and dZ1 in shared
// memory; then the block's threads share the 4801 parameter gradients, each a
// sum over the block's rows, and write them as one partial per block (summed
// in a fixed order by k_mlp_reduce, so the result is deterministic).
__global__ void __launch_bounds__(GT) k_mlp_grad(uint32_t batch, const float *__restrict__ X,
                                                 const float *__restrict__ target,
                                                 const uint32_t *__restrict__ idx,
                                                 const __nv_bfloat16 *__restrict__ w16,
                                                 float *partial, float *ploss) {
    extern __shared__ float sm[];
    float *W = sm;
    float *Xs = W + (NP + 3) / 4 * 4;
    float *H1 = Xs + GT * XS;
    float *H2 = H1 + GT * RS;
    float *DZ2 = H2 + GT * RS;
    float *DZ1 = DZ2 + GT * RS;
    float *DY = DZ1 + GT * RS;
    float *LS = DY + GT;
    load_weights(w16, W);
    __syncthreads();

    const int s = threadIdx.x;
    const uint32_t g = blockIdx.x * GT + s;
    const bool valid = g < batch;
    const uint64_t row = valid ? (idx ? idx[g] : g) : 0;
    float x[NF], h1[HID];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        x[k] = valid ? X[row * NF + k] : 0.f;
        Xs[s * XS + k] = x[k];
    }
#pragma unroll
    for (int i = 0; i < HID; ++i) {
        float z = W[O_B1 + i];
#pragma unroll
        for (int k = 0; k < NF; ++k) z = fmaf(W[O_W1 + i * NF + k], x[k], z);
        h1[i] = fmaxf(z, 0.f);
        H1[s * RS + i] = h1[i];
    }
    float y = W[O_B3];
    for (int j = 0; j < HID; ++j) {
        float z = W[O_B2 + j];
#pragma unroll
        for (int i = 0; i < HID; ++i) z = fmaf(W[O_W2 + j * HID + i], h1[i], z);
        const float h2 = fmaxf(z, 0.f);
        H2[s * RS + j] = h2;
        y = fmaf(W[O_W3 + j], h2, y);
    }
    const float res = valid ? y - target[row] : 0.f;
    const float dy = 2.f * res / (float)batch;
    DY[s] = dy;
    LS[s] = res * res;
    float dh[HID];
#pragma unroll
    for (int i = 0; i < HID; ++i) dh[i] = 0.f;
    for (int j = 0; j < HID; ++j) {
        const float dz = H2[s * RS + j] > 0.f ? dy * W[O_W3 + j] : 0.f;
        DZ2[s * RS + j] = dz;
#pragma unroll
        for (int i = 0; i < HID; ++i) dh[i] = fmaf(W[O_W2 + j * HID + i], dz, dh[i]);
    }
#pragma unroll
    for (int i = 0; i < HID; ++i) DZ1[s * RS + i] = h1[i] > 0.f ? dh[i] : 0.f;
    __syncthreads();

    float *out = partial + (size_t)blockIdx.x * NP;
    for (int o = threadIdx.x; o < NP; o += GT) {
        float acc = 0.f;
        if (o < O_B1) {
            const int i = o / NF, k = o % NF;
            for (int r = 0; r < GT; ++r) acc = fmaf(DZ1[r * RS + i], Xs[r * XS + k], acc);
        } else if (o < O_W2) {
            const int i = o - O_B1;
            for (int r = 0; r < GT; ++r) acc += DZ1[r * RS + i];
        } else if (o < O_B2) {
            const int j = (o - O_W2) / HID, i = (o - O_W2) % HID;
            for (int r = 0; r < GT; ++r) acc = fmaf(DZ2[r * RS + j], H1[r * RS + i], acc);
        } else if (o < O_W3) {
            const int j = o - O_B2;
            for (int r = 0; r < GT; ++r) acc += DZ2[r * RS + j];
        } else if (o < O_B3) {
            const int j = o - O_W3;
            for (int r = 0; r < GT; ++r) acc = fmaf(DY[r], H2[r * RS + j], acc);
        } else {
            for (int r = 0; r < GT; ++r) acc += DY[r];
        }
        out[o] = acc;
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int r = 0; r < GT; ++r) l += LS[r];
        ploss[blockIdx.x] = l;
    }
}

// grad[o] = sum over blocks of partial[b][o], in block order; grad[NP] = loss.
__global__ void k_mlp_reduce(uint32_t blocks, uint32_t batch, const float *__restrict__ partial,
                             const float *__restrict__ ploss, float *grad) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < NP) {
        float a = 0.f;
        for (uint32_t b = 0; b < blocks; ++b) a += partial[(size_t)b * NP + o];
        grad[o] = a;
    } else if (o == NP) {
        float a = 0.f;
        for (uint32_t b = 0; b < blocks; ++b) a += ploss[b];
        grad[NP] = a / (float)batch;
    }
}

// Adam (Kingma and Ba, 2015) on the float32 master parameters; c1, c2 are
// the bias corrections 1 / (1 - beta^step), and 1 - beta comes in rounded
// from double (1 - 0.999f in float32 is off by 1e-5 relative). The bf16 copy
// follows.
__global__ void k_adam(const float *__restrict__ grad, float *master, float *m, float *v,
                       __nv_bfloat16 *w16, float lr, float b1, float omb1, float b2, float omb2,
                       float eps, float c1, float c2) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= NP) return;
    const float g = grad[o];
    const float mo = b1 * m[o] + omb1 * g;
    const float vo = b2 * v[o] + omb2 * g * g;
    m[o] = mo;
    v[o] = vo;
    const float p = master[o] - lr * (mo * c1) / (sqrtf(vo * c2) + eps);
    master[o] = p;
    w16[o] = __float2bfloat16_rn(p);
}

__global__ void k_to_bf16(const float *__restrict__ p, __nv_bfloat16 *w16) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < NP) w16[o] = __float2bfloat16_rn(p[o]);
}

// ------------------------------------------------------------------ order
// Key of a score that sorts ascending as the score descends; -0 is +0, NaN
// goes last.
__global__ void k_score_keys(uint32_t n, const float *__restrict__ score, uint64_t *keys) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const float f = score[v];
        uint32_t k;
        if (f != f) {
            k = 0xffffffffu;
        } else {
            uint32_t b = __float_as_uint(f == 0.f ? 0.f : f);
            const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // ascending in f
            k = ~asc;
        }
        keys[v] = ((uint64_t)k << 32) | v;
    }
}

__global__ void k_key_ids(uint32_t n, const uint64_t *__restrict__ keys, uint32_t *order) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        order[v] = (uint32_t)keys[v];
}

int grid_for(uint64_t work, int block) {
    uint64_t g = (work + block - 1) / block;
    if (g > 152ull * 32) g = 152ull * 32;
    return (int)(g ? g : 1);
}

int read_u32(const uint32_t *d, cudaStream_t s, uint32_t *h) {
    PLL_TRY(cudaMemcpyAsync(h, d, 4, cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

}  // namespace

// Core numbers of the caller-space graph (deg already computed).
int core_numbers(const Graph &g, const uint32_t *d_deg, uint32_t *d_core, cudaStream_t s) {
    const uint32_t n = g.n;
    if (n == 0) return PLL_OK;
    DevMem m_cur, m_alive, m_ctl;
    PLL_CHECK(m_cur.alloc((size_t)n * 4));
    PLL_CHECK(m_alive.alloc(n));
    PLL_CHECK(m_ctl.alloc(sizeof(CoreCtl)));
    CoreCtl *h = nullptr;
    PLL_TRY(cudaMallocHost(&h, sizeof(CoreCtl)));
    struct HostFree {
        CoreCtl *p;
        ~HostFree() { cudaFreeHost(p); }
    } hf{h};
    k_core_init<<<grid_for(n, 256), 256, 0, s>>>(n, d_deg, m_cur.as<uint32_t>(), m_alive.as<uint8_t>());
    PLL_TRY(cudaGetLastError());
    uint32_t k = 0;
    // every pass removes a vertex or raises k past a degree, so the loop is finite
    const uint64_t max_passes = 2ull * n + 2;
    for (uint64_t pass = 0;; ++pass) {
        if (pass > max_passes) return PLL_E_CUDA;
        const CoreCtl init{0, 0, 0xffffffffu, 0};
        PLL_TRY(cudaMemcpyAsync(m_ctl.p, &init, sizeof(CoreCtl), cudaMemcpyHostToDevice, s));
        k_core_pass<<<grid_for(n, 256), 256, 0, s>>>(n, g.off, g.col, k, m_cur.as<uint32_t>(),
                                                     m_alive.as<uint8_t>(), d_core, m_ctl.as<CoreCtl>());
        PLL_TRY(cudaGetLastError());
        PLL_TRY(cudaMemcpyAsync(h, m_ctl.p, sizeof(CoreCtl), cudaMemcpyDeviceToHost, s));
        PLL_TRY(cudaStreamSynchronize(s));
        if (h->removed) continue;
        if (h->alive == 0) break;
        k = h->min_deg;
    }
    return PLL_OK;
}

}  // namespace pll

using namespace pll;

struct pll_mlp {
    int device = 0;
    uint32_t max_batch = 0, blocks = 0;
    float *master = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *w16 = nullptr;
    float *grad = nullptr;     // [NP + 1], the last one the loss
    float *partial = nullptr;  // [blocks][NP]
    float *ploss = nullptr;    // [blocks]
    uint64_t step = 0;
    void *mem = nullptr;
};

extern "C" {

PLL_API int pll_features(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                         uint32_t t, void *stream, float *feat, uint32_t *core,
                         uint64_t *two_hop) {
    cudaStream_t s = (cudaStream_t)stream;
    if (t > PLL_MAX_T) return PLL_E_RANGE;
    if (n > MAX_N || nnz >= 0xffffffffull) return PLL_E_RANGE;
    if ((n > 0 && (!offsets || !feat)) || (nnz > 0 && !cols) || (n == 0 && nnz)) return PLL_E_INVAL;
    if (n == 0) return PLL_OK;
    Graph g;
    g.n = n; g.nnz = nnz; g.off = offsets; g.col = cols;
    DevMem m_err;
    PLL_CHECK(m_err.alloc(4));
    PLL_TRY(cudaMemsetAsync(m_err.p, 0, 4, s));
    PLL_CHECK(prep_validate_csr(g, m_err.as<uint32_t>(), s));
    uint32_t h_err = 0;
    PLL_CHECK(read_u32(m_err.as<uint32_t>(), s, &h_err));
    if (h_err) return PLL_E_INVAL;

    DevMem m_deg, m_two, m_core;
    PLL_CHECK(m_deg.alloc((size_t)n * 4));
    uint64_t *d_two = two_hop;
    uint32_t *d_core = core;
    if (!d_two) { PLL_CHECK(m_two.alloc((size_t)n * 8)); d_two = m_two.as<uint64_t>(); }
    if (!d_core) { PLL_CHECK(m_core.alloc((size_t)n * 4)); d_core = m_core.as<uint32_t>(); }
    k_deg_twohop<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(
        n, offsets, cols, m_deg.as<uint32_t>(), reinterpret_cast<unsigned long long *>(d_two));
    PLL_TRY(cudaGetLastError());
    PLL_CHECK(core_numbers(g, m_deg.as<uint32_t>(), d_core, s));

    // bit-parallel labels of the Degree order (rank space)
    const uint32_t tp = bp_stride(t);
    DevMem m_order, m_inv, m_roff, m_rcol, m_inX, m_root, m_cnt, m_S, m_bpd, m_bpm;
    if (t) {
        PLL_CHECK(m_order.alloc((size_t)n * 4));
        PLL_CHECK(m_inv.alloc((size_t)n * 4));
        PLL_CHECK(prep_degree_order(g, m_order.as<uint32_t>(), s));
        PLL_CHECK(m_roff.alloc(((size_t)n + 1) * 4));
        PLL_CHECK(m_rcol.alloc(std::max<uint64_t>(nnz, 1) * 4));
        PLL_CHECK(prep_relabel(g, m_order.as<uint32_t>(), m_inv.as<uint32_t>(), m_roff.as<uint32_t>(),
                               m_rcol.as<uint32_t>(), s));
        PLL_CHECK(m_inX.alloc(n));
        PLL_TRY(cudaMemsetAsync(m_inX.p, 0, n, s));
        PLL_CHECK(m_root.alloc((size_t)t * 4));
        PLL_CHECK(m_cnt.alloc((size_t)t * 4));
        PLL_CHECK(m_S.alloc((size_t)t * BPW * 4));
        PLL_TRY(cudaMemsetAsync(m_S.p, 0xff, (size_t)t * BPW * 4, s));
        PLL_CHECK(prep_select_bp_roots(n, t, m_roff.as<uint32_t>(), m_rcol.as<uint32_t>(),
                                       m_inX.as<uint8_t>(), m_root.as<uint32_t>(), m_cnt.as<uint32_t>(),
                                       m_S.as<uint32_t>(), s));
        PLL_CHECK(m_bpd.alloc((size_t)n * tp));
        PLL_CHECK(m_bpm.alloc((size_t)n * t * 16));
        uint32_t levels = 0;
        PLL_TRY(cudaMemsetAsync(m_err.p, 0, 4, s));
        PLL_CHECK(bp_run(n, t, 1, m_roff.as<uint32_t>(), m_rcol.as<uint32_t>(), m_root.as<uint32_t>(),
                         m_cnt.as<uint32_t>(), m_S.as<uint32_t>(), m_bpd.as<uint8_t>(),
                         m_bpm.as<uint64_t>(), m_err.as<uint32_t>(), s, &levels));
        PLL_CHECK(read_u32(m_err.as<uint32_t>(), s, &h_err));
        if (h_err) return (h_err & ERR_DEPTH) ? PLL_E_RANGE : PLL_E_CUDA;
    }
    k_features_raw<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(
        n, t, tp, m_inv.as<uint32_t>(), m_deg.as<uint32_t>(),
        reinterpret_cast<const unsigned long long *>(d_two), d_core, m_bpd.as<uint8_t>(),
        m_bpm.as<uint64_t>(), feat);
    PLL_TRY(cudaGetLastError());
    DevMem m_mom;
    PLL_CHECK(m_mom.alloc(2 * NF * sizeof(double)));
    double *mean = m_mom.as<double>(), *ssd = mean + NF;
    PLL_TRY(cudaMemsetAsync(m_mom.p, 0, 2 * NF * sizeof(double), s));
    k_col_moments<<<grid_for(n, 256), 256, 0, s>>>(n, feat, mean, 0, mean);
    k_mean<<<1, 32, 0, s>>>(n, mean);
    k_col_moments<<<grid_for(n, 256), 256, 0, s>>>(n, feat, mean, 1, ssd);
    k_standardise<<<grid_for((uint64_t)n * NF, 256), 256, 0, s>>>(n, mean, ssd, feat);
    PLL_TRY(cudaGetLastError());
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

PLL_API int pll_hub_counts(const pll_index *idx, uint32_t *counts, float *log1p_counts, void *stream) {
    if (!idx || !counts) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = idx->n;
    if (n == 0) return PLL_OK;
    PLL_TRY(cudaMemsetAsync(counts, 0, (size_t)n * 4, s));
    if (idx->entries) {
        k_hub_counts<<<grid_for(idx->entries, 256), 256, 0, s>>>(idx->entries, idx->d_lab, idx->d_order,
                                                                  counts);
        PLL_TRY(cudaGetLastError());
    }
    if (log1p_counts) {
        k_log1p_counts<<<grid_for(n, 256), 256, 0, s>>>(n, counts, log1p_counts);
        PLL_TRY(cudaGetLastError());
    }
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

PLL_API int pll_order_from_scores(const float *scores, uint32_t n, uint32_t *order, void *stream) {
    if (n && (!scores || !order)) return PLL_E_INVAL;
    if (n == 0) return PLL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevMem m_keys, m_sorted, m_temp;
    PLL_CHECK(m_keys.alloc((size_t)n * 8));
    PLL_CHECK(m_sorted.alloc((size_t)n * 8));
    k_score_keys<<<grid_for(n, 256), 256, 0, s>>>(n, scores, m_keys.as<uint64_t>());
    PLL_TRY(cudaGetLastError());
    size_t tb = 0;
    PLL_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, m_keys.as<uint64_t>(), m_sorted.as<uint64_t>(),
                                           (int)n, 0, 64, s));
    PLL_CHECK(m_temp.alloc(tb));
    PLL_TRY(cub::DeviceRadixSort::SortKeys(m_temp.p, tb, m_keys.as<uint64_t>(), m_sorted.as<uint64_t>(),
                                           (int)n, 0, 64, s));
    k_key_ids<<<grid_for(n, 256), 256, 0, s>>>(n, m_sorted.as<uint64_t>(), order);
    PLL_TRY(cudaGetLastError());
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

PLL_API int pll_mlp_create(uint32_t max_batch, pll_mlp **out) {
    if (!out || max_batch == 0) return PLL_E_INVAL;
    *out = nullptr;
    pll_mlp *p = new (std::nothrow) pll_mlp();
    if (!p) return PLL_E_NOMEM;
    p->max_batch = max_batch;
    p->blocks = (max_batch + GT - 1) / GT;
    const size_t nf = 4 * (size_t)NP + (NP + 1) + (size_t)p->blocks * NP + p->blocks + 8;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->mem, nf * sizeof(float));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAD_SMEM);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (p->mem) cudaFree(p->mem);
        delete p;
        return e == cudaErrorMemoryAllocation ? PLL_E_NOMEM : cuda_status(e);
    }
    float *f = static_cast<float *>(p->mem);
    p->master = f;
    p->m = f + NP;
    p->v = f + 2 * NP;
    p->w16 = reinterpret_cast<__nv_bfloat16 *>(f + 3 * NP);  // NP bf16 fit in NP floats
    p->grad = f + 4 * NP;
    p->partial = p->grad + NP + 1;
    p->ploss = p->partial + (size_t)p->blocks * NP;
    if (cudaMemset(p->mem, 0, nf * sizeof(float)) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(p->mem);
        delete p;
        return PLL_E_CUDA;
    }
    *out = p;
    return PLL_OK;
}

PLL_API void pll_mlp_free(pll_mlp *p) {
    if (!p) return;
    if (p->mem) cudaFree(p->mem);
    delete p;
}

PLL_API int pll_mlp_set_params(pll_mlp *p, const float *host_params, void *stream) {
    if (!p || !host_params) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PLL_TRY(cudaMemcpyAsync(p->master, host_params, NP * sizeof(float), cudaMemcpyHostToDevice, s));
    PLL_TRY(cudaMemsetAsync(p->m, 0, 2 * NP * sizeof(float), s));
    k_to_bf16<<<(NP + 255) / 256, 256, 0, s>>>(p->master, p->w16);
    PLL_TRY(cudaGetLastError());
    PLL_TRY(cudaStreamSynchronize(s));
    p->step = 0;
    return PLL_OK;
}

PLL_API int pll_mlp_get_params(const pll_mlp *p, float *host_master, uint16_t *host_bf16) {
    if (!p || (!host_master && !host_bf16)) return PLL_E_INVAL;
    if (host_master) PLL_TRY(cudaMemcpy(host_master, p->master, NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (host_bf16) PLL_TRY(cudaMemcpy(host_bf16, p->w16, NP * 2, cudaMemcpyDeviceToHost));
    return PLL_OK;
}

PLL_API int pll_mlp_forward(const pll_mlp *p, const float *x, uint64_t n, float *y, void *stream) {
    if (!p || (n && (!x || !y))) return PLL_E_INVAL;
    if (n == 0) return PLL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_mlp_fwd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, p->w16, y);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

PLL_API int pll_mlp_grad(pll_mlp *p, const float *x, const float *target, const uint32_t *idx,
                         uint32_t batch, void *stream) {
    if (!p || !x || !target || batch == 0) return PLL_E_INVAL;
    if (batch > p->max_batch) return PLL_E_RANGE;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t blocks = (batch + GT - 1) / GT;
    k_mlp_grad<<<blocks, GT, GRAD_SMEM, s>>>(batch, x, target, idx, p->w16, p->partial, p->ploss);
    PLL_TRY(cudaGetLastError());
    k_mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, s>>>(blocks, batch, p->partial, p->ploss, p->grad);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

PLL_API int pll_mlp_read_grad(const pll_mlp *p, float *host_grad, float *host_loss, void *stream) {
    if (!p || (!host_grad && !host_loss)) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (host_grad) PLL_TRY(cudaMemcpyAsync(host_grad, p->grad, NP * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (host_loss) PLL_TRY(cudaMemcpyAsync(host_loss, p->grad + NP, sizeof(float), cudaMemcpyDeviceToHost, s));
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

PLL_API int pll_mlp_adam(pll_mlp *p, float lr, void *stream) {
    if (!p || !(lr > 0)) return PLL_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const double b1 = 0.9, b2 = 0.999;
    p->step++;
    const double c1 = 1.0 / (1.0 - std::pow(b1, (double)p->step));
    const double c2 = 1.0 / (1.0 - std::pow(b2, (double)p->step));
    k_adam<<<(NP + 255) / 256, 256, 0, s>>>(p->grad, p->master, p->m, p->v, p->w16, lr, (float)b1,
                                             (float)(1.0 - b1), (float)b2, (float)(1.0 - b2), 1e-8f,
                                             (float)c1, (float)c2);
    PLL_TRY(cudaGetLastError());
    return PLL_OK;
}

PLL_API int pll_mlp_train_step(pll_mlp *p, const float *x, const float *target, const uint32_t *idx,
                               uint32_t batch, float lr, void *stream) {
    PLL_CHECK(pll_mlp_grad(p, x, target, idx, batch, stream));
    return pll_mlp_adam(p, lr, stream);
}

PLL_API int pll_learned_order(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t nnz,
                              uint32_t t, const pll_mlp *p, uint32_t *order, void *stream) {
    if (!p || (n && !order)) return PLL_E_INVAL;
    if (n == 0) return PLL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevMem m_x, m_y;
    PLL_CHECK(m_x.alloc((size_t)n * NF * 4));
    PLL_CHECK(m_y.alloc((size_t)n * 4));
    PLL_CHECK(pll_features(offsets, cols, n, nnz, t, stream, m_x.as<float>(), nullptr, nullptr));
    PLL_CHECK(pll_mlp_forward(p, m_x.as<float>(), n, m_y.as<float>(), stream));
    PLL_CHECK(pll_order_from_scores(m_y.as<float>(), n, order, stream));
    PLL_TRY(cudaStreamSynchronize(s));
    return PLL_OK;
}

}  // extern "C"
