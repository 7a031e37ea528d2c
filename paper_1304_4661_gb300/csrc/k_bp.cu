// k_bp.cu -- bit-parallel BFSs (Alg. 3, Sec. 5.2) for all t roots at once.
//
// Alg. 3 walks one root's BFS with two queues and two edge lists per level:
// E0 (edges inside level L) updates S^0 of level L, then E1 (edges from level
// L to L+1) carries S^{-1} and S^0 down one level. Sec. 5.2 writes the same
// recurrence per vertex:
//   S^{-1}(v) = OR of S^{-1}(w) over neighbours w one level closer to r,
//   S^0(v)    = OR of S^0(w) over those w  OR  S^{-1}(w) over same-level w.
// Here that per-vertex form is evaluated as a pull: every vertex reads its
// neighbours' rows instead of being pushed to, so no atomics are needed, and
// all t roots advance level by level together. The state is vertex-major
// [n][t], one warp per vertex, each lane owning roots lane and lane + 32, so a
// neighbour's t distance bytes arrive in one coalesced load; a neighbour's
// 16-byte mask pair is read only for the roots where it is a parent (or a
// same-level neighbour).
//
// Per level L, two launches:
//   same-level pass (E0 of level L): S^0(u) |= S^{-1}(w) for u, w at level L;
//     S^0 is then final for level L and is stored minus S^{-1} (Sec. 5.1
//     defines S^0 as the members at difference exactly 0).
//   next-level pass (E1 of level L): every u still at distance 255 for root i
//     with some neighbour at level L joins level L+1 with the OR of those
//     neighbours' S^{-1} and S^0.
// The host loops until a next-level pass discovers nothing (from level 1 on:
// level 1 can hold only seeded members of S_r).
#include "pll_internal.cuh"

namespace pll {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__global__ void k_bp_seed(uint32_t t, const uint32_t *__restrict__ root,
                          const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ S,
                          uint8_t *bp_d, uint64_t *bp_m) {
    const uint32_t i = blockIdx.x, j = threadIdx.x;
    const uint32_t r = root[i];
    if (r == NONE) return;
    if (j == 0) bp_d[(size_t)r * t + i] = 0;
    if (j < cnt[i]) {
        uint32_t v = S[(size_t)i * BPW + j];
        bp_d[(size_t)v * t + i] = 1;
        bp_m[2 * ((size_t)v * t + i)] = 1ull << j;  // S^{-1}(v) = {v}
    }
}

// Loads neighbour ids 32 at a time and hands them to the whole warp.
template <class F>
__device__ __forceinline__ void for_each_neighbour(const uint32_t *__restrict__ rcol, uint32_t b,
                                                   uint32_t e, int lane, F &&f) {
    for (uint32_t x = b; x < e; x += 32) {
        uint32_t mine = (x + lane < e) ? rcol[x + lane] : 0;
        uint32_t cnt = (e - x) < 32 ? (e - x) : 32;
        for (uint32_t j = 0; j < cnt; ++j) f(__shfl_sync(FULL, mine, j));
    }
}

__global__ void k_bp_same_level(uint32_t n, uint32_t t, uint32_t L,
                                const uint32_t *__restrict__ roff, const uint32_t *__restrict__ rcol,
                                const uint8_t *__restrict__ bp_d, uint64_t *bp_m) {
    const int lane = threadIdx.x & 31;
    const uint32_t i0 = lane, i1 = lane + 32;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const size_t row = (size_t)u * t;
        const bool a0 = i0 < t && bp_d[row + i0] == L;
        const bool a1 = i1 < t && bp_d[row + i1] == L;
        if (!__any_sync(FULL, a0 || a1)) continue;
        uint64_t acc0 = 0, acc1 = 0;
        for_each_neighbour(rcol, roff[u], roff[u + 1], lane, [&](uint32_t w) {
            const size_t wr = (size_t)w * t;
            if (a0 && bp_d[wr + i0] == L) acc0 |= bp_m[2 * (wr + i0)];
            if (a1 && bp_d[wr + i1] == L) acc1 |= bp_m[2 * (wr + i1)];
        });
        if (a0) {
            uint64_t m1 = bp_m[2 * (row + i0)];
            bp_m[2 * (row + i0) + 1] = (bp_m[2 * (row + i0) + 1] | acc0) & ~m1;
        }
        if (a1) {
            uint64_t m1 = bp_m[2 * (row + i1)];
            bp_m[2 * (row + i1) + 1] = (bp_m[2 * (row + i1) + 1] | acc1) & ~m1;
        }
    }
}

__global__ void k_bp_next_level(uint32_t n, uint32_t t, uint32_t L,
                                const uint32_t *__restrict__ roff, const uint32_t *__restrict__ rcol,
                                uint8_t *bp_d, uint64_t *bp_m, uint32_t *changed, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    const uint32_t i0 = lane, i1 = lane + 32;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    bool any = false;
    for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const size_t row = (size_t)u * t;
        const bool a0 = i0 < t && bp_d[row + i0] == INF8;
        const bool a1 = i1 < t && bp_d[row + i1] == INF8;
        if (!__any_sync(FULL, a0 || a1)) continue;
        bool f0 = false, f1 = false;
        uint64_t m10 = 0, m00 = 0, m11 = 0, m01 = 0;
        for_each_neighbour(rcol, roff[u], roff[u + 1], lane, [&](uint32_t w) {
            const size_t wr = (size_t)w * t;
            if (a0 && bp_d[wr + i0] == L) {
                f0 = true;
                m10 |= bp_m[2 * (wr + i0)];
                m00 |= bp_m[2 * (wr + i0) + 1];
            }
            if (a1 && bp_d[wr + i1] == L) {
                f1 = true;
                m11 |= bp_m[2 * (wr + i1)];
                m01 |= bp_m[2 * (wr + i1) + 1];
            }
        });
        if (f0 || f1) {
            if (L + 1 >= INF8) {
                atomicOr(err, ERR_DEPTH);
                continue;
            }
            any = true;
        }
        if (f0) {
            bp_d[row + i0] = (uint8_t)(L + 1);
            bp_m[2 * (row + i0)] = m10;
            bp_m[2 * (row + i0) + 1] = m00;
        }
        if (f1) {
            bp_d[row + i1] = (uint8_t)(L + 1);
            bp_m[2 * (row + i1)] = m11;
            bp_m[2 * (row + i1) + 1] = m01;
        }
    }
    if (__any_sync(FULL, any) && lane == 0) atomicOr(changed, 1u);
}

}  // namespace

int bp_run(uint32_t n, uint32_t t, const uint32_t *d_roff, const uint32_t *d_rcol,
           const uint32_t *d_root, const uint32_t *d_cnt, const uint32_t *d_S, uint8_t *d_bp_d,
           uint64_t *d_bp_m, uint32_t *d_err, cudaStream_t s) {
    if (t == 0 || n == 0) return PLL_OK;
    if (t > PLL_MAX_T) return PLL_E_RANGE;
    const size_t nt = (size_t)n * t;
    PLL_TRY(cudaMemsetAsync(d_bp_d, 0xff, nt, s));
    PLL_TRY(cudaMemsetAsync(d_bp_m, 0, nt * 16, s));
    k_bp_seed<<<t, BPW, 0, s>>>(t, d_root, d_cnt, d_S, d_bp_d, d_bp_m);
    PLL_TRY(cudaGetLastError());
    DevMem flag;
    PLL_CHECK(flag.alloc(4));
    uint32_t *h_flag = nullptr;
    PLL_TRY(cudaMallocHost(&h_flag, 4));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = ((uint64_t)n * 32 + 255) / 256;
    int grid = (int)(want < (uint64_t)sms * 16 ? (want ? want : 1) : (uint64_t)sms * 16);
    int st = PLL_OK;
    for (uint32_t L = 0; L < INF8; ++L) {
        cudaError_t e = cudaMemsetAsync(flag.p, 0, 4, s);
        if (e == cudaSuccess) {
            k_bp_same_level<<<grid, 256, 0, s>>>(n, t, L, d_roff, d_rcol, d_bp_d, d_bp_m);
            k_bp_next_level<<<grid, 256, 0, s>>>(n, t, L, d_roff, d_rcol, d_bp_d, d_bp_m,
                                                 flag.as<uint32_t>(), d_err);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_flag, flag.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = cuda_status(e); break; }
        // level 1 may consist of the seeded members of S_r alone (nothing is
        // "discovered" from the root then), so it is always processed
        if (*h_flag == 0 && L >= 1) break;
    }
    cudaFreeHost(h_flag);
    return st;
}

}  // namespace pll
