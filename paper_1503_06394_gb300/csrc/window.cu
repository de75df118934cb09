// The gather-window plan of inner-loop variant 7 (step_window.cuh): for each
// tile of T consecutive rows, the index ranges its window copies and each
// stored entry's row in that window.  No paper counterpart: a data-layout
// step of this implementation, run once per matrix and panel width.
#include "cld_internal.cuh"
#include "step_window.cuh"

namespace cld {

namespace {

constexpr int kPlanThreads = 128;
constexpr int kSpanWords = kWinSpan / 32;

__device__ __forceinline__ int64_t block_min_max(int64_t v, bool want_max, int64_t* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const int64_t o = __shfl_xor_sync(0xffffffffu, v, off);
        v = want_max ? (o > v ? o : v) : (o < v ? o : v);
    }
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    int64_t r = scratch[0];
    for (int w = 1; w < kPlanThreads / 32; ++w) r = want_max ? (scratch[w] > r ? scratch[w] : r) : (scratch[w] < r ? scratch[w] : r);
    __syncthreads();
    return r;
}

}  // namespace

__global__ void __launch_bounds__(kPlanThreads) window_plan_kernel(const int64_t* __restrict__ rowptr,
                                                                  const int32_t* __restrict__ col, int64_t d, int T,
                                                                  int capx, int32_t* __restrict__ tab,
                                                                  int32_t* __restrict__ lcol) {
    __shared__ uint32_t bits[kSpanWords];
    __shared__ int64_t scratch[kPlanThreads / 32];
    __shared__ int nstart, nend, reject;
    __shared__ int64_t starts[kWinRanges], ends[kWinRanges];
    __shared__ int64_t rs[kWinRanges], roff[kWinRanges], rlen[kWinRanges];
    __shared__ int nr_final;

    const int64_t ntiles = (d + T - 1) / T;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = t * T;
        const int rows = (int)(d - r0 < T ? d - r0 : T);
        const int64_t k0 = rowptr[r0], k1 = rowptr[r0 + rows];
        // span of the columns and the own rows
        int64_t lo = r0, hi = r0 + rows - 1;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            const int64_t c = col[k];
            lo = c < lo ? c : lo;
            hi = c > hi ? c : hi;
        }
        lo = block_min_max(lo, false, scratch);
        hi = block_min_max(hi, true, scratch);
        int32_t* tt = tab + t * kWinTabInts;
        if (hi - lo + 1 > kWinSpan) {
            if (threadIdx.x == 0) tt[0] = 0;
            continue;  // uniform across the CTA
        }
        const int nwords = (int)((hi - lo) / 32) + 1;
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) bits[w] = 0u;
        if (threadIdx.x == 0) {
            nstart = 0;
            nend = 0;
            reject = 0;
        }
        __syncthreads();
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            const int p = (int)(col[k] - lo);
            atomicOr(&bits[p >> 5], 1u << (p & 31));
        }
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
            const int p = (int)(r0 + r - lo);
            atomicOr(&bits[p >> 5], 1u << (p & 31));
        }
        __syncthreads();
        // starts and ends (kWinGap < 32: neighbours reach one word either side)
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
            const uint32_t cur = bits[w];
            if (cur == 0u) continue;
            const uint64_t below = ((uint64_t)cur << 32) | (w > 0 ? bits[w - 1] : 0u);
            const uint64_t above = ((uint64_t)(w + 1 < nwords ? bits[w + 1] : 0u) << 32) | cur;
            constexpr uint64_t kNear = (1ull << (kWinGap + 1)) - 1ull;  // kWinGap + 1 rows
            for (int j = 0; j < 32; ++j) {
                if (!((cur >> j) & 1u)) continue;
                // rows p - kWinGap - 1 .. p - 1 sit at bits 31 + j - kWinGap .. 31 + j of `below`
                const bool is_start = ((below >> (32 + j - kWinGap - 1)) & kNear) == 0ull;
                // rows p + 1 .. p + kWinGap + 1 sit at bits j + 1 .. j + kWinGap + 1 of `above`
                const bool is_end = ((above >> (j + 1)) & kNear) == 0ull;
                const int64_t p = lo + (int64_t)w * 32 + j;
                if (is_start) {
                    const int i = atomicAdd(&nstart, 1);
                    if (i < kWinRanges) starts[i] = p;
                }
                if (is_end) {
                    const int i = atomicAdd(&nend, 1);
                    if (i < kWinRanges) ends[i] = p;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int nr = nstart;
            if (nr > kWinRanges || nr != nend || nr == 0) {
                reject = 1;
            } else {
                // the k-th start pairs with the k-th end in increasing order
                for (int a = 1; a < nr; ++a)
                    for (int b = a; b > 0 && starts[b] < starts[b - 1]; --b) {
                        const int64_t x = starts[b]; starts[b] = starts[b - 1]; starts[b - 1] = x;
                    }
                for (int a = 1; a < nr; ++a)
                    for (int b = a; b > 0 && ends[b] < ends[b - 1]; --b) {
                        const int64_t x = ends[b]; ends[b] = ends[b - 1]; ends[b - 1] = x;
                    }
                int64_t total = 0, own = -1;
                for (int k = 0; k < nr; ++k) {
                    rs[k] = starts[k];
                    rlen[k] = ends[k] - starts[k] + 1;
                    roff[k] = total;
                    if (r0 >= starts[k] && r0 <= ends[k]) own = total + (r0 - starts[k]);
                    total += rlen[k];
                }
                if (total > capx || own < 0) reject = 1;
                if (!reject) {
                    tt[0] = nr;
                    tt[1] = (int32_t)own;
                    for (int k = 0; k < kWinRanges; ++k) {
                        tt[2 + k] = k < nr ? (int32_t)rs[k] : 0;
                        tt[2 + kWinRanges + k] = k < nr ? (int32_t)rlen[k] : 0;
                    }
                }
                nr_final = nr;
            }
            if (reject) tt[0] = 0;
        }
        __syncthreads();
        if (!reject) {
            const int nr = nr_final;
            for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
                const int64_t c = col[k];
                int32_t w = 0;
                for (int q = 0; q < nr; ++q)
                    if (c >= rs[q] && c < rs[q] + rlen[q]) w = (int32_t)(roff[q] + (c - rs[q]));
                lcol[k] = w;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_window_plan(int panel, const int64_t* rowptr, const int32_t* col, int64_t d, int capx,
                               int32_t* tab, int32_t* lcol, int sms, cudaStream_t s) {
    const int T = 2048 / panel;
    const int64_t ntiles = (d + T - 1) / T;
    const int64_t full = (int64_t)sms * 8;
    const int grid = (int)(ntiles < full ? (ntiles > 0 ? ntiles : 1) : full);
    window_plan_kernel<<<grid, kPlanThreads, 0, s>>>(rowptr, col, d, T, capx, tab, lcol);
    return cudaGetLastError();
}

template <typename VT>
static int capx_vt(int panel) {
    switch (panel) {
        case 16: return window_ok<16, VT>() ? WindowLayout<16, VT, 2, WindowShape>::capx : 0;
        case 32: return window_ok<32, VT>() ? WindowLayout<32, VT, 2, WindowShape>::capx : 0;
        case 64: return window_ok<64, VT>() ? WindowLayout<64, VT, 2, WindowShape>::capx : 0;
        case 128: return window_ok<128, VT>() ? WindowLayout<128, VT, 2, WindowShape>::capx : 0;
        default: return 0;
    }
}

int window_capx(int panel, int dtype) {
    switch (dtype) {
        case 0: return capx_vt<float>(panel);
        case 1: return capx_vt<bf16_t>(panel);
        case 2: return capx_vt<double>(panel);
        default: return 0;
    }
}

}  // namespace cld
