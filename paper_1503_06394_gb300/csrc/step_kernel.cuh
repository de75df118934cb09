// Fused Chebyshev recurrence step (the hot loop of Algorithm 1, Sec. 2.2).
//
// One launch advances all probes of a panel by one degree:
//   w_{j+1} = 2 (scale * (X w_j) - shift * w_j) - w_{j-1},
//   scale = 2/(b-a), shift = (a+b)/(b-a), i.e. 2 At w_j - w_{j-1} with
//   At = (2X - (a+b) I)/(b-a) applied on the fly (X is never rewritten),
// and reduces t_{j+1,p} = v_p^T w_{j+1} for every probe p of the panel.
//
// Layout: the recurrence vectors of a panel are a d x P row-major FP32 block
// (probe index fastest, P in {4,...,128}).  A row of X is owned by a group of
// P/4 lanes; lane l of the group holds probes 4l..4l+3 as one float4, so every
// stored entry (i, k) costs one contiguous P*4-byte gather of row k of w_j
// (128 B, one L2 line, at P = 32).  Rows are dealt to groups round-robin
// (row = group id + r * #groups) so a warp's own-row loads and stores are
// contiguous.  Sign bits of the probes are read from a packed d x nw array
// (1 bit per probe) instead of materialising v.
//
// Moments: each lane accumulates its four v * w_{j+1} products in FP32 over
// its rows (every product is an exact sign flip), converts to FP64 and the
// CTA reduces them in a fixed order to one partial per probe; a later kernel
// sums the partials over CTAs in a fixed order, so results are deterministic.
#pragma once

#include "cld_internal.cuh"

namespace cld {

__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ldcs4(const float* p) {
    return __ldcs(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }


// Row product acc = sum_k X[row, k] * x[k, p0..p0+3] over the stored entries
// [k0, k1) of one row, for the four probes of this lane.
//
// IMPL 0: each lane loads the column index and value of 4 entries at a time
//         itself, then gathers those 4 rows (4 gathers in flight per group).
// IMPL 1 (2): the LPR lanes of the group load the next 8 (4) (index, value) pairs
//         cooperatively (one coalesced access per lane), broadcast them with
//         shuffles and issue all 8 (4) row gathers back to back; the indices of the
//         following chunk are loaded before the current chunk's gathers are
//         consumed.  CSR streams are read with the evict-first policy so they
//         do not displace gathered rows of w_j from L2.
//
// The shuffles of IMPL 1/2 name only the LPR lanes of the row's group
// (gmask): groups of one warp own rows of different lengths, so their chunk
// loops (and the last grid-stride round) diverge, and a full-warp mask would be
// undefined there.
template <int MP, int GATHER, int IMPL, typename VT>
__device__ __forceinline__ float4 row_product(int64_t k0, int64_t k1, const int32_t* __restrict__ col,
                                              const VT* __restrict__ val, const float* __restrict__ x,
                                              const uint32_t* __restrict__ vbits, int lig, int p0,
                                              int wsel, int bsh, float4 mask, unsigned gmask) {
    constexpr int LPR = MP / 4;
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (IMPL == 0) {
        constexpr int U = 4;
        for (int64_t k = k0; k < k1; k += U) {
            int c[U];
            float a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = k + u < k1;
                c[u] = ok ? __ldg(col + k + u) : -1;
                a[u] = ok ? load_val(val + k + u) : 0.f;
            }
            float4 xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (c[u] >= 0) {
                    if (GATHER == 1)
                        xv[u] = signs4(__ldg(vbits + (int64_t)c[u] * NW + wsel), bsh, mask);
                    else
                        xv[u] = __ldg(reinterpret_cast<const float4*>(x + (int64_t)c[u] * MP + p0));
                } else {
                    xv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                acc.x = fmaf(a[u], xv[u].x, acc.x);
                acc.y = fmaf(a[u], xv[u].y, acc.y);
                acc.z = fmaf(a[u], xv[u].z, acc.z);
                acc.w = fmaf(a[u], xv[u].w, acc.w);
            }
        }
    } else {
        constexpr int CH = IMPL == 1 ? 8 : 4;        // entries per chunk
        constexpr int E = LPR >= CH ? 1 : CH / LPR;  // entries held per lane
        int creg[E], cnext[E];
        float vreg[E], vnext[E];
        auto load_chunk = [&](int64_t kb, int* cr, float* vr) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = e * LPR + lig;  // entry of the chunk this lane loads
                const int64_t k = kb + idx;
                const bool ok = idx < CH && k < k1;
                cr[e] = ok ? __ldcs(col + k) : 0;
                vr[e] = ok ? load_val_cs(val + k) : 0.f;
            }
        };
        load_chunk(k0, creg, vreg);
        for (int64_t k = k0; k < k1; k += CH) {
            if (k + CH < k1) load_chunk(k + CH, cnext, vnext);
            float4 xv[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int c = __shfl_sync(gmask, creg[u / LPR], u % LPR, LPR);
                if (k + u < k1) {
                    if (GATHER == 1)
                        xv[u] = signs4(__ldg(vbits + (int64_t)c * NW + wsel), bsh, mask);
                    else
                        xv[u] = __ldg(reinterpret_cast<const float4*>(x + (int64_t)c * MP + p0));
                } else {
                    xv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const float av = __shfl_sync(gmask, vreg[u / LPR], u % LPR, LPR);
                acc.x = fmaf(av, xv[u].x, acc.x);
                acc.y = fmaf(av, xv[u].y, acc.y);
                acc.z = fmaf(av, xv[u].z, acc.z);
                acc.w = fmaf(av, xv[u].w, acc.w);
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                creg[e] = cnext[e];
                vreg[e] = vnext[e];
            }
        }
    }
    return acc;
}

// GATHER: 0 float rows of args.x, 1 probe signs.  PREV: 0 none, 1 v, 2 args.wprev.
// EPI: 0 plain product, 1 recurrence + moments.  IMPL: inner loop (row_product).
// The recurrence update of one row's four probes:
//   y = scale * (X w_j) - shift * w_j        (= At w_j; hi/lo constant pairs,
//                                             large terms first)
//   PREV 0: w_1 = y;  otherwise w_{j+1} = 2 y - w_{j-1}  (pv = w_{j-1}).
template <int PREV>
__device__ __forceinline__ float4 recurrence_update(float4 acc, float4 own, float4 pv, float scale,
                                                    float scale_lo, float shift, float shift_lo) {
    float4 y;
    y.x = fmaf(scale, acc.x, -shift * own.x) + fmaf(scale_lo, acc.x, -shift_lo * own.x);
    y.y = fmaf(scale, acc.y, -shift * own.y) + fmaf(scale_lo, acc.y, -shift_lo * own.y);
    y.z = fmaf(scale, acc.z, -shift * own.z) + fmaf(scale_lo, acc.z, -shift_lo * own.z);
    y.w = fmaf(scale, acc.w, -shift * own.w) + fmaf(scale_lo, acc.w, -shift_lo * own.w);
    if (PREV == 0) return y;
    float4 r;
    r.x = fmaf(2.f, y.x, -pv.x);
    r.y = fmaf(2.f, y.y, -pv.y);
    r.z = fmaf(2.f, y.z, -pv.z);
    r.w = fmaf(2.f, y.w, -pv.w);
    return r;
}

// Resident-CTA targets per variant (256 threads): 6 (40 registers), 3, 4.
template <int IMPL>
struct StepOccupancy { static constexpr int value = IMPL == 0 ? 6 : IMPL == 1 ? 3 : 4; };

template <int MP, typename VT, int GATHER, int PREV, int EPI, int IMPL>
__global__ void __launch_bounds__(kThreads, StepOccupancy<IMPL>::value) step_kernel(const StepArgs args);

template <int MP, typename VT, int GATHER, int PREV, int EPI, int IMPL>
__global__ void __launch_bounds__(kThreads, StepOccupancy<IMPL>::value) step_kernel(const StepArgs args) {
    constexpr int LPR = MP / 4;          // lanes per row
    constexpr int GPW = 32 / LPR;        // rows per warp
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    constexpr int WPB = kThreads / 32;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int lig = lane % LPR;
    const int g_in_w = lane / LPR;
    const int64_t gid = ((int64_t)blockIdx.x * WPB + warp) * GPW + g_in_w;
    const int64_t ngroups = (int64_t)gridDim.x * WPB * GPW;
    const int64_t d = args.d;

    const int p0 = 4 * lig;
    const int wsel = p0 >> 5;
    const int bsh = p0 & 31;
    const float4 mask = make_float4(p0 < args.mreal ? 1.f : 0.f, p0 + 1 < args.mreal ? 1.f : 0.f,
                                    p0 + 2 < args.mreal ? 1.f : 0.f, p0 + 3 < args.mreal ? 1.f : 0.f);

    const int64_t* __restrict__ rowptr = args.rowptr;
    const int32_t* __restrict__ col = args.col;
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const uint32_t* __restrict__ vbits = args.vbits;

    float scale = 1.f, scale_lo = 0.f, shift = 0.f, shift_lo = 0.f;
    if (EPI == 1) {
        scale = args.prm->scale_hi;
        scale_lo = args.prm->scale_lo;
        shift = args.prm->shift_hi;
        shift_lo = args.prm->shift_lo;
    }

    float4 tacc = make_float4(0.f, 0.f, 0.f, 0.f);

    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (g_in_w * LPR));
    int64_t k0 = 0, k1 = 0;
    if (IMPL != 0 && gid < d) {
        k0 = __ldg(rowptr + gid);
        k1 = __ldg(rowptr + gid + 1);
    }
    for (int64_t row = gid; row < d; row += ngroups) {
        float4 acc;
        if (IMPL == 0) {
            k0 = __ldg(rowptr + row);
            k1 = __ldg(rowptr + row + 1);
            acc = row_product<MP, GATHER, IMPL>(k0, k1, col, val, args.x, vbits, lig, p0, wsel, bsh, mask, gmask);
        } else {
            // row pointers of this group's next row, loaded ahead
            int64_t n0 = 0, n1 = 0;
            if (row + ngroups < d) {
                n0 = __ldg(rowptr + row + ngroups);
                n1 = __ldg(rowptr + row + ngroups + 1);
            }
            acc = row_product<MP, GATHER, IMPL>(k0, k1, col, val, args.x, vbits, lig, p0, wsel, bsh, mask, gmask);
            k0 = n0;
            k1 = n1;
        }
        float4 res;
        if (EPI == 0) {
            res = acc;
        } else {
            const float4 v = signs4(__ldg(vbits + row * NW + wsel), bsh, mask);
            const float4 own = (PREV == 0) ? v : ldg4(args.own + row * MP + p0);
            const float4 pv = (PREV == 2) ? ldcs4(args.wprev + row * MP + p0) : v;
            res = recurrence_update<PREV>(acc, own, pv, scale, scale_lo, shift, shift_lo);
            tacc.x = fmaf(v.x, res.x, tacc.x);
            tacc.y = fmaf(v.y, res.y, tacc.y);
            tacc.z = fmaf(v.z, res.z, tacc.z);
            tacc.w = fmaf(v.w, res.w, tacc.w);
        }
        st4(args.out + row * MP + p0, res);
    }

    if (EPI == 1) {
        __shared__ double red[WPB][MP];
        double t0 = tacc.x, t1 = tacc.y, t2 = tacc.z, t3 = tacc.w;
#pragma unroll
        for (int off = LPR; off < 32; off <<= 1) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, off);
            t1 += __shfl_xor_sync(0xffffffffu, t1, off);
            t2 += __shfl_xor_sync(0xffffffffu, t2, off);
            t3 += __shfl_xor_sync(0xffffffffu, t3, off);
        }
        if (g_in_w == 0) {
            red[warp][p0 + 0] = t0;
            red[warp][p0 + 1] = t1;
            red[warp][p0 + 2] = t2;
            red[warp][p0 + 3] = t3;
        }
        __syncthreads();
        for (int p = threadIdx.x; p < MP; p += kThreads) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < WPB; ++w) s += red[w][p];
            args.tpart[(int64_t)blockIdx.x * MP + p] = s;
        }
    }
}

template <int MP, typename VT, int IMPL>
cudaError_t launch_step_impl(StepKind kind, int grid, cudaStream_t s, const StepArgs& a) {
    switch (kind) {
        case kStepFirst: step_kernel<MP, VT, 1, 0, 1, IMPL><<<grid, kThreads, 0, s>>>(a); break;
        case kStepSecond: step_kernel<MP, VT, 0, 1, 1, IMPL><<<grid, kThreads, 0, s>>>(a); break;
        case kStepGeneral: step_kernel<MP, VT, 0, 2, 1, IMPL><<<grid, kThreads, 0, s>>>(a); break;
        case kProdBits: step_kernel<MP, VT, 1, 0, 0, IMPL><<<grid, kThreads, 0, s>>>(a); break;
        case kProdFloat: step_kernel<MP, VT, 0, 0, 0, IMPL><<<grid, kThreads, 0, s>>>(a); break;
        case kStepFirstFromFloat: step_kernel<MP, VT, 0, 0, 1, IMPL><<<grid, kThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int MP, typename VT>
cudaError_t launch_step_mp(StepKind kind, int grid, cudaStream_t s, const StepArgs& a) {
    switch (a.impl) {
        case 0: return launch_step_impl<MP, VT, 0>(kind, grid, s, a);
        case 1: return launch_step_impl<MP, VT, 1>(kind, grid, s, a);
        case 2: return launch_step_impl<MP, VT, 2>(kind, grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <typename VT>
cudaError_t launch_step_vt(int panel, StepKind kind, int grid, cudaStream_t s, const StepArgs& a) {
    switch (panel) {
        case 4: return launch_step_mp<4, VT>(kind, grid, s, a);
        case 8: return launch_step_mp<8, VT>(kind, grid, s, a);
        case 16: return launch_step_mp<16, VT>(kind, grid, s, a);
        case 32: return launch_step_mp<32, VT>(kind, grid, s, a);
        case 64: return launch_step_mp<64, VT>(kind, grid, s, a);
        case 128: return launch_step_mp<128, VT>(kind, grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int MP, typename VT>
int ctas_per_sm_mp(int impl) {
    int n = 0;
    cudaError_t e = impl == 0
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<MP, VT, 0, 2, 1, 0>, kThreads, 0)
        : impl == 1
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<MP, VT, 0, 2, 1, 1>, kThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<MP, VT, 0, 2, 1, 2>, kThreads, 0);
    if (e != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

template <typename VT>
int ctas_per_sm_vt(int panel, int impl) {
    switch (panel) {
        case 4: return ctas_per_sm_mp<4, VT>(impl);
        case 8: return ctas_per_sm_mp<8, VT>(impl);
        case 16: return ctas_per_sm_mp<16, VT>(impl);
        case 32: return ctas_per_sm_mp<32, VT>(impl);
        case 64: return ctas_per_sm_mp<64, VT>(impl);
        case 128: return ctas_per_sm_mp<128, VT>(impl);
        default: return 1;
    }
}

}  // namespace cld
