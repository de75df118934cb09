// Recurrence step with wide lanes (inner-loop variant 5).
//
// Same step as step_kernel (Algorithm 1, Sec. 2.2: w_{j+1} = 2 At w_j - w_{j-1}
// with At applied on the fly and t_{j+1,p} = v_p^T w_{j+1} reduced per CTA),
// with another mapping of probes to lanes: each lane owns 8 consecutive probes
// of a row (LPR = P / 8 lanes per row, P >= 8), so a gathered row slice is one
// 256-bit load and every per-entry cost (index and value loads, address,
// predicate) is paid once per 8 probes instead of once per 4.  Each lane keeps
// the gathers of 4 stored entries in flight.  Every row's sum is formed in
// entry order and the update uses the same operations as recurrence_update,
// so w_{j+1} is identical to the other variants'; only the moments' summation
// order differs.
#pragma once

#include "step_kernel.cuh"

namespace cld {

// 8 floats from a 32-byte aligned address through the read-only path.
__device__ __forceinline__ void ldg8(const float* p, float (&o)[8]) {
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
                 : "l"(p));
}

// +-1 (0 for a padded probe) for probes sh .. sh+7 of a sign word: bit = 1 -> -1.
__device__ __forceinline__ void signs8(uint32_t word, int sh, const float (&mk)[8], float (&s)[8]) {
    const uint32_t b = word >> sh;
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = __uint_as_float(0x3f800000u | (((b >> q) & 1u) << 31)) * mk[q];
}

// The update of recurrence_update for one probe (same operations, same order).
template <int PREV>
__device__ __forceinline__ float recurrence_update1(float acc, float own, float pv, float scale, float scale_lo,
                                                    float shift, float shift_lo) {
    const float y = fmaf(scale, acc, -shift * own) + fmaf(scale_lo, acc, -shift_lo * own);
    if (PREV == 0) return y;
    return fmaf(2.f, y, -pv);
}

template <int MP, typename VT, int GATHER, int PREV, int EPI>
__global__ void __launch_bounds__(kThreads, 3) step_kernel_wide(const StepArgs args) {
    pdl_wait();  // w_j, w_{j-1}, the signs and the parameters come from earlier kernels
    pdl_trigger();
    static_assert(MP >= 8, "wide lanes need at least 8 probes per panel");
    constexpr int PPL = 8;                 // probes per lane
    constexpr int LPR = MP / PPL;          // lanes per row
    constexpr int RPW = 32 / LPR;          // rows per warp
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    constexpr int WPB = kThreads / 32;
    constexpr int U = 4;                   // stored entries in flight per lane

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = lane % LPR;
    const int g_in_w = lane / LPR;
    const int64_t gid = ((int64_t)blockIdx.x * WPB + warp) * RPW + g_in_w;
    const int64_t ngroups = (int64_t)gridDim.x * WPB * RPW;
    const int q0 = sub * PPL;              // first probe of this lane
    const int wsel = q0 >> 5, bsh = q0 & 31;
    float mk[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) mk[q] = q0 + q < args.mreal ? 1.f : 0.f;
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const int64_t* __restrict__ rowptr = args.rowptr;
    const int64_t kend = value_end<VT>(rowptr, args.d);

    float scale = 1.f, scale_lo = 0.f, shift = 0.f, shift_lo = 0.f;
    if (EPI == 1) {
        scale = args.prm->scale_hi;
        scale_lo = args.prm->scale_lo;
        shift = args.prm->shift_hi;
        shift_lo = args.prm->shift_lo;
    }
    float tacc[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) tacc[q] = 0.f;

    for (int64_t row = gid; row < args.d; row += ngroups) {
        const int64_t k0 = __ldg(rowptr + row), k1 = __ldg(rowptr + row + 1);
        float acc[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) acc[q] = 0.f;
        // the row's product; EDGE: 16-bit value loads (a BF16 row that holds
        // the array's first or last entry), decided once per row
        auto row_product = [&](auto edge_tag) {
            constexpr bool EDGE = decltype(edge_tag)::value;
            for (int64_t k = k0; k < k1; k += U) {
                // indices and values first, then the gathers
                int c[U];
                uint32_t abits[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool ok = k + u < k1;
                    c[u] = ok ? __ldg(args.col + k + u) : -1;
                    abits[u] = ok ? load_bits(val, k + u, EDGE) : 0u;
                }
                float xv[U][PPL];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (c[u] >= 0) {
                        if (GATHER == 1)
                            signs8(__ldg(args.vbits + (int64_t)c[u] * NW + wsel), bsh, mk, xv[u]);
                        else
                            ldg8(args.x + (int64_t)c[u] * MP + q0, xv[u]);
                    } else {
#pragma unroll
                        for (int q = 0; q < PPL; ++q) xv[u][q] = 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float a = __uint_as_float(abits[u]);
#pragma unroll
                    for (int q = 0; q < PPL; ++q) acc[q] = fmaf(a, xv[u][q], acc[q]);
                }
            }
        };
        if (std::is_same<VT, bf16_t>::value && (k0 == 0 || k1 == kend))
            row_product(std::true_type{});
        else
            row_product(std::false_type{});
        float res[PPL];
        if (EPI == 0) {
#pragma unroll
            for (int q = 0; q < PPL; ++q) res[q] = acc[q];
        } else {
            float v[PPL], own[PPL], pv[PPL];
            signs8(__ldg(args.vbits + row * NW + wsel), bsh, mk, v);
            if (PREV == 0) {
#pragma unroll
                for (int q = 0; q < PPL; ++q) own[q] = v[q];
            } else {
                ldg8(args.own + row * MP + q0, own);
            }
            if (PREV == 2) {
                const float4 lo = ldcs4(args.wprev + row * MP + q0), hi = ldcs4(args.wprev + row * MP + q0 + 4);
                pv[0] = lo.x; pv[1] = lo.y; pv[2] = lo.z; pv[3] = lo.w;
                pv[4] = hi.x; pv[5] = hi.y; pv[6] = hi.z; pv[7] = hi.w;
            } else {
#pragma unroll
                for (int q = 0; q < PPL; ++q) pv[q] = v[q];
            }
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                res[q] = recurrence_update1<PREV>(acc[q], own[q], pv[q], scale, scale_lo, shift, shift_lo);
                tacc[q] = fmaf(v[q], res[q], tacc[q]);
            }
        }
        st4(args.out + row * MP + q0, make_float4(res[0], res[1], res[2], res[3]));
        st4(args.out + row * MP + q0 + 4, make_float4(res[4], res[5], res[6], res[7]));
    }

    if (EPI == 1) {
        // lanes with the same `sub` hold the same probes: fold them, then the
        // warps of the CTA in a fixed order
        __shared__ double red[WPB][MP];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            double t = tacc[q];
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (g_in_w == 0) red[warp][q0 + q] = t;
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

}  // namespace cld
