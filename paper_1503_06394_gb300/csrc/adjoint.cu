// Adjoint (reverse-mode gradient) of the Chebyshev-Hutchinson estimate with
// respect to the stored values of a symmetric B, the interval [a, b] held fixed.
// The paper has no gradient; this differentiates the recurrence of Sec. 2.2.
//
// With At = scale B - shift I (scale = 2/(b-a), shift = (a+b)/(b-a)),
// w_0 = v, w_1 = At v, w_{j+1} = 2 At w_j - w_{j-1} and
// Gamma_p = sum_j c_j v^T w_j, the adjoint vectors
//   lambda_{n+1} = lambda_{n+2} = 0,
//   lambda_i = c_i v + 2 At lambda_{i+1} - lambda_{i+2}   (i = n .. 1)
// give, for a stored entry (r, k),
//   dGamma_p / dB_rk = scale * (lambda_1[r] v[k] + 2 sum_{i=1}^{n-1} lambda_{i+1}[r] w_i[k]).
//
// Fused SDDMM: the pass that forms lambda_i over row k gathers lambda_{i+1}[r]
// for every stored (k, r) and holds w_i[k]; for a symmetric pattern that is the
// term of entry (r, k), so it is accumulated at the position of (k, r) in H and
// mapped through the transpose at the end (no extra gathers).
#include <math.h>

#include "step_staged.cuh"
#include "step_wide.cuh"

namespace cld {



// The per-entry probe sums of a 4-entry chunk are reduced across the LPR lanes
// of a row group with a reduce-scatter: after it, entry q's full sum sits in
// one lane (two entries per lane when LPR = 2, all four when LPR = 1).
// adj_owned_entries gives the entries a lane owns (-1: none).
template <int LPR>
__device__ __forceinline__ void adj_owned_entries(int lig, int& qa, int& qb) {
    if (LPR == 1) { qa = -1; qb = -1; }                      // handled as 4 entries below
    else if (LPR == 2) { qa = 2 * lig; qb = 2 * lig + 1; }
    else if (LPR == 4) { qa = lig; qb = -1; }
    else { qa = (lig & 1) == 0 && lig < 8 ? (lig >> 1) : -1; qb = -1; }
}

template <int LPR>
__device__ __forceinline__ void adj_reduce_scatter4(float (&dt)[4], int lig, unsigned gmask, float& sa, float& sb) {
    sa = 0.f;
    sb = 0.f;
    if constexpr (LPR == 2) {
        // lane 0 keeps entries 0,1; lane 1 keeps 2,3
        const bool hi = lig & 1;
        const float s0 = hi ? dt[0] : dt[2], s1 = hi ? dt[1] : dt[3];
        const float r0 = __shfl_xor_sync(gmask, s0, 1, LPR), r1 = __shfl_xor_sync(gmask, s1, 1, LPR);
        sa = (hi ? dt[2] : dt[0]) + r0;
        sb = (hi ? dt[3] : dt[1]) + r1;
    } else if constexpr (LPR >= 4) {
        // fold the upper lanes until 8 (or 4) remain
#pragma unroll
        for (int off = LPR / 2; off >= 8; off >>= 1) {
#pragma unroll
            for (int u = 0; u < 4; ++u) dt[u] += __shfl_xor_sync(gmask, dt[u], off, LPR);
        }
        constexpr int W = LPR >= 8 ? 8 : 4;
        // stage A over xor W/2: keep entries {0,1} or {2,3}
        const bool ha = (lig & (W / 2)) != 0;
        const float s0 = ha ? dt[0] : dt[2], s1 = ha ? dt[1] : dt[3];
        float k0 = (ha ? dt[2] : dt[0]) + __shfl_xor_sync(gmask, s0, W / 2, LPR);
        float k1 = (ha ? dt[3] : dt[1]) + __shfl_xor_sync(gmask, s1, W / 2, LPR);
        // stage B over xor W/4: keep one entry
        const bool hb = (lig & (W / 4)) != 0;
        const float snd = hb ? k0 : k1;
        float kk = (hb ? k1 : k0) + __shfl_xor_sync(gmask, snd, W / 4, LPR);
        // stage C (W = 8 only): finish over xor 1
        if (W == 8) kk += __shfl_xor_sync(gmask, kk, 1, LPR);
        sa = kk;
    }
}

// MODE 0: lambda_{i+1} = 0 (i = n): lambda_i = c_i v; no gather, no H term.
// MODE 1: lambda_{i+2} = 0 (i = n - 1).
// MODE 2: general.
// MODE 3: final pass: H[pos(k,r)] += sum_p lambda_in[r,p] v[k,p]; no lambda_out.
template <int MP, typename VT, int MODE>
// 6 resident CTAs per SM (40 registers, no spills): the pass is latency bound.
__global__ void __launch_bounds__(kThreads, 6) adjoint_kernel(const AdjArgs args) {
    pdl_wait();  // lambda_{i+1}, lambda_{i+2}, H and w_i come from earlier kernels
    pdl_trigger();
    constexpr int LPR = MP / 4;
    constexpr int GPW = 32 / LPR;
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    constexpr int WPB = kThreads / 32;
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int lig = lane % LPR;
    const int g_in_w = lane / LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (g_in_w * LPR));
    const int64_t gid = ((int64_t)blockIdx.x * WPB + warp) * GPW + g_in_w;
    const int64_t ngroups = (int64_t)gridDim.x * WPB * GPW;
    const int p0 = 4 * lig, wsel = p0 >> 5, bsh = p0 & 31;
    const float4 mask = make_float4(p0 < args.mreal ? 1.f : 0.f, p0 + 1 < args.mreal ? 1.f : 0.f,
                                    p0 + 2 < args.mreal ? 1.f : 0.f, p0 + 3 < args.mreal ? 1.f : 0.f);
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const float scale = args.prm->scale_hi, scale_lo = args.prm->scale_lo;
    const float shift = args.prm->shift_hi, shift_lo = args.prm->shift_lo;
    const float ci = MODE == 3 ? 0.f : (float)args.coeffs[args.ci];
    const float hfac = MODE == 3 ? 1.f : 2.f;

    for (int64_t row = gid; row < args.d; row += ngroups) {
        const float4 v = signs4(__ldg(args.vbits + row * NW + wsel), bsh, mask);
        if (MODE == 0) {
            *reinterpret_cast<float4*>(args.lam_out + row * MP + p0) =
                make_float4(ci * v.x, ci * v.y, ci * v.z, ci * v.w);
            continue;
        }
        const float4 wk = MODE == 3 ? v : __ldg(reinterpret_cast<const float4*>(args.w + row * MP + p0));
        const int64_t k0 = __ldg(args.rowptr + row), k1 = __ldg(args.rowptr + row + 1);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t k = k0; k < k1; k += U) {
            // this lane's share of the H updates of the chunk, loaded up front
            int qa, qb;  // entries owned (qb < 0: one entry)
            adj_owned_entries<LPR>(lig, qa, qb);
            float ha = 0.f, hb = 0.f, h1[U];
            if (LPR == 1) {
#pragma unroll
                for (int u = 0; u < U; ++u) h1[u] = k + u < k1 ? args.H[k + u] : 0.f;
            }
            if (qa >= 0 && k + qa < k1) ha = args.H[k + qa];
            if (qb >= 0 && k + qb < k1) hb = args.H[k + qb];
            int c[U];
            float a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = k + u < k1;
                c[u] = ok ? __ldg(args.col + k + u) : -1;
                a[u] = ok ? load_val(val + k + u) : 0.f;
            }
            float4 xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                xv[u] = c[u] >= 0 ? __ldg(reinterpret_cast<const float4*>(args.lam_in + (int64_t)c[u] * MP + p0))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            float dt[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                acc.x = fmaf(a[u], xv[u].x, acc.x);
                acc.y = fmaf(a[u], xv[u].y, acc.y);
                acc.z = fmaf(a[u], xv[u].z, acc.z);
                acc.w = fmaf(a[u], xv[u].w, acc.w);
                float t = xv[u].x * wk.x;
                t = fmaf(xv[u].y, wk.y, t);
                t = fmaf(xv[u].z, wk.z, t);
                dt[u] = fmaf(xv[u].w, wk.w, t);
            }
            if (LPR == 1) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (k + u < k1) args.H[k + u] = fmaf(hfac, dt[u], h1[u]);
            }
            float sa, sb;
            adj_reduce_scatter4<LPR>(dt, lig, gmask, sa, sb);
            if (qa >= 0 && k + qa < k1) args.H[k + qa] = fmaf(hfac, sa, ha);
            if (qb >= 0 && k + qb < k1) args.H[k + qb] = fmaf(hfac, sb, hb);
        }
        if (MODE == 3) continue;
        const float4 own = __ldg(reinterpret_cast<const float4*>(args.lam_in + row * MP + p0));
        float4 y;
        y.x = fmaf(scale, acc.x, -shift * own.x) + fmaf(scale_lo, acc.x, -shift_lo * own.x);
        y.y = fmaf(scale, acc.y, -shift * own.y) + fmaf(scale_lo, acc.y, -shift_lo * own.y);
        y.z = fmaf(scale, acc.z, -shift * own.z) + fmaf(scale_lo, acc.z, -shift_lo * own.z);
        y.w = fmaf(scale, acc.w, -shift * own.w) + fmaf(scale_lo, acc.w, -shift_lo * own.w);
        float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MODE == 2) pv = __ldcs(reinterpret_cast<const float4*>(args.lam_prev + row * MP + p0));
        float4 out;
        out.x = fmaf(ci, v.x, fmaf(2.f, y.x, -pv.x));
        out.y = fmaf(ci, v.y, fmaf(2.f, y.y, -pv.y));
        out.z = fmaf(ci, v.z, fmaf(2.f, y.z, -pv.z));
        out.w = fmaf(ci, v.w, fmaf(2.f, y.w, -pv.w));
        *reinterpret_cast<float4*>(args.lam_out + row * MP + p0) = out;
    }
}

// The same reverse step with wide lanes (the forward's variant 5): each lane
// owns 8 consecutive probes of a row (LPR = P / 8 lanes per row, P >= 8),
// gathers lambda_{i+1} rows with 256-bit loads, and forms its 8-probe share
// of each entry's dot product before the reduce-scatter over the row's lanes.
template <int MP, typename VT, int MODE>
__global__ void __launch_bounds__(kThreads, 3) adjoint_kernel_wide(const AdjArgs args) {
    pdl_wait();  // lambda_{i+1}, lambda_{i+2}, H and w_i come from earlier kernels
    pdl_trigger();
    static_assert(MP >= 8, "wide lanes need at least 8 probes per panel");
    constexpr int PPL = 8;
    constexpr int LPR = MP / PPL;
    constexpr int RPW = 32 / LPR;
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    constexpr int WPB = kThreads / 32;
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = lane % LPR;
    const int g_in_w = lane / LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (g_in_w * LPR));
    const int64_t gid = ((int64_t)blockIdx.x * WPB + warp) * RPW + g_in_w;
    const int64_t ngroups = (int64_t)gridDim.x * WPB * RPW;
    const int q0 = sub * PPL, wsel = q0 >> 5, bsh = q0 & 31;
    float mk[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) mk[q] = q0 + q < args.mreal ? 1.f : 0.f;
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const int64_t kend = value_end<VT>(args.rowptr, args.d);
    const float scale = args.prm->scale_hi, scale_lo = args.prm->scale_lo;
    const float shift = args.prm->shift_hi, shift_lo = args.prm->shift_lo;
    const float ci = MODE == 3 ? 0.f : (float)args.coeffs[args.ci];
    const float hfac = MODE == 3 ? 1.f : 2.f;

    for (int64_t row = gid; row < args.d; row += ngroups) {
        float v[PPL];
        signs8(__ldg(args.vbits + row * NW + wsel), bsh, mk, v);
        if (MODE == 0) {
            st4(args.lam_out + row * MP + q0, make_float4(ci * v[0], ci * v[1], ci * v[2], ci * v[3]));
            st4(args.lam_out + row * MP + q0 + 4, make_float4(ci * v[4], ci * v[5], ci * v[6], ci * v[7]));
            continue;
        }
        float wk[PPL];
        if (MODE == 3) {
#pragma unroll
            for (int q = 0; q < PPL; ++q) wk[q] = v[q];
        } else {
            ldg8(args.w + row * MP + q0, wk);
        }
        const int64_t k0 = __ldg(args.rowptr + row), k1 = __ldg(args.rowptr + row + 1);
        float acc[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) acc[q] = 0.f;
        // the row's sweep; EDGE: 16-bit value loads (a BF16 row that holds the
        // array's first or last entry), decided once per row (all lanes of the
        // row's group take the same branch)
        auto row_sweep = [&](auto edge_tag) {
            constexpr bool EDGE = decltype(edge_tag)::value;
            for (int64_t k = k0; k < k1; k += U) {
                // this lane's share of the H updates of the chunk, loaded up front
                int qa, qb;
                adj_owned_entries<LPR>(sub, qa, qb);
                float ha = 0.f, hb = 0.f, h1[U];
                if (LPR == 1) {
#pragma unroll
                    for (int u = 0; u < U; ++u) h1[u] = k + u < k1 ? args.H[k + u] : 0.f;
                }
                if (qa >= 0 && k + qa < k1) ha = args.H[k + qa];
                if (qb >= 0 && k + qb < k1) hb = args.H[k + qb];
                int c[U];
                float a[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool ok = k + u < k1;
                    c[u] = ok ? __ldg(args.col + k + u) : -1;
                    a[u] = ok ? __uint_as_float(load_bits(val, k + u, EDGE)) : 0.f;
                }
                float xv[U][PPL];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (c[u] >= 0) {
                        ldg8(args.lam_in + (int64_t)c[u] * MP + q0, xv[u]);
                    } else {
#pragma unroll
                        for (int q = 0; q < PPL; ++q) xv[u][q] = 0.f;
                    }
                }
                float dt[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    float t = xv[u][0] * wk[0];
#pragma unroll
                    for (int q = 0; q < PPL; ++q) {
                        acc[q] = fmaf(a[u], xv[u][q], acc[q]);
                        if (q > 0) t = fmaf(xv[u][q], wk[q], t);
                    }
                    dt[u] = t;
                }
                if (LPR == 1) {
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (k + u < k1) args.H[k + u] = fmaf(hfac, dt[u], h1[u]);
                }
                float sa, sb;
                adj_reduce_scatter4<LPR>(dt, sub, gmask, sa, sb);
                if (qa >= 0 && k + qa < k1) args.H[k + qa] = fmaf(hfac, sa, ha);
                if (qb >= 0 && k + qb < k1) args.H[k + qb] = fmaf(hfac, sb, hb);
            }
        };
        if (std::is_same<VT, bf16_t>::value && (k0 == 0 || k1 == kend))
            row_sweep(std::true_type{});
        else
            row_sweep(std::false_type{});
        if (MODE == 3) continue;
        float own[PPL];
        ldg8(args.lam_in + row * MP + q0, own);
        float pv[PPL];
        if (MODE == 2) {
            const float4 lo = __ldcs(reinterpret_cast<const float4*>(args.lam_prev + row * MP + q0));
            const float4 hi = __ldcs(reinterpret_cast<const float4*>(args.lam_prev + row * MP + q0 + 4));
            pv[0] = lo.x; pv[1] = lo.y; pv[2] = lo.z; pv[3] = lo.w;
            pv[4] = hi.x; pv[5] = hi.y; pv[6] = hi.z; pv[7] = hi.w;
        } else {
#pragma unroll
            for (int q = 0; q < PPL; ++q) pv[q] = 0.f;
        }
        float out[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const float y = fmaf(scale, acc[q], -shift * own[q]) + fmaf(scale_lo, acc[q], -shift_lo * own[q]);
            out[q] = fmaf(ci, v[q], fmaf(2.f, y, -pv[q]));
        }
        st4(args.lam_out + row * MP + q0, make_float4(out[0], out[1], out[2], out[3]));
        st4(args.lam_out + row * MP + q0 + 4, make_float4(out[4], out[5], out[6], out[7]));
    }
}

// The reverse step with staged tiles (the form of the forward's variant 6):
// the producer warp of step_kernel_staged copies each tile's row pointers,
// indices, values and per-entry accumulators H, its rows of w_i,
// lambda_{i+1} (the row's own entry) and lambda_{i+2}, and its sign words
// into a ring of shared-memory stages; the consumer warps run the row sweep
// of adjoint_kernel_wide on them, gathering only lambda_{i+1} rows from
// global memory, and write H and lambda_i back to global memory.  MODE 1..3
// (MODE 0 has no gathers and runs the wide form).
template <int MP, typename VT, int MODE, class C>
struct AdjStagedSizes {
    using G = StagedGeom<MP, C::NC>;
    static constexpr bool kW = MODE != 3;       // w_i rows (MODE 3 uses v)
    static constexpr bool kOwn = MODE != 3;     // lambda_{i+1} rows
    static constexpr bool kPrev = MODE == 2;    // lambda_{i+2} rows
    static constexpr int rp_bytes = staged_up16((G::T + 2) * 8);
    // indices, H accumulators and values of capr entries a row, then the rows
    static constexpr int stage_of(int capr) {
        return staged_up16(rp_bytes + 2 * staged_up16(capr * G::T * 4) + staged_up16(capr * G::T * (int)sizeof(VT)) +
                           ((kW ? 1 : 0) + (kOwn ? 1 : 0) + (kPrev ? 1 : 0)) * G::T * MP * 4 +
                           staged_up16(G::T * G::NW * 4));
    }
    static constexpr int static_of(int) { return 512; }
};

template <int MP, typename VT, int MODE, class C>
struct AdjStagedLayout {
    using G = StagedGeom<MP, C::NC>;
    using Z = AdjStagedSizes<MP, VT, MODE, C>;
    using R = StagedRing<Z, C>;
    static constexpr bool kW = Z::kW, kOwn = Z::kOwn, kPrev = Z::kPrev;
    static constexpr int CAP = R::capr * G::T;  // stored entries a stage holds
    static constexpr int rp = 0;
    static constexpr int col = rp + Z::rp_bytes;
    static constexpr int h = col + staged_up16(CAP * 4);
    static constexpr int val = h + staged_up16(CAP * 4);
    static constexpr int w = val + staged_up16(CAP * (int)sizeof(VT));
    static constexpr int own = w + (kW ? G::T * MP * 4 : 0);
    static constexpr int prev = own + (kOwn ? G::T * MP * 4 : 0);
    static constexpr int sg = prev + (kPrev ? G::T * MP * 4 : 0);
    static constexpr int stage = staged_up16(sg + staged_up16(G::T * G::NW * 4));
    static constexpr int NS = R::ns;
    static constexpr int bytes = NS * stage;
    static_assert(stage == Z::stage_of(R::capr), "stage regions and stage_of disagree");
};

template <int MP, typename VT, int MODE, class C>
__global__ void __launch_bounds__(C::threads, C::MINB) adjoint_kernel_staged(const AdjArgs args) {
    static_assert(MP >= 8 && MODE >= 1 && MODE <= 3, "staged reverse steps: panels of 8 or more, MODE 1..3");
    using G = StagedGeom<MP, C::NC>;
    using S = AdjStagedLayout<MP, VT, MODE, C>;
    constexpr int PPL = G::PPL, LPR = G::LPR, RPW = G::RPW, T = G::T, NW = G::NW, NS = S::NS;
    constexpr int U = 4;
    constexpr int NC = C::NC;

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2 * NS];
    __shared__ int64_t hdr_kc[NS], hdr_kv[NS];
    __shared__ int hdr_staged[NS];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[NS + s]); };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full(s), 32);
            mbar_init(empty(s), NC);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();  // lambda_{i+1}, lambda_{i+2}, H and w_i come from earlier kernels
    pdl_trigger();

    const int64_t d = args.d;
    const int64_t ntiles = (d + T - 1) / T;
    const int64_t mine = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const int64_t* __restrict__ rowptr = args.rowptr;

    if (warp == NC) {
        const int64_t nnz = __ldg(rowptr + d);
        staged_producer_loop<NS, T>(lane, mine, d, rowptr, args.withhold_tile, args.err, bars,
                                    [&](int s, uint32_t bar, int64_t r0, int rows, int64_t k0, int64_t k1) {
            staged_fill_tile<MP, NW, VT>(lane, smem + s * S::stage, bar, r0, rows, 0, d, k0, k1, nnz, S::CAP, rowptr,
                                         args.col, val, args.H, S::kW ? args.w : nullptr,
                                         S::kOwn ? args.lam_in : nullptr, S::kPrev ? args.lam_prev : nullptr,
                                         args.vbits, S::rp, S::col, S::val, S::h, S::w, S::own, S::prev, S::sg,
                                         hdr_kc[s], hdr_kv[s], hdr_staged[s]);
        });
    } else {
        const int sub = lane % LPR;
        const int g_in_w = lane / LPR;
        const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (g_in_w * LPR));
        const int lr = warp * RPW + g_in_w;
        const int q0 = sub * PPL, wsel = q0 >> 5, bsh = q0 & 31;
        float mk[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) mk[q] = q0 + q < args.mreal ? 1.f : 0.f;
        const int64_t kend = value_end<VT>(rowptr, d);
        const float scale = args.prm->scale_hi, scale_lo = args.prm->scale_lo;
        const float shift = args.prm->shift_hi, shift_lo = args.prm->shift_lo;
        const float ci = MODE == 3 ? 0.f : (float)args.coeffs[args.ci];
        const float hfac = MODE == 3 ? 1.f : 2.f;
        int qa, qb;  // entries of a chunk whose H update this lane owns
        adj_owned_entries<LPR>(sub, qa, qb);

        for (int64_t i = 0; i < mine; ++i) {
            const int s = (int)(i % NS);
            if (!__all_sync(0xffffffffu, mbar_wait(full(s), (uint32_t)((i / NS) & 1)))) {
                if (lane == 0) atomicOr(args.err, 2u);
                break;
            }
            const int64_t r0 = ((int64_t)blockIdx.x + i * gridDim.x) * T;
            const int rows = (int)(d - r0 < T ? d - r0 : T);
            const unsigned char* st = smem + s * S::stage;
            if (lr < rows) {
                const int64_t row = r0 + lr;
                float v[PPL];
                signs8(reinterpret_cast<const uint32_t*>(st + S::sg)[lr * NW + wsel], bsh, mk, v);
                float wk[PPL];
                if (MODE == 3) {
#pragma unroll
                    for (int q = 0; q < PPL; ++q) wk[q] = v[q];
                } else {
                    const float4* w4 = reinterpret_cast<const float4*>(st + S::w + (lr * MP + q0) * 4);
                    const float4 a = w4[0], b = w4[1];
                    wk[0] = a.x; wk[1] = a.y; wk[2] = a.z; wk[3] = a.w;
                    wk[4] = b.x; wk[5] = b.y; wk[6] = b.z; wk[7] = b.w;
                }
                const int64_t* rp = reinterpret_cast<const int64_t*>(st + S::rp);
                const int64_t k0 = rp[lr], k1 = rp[lr + 1];
                float acc[PPL];
#pragma unroll
                for (int q = 0; q < PPL; ++q) acc[q] = 0.f;
                // one chunk of U entries starting at global entry k: their
                // indices c, value bits ab and H values (h1 for LPR == 1, else
                // this lane's owned entries ha / hb) are given
                auto chunk = [&](int64_t k, const int (&c)[U], const uint32_t (&ab)[U], const float (&h1)[U],
                                 float ha, float hb) {
                    float xv[U][PPL];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (c[u] >= 0) {
                            ldg8(args.lam_in + (int64_t)c[u] * MP + q0, xv[u]);
                        } else {
#pragma unroll
                            for (int q = 0; q < PPL; ++q) xv[u][q] = 0.f;
                        }
                    }
                    float dt[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const float a = __uint_as_float(ab[u]);
                        float t = xv[u][0] * wk[0];
#pragma unroll
                        for (int q = 0; q < PPL; ++q) {
                            acc[q] = fmaf(a, xv[u][q], acc[q]);
                            if (q > 0) t = fmaf(xv[u][q], wk[q], t);
                        }
                        dt[u] = t;
                    }
                    if (LPR == 1) {
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            if (k + u < k1) args.H[k + u] = fmaf(hfac, dt[u], h1[u]);
                    }
                    float sa, sb;
                    adj_reduce_scatter4<LPR>(dt, sub, gmask, sa, sb);
                    if (qa >= 0 && k + qa < k1) args.H[k + qa] = fmaf(hfac, sa, ha);
                    if (qb >= 0 && k + qb < k1) args.H[k + qb] = fmaf(hfac, sb, hb);
                };
                if (hdr_staged[s]) {
                    const int32_t* cs = reinterpret_cast<const int32_t*>(st + S::col);
                    const float* hs = reinterpret_cast<const float*>(st + S::h);
                    const VT* vs = reinterpret_cast<const VT*>(st + S::val);
                    const int64_t kc = hdr_kc[s];
                    const int dv = (int)(kc - hdr_kv[s]);
                    const int e1 = (int)(k1 - kc);
                    for (int e = (int)(k0 - kc); e < e1; e += U) {
                        int c[U];
                        uint32_t ab[U];
                        float h1[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const bool ok = e + u < e1;
                            c[u] = ok ? cs[e + u] : -1;
                            ab[u] = ok ? smem_val_bits<VT>(vs + e + u + dv) : 0u;
                            h1[u] = (LPR == 1 && ok) ? hs[e + u] : 0.f;
                        }
                        const float ha = (qa >= 0 && e + qa < e1) ? hs[e + qa] : 0.f;
                        const float hb = (qb >= 0 && e + qb < e1) ? hs[e + qb] : 0.f;
                        chunk(kc + e, c, ab, h1, ha, hb);
                    }
                } else {
                    const bool edge = std::is_same<VT, bf16_t>::value && (k0 == 0 || k1 == kend);
                    for (int64_t k = k0; k < k1; k += U) {
                        int c[U];
                        uint32_t ab[U];
                        float h1[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const bool ok = k + u < k1;
                            c[u] = ok ? __ldg(args.col + k + u) : -1;
                            ab[u] = ok ? load_bits(val, k + u, edge) : 0u;
                            h1[u] = (LPR == 1 && ok) ? args.H[k + u] : 0.f;
                        }
                        const float ha = (qa >= 0 && k + qa < k1) ? args.H[k + qa] : 0.f;
                        const float hb = (qb >= 0 && k + qb < k1) ? args.H[k + qb] : 0.f;
                        chunk(k, c, ab, h1, ha, hb);
                    }
                }
                if (MODE != 3) {
                    float own[PPL], pv[PPL];
                    const float4* o4 = reinterpret_cast<const float4*>(st + S::own + (lr * MP + q0) * 4);
                    {
                        const float4 a = o4[0], b = o4[1];
                        own[0] = a.x; own[1] = a.y; own[2] = a.z; own[3] = a.w;
                        own[4] = b.x; own[5] = b.y; own[6] = b.z; own[7] = b.w;
                    }
                    if (MODE == 2) {
                        const float4* p4 = reinterpret_cast<const float4*>(st + S::prev + (lr * MP + q0) * 4);
                        const float4 a = p4[0], b = p4[1];
                        pv[0] = a.x; pv[1] = a.y; pv[2] = a.z; pv[3] = a.w;
                        pv[4] = b.x; pv[5] = b.y; pv[6] = b.z; pv[7] = b.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < PPL; ++q) pv[q] = 0.f;
                    }
                    float out[PPL];
#pragma unroll
                    for (int q = 0; q < PPL; ++q) {
                        const float y = fmaf(scale, acc[q], -shift * own[q]) + fmaf(scale_lo, acc[q], -shift_lo * own[q]);
                        out[q] = fmaf(ci, v[q], fmaf(2.f, y, -pv[q]));
                    }
                    st4(args.lam_out + row * MP + q0, make_float4(out[0], out[1], out[2], out[3]));
                    st4(args.lam_out + row * MP + q0 + 4, make_float4(out[4], out[5], out[6], out[7]));
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty(s));
        }
    }
    __syncthreads();
}

// Shape of the staged reverse step: as the forward's variant 6.
using AdjStagedCfg = StagedCfg<4, 8, 3>;

template <int MP, typename VT, int MODE>
static cudaError_t launch_adj_staged_one(int grid, cudaStream_t s, const AdjArgs& a) {
    using C = AdjStagedCfg;
    constexpr auto kern = adjoint_kernel_staged<MP, VT, MODE, C>;
    constexpr int smem = AdjStagedLayout<MP, VT, MODE, C>::bytes;
    cudaError_t e = smem_opt_in<kern>(smem, C::MINB);
    if (e != cudaSuccess || grid == 0) return e;
    return launch_pdl(kern, grid, smem, s, a, C::threads);
}

template <int MP, typename VT>
static cudaError_t launch_adj_wide_mp(int mode, int grid, cudaStream_t s, const AdjArgs& a) {
    if constexpr (MP >= 8) {
        switch (mode) {
            case 0: return launch_pdl(adjoint_kernel_wide<MP, VT, 0>, grid, 0, s, a);
            case 1: return launch_pdl(adjoint_kernel_wide<MP, VT, 1>, grid, 0, s, a);
            case 2: return launch_pdl(adjoint_kernel_wide<MP, VT, 2>, grid, 0, s, a);
            case 3: return launch_pdl(adjoint_kernel_wide<MP, VT, 3>, grid, 0, s, a);
            default: return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int MP, typename VT>
static cudaError_t launch_adj_mp(int mode, int grid, cudaStream_t s, const AdjArgs& a) {
    switch (mode) {
        case 0: return launch_pdl(adjoint_kernel<MP, VT, 0>, grid, 0, s, a);
        case 1: return launch_pdl(adjoint_kernel<MP, VT, 1>, grid, 0, s, a);
        case 2: return launch_pdl(adjoint_kernel<MP, VT, 2>, grid, 0, s, a);
        case 3: return launch_pdl(adjoint_kernel<MP, VT, 3>, grid, 0, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int MP, typename VT>
static cudaError_t launch_adj_staged_mp(int mode, int grid, cudaStream_t s, const AdjArgs& a) {
    if constexpr (MP >= 8) {
        // bulk copies need 16-byte aligned CSR arrays; MODE 0 has no gathers
        const bool aligned = (reinterpret_cast<uintptr_t>(a.rowptr) % 16 == 0) &&
                             (reinterpret_cast<uintptr_t>(a.col) % 16 == 0) &&
                             (reinterpret_cast<uintptr_t>(a.val) % 16 == 0) &&
                             (reinterpret_cast<uintptr_t>(a.H) % 16 == 0);
        if (mode == 0 || !aligned || a.err == nullptr) return launch_adj_wide_mp<MP, VT>(mode, grid, s, a);
        switch (mode) {
            case 1: return launch_adj_staged_one<MP, VT, 1>(grid, s, a);
            case 2: return launch_adj_staged_one<MP, VT, 2>(grid, s, a);
            case 3: return launch_adj_staged_one<MP, VT, 3>(grid, s, a);
            default: return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename VT>
static cudaError_t launch_adj_vt(int panel, int mode, int grid, cudaStream_t s, const AdjArgs& a, int form) {
    if (form == 2) {
        switch (panel) {
            case 8: return launch_adj_staged_mp<8, VT>(mode, grid, s, a);
            case 16: return launch_adj_staged_mp<16, VT>(mode, grid, s, a);
            case 32: return launch_adj_staged_mp<32, VT>(mode, grid, s, a);
            case 64: return launch_adj_staged_mp<64, VT>(mode, grid, s, a);
            case 128: return launch_adj_staged_mp<128, VT>(mode, grid, s, a);
            default: return cudaErrorInvalidValue;
        }
    }
    if (form == 1) {
        switch (panel) {
            case 8: return launch_adj_wide_mp<8, VT>(mode, grid, s, a);
            case 16: return launch_adj_wide_mp<16, VT>(mode, grid, s, a);
            case 32: return launch_adj_wide_mp<32, VT>(mode, grid, s, a);
            case 64: return launch_adj_wide_mp<64, VT>(mode, grid, s, a);
            case 128: return launch_adj_wide_mp<128, VT>(mode, grid, s, a);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (panel) {
        case 4: return launch_adj_mp<4, VT>(mode, grid, s, a);
        case 8: return launch_adj_mp<8, VT>(mode, grid, s, a);
        case 16: return launch_adj_mp<16, VT>(mode, grid, s, a);
        case 32: return launch_adj_mp<32, VT>(mode, grid, s, a);
        case 64: return launch_adj_mp<64, VT>(mode, grid, s, a);
        case 128: return launch_adj_mp<128, VT>(mode, grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

// G[pos(r,k)] = gscale * H[pos(k,r)]: for every stored (r, k), the first stored
// (k, r) of row k.  flags bit 16: the pattern is not symmetric.
__global__ void adjoint_gather_kernel(int64_t d, const int64_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ col, const float* __restrict__ H,
                                      double gscale, float* __restrict__ G, uint32_t* flags) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < d;
         r += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t pos = rowptr[r]; pos < rowptr[r + 1]; ++pos) {
            const int64_t k = col[pos];
            int64_t hit = -1;
            for (int64_t q = rowptr[k]; q < rowptr[k + 1]; ++q)
                if (col[q] == r) { hit = q; break; }
            if (hit < 0) {
                atomicOr(flags, 0x10000u);
                G[pos] = 0.f;
            } else {
                G[pos] = (float)(gscale * (double)H[hit]);
            }
        }
    }
}

template <int MP, typename VT>
static int adj_ctas_mp(int form) {
    int n = 0;
    cudaError_t e;
    if constexpr (MP >= 8) {
        if (form == 2) {
            using C = AdjStagedCfg;
            constexpr auto kern = adjoint_kernel_staged<MP, VT, 2, C>;
            constexpr int smem = AdjStagedLayout<MP, VT, 2, C>::bytes;
            e = smem_opt_in<kern>(smem, C::MINB);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, C::threads, smem);
        } else {
            e = form == 1
                    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_kernel_wide<MP, VT, 2>, kThreads, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_kernel<MP, VT, 2>, kThreads, 0);
        }
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_kernel<MP, VT, 2>, kThreads, 0);
    }
    if (e != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

template <typename VT>
static int adj_ctas_vt(int panel, int form) {
    switch (panel) {
        case 4: return adj_ctas_mp<4, VT>(0);
        case 8: return adj_ctas_mp<8, VT>(form);
        case 16: return adj_ctas_mp<16, VT>(form);
        case 32: return adj_ctas_mp<32, VT>(form);
        case 64: return adj_ctas_mp<64, VT>(form);
        case 128: return adj_ctas_mp<128, VT>(form);
        default: return 1;
    }
}

int adjoint_ctas_per_sm(int panel, int dtype, int form) {
    switch (dtype) {
        case 0: return adj_ctas_vt<float>(panel, form);
        case 1: return adj_ctas_vt<bf16_t>(panel, form);
        case 2: return adj_ctas_vt<double>(panel, form);
        default: return 1;
    }
}

cudaError_t launch_adjoint(int panel, int dtype, int mode, int grid, cudaStream_t s, const AdjArgs& a, int form) {
    switch (dtype) {
        case 0: return launch_adj_vt<float>(panel, mode, grid, s, a, form);
        case 1: return launch_adj_vt<bf16_t>(panel, mode, grid, s, a, form);
        case 2: return launch_adj_vt<double>(panel, mode, grid, s, a, form);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_gather(int64_t d, const int64_t* rowptr, const int32_t* col, const float* H,
                                  double gscale, float* G, uint32_t* flags, int grid, cudaStream_t s) {
    adjoint_gather_kernel<<<grid, kThreads, 0, s>>>(d, rowptr, col, H, gscale, G, flags);
    return cudaGetLastError();
}

}  // namespace cld
