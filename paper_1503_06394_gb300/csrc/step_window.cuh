// Recurrence step with staged gather windows (inner-loop variant 7).
//
// The step of step_kernel_staged (Algorithm 1, Sec. 2.2: w_{j+1} =
// 2 At w_j - w_{j-1}, t_{j+1,p} = v_p^T w_{j+1}) for symmetric positive
// definite matrices whose rows reach few, compact index ranges: stencils and
// point clouds numbered by cell.  The columns that a tile of T consecutive
// rows gathers then form a handful of contiguous ranges (a grid tile: the
// rows above, beside and below it; a cell-ordered point cloud: three rows of
// cells), so the producer warp copies those ranges of w_j into the stage with
// bulk copies (TMA) and every gather becomes a shared-memory read: the
// gathers leave the chain of L1 / L2 latencies that bounds variant 6 on these
// matrices.
//
// * A plan (window_plan_kernel, once per matrix and panel width) gives each
//   tile up to kWinRanges ranges (gaps of up to kWinGap rows merged, the
//   tile's own rows always included) and each stored entry its row in the
//   concatenated ranges (`lcol`, an int32 array parallel to col).  A tile
//   whose columns span more than 65536 rows, need more ranges, or more rows
//   than a stage's window holds is not windowed: it is staged as in variant 6
//   and its consumers gather from global memory.
// * A stage holds the tile's row pointers, lcol (or col) and values, the
//   window (whose rows include w_j's own rows: for an SPD step x = w_j), the
//   rows of w_{j-1} and the sign words.
// * Consumers read their 8 probes of a row as two 16-byte halves; lanes whose
//   lane index has bit 2 set keep the halves swapped in all their registers
//   (gathers, own and w_{j-1} rows, signs, results, moments), which makes the
//   window and row reads free of bank conflicts at 32 and more probes without
//   a select per entry; the moments are put back in probe order once, before
//   the cross-lane fold.
//
// Row sums are formed in entry order with the update of recurrence_update, so
// w_{j+1} is identical to the other variants'.  Waits are bounded and report
// through args.err as in variant 6.
#pragma once

#include "step_staged.cuh"

namespace cld {

constexpr int kWinRanges = 4;     // index ranges a tile's window may hold
constexpr int kWinGap = 16;       // gaps of up to this many rows are copied, not split
constexpr int kWinSpan = 65536;   // a tile whose columns span more rows is not windowed

// Plan table of one tile (kWinTabInts ints): [0] ranges (0: not windowed),
// [1] window row of the tile's first row, [2 + k] first row of range k,
// [2 + kWinRanges + k] rows of range k (ranges in increasing order).

// Shape: one producer warp, NC consumer warps, U entries in flight per lane,
// MINB resident CTAs per SM; a CTA's share of shared memory is half the SM's
// largest carveout (the window's reads do not need L1).
template <int U_, int NC_, int MINB_>
struct WindowCfg {
    static constexpr int U = U_;
    static constexpr int NC = NC_;
    static constexpr int MINB = MINB_;
    static constexpr int threads = 32 * (NC + 1);
    static constexpr int cta_bytes = 228 * 1024 / MINB - 1024;
};

// Stage layout: row pointers, CAP indices, CAP values, w_{j-1} rows, sign
// words, then the window (capx rows of MP floats) with what is left of the
// CTA's share over two stages.
template <int MP, typename VT, int PREV, class C>
struct WindowLayout {
    using G = StagedGeom<MP, C::NC>;
    static constexpr int T = G::T;
    static constexpr int CAP = 16 * T;
    static constexpr int NS = 2;
    static constexpr int kStatic = C::NC * MP * 8 + 1024;  // moment partials, barriers, headers (upper bound)
    static constexpr int rp = 0;
    static constexpr int col = rp + staged_up16((T + 2) * 8);
    static constexpr int val = col + staged_up16(CAP * 4);
    static constexpr int prev = val + staged_up16(CAP * (int)sizeof(VT));
    static constexpr int sg = prev + (PREV == 2 ? T * MP * 4 : 0);
    static constexpr int win = sg + staged_up16(T * G::NW * 4);
    static constexpr int capx = ((C::cta_bytes - kStatic) / NS - win) / (MP * 4);  // window rows
    static constexpr int stage = staged_up16(win + capx * MP * 4);
    static constexpr int bytes = NS * stage;
    // windows at this shape: room for at least three tiles of rows
    static constexpr bool ok = capx >= 3 * T;
};

// The shape used by the dispatcher.
using WindowShape = WindowCfg<4, 8, 2>;

// Whether a panel of MP probes and value type VT has windows (checked on the
// general step's layout, whose window is the smallest).
template <int MP, typename VT>
constexpr bool window_ok() {
    if constexpr (MP >= 16) return WindowLayout<MP, VT, 2, WindowShape>::ok;
    else return false;
}

// Registers the bytes of copies on a stage's mbarrier without arriving.
__device__ __forceinline__ void mbar_expect_tx_only(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// This lane's 8 probes of a row in shared memory at `p` (16-byte aligned),
// the two 16-byte halves in slot order: half `sw` in slots 0..3.
__device__ __forceinline__ void lds8_slots(const unsigned char* p, int sw, float (&o)[8]) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = q[sw], b = q[sw ^ 1];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}

// The same from global memory (read-only path).
__device__ __forceinline__ void ldg8_slots(const float* p, int sw, float (&o)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p + 4 * sw));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p + 4 * (sw ^ 1)));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}

// +-1 (0 for a padded probe) of the 8 probes at bit `sh` of a sign word, in
// slot order (the two groups of 4 bits swapped when sw = 1); mk in slot order.
__device__ __forceinline__ void signs8_slots(uint32_t word, int sh, int sw, const float (&mk)[8], float (&s)[8]) {
    uint32_t b = (word >> sh) & 0xffu;
    if (sw) b = ((b >> 4) | (b << 4)) & 0xffu;
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = __uint_as_float(0x3f800000u | (((b >> q) & 1u) << 31)) * mk[q];
}

template <int MP, typename VT, int PREV, class C>
__global__ void __launch_bounds__(C::threads, C::MINB) step_kernel_window(const StepArgs args) {
    static_assert(MP >= 16 && (PREV == 1 || PREV == 2), "windows: 16 or more probes, steps j >= 1");
    using G = StagedGeom<MP, C::NC>;
    using S = WindowLayout<MP, VT, PREV, C>;
    static_assert(S::ok, "a window must hold at least three tiles of rows");
    constexpr int PPL = G::PPL, LPR = G::LPR, RPW = G::RPW, T = G::T, NW = G::NW, NS = S::NS;
    constexpr int U = C::U, NC = C::NC;
    constexpr bool kMask = PREV != 2;  // v enters the result of step 1

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2 * NS];
    __shared__ int64_t hdr_kc[NS], hdr_kv[NS];
    __shared__ int hdr_staged[NS], hdr_win[NS], hdr_own[NS];
    __shared__ double red[NC][MP];

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
    pdl_wait();  // w_j, w_{j-1}, the signs, the plan and the parameters come from earlier kernels

    const int64_t d = args.d;
    const int64_t ntiles = (d + T - 1) / T;
    const int64_t mine = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const int64_t* __restrict__ rowptr = args.rowptr;

    if (warp == NC) {
        // ------------------------------------------------------------ producer
        const int64_t nnz = __ldg(rowptr + d);
        int64_t started = 0, withheld_it = -1;
        bool ok = true;
        int64_t k0 = 0, k1 = 0;
        int32_t tv = 0;  // lane j < 2 + 2 kWinRanges: int j of the tile's plan row
        auto prefetch = [&](int64_t t) {
            const int64_t r0 = t * T;
            k0 = __ldg(rowptr + r0);
            k1 = __ldg(rowptr + (r0 + T < d ? r0 + T : d));
            tv = lane < 2 + 2 * kWinRanges ? __ldg(args.wtab + t * kWinTabInts + lane) : 0;
        };
        if (mine > 0) prefetch(blockIdx.x);
        for (int64_t i = 0; i < mine; ++i) {
            const int s = (int)(i % NS);
            const int64_t use = i / NS;
            if (use >= 1 && !__all_sync(0xffffffffu, mbar_wait(empty(s), (uint32_t)((use + 1) & 1)))) {
                ok = false;
                break;
            }
            const int64_t t = (int64_t)blockIdx.x + i * gridDim.x;
            const int64_t r0 = t * T;
            const int rows = (int)(d - r0 < T ? d - r0 : T);
            unsigned char* st = smem + s * S::stage;
            // the tile's plan row, broadcast from the lanes that loaded it
            const int nr = __shfl_sync(0xffffffffu, tv, 0);
            const int own_off = __shfl_sync(0xffffffffu, tv, 1);
            int rstart[kWinRanges], rlen[kWinRanges];
#pragma unroll
            for (int k = 0; k < kWinRanges; ++k) {
                rstart[k] = __shfl_sync(0xffffffffu, tv, 2 + k);
                rlen[k] = __shfl_sync(0xffffffffu, tv, 2 + kWinRanges + k);
            }
            if (args.withhold_tile == t + 1) {
                withheld_it = i;  // neither copies nor arrivals for this stage
            } else if (nr > 0) {
                // the window's ranges first, registered without an arrival
                // (the phase cannot complete before lane 0 arrives below)
                if (lane == 0) {
                    hdr_win[s] = nr;
                    hdr_own[s] = own_off;
                    uint32_t wbytes = 0;
#pragma unroll
                    for (int k = 0; k < kWinRanges; ++k)
                        if (k < nr) wbytes += (uint32_t)rlen[k] * MP * 4u;
                    mbar_expect_tx_only(full(s), wbytes);
                    int off = 0;
#pragma unroll
                    for (int k = 0; k < kWinRanges; ++k) {
                        if (k < nr) {
                            bulk_g2s(smem_u32(st + S::win + (size_t)off * MP * 4), args.x + (int64_t)rstart[k] * MP,
                                     (uint32_t)rlen[k] * MP * 4u, full(s));
                            off += rlen[k];
                        }
                    }
                }
                staged_fill_tile<MP, NW, VT>(lane, st, full(s), r0, rows, 0, d, k0, k1, nnz, S::CAP, rowptr,
                                             args.lcol, val, nullptr, nullptr, nullptr,
                                             PREV == 2 ? args.wprev : nullptr, args.vbits, S::rp, S::col, S::val,
                                             -1, -1, -1, S::prev, S::sg, hdr_kc[s], hdr_kv[s], hdr_staged[s]);
            } else {
                // not windowed: global columns, the own rows at window row 0
                if (lane == 0) {
                    hdr_win[s] = 0;
                    hdr_own[s] = 0;
                }
                staged_fill_tile<MP, NW, VT>(lane, st, full(s), r0, rows, 0, d, k0, k1, nnz, S::CAP, rowptr,
                                             args.col, val, nullptr, args.own, nullptr,
                                             PREV == 2 ? args.wprev : nullptr, args.vbits, S::rp, S::col, S::val,
                                             -1, S::win, -1, S::prev, S::sg, hdr_kc[s], hdr_kv[s], hdr_staged[s]);
            }
            started = i + 1;
            if (i + 1 < mine) prefetch(t + gridDim.x);
        }
        if (!ok) {
            if (lane == 0) atomicOr(args.err, 1u);
            for (int64_t j = started > NS ? started - NS : 0; j < started; ++j)
                if (j != withheld_it) mbar_wait(full((int)(j % NS)), (uint32_t)((j / NS) & 1));
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int sub = lane % LPR;
        const int g_in_w = lane / LPR;
        const int lr = warp * RPW + g_in_w;  // this lane's row within a tile
        const int q0 = sub * PPL;
        const int wsel = q0 >> 5, bsh = q0 & 31;
        const int sw = (lane >> 2) & 1;  // slots 0..3 hold probes q0 + 4 sw ..
        float mk[PPL];                   // in slot order
#pragma unroll
        for (int q = 0; q < PPL; ++q) mk[q] = (!kMask || q0 + (q ^ (4 * sw)) < args.mreal) ? 1.f : 0.f;
        const int64_t kend = value_end<VT>(rowptr, d);
        const float scale = args.prm->scale_hi, scale_lo = args.prm->scale_lo;
        const float shift = args.prm->shift_hi, shift_lo = args.prm->shift_lo;
        float tacc[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) tacc[q] = 0.f;

        for (int64_t i = 0; i < mine; ++i) {
            const int s = (int)(i % NS);
            if (!__all_sync(0xffffffffu, mbar_wait(full(s), (uint32_t)((i / NS) & 1)))) {
                if (lane == 0) atomicOr(args.err, 2u);
                break;
            }
            const int64_t r0 = ((int64_t)blockIdx.x + i * gridDim.x) * T;
            const int rows = (int)(d - r0 < T ? d - r0 : T);
            const unsigned char* st = smem + s * S::stage;
            const bool win = hdr_win[s] > 0;
            const unsigned char* wb = st + S::win + q0 * 4;  // this lane's probes of window row 0
            if (lr < rows) {
                const int64_t* rp = reinterpret_cast<const int64_t*>(st + S::rp);
                const int64_t k0 = rp[lr], k1 = rp[lr + 1];
                float acc[PPL];
#pragma unroll
                for (int q = 0; q < PPL; ++q) acc[q] = 0.f;
                // gathers of U entries (window rows or global columns in c)
                auto consume = [&](const int (&c)[U], const uint32_t (&ab)[U]) {
                    float xv[U][PPL];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (c[u] >= 0) {
                            if (win)
                                lds8_slots(wb + (size_t)c[u] * MP * 4, sw, xv[u]);
                            else
                                ldg8_slots(args.x + (int64_t)c[u] * MP + q0, sw, xv[u]);
                        } else {
#pragma unroll
                            for (int q = 0; q < PPL; ++q) xv[u][q] = 0.f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const float a = __uint_as_float(ab[u]);
#pragma unroll
                        for (int q = 0; q < PPL; ++q) acc[q] = fmaf(a, xv[u][q], acc[q]);
                    }
                };
                if (hdr_staged[s]) {
                    const int32_t* cs = reinterpret_cast<const int32_t*>(st + S::col);
                    const VT* vs = reinterpret_cast<const VT*>(st + S::val);
                    const int e0 = (int)(k0 - hdr_kc[s]), e1 = (int)(k1 - hdr_kc[s]);
                    const int dv = (int)(hdr_kc[s] - hdr_kv[s]);
                    for (int e = e0; e < e1; e += U) {
                        int c[U];
                        uint32_t ab[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const bool ok = e + u < e1;
                            c[u] = ok ? cs[e + u] : -1;
                            ab[u] = ok ? smem_val_bits<VT>(vs + e + u + dv) : 0u;
                        }
                        consume(c, ab);
                    }
                } else {
                    const int32_t* gc = win ? args.lcol : args.col;
                    const bool edge = std::is_same<VT, bf16_t>::value && (k0 == 0 || k1 == kend);
                    for (int64_t k = k0; k < k1; k += U) {
                        int c[U];
                        uint32_t ab[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const bool ok = k + u < k1;
                            c[u] = ok ? __ldg(gc + k + u) : -1;
                            ab[u] = ok ? load_bits(val, k + u, edge) : 0u;
                        }
                        consume(c, ab);
                    }
                }
                float v[PPL], own[PPL], pv[PPL], res[PPL];
                signs8_slots(reinterpret_cast<const uint32_t*>(st + S::sg)[lr * NW + wsel], bsh, sw, mk, v);
                lds8_slots(wb + (size_t)(hdr_own[s] + lr) * MP * 4, sw, own);
                if (PREV == 2) {
                    lds8_slots(st + S::prev + (lr * MP + q0) * 4, sw, pv);
                } else {
#pragma unroll
                    for (int q = 0; q < PPL; ++q) pv[q] = v[q];
                }
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    res[q] = recurrence_update1<PREV>(acc[q], own[q], pv[q], scale, scale_lo, shift, shift_lo);
                    tacc[q] = fmaf(v[q], res[q], tacc[q]);
                }
                float* o = args.out + (r0 + lr) * MP + q0;
                st4(o + 4 * sw, make_float4(res[0], res[1], res[2], res[3]));
                st4(o + 4 * (sw ^ 1), make_float4(res[4], res[5], res[6], res[7]));
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty(s));
        }
        // the moments back in probe order, then the lanes with the same `sub`
        // (the same probes) folded
        float tq[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) tq[q] = sw ? tacc[q ^ 4] : tacc[q];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            double t = tq[q];
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (g_in_w == 0) red[warp][q0 + q] = t;
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < MP; p += blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NC; ++w) s += red[w][p];
        args.tpart[(int64_t)blockIdx.x * MP + p] = s;
    }
}

}  // namespace cld
