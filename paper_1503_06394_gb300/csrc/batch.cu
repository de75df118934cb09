// Batched estimates: many independent matrices of uneven size in one pass per
// degree step.  The batch is one block-diagonal CSR with global indices; block
// b holds rows [blk_rows[b], blk_rows[b+1]) and has its own interval, probe
// key (seed + b, counter = local row), moments and result, so block b gives
// the same estimate as a single-matrix call with seed + b.
//
// Work is a static queue of row tiles that never span two blocks; a CTA takes
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... (deterministic) and reduces
// each tile's moment partials itself; a segmented reduction then sums each
// block's tiles in tile order.
#include <math.h>

#include "step_staged.cuh"
#include "step_wide.cuh"

namespace cld {

template <int MP, typename VT, int GATHER, int PREV, int IMPL>
__global__ void __launch_bounds__(kThreads, (StepOccupancy<IMPL, GATHER>::value))
    batch_step_kernel(const BatchStepArgs ba) {
    pdl_wait();  // w_j, w_{j-1}, the signs, tiles and parameters come from earlier kernels
    pdl_trigger();
    constexpr int LPR = MP / 4;
    constexpr int GPW = 32 / LPR;
    constexpr int WPB = kThreads / 32;
    const StepArgs& args = ba.s;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int lig = lane % LPR;
    const int g_in_w = lane / LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (g_in_w * LPR));
    const int gloc = warp * GPW + g_in_w;  // group within the CTA
    const int gcta = WPB * GPW;            // groups per CTA
    const int p0 = 4 * lig, wsel = p0 >> 5, bsh = p0 & 31;
    const float4 mask = make_float4(p0 < args.mreal ? 1.f : 0.f, p0 + 1 < args.mreal ? 1.f : 0.f,
                                    p0 + 2 < args.mreal ? 1.f : 0.f, p0 + 3 < args.mreal ? 1.f : 0.f);
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    __shared__ double red[WPB][MP];
    extern __shared__ float4 ring[];

    for (int64_t t = blockIdx.x; t < ba.ntiles; t += gridDim.x) {
        const Tile tl = ba.tiles[t];
        const Params* P = ba.bprm + tl.blk;
        const float scale = P->scale_hi, scale_lo = P->scale_lo, shift = P->shift_hi, shift_lo = P->shift_lo;
        float4 tacc = make_float4(0.f, 0.f, 0.f, 0.f);
        auto finish = [&](int64_t row, const float4& acc, const RowOperands& o) {
            const float4 res = recurrence_update<PREV>(acc, o.own, o.pv, scale, scale_lo, shift, shift_lo);
            tacc.x = fmaf(o.v.x, res.x, tacc.x);
            tacc.y = fmaf(o.v.y, res.y, tacc.y);
            tacc.z = fmaf(o.v.z, res.z, tacc.z);
            tacc.w = fmaf(o.v.w, res.w, tacc.w);
            st4(args.out + row * MP + p0, res);
        };
        rows_all<MP, GATHER, PREV, 1, IMPL>(args, val, tl.lo + gloc, tl.hi, gcta, lig, p0, wsel, bsh, mask, gmask,
                                            ring, finish);
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
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < WPB; ++w) sum += red[w][p];
            ba.tpart[t * MP + p] = sum;
        }
        __syncthreads();
    }
}

// The tile-queue step with wide lanes (variant 5 for batches): each lane owns
// 8 consecutive probes of a row (P / 8 lanes per row, P >= 8), gathers row
// slices with 256-bit loads and keeps 4 stored entries in flight; BF16 values
// are read as the 4-byte words that hold them (16-bit loads in the rows that
// hold the array's first or last entry).  Each row's sum is formed in entry
// order and updated with the same operations as batch_step_kernel, so w_{j+1}
// is identical; only the moments' summation order differs.
template <int MP, typename VT, int GATHER, int PREV>
__global__ void __launch_bounds__(kThreads, 3) batch_step_kernel_wide(const BatchStepArgs ba) {
    pdl_wait();  // w_j, w_{j-1}, the signs, tiles and parameters come from earlier kernels
    pdl_trigger();
    static_assert(MP >= 8, "wide lanes need at least 8 probes per panel");
    constexpr int PPL = 8;             // probes per lane
    constexpr int LPR = MP / PPL;      // lanes per row
    constexpr int RPW = 32 / LPR;      // rows per warp
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    constexpr int WPB = kThreads / 32;
    constexpr int U = 4;               // stored entries in flight per lane
    const StepArgs& args = ba.s;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = lane % LPR;
    const int g_in_w = lane / LPR;
    const int gloc = warp * RPW + g_in_w;  // row group within the CTA
    const int gcta = WPB * RPW;            // row groups per CTA
    const int q0 = sub * PPL, wsel = q0 >> 5, bsh = q0 & 31;
    float mk[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) mk[q] = q0 + q < args.mreal ? 1.f : 0.f;
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const int64_t* __restrict__ rowptr = args.rowptr;
    const int64_t kend = value_end<VT>(rowptr, args.d);
    __shared__ double red[WPB][MP];

    for (int64_t t = blockIdx.x; t < ba.ntiles; t += gridDim.x) {
        const Tile tl = ba.tiles[t];
        const Params* P = ba.bprm + tl.blk;
        const float scale = P->scale_hi, scale_lo = P->scale_lo, shift = P->shift_hi, shift_lo = P->shift_lo;
        float tacc[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) tacc[q] = 0.f;
        for (int64_t row = tl.lo + gloc; row < tl.hi; row += gcta) {
            const int64_t k0 = __ldg(rowptr + row), k1 = __ldg(rowptr + row + 1);
            float acc[PPL];
#pragma unroll
            for (int q = 0; q < PPL; ++q) acc[q] = 0.f;
            auto row_product = [&](auto edge_tag) {
                constexpr bool EDGE = decltype(edge_tag)::value;
                for (int64_t k = k0; k < k1; k += U) {
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
            float v[PPL], own[PPL], pv[PPL], res[PPL];
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
            st4(args.out + row * MP + q0, make_float4(res[0], res[1], res[2], res[3]));
            st4(args.out + row * MP + q0 + 4, make_float4(res[4], res[5], res[6], res[7]));
        }
        // lanes with the same `sub` hold the same probes: fold them, then the
        // warps of the CTA in a fixed order, into this tile's partials
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            double tq = tacc[q];
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1) tq += __shfl_xor_sync(0xffffffffu, tq, off);
            if (g_in_w == 0) red[warp][q0 + q] = tq;
        }
        __syncthreads();
        for (int p = threadIdx.x; p < MP; p += kThreads) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < WPB; ++w) sum += red[w][p];
            ba.tpart[t * MP + p] = sum;
        }
        __syncthreads();
    }
}

template <int MP, typename VT>
static cudaError_t launch_batch_wide(StepKind kind, int grid, cudaStream_t s, const BatchStepArgs& a) {
    if (grid == 0) return cudaSuccess;  // no dynamic shared memory to opt in
    switch (kind) {
        case kStepFirst: return launch_pdl(batch_step_kernel_wide<MP, VT, 1, 0>, grid, 0, s, a);
        case kStepSecond: return launch_pdl(batch_step_kernel_wide<MP, VT, 0, 1>, grid, 0, s, a);
        case kStepGeneral: return launch_pdl(batch_step_kernel_wide<MP, VT, 0, 2>, grid, 0, s, a);
        case kStepFirstFromFloat: return launch_pdl(batch_step_kernel_wide<MP, VT, 0, 0>, grid, 0, s, a);
        default: return cudaErrorInvalidValue;
    }
}

// The tile-queue step with staged tiles (variant 6 for batches): the CTA's
// queue tiles (tile blockIdx.x, then every gridDim.x-th) are cut into
// sub-tiles of T = 2048 / P rows, which the producer warp stages into the
// ring as step_kernel_staged does (the copies of row-indexed arrays start up
// to 3 rows early, at a multiple of 4, since tiles start where blocks do);
// the consumer warps compute them with 8 probes per lane and the block's own
// interval.  Each queue tile's moments are folded per warp into one of NS + 1
// shared slots; the warp that arrives last (a shared counter) sums the slot
// over the warps in a fixed order into the tile's partials, so no consumer
// ever waits for another (a stalled wait cannot hang the CTA), and a slot is
// reused only NS + 1 tiles later, when every warp is past that tile.
template <int MP, typename VT, int GATHER, int PREV, class C>
__global__ void __launch_bounds__(C::threads, C::MINB) batch_step_kernel_staged(const BatchStepArgs ba) {
    static_assert(MP >= 8, "staged tiles need at least 8 probes per panel");
    using G = StagedGeom<MP, C::NC>;
    using S = StagedLayout<MP, VT, PREV, 1, C, true>;
    constexpr int PPL = G::PPL, LPR = G::LPR, RPW = G::RPW, T = G::T, NW = G::NW, NS = S::NS;
    constexpr int U = C::U, NC = C::NC, NSLOT = NS + 1;
    constexpr bool kMask = GATHER == 1 || PREV != 2;

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2 * NS];
    __shared__ int64_t hdr_kc[NS], hdr_kv[NS];
    __shared__ int hdr_staged[NS];
    __shared__ double red[NSLOT][NC][MP];
    __shared__ int red_cnt[NSLOT];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[NS + s]); };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full(s), 32);
            mbar_init(empty(s), NC);
        }
        for (int k = 0; k < NSLOT; ++k) red_cnt[k] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();  // w_j, w_{j-1}, the signs, tiles and parameters come from earlier kernels
    // No early trigger: the next kernel's CTAs are placed when this one ends,
    // on SMs whose shared-memory carveout can then follow that kernel's
    // (placed early, they run with this kernel's carveout and its smaller L1).

    const StepArgs& args = ba.s;
    const int64_t d = args.d;
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const int64_t* __restrict__ rowptr = args.rowptr;

    if (warp == NC) {
        // ------------------------------------------------------------ producer
        const int64_t nnz = __ldg(rowptr + d);
        int64_t t = blockIdx.x;
        Tile tl{};
        int64_t r0 = 0, k0 = 0, k1 = 0;
        auto rows_at = [&](int64_t r) { return (int)(tl.hi - r < T ? tl.hi - r : T); };
        if (t < ba.ntiles) {
            tl = ba.tiles[t];
            r0 = tl.lo;
            k0 = __ldg(rowptr + r0);
            k1 = __ldg(rowptr + r0 + rows_at(r0));
        }
        int64_t it = 0;
        bool ok = true;
        while (t < ba.ntiles) {
            const int s = (int)(it % NS);
            const int64_t use = it / NS;
            if (use >= 1 && !__all_sync(0xffffffffu, mbar_wait(empty(s), (uint32_t)((use + 1) & 1)))) {
                ok = false;
                break;
            }
            const int rows = rows_at(r0);
            staged_fill_tile<MP, NW, VT>(lane, smem + s * S::stage, full(s), r0, rows, (int)(r0 & 3), d, k0, k1, nnz,
                                         S::CAP, rowptr, args.col, val, nullptr, PREV != 0 ? args.own : nullptr,
                                         PREV == 2 ? args.wprev : nullptr, nullptr, args.vbits, S::rp, S::col,
                                         S::val, -1, S::own, S::prev, -1, S::sg, hdr_kc[s], hdr_kv[s],
                                         hdr_staged[s]);
            ++it;
            // the next sub-tile (of this queue tile, or the CTA's next one) and
            // its entry bounds, loaded while the stage fills
            r0 += T;
            if (r0 >= tl.hi) {
                t += gridDim.x;
                if (t >= ba.ntiles) break;
                tl = ba.tiles[t];
                r0 = tl.lo;
            }
            k0 = __ldg(rowptr + r0);
            k1 = __ldg(rowptr + r0 + rows_at(r0));
        }
        if (!ok) {
            if (lane == 0) atomicOr(args.err, 1u);
            for (int64_t j = it > NS ? it - NS : 0; j < it; ++j)
                mbar_wait(full((int)(j % NS)), (uint32_t)((j / NS) & 1));
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int sub = lane % LPR;
        const int g_in_w = lane / LPR;
        const int lr = warp * RPW + g_in_w;  // this lane's row within a sub-tile
        const int q0 = sub * PPL;
        const int wsel = q0 >> 5, bsh = q0 & 31;
        float mk[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) mk[q] = (!kMask || q0 + q < args.mreal) ? 1.f : 0.f;
        const int64_t kend = value_end<VT>(rowptr, d);
        int64_t it = 0, qt = 0;  // sub-tiles and queue tiles taken
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ba.ntiles && ok; t += gridDim.x, ++qt) {
            const Tile tl = ba.tiles[t];
            const Params* P = ba.bprm + tl.blk;
            const float scale = P->scale_hi, scale_lo = P->scale_lo, shift = P->shift_hi, shift_lo = P->shift_lo;
            float tacc[PPL];
#pragma unroll
            for (int q = 0; q < PPL; ++q) tacc[q] = 0.f;
            for (int64_t r0 = tl.lo; r0 < tl.hi; r0 += T, ++it) {
                const int s = (int)(it % NS);
                if (!__all_sync(0xffffffffu, mbar_wait(full(s), (uint32_t)((it / NS) & 1)))) {
                    if (lane == 0) atomicOr(args.err, 2u);
                    ok = false;
                    break;
                }
                const int rows = (int)(tl.hi - r0 < T ? tl.hi - r0 : T);
                const int pre = (int)(r0 & 3);
                const unsigned char* st = smem + s * S::stage;
                if (lr < rows) {
                    const int sl = pre + lr;  // staged row
                    const int64_t* rp = reinterpret_cast<const int64_t*>(st + S::rp);
                    const int64_t k0 = rp[sl], k1 = rp[sl + 1];
                    float acc[PPL];
#pragma unroll
                    for (int q = 0; q < PPL; ++q) acc[q] = 0.f;
                    auto consume = [&](const int (&c)[U], const uint32_t (&ab)[U]) {
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
                                const bool okk = e + u < e1;
                                c[u] = okk ? cs[e + u] : -1;
                                ab[u] = okk ? smem_val_bits<VT>(vs + e + u + dv) : 0u;
                            }
                            consume(c, ab);
                        }
                    } else {
                        const bool edge = std::is_same<VT, bf16_t>::value && (k0 == 0 || k1 == kend);
                        for (int64_t k = k0; k < k1; k += U) {
                            int c[U];
                            uint32_t ab[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const bool okk = k + u < k1;
                                c[u] = okk ? __ldg(args.col + k + u) : -1;
                                ab[u] = okk ? load_bits(val, k + u, edge) : 0u;
                            }
                            consume(c, ab);
                        }
                    }
                    float v[PPL], own[PPL], pv[PPL], res[PPL];
                    signs8(reinterpret_cast<const uint32_t*>(st + S::sg)[sl * NW + wsel], bsh, mk, v);
                    if (PREV == 0) {
#pragma unroll
                        for (int q = 0; q < PPL; ++q) own[q] = v[q];
                    } else {
                        const float4* o4 = reinterpret_cast<const float4*>(st + S::own + (sl * MP + q0) * 4);
                        const float4 a = o4[0], b = o4[1];
                        own[0] = a.x; own[1] = a.y; own[2] = a.z; own[3] = a.w;
                        own[4] = b.x; own[5] = b.y; own[6] = b.z; own[7] = b.w;
                    }
                    if (PREV == 2) {
                        const float4* p4 = reinterpret_cast<const float4*>(st + S::prev + (sl * MP + q0) * 4);
                        const float4 a = p4[0], b = p4[1];
                        pv[0] = a.x; pv[1] = a.y; pv[2] = a.z; pv[3] = a.w;
                        pv[4] = b.x; pv[5] = b.y; pv[6] = b.z; pv[7] = b.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < PPL; ++q) pv[q] = v[q];
                    }
#pragma unroll
                    for (int q = 0; q < PPL; ++q) {
                        res[q] = recurrence_update1<PREV>(acc[q], own[q], pv[q], scale, scale_lo, shift, shift_lo);
                        tacc[q] = fmaf(v[q], res[q], tacc[q]);
                    }
                    const int64_t row = r0 + lr;
                    st4(args.out + row * MP + q0, make_float4(res[0], res[1], res[2], res[3]));
                    st4(args.out + row * MP + q0 + 4, make_float4(res[4], res[5], res[6], res[7]));
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty(s));
            }
            if (!ok) break;
            // this warp's share of the tile's moments into slot qt mod NSLOT;
            // the last warp to arrive sums the slot in warp order
            const int slot = (int)(qt % NSLOT);
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                double tq = tacc[q];
#pragma unroll
                for (int off = LPR; off < 32; off <<= 1) tq += __shfl_xor_sync(0xffffffffu, tq, off);
                if (g_in_w == 0) red[slot][warp][q0 + q] = tq;
            }
            __syncwarp();
            __threadfence_block();
            int last = 0;
            if (lane == 0) last = atomicAdd(&red_cnt[slot], 1) == NC - 1;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence_block();
                for (int p = lane; p < MP; p += 32) {
                    double sum = 0.0;
#pragma unroll
                    for (int w = 0; w < NC; ++w) sum += red[slot][w][p];
                    ba.tpart[t * MP + p] = sum;
                }
                __syncwarp();
                if (lane == 0) red_cnt[slot] = 0;
            }
        }
    }
    __syncthreads();
}

template <int MP, typename VT, int GATHER, int PREV>
static cudaError_t launch_one_batch_staged(int grid, cudaStream_t s, const BatchStepArgs& a) {
    using C = StagedCfg<4, 8, 3>;
    constexpr auto kern = batch_step_kernel_staged<MP, VT, GATHER, PREV, C>;
    constexpr int smem = StagedLayout<MP, VT, PREV, 1, C, true>::bytes;
    cudaError_t e = smem_opt_in<kern>(smem, C::MINB);
    if (e != cudaSuccess || grid == 0) return e;
    return launch_pdl(kern, grid, smem, s, a, C::threads);
}

template <int MP, typename VT>
static cudaError_t launch_batch_staged(StepKind kind, int grid, cudaStream_t s, const BatchStepArgs& a) {
    // bulk copies need 16-byte aligned CSR arrays; otherwise the wide lanes
    const bool aligned = (reinterpret_cast<uintptr_t>(a.s.rowptr) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(a.s.col) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(a.s.val) % 16 == 0);
    if (!aligned || a.s.err == nullptr) return launch_batch_wide<MP, VT>(kind, grid, s, a);
    switch (kind) {
        case kStepFirst: return launch_one_batch_staged<MP, VT, 1, 0>(grid, s, a);
        case kStepSecond: return launch_one_batch_staged<MP, VT, 0, 1>(grid, s, a);
        case kStepGeneral: return launch_one_batch_staged<MP, VT, 0, 2>(grid, s, a);
        case kStepFirstFromFloat: return launch_one_batch_staged<MP, VT, 0, 0>(grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int MP, typename VT, int GATHER, int PREV, int IMPL>
static cudaError_t launch_one_batch(int grid, cudaStream_t s, const BatchStepArgs& a) {
    constexpr auto kern = batch_step_kernel<MP, VT, GATHER, PREV, IMPL>;
    constexpr int smem = step_smem<IMPL, GATHER>();
    cudaError_t e = smem_opt_in<kern>(smem);
    if (e != cudaSuccess || grid == 0) return e;  // grid 0: opt in only
    return launch_pdl(kern, grid, smem, s, a);
}

template <int MP, typename VT, int IMPL>
static cudaError_t launch_batch_impl(StepKind kind, int grid, cudaStream_t s, const BatchStepArgs& a) {
    switch (kind) {
        case kStepFirst: return launch_one_batch<MP, VT, 1, 0, IMPL>(grid, s, a);
        case kStepSecond: return launch_one_batch<MP, VT, 0, 1, IMPL>(grid, s, a);
        case kStepGeneral: return launch_one_batch<MP, VT, 0, 2, IMPL>(grid, s, a);
        case kStepFirstFromFloat: return launch_one_batch<MP, VT, 0, 0, IMPL>(grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int MP, typename VT>
static cudaError_t launch_batch_mp(StepKind kind, int grid, cudaStream_t s, const BatchStepArgs& a) {
    switch (a.s.impl) {
        case 0: return launch_batch_impl<MP, VT, 0>(kind, grid, s, a);
        case 1: return launch_batch_impl<MP, VT, 1>(kind, grid, s, a);
        case 2: return launch_batch_impl<MP, VT, 2>(kind, grid, s, a);
        case 3: return launch_batch_impl<MP, VT, 3>(kind, grid, s, a);
        case 4: return launch_batch_impl<MP, VT, 4>(kind, grid, s, a);
        case 5:
            if constexpr (MP >= 8) return launch_batch_wide<MP, VT>(kind, grid, s, a);
            else return launch_batch_impl<MP, VT, 0>(kind, grid, s, a);  // wide lanes need 8 probes
        case 6:
            if constexpr (MP >= 8) return launch_batch_staged<MP, VT>(kind, grid, s, a);
            else return launch_batch_impl<MP, VT, 0>(kind, grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <typename VT>
static cudaError_t launch_batch_vt(int panel, StepKind kind, int grid, cudaStream_t s, const BatchStepArgs& a) {
    switch (panel) {
        case 4: return launch_batch_mp<4, VT>(kind, grid, s, a);
        case 8: return launch_batch_mp<8, VT>(kind, grid, s, a);
        case 16: return launch_batch_mp<16, VT>(kind, grid, s, a);
        case 32: return launch_batch_mp<32, VT>(kind, grid, s, a);
        case 64: return launch_batch_mp<64, VT>(kind, grid, s, a);
        case 128: return launch_batch_mp<128, VT>(kind, grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_step(int panel, int dtype, StepKind kind, int grid, cudaStream_t s,
                              const BatchStepArgs& a) {
    switch (dtype) {
        case 0: return launch_batch_vt<float>(panel, kind, grid, s, a);
        case 1: return launch_batch_vt<bf16_t>(panel, kind, grid, s, a);
        case 2: return launch_batch_vt<double>(panel, kind, grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- probe signs
// Row i of block b: key = seed + b, counter = (local row lo, hi, panel, 0).
__global__ void batch_probe_bits_kernel(const Tile* __restrict__ tiles, int64_t ntiles, int nw, uint32_t panel,
                                        const Params* __restrict__ bprm, const int64_t* __restrict__ blk_rows,
                                        uint32_t* __restrict__ vbits) {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const uint32_t k0 = bprm[tl.blk].key_lo, k1 = bprm[tl.blk].key_hi;
        const int64_t base = blk_rows[tl.blk];
        for (int64_t i = tl.lo + threadIdx.x; i < tl.hi; i += blockDim.x) {
            const uint64_t u = (uint64_t)(i - base);
            const uint4 r = philox4x32_10(make_uint4((uint32_t)u, (uint32_t)(u >> 32), panel, 0u), k0, k1);
            const uint32_t w[4] = {r.x, r.y, r.z, r.w};
            for (int q = 0; q < nw; ++q) vbits[i * nw + q] = w[q];
        }
    }
}

// bprm[b].key = seed + b
__global__ void batch_set_seed_kernel(Params* bprm, int nb, uint64_t seed) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const uint64_t k = seed + (uint64_t)b;
        bprm[b].key_lo = (uint32_t)k;
        bprm[b].key_hi = (uint32_t)(k >> 32);
    }
}

// bprm[b] interval from host arrays already copied to dev_ab (a_0, b_0, a_1, b_1, ...)
__global__ void batch_set_intervals_kernel(Params* bprm, int nb, const double* ab) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const double a = ab[2 * b], bb = ab[2 * b + 1];
        set_affine(bprm + b, a, bb);
        bprm[b].interval_ok = (a > 0.0 && a < bb && isfinite(a) && isfinite(bb)) ? 1 : 0;
    }
}

// ---------------------------------------------------------------- moments
// T[b][(s+1) M + pbase + p] = sum over the tiles of block b (ascending) of
// tpart[s][tile][p].  Grid (nb, nsteps); thread (p, q) sums every nq-th tile.
__global__ void batch_reduce_kernel(const double* __restrict__ tpart, int64_t ntiles,
                                    const int64_t* __restrict__ tile_start, int panel, int mreal, int n, int M,
                                    int pbase, double* __restrict__ T) {
    const int b = blockIdx.x;
    const int p = threadIdx.x % panel, q = threadIdx.x / panel, nq = kThreads / panel;
    __shared__ double part[kThreads];
    for (int s = blockIdx.y; s < n; s += gridDim.y) {
        const double* base = tpart + (int64_t)s * ntiles * panel;
        double acc = 0.0;
        for (int64_t t = tile_start[b] + q; t < tile_start[b + 1]; t += nq) acc += base[t * panel + p];
        part[threadIdx.x] = acc;
        __syncthreads();
        if (q == 0 && p < mreal) {
            double sum = 0.0;
            for (int r = 0; r < nq; ++r) sum += part[r * panel + p];
            T[(size_t)b * (n + 1) * M + (size_t)(s + 1) * M + pbase + p] = sum;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- intervals
// SPD blocks: Gershgorin per block; one CTA per block.
template <typename VT>
__global__ void batch_gershgorin_kernel(const int64_t* __restrict__ blk_rows, const int64_t* __restrict__ rowptr,
                                        const int32_t* __restrict__ col, const VT* __restrict__ val, Params* bprm,
                                        uint32_t* flags) {
    __shared__ double shl[kThreads], shh[kThreads];
    const int b = blockIdx.x;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = blk_rows[b] + threadIdx.x; i < blk_rows[b + 1]; i += blockDim.x) {
        double dg = 0.0, r = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const double v = load_val_f64(val + k);
            if (col[k] == i) dg += v; else r += fabs(v);
        }
        lo = fmin(lo, dg - r);
        hi = fmax(hi, dg + r);
    }
    shl[threadIdx.x] = lo;
    shh[threadIdx.x] = hi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            shl[threadIdx.x] = fmin(shl[threadIdx.x], shl[threadIdx.x + o]);
            shh[threadIdx.x] = fmax(shh[threadIdx.x], shh[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double a = shl[0], bb = shh[0];
        const int ok = finish_interval(a, bb, blk_rows[b + 1] - blk_rows[b]) ? 1 : 0;
        set_affine(bprm + b, a, bb);
        bprm[b].interval_ok = ok;
        if (!ok) atomicOr(flags, 0x100u);
    }
}

// General blocks: [alpha beta, ||C_b||_1 ||C_b||_inf] per block from C and C^T rows.
template <typename VT>
__global__ void batch_general_bounds_kernel(const int64_t* __restrict__ blk_rows, const int64_t* __restrict__ rowptr,
                                            const int32_t* __restrict__ col, const VT* __restrict__ val,
                                            const int64_t* __restrict__ rowptrT, const int32_t* __restrict__ colT,
                                            const VT* __restrict__ valT, Params* bprm, uint32_t* flags) {
    __shared__ double sh[4][kThreads];
    const int b = blockIdx.x;
    double amin = INFINITY, rmax = 0.0, bmin = INFINITY, cmax = 0.0;
    for (int64_t i = blk_rows[b] + threadIdx.x; i < blk_rows[b + 1]; i += blockDim.x) {
        double dg = 0.0, r = 0.0, tot = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const double v = load_val_f64(val + k);
            tot += fabs(v);
            if (col[k] == i) dg += v; else r += fabs(v);
        }
        amin = fmin(amin, fabs(dg) - r);
        rmax = fmax(rmax, tot);
        double dgT = 0.0, s = 0.0, totT = 0.0;
        for (int64_t k = rowptrT[i]; k < rowptrT[i + 1]; ++k) {
            const double v = load_val_f64(valT + k);
            totT += fabs(v);
            if (colT[k] == i) dgT += v; else s += fabs(v);
        }
        bmin = fmin(bmin, fabs(dgT) - s);
        cmax = fmax(cmax, totT);
    }
    sh[0][threadIdx.x] = amin; sh[1][threadIdx.x] = rmax;
    sh[2][threadIdx.x] = bmin; sh[3][threadIdx.x] = cmax;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] = fmin(sh[0][threadIdx.x], sh[0][threadIdx.x + o]);
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double a = (sh[0][0] > 0.0 && sh[2][0] > 0.0) ? sh[0][0] * sh[2][0] : 0.0;
        double bb = sh[1][0] * sh[3][0];
        const int ok = finish_interval(a, bb, blk_rows[b + 1] - blk_rows[b]) ? 1 : 0;
        set_affine(bprm + b, a, bb);
        bprm[b].interval_ok = ok;
        if (!ok) atomicOr(flags, 0x100u);
    }
}

// Columns of block b must stay inside [blk_rows[b], blk_rows[b+1]) (flags bit 3).
__global__ void batch_check_blocks_kernel(const Tile* __restrict__ tiles, int64_t ntiles,
                                          const int64_t* __restrict__ blk_rows, const int64_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ col, uint32_t* flags) {
    uint32_t f = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const int64_t lo = blk_rows[tl.blk], hi = blk_rows[tl.blk + 1];
        for (int64_t i = tl.lo + threadIdx.x; i < tl.hi; i += blockDim.x)
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
                if (col[k] < lo || col[k] >= hi) f |= 8u;
    }
    if (f) atomicOr(flags, f);
}

cudaError_t launch_batch_aux(int what, int nb, int grid, cudaStream_t s, const BatchAuxArgs& a) {
    switch (what) {
        case 0: batch_set_seed_kernel<<<(nb + 255) / 256, 256, 0, s>>>(a.bprm, nb, a.seed); break;
        case 1: batch_set_intervals_kernel<<<(nb + 255) / 256, 256, 0, s>>>(a.bprm, nb, a.ab); break;
        case 2:
            batch_probe_bits_kernel<<<grid, kThreads, 0, s>>>(a.tiles, a.ntiles, a.nw, a.panel, a.bprm, a.blk_rows,
                                                              a.vbits);
            break;
        case 3: {
            dim3 g(nb, a.nsteps < 65535 ? a.nsteps : 65535);
            batch_reduce_kernel<<<g, kThreads, 0, s>>>(a.tpart, a.ntiles, a.tile_start, a.panel_width, a.mreal,
                                                       a.n, a.M, a.pbase, a.T);
            break;
        }
        case 4:
            switch (a.dtype) {
                case 0: batch_gershgorin_kernel<float><<<nb, kThreads, 0, s>>>(a.blk_rows, a.rowptr, a.col,
                                                                                static_cast<const float*>(a.val), a.bprm, a.flags); break;
                case 1: batch_gershgorin_kernel<bf16_t><<<nb, kThreads, 0, s>>>(a.blk_rows, a.rowptr, a.col,
                                                                                 static_cast<const bf16_t*>(a.val), a.bprm, a.flags); break;
                case 2: batch_gershgorin_kernel<double><<<nb, kThreads, 0, s>>>(a.blk_rows, a.rowptr, a.col,
                                                                                 static_cast<const double*>(a.val), a.bprm, a.flags); break;
                default: return cudaErrorInvalidValue;
            }
            break;
        case 5:
            switch (a.dtype) {
                case 0: batch_general_bounds_kernel<float><<<nb, kThreads, 0, s>>>(a.blk_rows, a.rowptr, a.col,
                            static_cast<const float*>(a.val), a.rowptrT, a.colT, static_cast<const float*>(a.valT), a.bprm, a.flags); break;
                case 1: batch_general_bounds_kernel<bf16_t><<<nb, kThreads, 0, s>>>(a.blk_rows, a.rowptr, a.col,
                            static_cast<const bf16_t*>(a.val), a.rowptrT, a.colT, static_cast<const bf16_t*>(a.valT), a.bprm, a.flags); break;
                case 2: batch_general_bounds_kernel<double><<<nb, kThreads, 0, s>>>(a.blk_rows, a.rowptr, a.col,
                            static_cast<const double*>(a.val), a.rowptrT, a.colT, static_cast<const double*>(a.valT), a.bprm, a.flags); break;
                default: return cudaErrorInvalidValue;
            }
            break;
        case 6:
            batch_check_blocks_kernel<<<grid, kThreads, 0, s>>>(a.tiles, a.ntiles, a.blk_rows, a.rowptr, a.col, a.flags);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cld
