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
