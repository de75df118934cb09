// Recurrence step with staged tiles (inner-loop variant 6).
//
// The same step as step_kernel and step_kernel_wide (Algorithm 1, Sec. 2.2:
// w_{j+1} = 2 At w_j - w_{j-1} with At applied on the fly, t_{j+1,p} =
// v_p^T w_{j+1} reduced per CTA), for matrices whose gathers hit the caches
// (stencils, point clouds numbered by cell, small blocks).  There a row's
// cost is its chain of dependent loads -- row pointers, then the indices and
// values of each chunk, then the gathers, then the own row, the w_{j-1} row
// and the sign word -- not bandwidth.  Here everything but the gathers is
// streamed into shared memory ahead of use:
//
// * a CTA owns tiles of T = 2048 / P consecutive rows (tile blockIdx.x, then
//   every gridDim.x-th); one producer warp copies a tile's row pointers,
//   stored indices and values, own rows of w_j, rows of w_{j-1} and sign words
//   into a ring of NS (2 to 4) shared-memory stages with bulk asynchronous
//   copies (TMA, cp.async.bulk) that complete on the stage's "full" mbarrier,
//   up to NS - 1 tiles ahead of the consumers, while
// * eight consumer warps compute the tiles in order with the wide-lane
//   mapping of variant 5 (8 consecutive probes per lane, P / 8 lanes per
//   row, 4 gathers of 32 bytes in flight per lane), write w_{j+1} to global
//   memory and release the stage on its "empty" mbarrier.  (Two groups of 4
//   probes per lane, one in each half of the panel, made the shared-memory
//   reads contiguous but took two 16-byte gathers per entry instead of one
//   32-byte gather: slower, the L1 data path being the busiest unit.)
//
// A tile whose entries do not fit the stage (more than 16 per row on
// average; 12 for the shapes whose stages are cut to keep L1, StagedRing) is
// staged without its indices and values, which the consumers then read from
// global memory.  Bulk copies need 16-byte aligned addresses
// and sizes: the index and value ranges are widened to 16-byte boundaries
// (neighbouring rows' entries, never read), and the bytes that would pass
// the end of the row-pointer, index or value array are copied by plain loads
// instead.  The launcher uses this variant only when rowptr, col and val are
// 16-byte aligned.  Every mbarrier wait is bounded and taken by all lanes of
// a warp, which go on only if all of them saw the phase: a wait that gives up
// sets args.err and the CTA winds down (the producer first waits, bounded,
// for the copies still in flight).  Row sums are formed in entry order with
// the update of recurrence_update, so w_{j+1} is identical to the other
// variants'.
#pragma once

#include "async_copy.cuh"
#include "step_wide.cuh"

namespace cld {

// Shape of one configuration: U stored entries in flight per lane, NC
// consumer warps per CTA (and one producer warp), MINB resident CTAs per SM.
template <int U_, int NC_, int MINB_>
struct StagedCfg {
    static constexpr int U = U_;
    static constexpr int NC = NC_;
    static constexpr int MINB = MINB_;
    static constexpr int threads = 32 * (NC + 1);
    // Shared memory (ring and static) one CTA may hold: MINB CTAs, with the
    // 1 KB the runtime reserves for each, fit the 196 KB shared-memory
    // carveout, so the SM keeps 60 KB of L1 for the gathers' lines in flight.
    // The next carveout (228 KB, 28 KB of L1) halved the speed of a batched
    // general step whose gathers miss L1.
    static constexpr int cta_bytes = 196 * 1024 / MINB - 1024;
};

template <int MP, int NC>
struct StagedGeom {
    static constexpr int PPL = 8;                      // probes per lane
    static constexpr int LPR = MP / PPL;               // lanes per row
    static constexpr int RPW = 32 / LPR;               // rows per consumer warp
    static constexpr int T = NC * RPW;                 // rows per tile (256 NC / MP)
    static constexpr int NW = MP <= 32 ? 1 : MP / 32;  // sign words per row
};

__host__ __device__ constexpr int staged_up16(int x) { return (x + 15) / 16 * 16; }

// Ring shape from a stage's size at a given entry capacity (`stage_of(capr)`:
// bytes of one stage holding capr stored entries a row) and the static shared
// memory at a given stage count (`static_of(ns)`, an upper bound): 16 entries a
// row if three stages fit the CTA's share, or if two do and 12 entries would
// not make room for a third; else 12 if two stages fit; else 16 (the CTA then
// takes more than its share and the SM holds fewer CTAs or less L1); then as
// many stages (2 to 4) as fit.  (The third stage measured 2 % faster on the
// five-point grid at 64 probes, whose rows hold 5 entries.)  Tiles with more
// entries than the capacity read their indices and values from global memory.
template <class L, class C>
struct StagedRing {
    static constexpr bool fits(int capr, int ns) { return ns * L::stage_of(capr) + L::static_of(ns) <= C::cta_bytes; }
    static constexpr int capr = fits(16, 3) || (fits(16, 2) && !fits(12, 3)) ? 16 : fits(12, 2) ? 12 : 16;
    static constexpr int ns = fits(capr, 4) ? 4 : fits(capr, 3) ? 3 : 2;
};

// Sizes of the forward step's stage (at a given entry capacity) and static
// shared memory (at a given stage count).  BATCH: the tile-queue kernel, whose
// stages hold 3 rows beyond the tile's T (its copies start up to 3 rows early
// to sit on 16-byte boundaries) and whose static memory holds NS + 1 moment
// slots.
template <int MP, typename VT, int PREV, int EPI, class C, bool BATCH>
struct StagedSizes {
    using G = StagedGeom<MP, C::NC>;
    static constexpr int TR = G::T + (BATCH ? 3 : 0);  // rows a stage holds
    static constexpr bool kOwn = EPI == 1 && PREV != 0;
    static constexpr bool kPrev = EPI == 1 && PREV == 2;
    static constexpr bool kSigns = EPI == 1;
    static constexpr int rp_bytes = staged_up16((TR + 2) * 8);  // TR + 2 row pointers
    static constexpr int stage_of(int capr) {
        return staged_up16(rp_bytes + staged_up16(capr * G::T * 4) + staged_up16(capr * G::T * (int)sizeof(VT)) +
                           (kOwn ? TR * MP * 4 : 0) + (kPrev ? TR * MP * 4 : 0) +
                           (kSigns ? staged_up16(TR * G::NW * 4) : 0));
    }
    static constexpr int static_of(int ns) { return (kSigns ? (BATCH ? ns + 1 : 1) * C::NC * MP * 8 : 0) + 512; }
};

// Byte offsets of one stage's regions, the stages of the ring and the dynamic
// shared memory.
template <int MP, typename VT, int PREV, int EPI, class C, bool BATCH = false>
struct StagedLayout {
    using G = StagedGeom<MP, C::NC>;
    using Z = StagedSizes<MP, VT, PREV, EPI, C, BATCH>;
    using R = StagedRing<Z, C>;
    static constexpr int TR = Z::TR;
    static constexpr bool kOwn = Z::kOwn, kPrev = Z::kPrev, kSigns = Z::kSigns;
    static constexpr int CAP = R::capr * G::T;                            // stored entries a stage holds
    static constexpr int rp = 0;
    static constexpr int col = rp + Z::rp_bytes;                          // CAP indices
    static constexpr int val = col + staged_up16(CAP * 4);                // CAP values
    static constexpr int own = val + staged_up16(CAP * (int)sizeof(VT));
    static constexpr int prev = own + (kOwn ? TR * MP * 4 : 0);           // TR x P floats each
    static constexpr int sg = prev + (kPrev ? TR * MP * 4 : 0);           // TR x NW sign words
    static constexpr int stage = staged_up16(sg + (kSigns ? staged_up16(TR * G::NW * 4) : 0));
    static constexpr int NS = R::ns;
    static constexpr int bytes = NS * stage;
    static_assert(stage == Z::stage_of(R::capr), "stage regions and stage_of disagree");
};

template <typename VT>
__device__ __forceinline__ uint32_t smem_val_bits(const VT* p);
template <>
__device__ __forceinline__ uint32_t smem_val_bits<float>(const float* p) {
    return __float_as_uint(*p);
}
template <>
__device__ __forceinline__ uint32_t smem_val_bits<double>(const double* p) {
    return __float_as_uint((float)*p);
}
template <>
__device__ __forceinline__ uint32_t smem_val_bits<bf16_t>(const bf16_t* p) {
    return (uint32_t)(*reinterpret_cast<const unsigned short*>(p)) << 16;
}

// Bounds and copies of one tile for the producer warp: row pointers
// r0 - pre .. r0 + rows, the stored indices and values of entries [k0, k1)
// (and, with H, the per-entry FP32 accumulators of the same range), up to
// three blocks of `pre + rows` x MP floats starting at row r0 - pre, and those
// rows' sign words, into the stage at `st` (byte offsets o_*; a null source
// or a negative offset: not staged).  pre (0 .. 3) puts row-indexed copies on
// 16-byte boundaries when r0 is not a multiple of 4 (batch tiles); the pre
// rows are copied, never used.  Lane 0 registers the bytes on the stage's mbarrier and issues the
// bulk copies; lanes 1 .. 15 copy what the bulk copies must leave out at the
// ends of the arrays; every lane then arrives once (the barrier expects 32).
// The index range is widened to 16-byte boundaries; if it holds more than
// cap entries, indices, values and H stay in global memory (hdr_staged = 0).
template <int MP, int NW, typename VT>
__device__ __forceinline__ void staged_fill_tile(int lane, unsigned char* st, uint32_t bar, int64_t r0, int rows,
                                                 int pre, int64_t d, int64_t k0, int64_t k1, int64_t nnz, int cap,
                                                 const int64_t* rowptr, const int32_t* col, const VT* val,
                                                 const float* H, const float* v0, const float* v1, const float* v2,
                                                 const uint32_t* vbits, int o_rp, int o_col, int o_val, int o_h,
                                                 int o_v0, int o_v1, int o_v2, int o_sg, int64_t& hdr_kc,
                                                 int64_t& hdr_kv, int& hdr_staged) {
    constexpr int UV = 16 / (int)sizeof(VT);  // values per 16 bytes
    const int64_t ra = r0 - pre;  // first staged row
    const int nrow = rows + pre;  // staged rows
    // row pointers ra .. r0 + rows
    uint32_t rp_bulk = (uint32_t)(nrow + 1) * 8u;
    bool rp_tail = false;
    if (rp_bulk & 15u) {
        if (r0 + rows + 1 <= d) {
            rp_bulk += 8u;  // one more (valid) row pointer
        } else {
            rp_bulk -= 8u;  // the last one by a plain load
            rp_tail = true;
        }
    }
    // index and value ranges widened to 16-byte boundaries, clamped at nnz
    const int64_t ka = k0 & ~(int64_t)3, kz = (k1 + 3) & ~(int64_t)3;
    const int64_t kzb = kz <= nnz ? kz : (nnz & ~(int64_t)3);
    const int64_t kva = k0 & ~(int64_t)(UV - 1), kvz = (k1 + UV - 1) & ~(int64_t)(UV - 1);
    const int64_t kvzb = kvz <= nnz ? kvz : (nnz & ~(int64_t)(UV - 1));
    const bool staged = kz - ka <= cap && kvz - kva <= cap;
    const uint32_t col_bytes = staged ? (uint32_t)(kzb - ka) * 4u : 0u;
    const uint32_t h_bytes = H != nullptr ? col_bytes : 0u;
    const uint32_t val_bytes = staged ? (uint32_t)(kvzb - kva) * (uint32_t)sizeof(VT) : 0u;
    const uint32_t vec_bytes = (uint32_t)nrow * MP * 4u;
    const uint32_t sg_bytes = o_sg >= 0 ? (uint32_t)staged_up16(nrow * NW * 4) : 0u;
    if (lane == 0) {
        hdr_kc = ka;
        hdr_kv = kva;
        hdr_staged = staged ? 1 : 0;
        const uint32_t tx = rp_bulk + col_bytes + h_bytes + val_bytes + (v0 ? vec_bytes : 0u) +
                            (v1 ? vec_bytes : 0u) + (v2 ? vec_bytes : 0u) + sg_bytes;
        mbar_expect_tx(bar, tx);
        bulk_g2s(smem_u32(st + o_rp), rowptr + ra, rp_bulk, bar);
        if (col_bytes) bulk_g2s(smem_u32(st + o_col), col + ka, col_bytes, bar);
        if (h_bytes) bulk_g2s(smem_u32(st + o_h), H + ka, h_bytes, bar);
        if (val_bytes) bulk_g2s(smem_u32(st + o_val), val + kva, val_bytes, bar);
        if (v0) bulk_g2s(smem_u32(st + o_v0), v0 + ra * MP, vec_bytes, bar);
        if (v1) bulk_g2s(smem_u32(st + o_v1), v1 + ra * MP, vec_bytes, bar);
        if (v2) bulk_g2s(smem_u32(st + o_v2), v2 + ra * MP, vec_bytes, bar);
        if (sg_bytes) bulk_g2s(smem_u32(st + o_sg), vbits + ra * NW, sg_bytes, bar);
    } else {
        if (lane == 1 && rp_tail) reinterpret_cast<int64_t*>(st + o_rp)[nrow] = __ldg(rowptr + r0 + rows);
        if (staged && lane >= 2 && lane < 6) {
            const int64_t e = kzb + (lane - 2);
            if (e < k1) {
                reinterpret_cast<int32_t*>(st + o_col)[e - ka] = __ldg(col + e);
                if (H != nullptr) reinterpret_cast<float*>(st + o_h)[e - ka] = H[e];
            }
        }
        if (staged && lane >= 8 && lane < 8 + UV) {
            const int64_t e = kvzb + (lane - 8);
            if (e < k1) {
                const unsigned short* src = reinterpret_cast<const unsigned short*>(val + e);
                unsigned short* dst = reinterpret_cast<unsigned short*>(st + o_val + (e - kva) * sizeof(VT));
#pragma unroll
                for (int h = 0; h < (int)sizeof(VT) / 2; ++h) dst[h] = __ldg(src + h);
            }
        }
        mbar_arrive(bar);
    }
}

// The producer warp's loop over the CTA's tiles (blockIdx.x, then every
// gridDim.x-th): wait until the stage is free (bounded, all lanes), fill it
// with fill(stage, tile, r0, rows, k0, k1), and load the next tile's entry
// bounds while the copies fly.  A tile equal to withhold_tile - 1 is neither
// copied nor announced (a testing aid: its consumers' waits run out).  If a
// wait gives up: set bit 0 of *err and wait (bounded) for the copies of the
// last NS iterations, which may still be in flight.
template <int NS, int T, class Fill>
__device__ __forceinline__ void staged_producer_loop(int lane, int64_t mine, int64_t d, const int64_t* rowptr,
                                                     int64_t withhold_tile, uint32_t* err, const uint64_t* bars,
                                                     Fill&& fill) {
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[NS + s]); };
    int64_t started = 0;       // iterations whose stage was filled (or withheld)
    int64_t withheld_it = -1;  // the iteration of the withheld tile, if any
    bool ok = true;
    int64_t k0 = 0, k1 = 0;
    if (mine > 0) {
        const int64_t r0 = (int64_t)blockIdx.x * T;
        k0 = __ldg(rowptr + r0);
        k1 = __ldg(rowptr + (r0 + T < d ? r0 + T : d));
    }
    for (int64_t i = 0; i < mine; ++i) {
        const int s = (int)(i % NS);
        const int64_t use = i / NS;  // how often stage s was filled before
        // every lane waits; the warp goes on only if all of them saw the phase
        if (use >= 1 && !__all_sync(0xffffffffu, mbar_wait(empty(s), (uint32_t)((use + 1) & 1)))) {
            ok = false;
            break;
        }
        const int64_t t = (int64_t)blockIdx.x + i * gridDim.x;
        const int64_t r0 = t * T;
        const int rows = (int)(d - r0 < T ? d - r0 : T);
        if (withhold_tile == t + 1) {
            withheld_it = i;  // neither copies nor arrivals for this stage
        } else {
            fill(s, full(s), r0, rows, k0, k1);
        }
        started = i + 1;
        // bounds of the next tile, loaded while the stage fills
        if (i + 1 < mine) {
            const int64_t rn = (t + gridDim.x) * T;
            k0 = __ldg(rowptr + rn);
            k1 = __ldg(rowptr + (rn + T < d ? rn + T : d));
        }
    }
    if (!ok) {
        if (lane == 0) atomicOr(err, 1u);
        for (int64_t j = started > NS ? started - NS : 0; j < started; ++j)
            if (j != withheld_it) mbar_wait(full((int)(j % NS)), (uint32_t)((j / NS) & 1));
    }
}

template <int MP, typename VT, int GATHER, int PREV, int EPI, class C>
__global__ void __launch_bounds__(C::threads, C::MINB) step_kernel_staged(const StepArgs args) {
    static_assert(MP >= 8, "staged tiles need at least 8 probes per panel");
    using G = StagedGeom<MP, C::NC>;
    using S = StagedLayout<MP, VT, PREV, EPI, C>;
    constexpr int PPL = G::PPL, LPR = G::LPR, RPW = G::RPW, T = G::T, NW = G::NW, NS = S::NS;
    constexpr int U = C::U;                   // stored entries in flight per lane
    constexpr int NC = C::NC;                 // consumer warps
    // padded probes: signs are masked where v itself enters the result
    constexpr bool kMask = GATHER == 1 || (EPI == 1 && PREV != 2);

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2 * NS];  // full[0 .. NS), empty[0 .. NS)
    __shared__ int64_t hdr_kc[NS], hdr_kv[NS];      // first staged index / value entry
    __shared__ int hdr_staged[NS];
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
    pdl_wait();  // w_j, w_{j-1}, the signs and the parameters come from earlier kernels
    // No early trigger: the next kernel's CTAs are placed when this one ends,
    // with their own shared-memory carveout (batched general steps alternate
    // this kernel with the batched C^T step, whose carveout differs).

    const int64_t d = args.d;
    const int64_t ntiles = (d + T - 1) / T;
    const int64_t mine = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const VT* __restrict__ val = static_cast<const VT*>(args.val);
    const int64_t* __restrict__ rowptr = args.rowptr;

    if (warp == NC) {
        // ------------------------------------------------------------ producer
        const int64_t nnz = __ldg(rowptr + d);
        staged_producer_loop<NS, T>(lane, mine, d, rowptr, args.withhold_tile, args.err, bars,
                                    [&](int s, uint32_t bar, int64_t r0, int rows, int64_t k0, int64_t k1) {
            staged_fill_tile<MP, NW, VT>(lane, smem + s * S::stage, bar, r0, rows, 0, d, k0, k1, nnz, S::CAP, rowptr,
                                         args.col, val, nullptr, S::kOwn ? args.own : nullptr,
                                         S::kPrev ? args.wprev : nullptr, nullptr, args.vbits, S::rp, S::col,
                                         S::val, -1, S::own, S::prev, -1, S::kSigns ? S::sg : -1, hdr_kc[s],
                                         hdr_kv[s], hdr_staged[s]);
        });
    } else {
        // ------------------------------------------------------------ consumers
        const int sub = lane % LPR;
        const int g_in_w = lane / LPR;
        const int lr = warp * RPW + g_in_w;  // this lane's row within a tile
        const int q0 = sub * PPL;
        const int wsel = q0 >> 5, bsh = q0 & 31;
        float mk[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) mk[q] = (!kMask || q0 + q < args.mreal) ? 1.f : 0.f;
        const int64_t kend = value_end<VT>(rowptr, d);
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
                const int64_t* rp = reinterpret_cast<const int64_t*>(st + S::rp);
                const int64_t k0 = rp[lr], k1 = rp[lr + 1];
                float acc[PPL];
#pragma unroll
                for (int q = 0; q < PPL; ++q) acc[q] = 0.f;
                // gathers of U entries whose indices and value bits are in c / ab
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
                    const int dv = (int)(hdr_kc[s] - hdr_kv[s]);  // value slot = index slot + dv
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
                    const bool edge = std::is_same<VT, bf16_t>::value && (k0 == 0 || k1 == kend);
                    for (int64_t k = k0; k < k1; k += U) {
                        int c[U];
                        uint32_t ab[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const bool ok = k + u < k1;
                            c[u] = ok ? __ldg(args.col + k + u) : -1;
                            ab[u] = ok ? load_bits(val, k + u, edge) : 0u;
                        }
                        consume(c, ab);
                    }
                }
                float res[PPL];
                if (EPI == 0) {
#pragma unroll
                    for (int q = 0; q < PPL; ++q) res[q] = acc[q];
                } else {
                    float v[PPL], own[PPL], pv[PPL];
                    const uint32_t* sg = reinterpret_cast<const uint32_t*>(st + S::sg);
                    signs8(sg[lr * NW + wsel], bsh, mk, v);
                    if (S::kOwn) {
                        const float4* o4 = reinterpret_cast<const float4*>(st + S::own + (lr * MP + q0) * 4);
                        const float4 a = o4[0], b = o4[1];
                        own[0] = a.x; own[1] = a.y; own[2] = a.z; own[3] = a.w;
                        own[4] = b.x; own[5] = b.y; own[6] = b.z; own[7] = b.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < PPL; ++q) own[q] = v[q];
                    }
                    if (S::kPrev) {
                        const float4* p4 = reinterpret_cast<const float4*>(st + S::prev + (lr * MP + q0) * 4);
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
                }
                const int64_t row = r0 + lr;
                st4(args.out + row * MP + q0, make_float4(res[0], res[1], res[2], res[3]));
                st4(args.out + row * MP + q0 + 4, make_float4(res[4], res[5], res[6], res[7]));
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty(s));
        }
        if (EPI == 1) {
            // lanes with the same `sub` hold the same probes: fold them
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                double t = tacc[q];
#pragma unroll
                for (int off = LPR; off < 32; off <<= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
                if (g_in_w == 0) red[warp][q0 + q] = t;
            }
        }
    }
    __syncthreads();
    if (EPI == 1) {
        // the consumer warps of the CTA in a fixed order
        for (int p = threadIdx.x; p < MP; p += blockDim.x) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NC; ++w) s += red[w][p];
            args.tpart[(int64_t)blockIdx.x * MP + p] = s;
        }
    }
}

}  // namespace cld
