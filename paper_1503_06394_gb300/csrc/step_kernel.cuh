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

#include <atomic>

#include "cld_internal.cuh"

namespace cld {

__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ldcs4(const float* p) {
    return __ldcs(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }


// Column indices and values of the chunk of CH stored entries starting at kb
// (entries at or beyond k1 read as column 0, value 0), spread over the LPR
// lanes of a row's group: lane lig holds entries e * LPR + lig, e < E.  CSR
// streams are read with the evict-first policy so they do not displace
// gathered rows of w_j from L2.
template <int CH, int E, int LPR, typename VT>
__device__ __forceinline__ void load_chunk(int64_t kb, int64_t k1, const int32_t* __restrict__ col,
                                           const VT* __restrict__ val, int lig, int (&cr)[E], float (&vr)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = e * LPR + lig;  // entry of the chunk this lane loads
        const int64_t k = kb + idx;
        const bool ok = idx < CH && k < k1;
        cr[e] = ok ? __ldcs(col + k) : 0;
        vr[e] = ok ? load_val_cs(val + k) : 0.f;
    }
}

// Row product over [k0, k1) in chunks of CH entries whose first chunk is
// already in (creg, vreg): the pairs are broadcast with group-masked shuffles,
// all CH row gathers are issued back to back, and the next chunk's pairs are
// loaded before the current chunk's gathers are consumed.
template <int MP, int GATHER, int CH, int E, typename VT>
__device__ __forceinline__ float4 chunk_product(int64_t k0, int64_t k1, int (&creg)[E], float (&vreg)[E],
                                                const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                const float* __restrict__ x, const uint32_t* __restrict__ vbits,
                                                int lig, int p0, int wsel, int bsh, float4 mask, unsigned gmask) {
    constexpr int LPR = MP / 4;
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int cnext[E];
    float vnext[E];
    for (int64_t k = k0; k < k1; k += CH) {
        if (k + CH < k1) load_chunk<CH, E, LPR>(k + CH, k1, col, val, lig, cnext, vnext);
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
    return acc;
}

// Entries per chunk of the cooperative variants (1: 8, 2: 4).
template <int IMPL>
struct ChunkSize { static constexpr int value = IMPL == 2 ? 4 : 8; };

// acc += sum over the stored entries [k0, k1) of one row, in entry order:
// each lane loads the (index, value) pairs of 4 entries at a time itself, then
// gathers those 4 rows (4 gathers in flight per group).  The whole row product
// of variant 0, and the entries past the staged chunk of the ring variants.
template <int MP, int GATHER, typename VT>
__device__ __forceinline__ float4 tail_product(float4 acc, int64_t k0, int64_t k1, const int32_t* __restrict__ col,
                                               const VT* __restrict__ val, const float* __restrict__ x,
                                               const uint32_t* __restrict__ vbits, int p0, int wsel, int bsh,
                                               float4 mask) {
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
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
    return acc;
}

// Row product acc = sum_k X[row, k] * x[k, p0..p0+3] over the stored entries
// [k0, k1) of one row, for the four probes of this lane.
//
// IMPL 0: tail_product over the whole row.
// IMPL 1 (2): the LPR lanes of the group load the next 8 (4) (index, value) pairs
//         cooperatively (one coalesced access per lane) and chunk_product
//         consumes them.
// IMPL 3 and 4 (the shared-memory ring) do not go through row_product; see
// rows_ring.
//
// The shuffles of the cooperative variants name only the LPR lanes of the
// row's group (gmask): groups of one warp own rows of different lengths, so
// their chunk loops (and the last grid-stride round) diverge, and a full-warp
// mask would be undefined there.
template <int MP, int GATHER, int IMPL, typename VT>
__device__ __forceinline__ float4 row_product(int64_t k0, int64_t k1, const int32_t* __restrict__ col,
                                              const VT* __restrict__ val, const float* __restrict__ x,
                                              const uint32_t* __restrict__ vbits, int lig, int p0,
                                              int wsel, int bsh, float4 mask, unsigned gmask) {
    constexpr int LPR = MP / 4;
    if constexpr (IMPL == 0) {
        return tail_product<MP, GATHER>(make_float4(0.f, 0.f, 0.f, 0.f), k0, k1, col, val, x, vbits, p0, wsel, bsh,
                                        mask);
    } else {
        constexpr int CH = ChunkSize<IMPL>::value;
        constexpr int E = LPR >= CH ? 1 : CH / LPR;  // entries held per lane
        int creg[E];
        float vreg[E];
        load_chunk<CH, E, LPR>(k0, k1, col, val, lig, creg, vreg);
        return chunk_product<MP, GATHER, CH, E>(k0, k1, creg, vreg, col, val, x, vbits, lig, p0, wsel, bsh, mask,
                                                gmask);
    }
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

// Epilogue operands of one row that do not depend on its gathers: the signs
// v of the row, w_j's own row ("own"; v when PREV is 0) and w_{j-1} ("pv";
// v when PREV is 0 or 1).
struct RowOperands {
    float4 v, own, pv;
};

template <int MP, int PREV, int EPI>
__device__ __forceinline__ RowOperands row_operands(const StepArgs& args, int64_t row, int p0, int wsel, int bsh,
                                                    float4 mask) {
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    RowOperands o;
    if (EPI == 0) {
        o.v = o.own = o.pv = make_float4(0.f, 0.f, 0.f, 0.f);
        return o;
    }
    o.v = signs4(__ldg(args.vbits + row * NW + wsel), bsh, mask);
    o.own = (PREV == 0) ? o.v : ldg4(args.own + row * MP + p0);
    o.pv = (PREV == 2) ? ldcs4(args.wprev + row * MP + p0) : o.v;
    return o;
}

// Rows first, first + stride, ... below end, one per group (variants 0-2):
// each row's pointers (IMPL 1/2: loaded one row ahead), its product, then its
// epilogue operands and finish(row, acc, operands).
template <int MP, int GATHER, int PREV, int EPI, int IMPL, typename VT, class Finish>
__device__ __forceinline__ void rows_plain(const StepArgs& args, const VT* __restrict__ val, int64_t first,
                                           int64_t end, int64_t stride, int lig, int p0, int wsel, int bsh,
                                           float4 mask, unsigned gmask, Finish&& finish) {
    const int64_t* __restrict__ rowptr = args.rowptr;
    int64_t k0 = 0, k1 = 0;
    if (IMPL != 0 && first < end) {
        k0 = __ldg(rowptr + first);
        k1 = __ldg(rowptr + first + 1);
    }
    for (int64_t row = first; row < end; row += stride) {
        float4 acc;
        if (IMPL == 0) {
            k0 = __ldg(rowptr + row);
            k1 = __ldg(rowptr + row + 1);
            acc = row_product<MP, GATHER, IMPL>(k0, k1, args.col, val, args.x, args.vbits, lig, p0, wsel, bsh, mask,
                                                gmask);
        } else {
            // row pointers of this group's next row, loaded ahead
            int64_t n0 = 0, n1 = 0;
            if (row + stride < end) {
                n0 = __ldg(rowptr + row + stride);
                n1 = __ldg(rowptr + row + stride + 1);
            }
            acc = row_product<MP, GATHER, IMPL>(k0, k1, args.col, val, args.x, args.vbits, lig, p0, wsel, bsh, mask,
                                                gmask);
            k0 = n0;
            k1 = n1;
        }
        finish(row, acc, row_operands<MP, PREV, EPI>(args, row, p0, wsel, bsh, mask));
    }
}

// ---------------------------------------------------------------- ring
// Variants 3 and 4 stage the operands of a row in shared memory with
// cp.async (16 bytes per lane per row: the lane's four probes) instead of
// holding loads in flight in registers, so a group keeps the next row's
// gathers in flight while it consumes the current one without the register
// cost that would lower occupancy.  Per group and row: the first RC stored
// entries' rows of w_j (or, for sign gathers, the 4-byte sign word of each),
// w_j's own row and w_{j-1}'s row go to one of two stages; entries past RC are
// gathered directly (tail_product, same order).
template <int IMPL>
struct RingChunk { static constexpr int value = IMPL == 3 ? 5 : 8; };

// Dynamic shared memory of the ring variants (two stages of RC + 2 slots of
// 16 bytes per thread); 0 for the others.
__host__ __device__ constexpr int ring_bytes(int impl) {
    return impl == 3 ? 2 * (5 + 2) * kThreads * 16 : impl == 4 ? 2 * (8 + 2) * kThreads * 16 : 0;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rows first, first + stride, ... below end through the ring.  At the top
// of the iteration for row r the copies of r are in flight or done, the pairs
// and sign word of r + stride are in registers and the pointers of
// r + 2 stride too; the iteration issues the copies of r + stride, loads the
// pairs of r + 2 stride, waits for r's copies (leaving r + stride's in
// flight), and consumes r.  Each thread reads only the slots it copied, so
// its own cp.async.wait_group orders them; a slot is rewritten only by the
// same thread after its value was consumed (in-order issue).
template <int MP, int GATHER, int PREV, int EPI, int RC, typename VT, class Finish>
__device__ __forceinline__ void rows_ring(const StepArgs& args, const VT* __restrict__ val, int64_t first,
                                          int64_t end, int64_t stride, int lig, int p0, int wsel, int bsh,
                                          float4 mask, unsigned gmask, float4* ring, Finish&& finish) {
    constexpr int LPR = MP / 4;
    constexpr int NW = MP <= 32 ? 1 : MP / 32;
    constexpr int E = (RC + LPR - 1) / LPR;  // staged entries whose pairs a lane holds
    constexpr int SL = RC + 2;               // slots per stage
    constexpr bool kOwn = EPI == 1 && PREV != 0;
    constexpr bool kPrev = PREV == 2;
    const int64_t* __restrict__ rowptr = args.rowptr;
    auto slot = [&](int st, int q) -> float4* { return ring + (st * SL + q) * kThreads + threadIdx.x; };
    auto issue = [&](int st, int64_t row, int64_t k0, int64_t k1, const int (&cr)[E]) {
#pragma unroll
        for (int q = 0; q < RC; ++q) {
            const int c = __shfl_sync(gmask, cr[q / LPR], q % LPR, LPR);
            if (k0 + q < k1) {
                if (GATHER == 1)
                    cp_async4(slot(st, q), args.vbits + (int64_t)c * NW + wsel);
                else
                    cp_async16(slot(st, q), args.x + (int64_t)c * MP + p0);
            }
        }
        if (kOwn) cp_async16(slot(st, RC), args.own + row * MP + p0);
        if (kPrev) cp_async16(slot(st, RC + 1), args.wprev + row * MP + p0);
    };
    int64_t k0 = 0, k1 = 0, n0 = 0, n1 = 0, m0 = 0, m1 = 0;
    int cr[E], cn[E];
    float vr[E], vn[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        cr[e] = cn[e] = 0;
        vr[e] = vn[e] = 0.f;
    }
    uint32_t wr = 0, wn = 0;
    if (first < end) {
        k0 = __ldg(rowptr + first);
        k1 = __ldg(rowptr + first + 1);
        load_chunk<RC, E, LPR>(k0, k1, args.col, val, lig, cr, vr);
        if (EPI == 1) wr = __ldg(args.vbits + first * NW + wsel);
        issue(0, first, k0, k1, cr);
        if (first + stride < end) {
            n0 = __ldg(rowptr + first + stride);
            n1 = __ldg(rowptr + first + stride + 1);
            load_chunk<RC, E, LPR>(n0, n1, args.col, val, lig, cn, vn);
            if (EPI == 1) wn = __ldg(args.vbits + (first + stride) * NW + wsel);
            if (first + 2 * stride < end) {
                m0 = __ldg(rowptr + first + 2 * stride);
                m1 = __ldg(rowptr + first + 2 * stride + 1);
            }
        }
    }
    cp_async_commit();
    int st = 0;
    for (int64_t r = first; r < end; r += stride, st ^= 1) {
        const int64_t nr = r + stride;
        if (nr < end) issue(st ^ 1, nr, n0, n1, cn);
        cp_async_commit();
        int c2[E];
        float v2[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            c2[e] = 0;
            v2[e] = 0.f;
        }
        uint32_t w2 = 0;
        int64_t q0 = 0, q1 = 0;
        if (nr + stride < end) {
            load_chunk<RC, E, LPR>(m0, m1, args.col, val, lig, c2, v2);
            if (EPI == 1) w2 = __ldg(args.vbits + (nr + stride) * NW + wsel);
            if (nr + 2 * stride < end) {
                q0 = __ldg(rowptr + nr + 2 * stride);
                q1 = __ldg(rowptr + nr + 2 * stride + 1);
            }
        }
        cp_async_wait<1>();
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < RC; ++q) {
            const float av = __shfl_sync(gmask, vr[q / LPR], q % LPR, LPR);
            if (k0 + q < k1) {
                const float4 xv = GATHER == 1 ? signs4(*reinterpret_cast<const uint32_t*>(slot(st, q)), bsh, mask)
                                              : *slot(st, q);
                acc.x = fmaf(av, xv.x, acc.x);
                acc.y = fmaf(av, xv.y, acc.y);
                acc.z = fmaf(av, xv.z, acc.z);
                acc.w = fmaf(av, xv.w, acc.w);
            }
        }
        if (k0 + RC < k1)
            acc = tail_product<MP, GATHER>(acc, k0 + RC, k1, args.col, val, args.x, args.vbits, p0, wsel, bsh, mask);
        RowOperands o;
        if (EPI == 0) {
            o.v = o.own = o.pv = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            o.v = signs4(wr, bsh, mask);
            o.own = kOwn ? *slot(st, RC) : o.v;
            o.pv = kPrev ? *slot(st, RC + 1) : o.v;
        }
        finish(r, acc, o);
        k0 = n0;
        k1 = n1;
        n0 = m0;
        n1 = m1;
        m0 = q0;
        m1 = q1;
        wr = wn;
        wn = w2;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            vr[e] = vn[e];
            cn[e] = c2[e];
            vn[e] = v2[e];
        }
    }
    cp_async_wait<0>();
}

// The row loop of variant IMPL.
template <int MP, int GATHER, int PREV, int EPI, int IMPL, typename VT, class Finish>
__device__ __forceinline__ void rows_all(const StepArgs& args, const VT* __restrict__ val, int64_t first,
                                         int64_t end, int64_t stride, int lig, int p0, int wsel, int bsh,
                                         float4 mask, unsigned gmask, float4* ring, Finish&& finish) {
    if constexpr (IMPL >= 3)
        rows_ring<MP, GATHER, PREV, EPI, RingChunk<IMPL>::value>(args, val, first, end, stride, lig, p0, wsel, bsh,
                                                                 mask, gmask, ring, finish);
    else
        rows_plain<MP, GATHER, PREV, EPI, IMPL>(args, val, first, end, stride, lig, p0, wsel, bsh, mask, gmask,
                                                finish);
}

// Resident-CTA targets per variant (256 threads): 6 (40 registers), 3, 4;
// the ring variants are bounded by their shared memory (3 and 2 CTAs).
template <int IMPL, int GATHER = 0>
struct StepOccupancy {
    static constexpr int value = IMPL == 0 ? 6 : IMPL == 1 ? 3 : IMPL == 2 ? 4 : IMPL == 3 ? 3 : 2;
};

// Dynamic shared memory of one instantiation.
template <int IMPL, int GATHER>
constexpr int step_smem() { return ring_bytes(IMPL); }

// Opts kernel K into `bytes` of dynamic shared memory on the current device,
// once per device (the attributes are per device; ordinals >= 64 set them on
// every call), before the first launch or occupancy query.  Needed when the
// dynamic and static shared memory together pass 48 KB; the static size is
// read from the kernel's attributes.  With `ctas` > 0 it also asks for the
// smallest shared-memory carveout that holds `ctas` CTAs per SM (dynamic +
// static + the per-CTA reservation each; fewer if the SM cannot hold that
// many): left to itself the driver may take a smaller one (more L1, or room
// for a kernel launched early beside it), and a kernel whose grid assumes
// `ctas` resident CTAs per SM then runs in 1.5 waves.
template <auto K>
cudaError_t smem_opt_in(int bytes, int ctas = 0) {
    if (ctas == 0 && bytes <= 48 * 1024) return cudaSuccess;
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit != 0 && (done.load(std::memory_order_acquire) & bit) != 0) return cudaSuccess;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, K);
    if (e != cudaSuccess) return e;
    const long long stat = (long long)fa.sharedSizeBytes;
    if (bytes + stat > 48 * 1024) {
        e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    if (ctas > 0) {
        int per_sm = 0, reserved = 0;
        e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e != cudaSuccess) return e;
        const long long per_cta = bytes + stat + reserved;
        long long want = ctas;  // as many of `ctas` as the SM can hold
        while (want > 1 && want * per_cta > per_sm) --want;
        long long pct = per_sm > 0 ? (100 * want * per_cta + per_sm - 1) / per_sm : 100;
        if (pct > 100) pct = 100;
        e = cudaFuncSetAttribute(K, cudaFuncAttributePreferredSharedMemoryCarveout, (int)pct);
        if (e != cudaSuccess) return e;
    }
    if (bit != 0) done.fetch_or(bit, std::memory_order_acq_rel);
    return cudaSuccess;
}

template <int MP, typename VT, int GATHER, int PREV, int EPI, int IMPL>
__global__ void __launch_bounds__(kThreads, (StepOccupancy<IMPL, GATHER>::value)) step_kernel(const StepArgs args);

template <int MP, typename VT, int GATHER, int PREV, int EPI, int IMPL>
__global__ void __launch_bounds__(kThreads, (StepOccupancy<IMPL, GATHER>::value)) step_kernel(const StepArgs args) {
    pdl_wait();  // w_j, w_{j-1}, the signs and the parameters come from earlier kernels
    pdl_trigger();
    constexpr int LPR = MP / 4;          // lanes per row
    constexpr int GPW = 32 / LPR;        // rows per warp
    constexpr int WPB = kThreads / 32;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int lig = lane % LPR;
    const int g_in_w = lane / LPR;
    const int64_t gid = ((int64_t)blockIdx.x * WPB + warp) * GPW + g_in_w;
    const int64_t ngroups = (int64_t)gridDim.x * WPB * GPW;

    const int p0 = 4 * lig;
    const int wsel = p0 >> 5;
    const int bsh = p0 & 31;
    const float4 mask = make_float4(p0 < args.mreal ? 1.f : 0.f, p0 + 1 < args.mreal ? 1.f : 0.f,
                                    p0 + 2 < args.mreal ? 1.f : 0.f, p0 + 3 < args.mreal ? 1.f : 0.f);
    const VT* __restrict__ val = static_cast<const VT*>(args.val);

    float scale = 1.f, scale_lo = 0.f, shift = 0.f, shift_lo = 0.f;
    if (EPI == 1) {
        scale = args.prm->scale_hi;
        scale_lo = args.prm->scale_lo;
        shift = args.prm->shift_hi;
        shift_lo = args.prm->shift_lo;
    }

    float4 tacc = make_float4(0.f, 0.f, 0.f, 0.f);
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (g_in_w * LPR));
    auto finish = [&](int64_t row, const float4& acc, const RowOperands& o) {
        float4 res;
        if (EPI == 0) {
            res = acc;
        } else {
            res = recurrence_update<PREV>(acc, o.own, o.pv, scale, scale_lo, shift, shift_lo);
            tacc.x = fmaf(o.v.x, res.x, tacc.x);
            tacc.y = fmaf(o.v.y, res.y, tacc.y);
            tacc.z = fmaf(o.v.z, res.z, tacc.z);
            tacc.w = fmaf(o.v.w, res.w, tacc.w);
        }
        st4(args.out + row * MP + p0, res);
    };
    extern __shared__ float4 ring[];
    rows_all<MP, GATHER, PREV, EPI, IMPL>(args, val, gid, args.d, ngroups, lig, p0, wsel, bsh, mask, gmask, ring,
                                          finish);

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

}  // namespace cld
