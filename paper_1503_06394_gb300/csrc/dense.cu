// Dense kernel-matrix path: the recurrence step w_{j+1} = 2 At w_j - w_{j-1}
// (Sec. 2.2) when B is a dense d x d matrix stored in BF16, as a tensor-core
// GEMM on sm_103a (tcgen05 + TMA + TMEM).
//
// Work: 128-row tiles of the output (the MMA M) times all P probes (the MMA
// N), each over K = d in blocks of 64 columns.  The (tile, K block) units are
// split evenly over a persistent grid of as many CTAs as fit the GPU at once
// (stream-K): each CTA takes a contiguous range of units, so one holds whole
// tiles or pieces of up to a few.  (One CTA per tile left 48 of 152 SMs with
// a single CTA at d = 32768, and one CTA's ring cannot keep an SM's share of
// HBM busy: 88 % of the copy peak, 95 % when every SM held two.)
//
// Per CTA (192 threads): warp 4 brings each unit's B tile (128 rows x 64
// columns, 128-byte swizzled) and W_j tiles to shared memory by TMA through
// a ring of stages; warp 5 issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32
// in TMEM) and tcgen05.commit frees each stage; warps 0-3 (the four TMEM lane
// quarters) read a finished piece's accumulators and either apply the
// recurrence epilogue (a whole tile) or store the piece's 128 x P partial sums
// to the workspace.  The CTA that completes a tile's last piece (a per-tile
// counter) adds the pieces in piece order and applies the epilogue, so no CTA
// waits for another and the sums do not depend on which finishes last.  At
// 32 and 64 probes TMEM holds two accumulator sets, so a piece's MMAs overlap
// the previous piece's epilogue.
//
// W_j enters the MMA as an exact three-way BF16 split, w = hi + mid + lo
// (hi = bf16(w), mid = bf16(w - hi), lo = bf16(w - hi - mid)): the MMA runs
// once per part, so B (w_hi + w_mid + w_lo) is accumulated in FP32 with about
// 24 significant bits of w, the accuracy of the FP32 recurrence.  The split is
// stored probe-major ([part][probe][row]), the K-major layout of the MMA's B
// operand, and double-buffered across steps.
//
// Every mbarrier wait is bounded; a wait that gives up sets *err, the roles
// wind down (their later waits give up too), and the CTA frees its TMEM once
// the MMAs it issued have completed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "cld_internal.cuh"

namespace cld {

constexpr int kDRows = 128;     // MMA M: rows of a tile
constexpr int kDK = 64;         // K per unit and stage: 64 BF16 = 128 bytes, one swizzle atom
constexpr int kDSplit = 3;      // parts of the BF16 split of W
constexpr int kDEpi = 128;      // epilogue threads: warps 0-3, one TMEM lane (tile row) each
constexpr int kDThreads = 192;  // + warp 4 (TMA producer) + warp 5 (MMA issuer)

struct DenseArgs {
    int64_t d;
    const float* own;        // W_j, d x P (PREV != 0)
    const float* wprev;      // W_{j-1} (PREV == 2)
    float* out;              // W_{j+1}
    __nv_bfloat16* xt_out;   // split of W_{j+1}: [3][P][dx]
    int64_t dx;              // row length of the split buffers
    const uint32_t* vbits;
    double* tpart;           // [ntiles][P]
    const Params* prm;
    int mreal;
    uint32_t* err;
    float* part;             // pieces' partial sums [ntiles][smax][128][P]
    int* cnt;                // per tile: pieces finished in this step (0 between steps)
    int smax;                // piece slots per tile
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"(map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (SBO), version 1 (sm_100 family).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4)                      // D format F32
           | (1u << 7)                    // A format BF16
           | (1u << 10)                   // B format BF16
           | ((uint32_t)(n >> 3) << 17)   // N
           | ((uint32_t)(m >> 4) << 24);  // M
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ the step
template <int P>
struct DenseSmem {
    // ring depth: 3 at P = 32 leaves room for two CTAs per SM (4 stages,
    // one CTA per SM, measured 35 % slower); 4 at P = 64; 2 at 128
    static constexpr int kStages = P == 32 ? 3 : P == 64 ? 4 : 2;
    static constexpr int kA = kDRows * kDK * 2;        // 16 KB
    static constexpr int kX = kDSplit * P * kDK * 2;   // 3 parts x P rows x 128 B
    static constexpr int kStage = kA + kX;
    // The i-th K block of a piece goes to TMEM accumulator i mod kAcc; the
    // kAcc accumulators are added in FP32 (round to nearest) in the epilogue.
    // The tensor cores' accumulation rounds each addition in a way that does
    // not average out: the error grows with the additions into one accumulator
    // that follow a large term (it showed as a probe-independent moment bias,
    // logdet -1.15 instead of about -0.02 for a near-identity d = 32768
    // matrix, -0.31 with 4 accumulators, -0.10 with 16).  So each tile also
    // takes its K blocks starting after its diagonal block, which comes last:
    // the large diagonal products meet few later additions.  (16 accumulators
    // need 512 TMEM columns, one CTA per SM: 35 % slower.)
    static constexpr int kAcc = 4;
    static constexpr int kBufs = P == 128 ? 1 : 2;  // accumulator sets (TMEM: 512 columns per SM)
    static constexpr uint32_t kTmemCols = (uint32_t)(kBufs * kAcc * P);  // 256, 512, 512
    static constexpr int kTr = kDRows * (P + 1) * 4;  // moment transpose [128][P+1]
    static constexpr int kBars = 2 * kStages + 2 * kBufs + 1;
    static constexpr int kBytes = kStage * kStages + kTr + 1024 /*align*/ + kBars * 8 + 32;
    // resident CTAs per SM the grid is sized for: two at 32 probes (shared
    // memory with the 1 KB per-CTA reservation, 2 x 256 TMEM columns, and the
    // launch bounds' register cap), one otherwise
    static constexpr int kPerSM = P == 32 ? 2 : 1;
    static_assert(kPerSM * (kBytes + 1024) <= 233472, "shared memory of the CTAs an SM holds");
    static_assert(kPerSM * kTmemCols <= 512, "TMEM columns of the CTAs an SM holds");
};

// Unit range of CTA c of G over U units, and the CTA holding unit x.
__host__ __device__ inline int64_t dense_u0(int64_t U, int64_t c, int64_t G) { return U * c / G; }
__host__ __device__ inline int64_t dense_owner(int64_t U, int64_t G, int64_t x) {
    int64_t c = x * G / U;
    while (c + 1 < G && dense_u0(U, c + 1, G) <= x) ++c;
    while (c > 0 && dense_u0(U, c, G) > x) --c;
    return c;
}

template <int P, int PREV>
__global__ void __launch_bounds__(kDThreads, DenseSmem<P>::kPerSM)
    dense_step_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                      const DenseArgs args) {
    using S = DenseSmem<P>;
    constexpr int NS = S::kStages;
    constexpr int kAcc = S::kAcc, kBufs = S::kBufs;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned ring (swizzle atoms)
    uint8_t* gbase = smem_raw + (base - raw);
    float* tr = reinterpret_cast<float*>(gbase + S::kStage * NS);  // [128][P+1]
    const uint32_t bars = base + S::kStage * NS + S::kTr;
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (NS + s); };
    auto accf = [&](int b) { return bars + 8u * (2 * NS + b); };
    auto acce = [&](int b) { return bars + 8u * (2 * NS + kBufs + b); };
    const uint32_t done = bars + 8u * (2 * NS + 2 * kBufs);
    uint8_t* misc = gbase + S::kStage * NS + S::kTr + S::kBars * 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(misc);
    int* fail = reinterpret_cast<int*>(misc + 4);
    int* lastflag = reinterpret_cast<int*>(misc + 8);
    volatile int* votes = reinterpret_cast<volatile int*>(misc + 16);  // one per epilogue warp

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t d = args.d;
    const int64_t ntiles = (d + kDRows - 1) / kDRows;
    const int nk = (int)((d + kDK - 1) / kDK);
    const int64_t U = ntiles * nk, G = gridDim.x;
    const int64_t u0 = dense_u0(U, blockIdx.x, G), u1 = dense_u0(U, blockIdx.x + 1, G);

    if (threadIdx.x == 0) {
        *fail = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), kDEpi / 32);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // TMEM: kBufs x kAcc x P FP32 columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(S::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // the next step may be scheduled now: its CTAs take an SM's place as ours
    // leave, and stream their first B tiles while ours finish
    pdl_trigger();

    if (warp == 4) {
        if (lane == 0) {
            // producer: unit u = tile u / nk, its (u mod nk)-th K block in the
            // tile's order, (kfirst + i) mod nk, so that the diagonal blocks
            // (columns row0 .. row0 + 127) come last
            auto kblock = [&](int64_t u) {
                const int64_t row0 = (u / nk) * kDRows;
                const int kfirst = (int)(((row0 + kDRows) / kDK) % nk);
                return (int)((kfirst + u % nk) % nk);
            };
            // the first ring fill's B tiles (written by no earlier kernel)
            // before waiting for the predecessor; then their W_j tiles
            const int64_t pre = u1 - u0 < NS ? u1 - u0 : NS;
            for (int64_t g = 0; g < pre; ++g) {
                const int s = (int)g;
                mbar_expect_tx(full(s), S::kStage);
                tma_load_2d(base + S::kStage * s, &tmA, full(s), kblock(u0 + g) * kDK, (int)(((u0 + g) / nk) * kDRows));
            }
            pdl_wait();
            for (int64_t g = 0; g < pre; ++g) {
                const uint32_t sa = base + S::kStage * (int)g;
                for (int q = 0; q < kDSplit; ++q)
                    tma_load_2d(sa + S::kA + q * P * kDK * 2, &tmX, full((int)g), kblock(u0 + g) * kDK, q * P);
            }
            int64_t issued = pre;
            for (int64_t g = pre; u0 + g < u1; ++g) {
                const int64_t u = u0 + g;
                const int64_t row0 = (u / nk) * kDRows;
                const int kx = kblock(u);
                const int s = (int)(g % NS);
                if (!mbar_wait(empty(s), (uint32_t)(((g / NS) - 1) & 1))) {
                    atomicExch(fail, 1);
                    break;
                }
                mbar_expect_tx(full(s), S::kStage);
                const uint32_t sa = base + S::kStage * s;
                tma_load_2d(sa, &tmA, full(s), kx * kDK, (int)row0);
                for (int q = 0; q < kDSplit; ++q)
                    tma_load_2d(sa + S::kA + q * P * kDK * 2, &tmX, full(s), kx * kDK, q * P);
                issued = g + 1;
            }
            if (*fail)  // copies in flight land before the CTA exits (bounded)
                for (int64_t g = issued > NS ? issued - NS : 0; g < issued; ++g)
                    mbar_wait(full((int)(g % NS)), (uint32_t)((g / NS) & 1));
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer: one piece (the CTA's units of one tile) per
            // accumulator set
            constexpr uint32_t idesc = idesc_bf16(kDRows, P);
            int64_t g = 0;
            int piece = 0;
            bool ok = true;
            for (int64_t ps = u0; ps < u1 && ok; ++piece) {
                const int64_t t = ps / nk;
                const int64_t pe = (t + 1) * nk < u1 ? (t + 1) * nk : u1;
                const int b = piece % kBufs, use = piece / kBufs;
                if (use >= 1 && !mbar_wait(acce(b), (uint32_t)((use - 1) & 1))) {
                    atomicExch(fail, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int64_t u = ps; u < pe; ++u, ++g) {
                    const int s = (int)(g % NS);
                    if (!mbar_wait(full(s), (uint32_t)((g / NS) & 1))) {
                        atomicExch(fail, 1);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = base + S::kStage * s;
                    const int i = (int)(u - ps);  // index within the piece
                    const uint32_t dcol = tmem + (uint32_t)((b * kAcc + i % kAcc) * P);
#pragma unroll
                    for (int kk = 0; kk < kDK / 16; ++kk) {
                        const uint64_t ad = smem_desc_sw128(sa + kk * 32);
#pragma unroll
                        for (int q = 0; q < kDSplit; ++q) {
                            const uint64_t bd = smem_desc_sw128(sa + S::kA + q * P * kDK * 2 + kk * 32);
                            // the first MMA of an accumulator in a piece overwrites
                            umma_bf16(dcol, ad, bd, idesc, (i >= kAcc || kk != 0 || q != 0) ? 1u : 0u);
                        }
                    }
                    umma_commit(empty(s));
                }
                if (!ok) break;
                umma_commit(accf(b));  // arrives once the piece's MMAs have completed
                ps = pe;
            }
            umma_commit(done);  // every MMA issued above has completed
        }
    } else {
        // epilogue warps: thread = TMEM lane = row of the tile; they read
        // w_j, w_{j-1} and the signs and write w_{j+1}, its split, the
        // partial sums and the counters: after the predecessor
        pdl_wait();
        constexpr int NW = P <= 32 ? 1 : P / 32;
        const float scale = args.prm->scale_hi, scale_lo = args.prm->scale_lo;
        const float shift = args.prm->shift_hi, shift_lo = args.prm->shift_lo;
        const uint32_t lanebase = tmem + ((uint32_t)(warp * 32) << 16);
        int piece = 0;
        for (int64_t ps = u0; ps < u1; ++piece) {
            const int64_t t = ps / nk;
            const int64_t pe = (t + 1) * nk < u1 ? (t + 1) * nk : u1;
            const int b = piece % kBufs, use = piece / kBufs;
            const int nacc = (int)(pe - ps < kAcc ? pe - ps : kAcc);  // accumulators written
            // the four warps decide together (a warp leaving alone would
            // strand the others at the named barriers below)
            const bool okw = __all_sync(0xffffffffu, mbar_wait(accf(b), (uint32_t)(use & 1)));
            if (lane == 0) votes[warp] = okw ? 1 : 0;
            asm volatile("bar.sync 1, %0;" ::"r"(kDEpi) : "memory");
            const bool ok = votes[0] && votes[1] && votes[2] && votes[3];
            asm volatile("bar.sync 1, %0;" ::"r"(kDEpi) : "memory");
            if (!ok) {
                atomicExch(fail, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int64_t row = t * kDRows + threadIdx.x;
            const bool live = row < d;
            const bool whole = ps == t * nk && pe == (t + 1) * nk;
            // the recurrence epilogue of columns c0 .. c0 + 31 from the tile
            // sums acc (w_{j+1} rows, its split, the moment terms)
            auto finish = [&](int c0, const float (&acc)[32]) {
                if (live) {
                    const uint32_t word = __ldg(args.vbits + row * NW + c0 / 32);
#pragma unroll
                    for (int qg = 0; qg < 32; qg += 4) {
                        float4 o4 = make_float4(0.f, 0.f, 0.f, 0.f), p4 = o4;
                        if (PREV != 0) o4 = __ldg(reinterpret_cast<const float4*>(args.own + row * P + c0 + qg));
                        if (PREV == 2) p4 = __ldg(reinterpret_cast<const float4*>(args.wprev + row * P + c0 + qg));
                        const float ov[4] = {o4.x, o4.y, o4.z, o4.w}, pvv[4] = {p4.x, p4.y, p4.z, p4.w};
                        float wv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int q = qg + e, p = c0 + q;
                            const float vm = p < args.mreal ? 1.f : 0.f;
                            const float v = vm * __uint_as_float(0x3f800000u | (((word >> q) & 1u) << 31));
                            const float own = PREV == 0 ? v : ov[e];
                            const float y = fmaf(scale, acc[q], -shift * own) + fmaf(scale_lo, acc[q], -shift_lo * own);
                            const float w = PREV == 0 ? y : fmaf(2.f, y, -(PREV == 1 ? v : pvv[e]));
                            wv[e] = w;
                            const __nv_bfloat16 hi = __float2bfloat16_rn(w);
                            const float r1 = w - __bfloat162float(hi);
                            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
                            const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
                            args.xt_out[(0 * P + p) * args.dx + row] = hi;
                            args.xt_out[(1 * P + p) * args.dx + row] = mid;
                            args.xt_out[(2 * P + p) * args.dx + row] = lo;
                            tr[threadIdx.x * (P + 1) + p] = v * w;
                        }
                        *reinterpret_cast<float4*>(args.out + row * P + c0 + qg) = make_float4(wv[0], wv[1], wv[2], wv[3]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q) tr[threadIdx.x * (P + 1) + c0 + q] = 0.f;
                }
            };
            // this piece's sums of columns c0 .. c0 + 31: the written
            // accumulators added in a fixed order
            auto piece_sums = [&](int c0, float (&acc)[32]) {
                tmem_ld32(lanebase + (uint32_t)(b * kAcc * P + c0), acc);
#pragma unroll 1
                for (int a = 1; a < nacc; ++a) {
                    float part[32];
                    tmem_ld32(lanebase + (uint32_t)((b * kAcc + a) * P + c0), part);
#pragma unroll
                    for (int q = 0; q < 32; ++q) acc[q] += part[q];
                }
            };
            auto release = [&]() {  // TMEM set b read: the MMA issuer may refill it
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(acce(b));
            };
            bool fin = whole;
            if (whole) {
#pragma unroll 1
                for (int c0 = 0; c0 < P; c0 += 32) {
                    float acc[32];
                    piece_sums(c0, acc);
                    finish(c0, acc);
                }
                release();
            } else {
                // a piece of a shared tile: its partial sums to slot
                // (this CTA - the tile's first CTA), then the tile's counter
                const int64_t cfirst = dense_owner(U, G, t * nk);
                const int np = (int)(dense_owner(U, G, (t + 1) * nk - 1) - cfirst + 1);
                const int slot = (int)(blockIdx.x - cfirst);
                float* mine = args.part + ((t * args.smax + slot) * kDRows + threadIdx.x) * P;
#pragma unroll 1
                for (int c0 = 0; c0 < P; c0 += 32) {
                    float acc[32];
                    piece_sums(c0, acc);
#pragma unroll
                    for (int q = 0; q < 32; q += 4)
                        *reinterpret_cast<float4*>(mine + c0 + q) = make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
                }
                release();
                __threadfence();
                asm volatile("bar.sync 1, %0;" ::"r"(kDEpi) : "memory");
                if (threadIdx.x == 0) *lastflag = atomicAdd(args.cnt + t, 1) == np - 1 ? 1 : 0;
                asm volatile("bar.sync 1, %0;" ::"r"(kDEpi) : "memory");
                fin = *lastflag != 0;
                if (fin) {
                    // the tile's last piece: all pieces, added in slot order
                    __threadfence();
                    if (threadIdx.x == 0) args.cnt[t] = 0;  // ready for the next step
                    const float* first = args.part + ((t * args.smax) * kDRows + threadIdx.x) * P;
#pragma unroll 1
                    for (int c0 = 0; c0 < P; c0 += 32) {
                        float acc[32];
#pragma unroll
                        for (int q = 0; q < 32; q += 4) {
                            const float4 a = __ldcg(reinterpret_cast<const float4*>(first + c0 + q));
                            acc[q] = a.x; acc[q + 1] = a.y; acc[q + 2] = a.z; acc[q + 3] = a.w;
                        }
#pragma unroll 1
                        for (int k = 1; k < np; ++k) {
                            const float* src = first + (int64_t)k * kDRows * P;
#pragma unroll
                            for (int q = 0; q < 32; q += 4) {
                                const float4 a = __ldcg(reinterpret_cast<const float4*>(src + c0 + q));
                                acc[q] += a.x; acc[q + 1] += a.y; acc[q + 2] += a.z; acc[q + 3] += a.w;
                            }
                        }
                        finish(c0, acc);
                    }
                }
            }
            if (fin) {
                // the tile's moment terms summed over its rows in order
                asm volatile("bar.sync 1, %0;" ::"r"(kDEpi) : "memory");
                for (int p = threadIdx.x; p < P; p += kDEpi) {
                    double s = 0.0;
                    for (int r = 0; r < kDRows; ++r) s += (double)tr[r * (P + 1) + p];
                    args.tpart[t * P + p] = s;
                }
                asm volatile("bar.sync 1, %0;" ::"r"(kDEpi) : "memory");
            }
            ps = pe;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *fail) atomicOr(args.err, 1u);
    // free TMEM once the MMAs issued have completed (bounded)
    if (warp == 0) {
        mbar_wait(done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols));
    }
}

// Split of the probe signs for the first step: hi = v (0 for padded probes),
// mid = lo = 0; rows >= d (up to dx) are 0.
__global__ void dense_sign_split_kernel(int64_t d, int64_t dx, int P, int mreal, const uint32_t* __restrict__ vbits,
                                        __nv_bfloat16* __restrict__ xt) {
    const int nw = P <= 32 ? 1 : P / 32;
    const int64_t total = (int64_t)kDSplit * P * dx;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx % dx;
        const int64_t pq = idx / dx;
        const int p = (int)(pq % P), q = (int)(pq / P);
        float v = 0.f;
        if (q == 0 && r < d && p < mreal) {
            const uint32_t word = vbits[r * nw + p / 32];
            v = ((word >> (p % 32)) & 1u) ? -1.f : 1.f;
        }
        xt[idx] = __float2bfloat16_rn(v);
    }
}

// Gershgorin bounds of a dense BF16 matrix: per-CTA min/max of
// B_ii -+ sum_{k != i} |B_ik| (one row per thread), then one CTA finishes.
__global__ void dense_gershgorin_kernel(int64_t d, int64_t ld, const __nv_bfloat16* __restrict__ B,
                                        double* partial) {
    __shared__ double shl[kThreads], shh[kThreads];
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        double r = 0.0;
        for (int64_t k = 0; k < d; ++k)
            if (k != i) r += fabs((double)__bfloat162float(B[i * ld + k]));
        const double dg = (double)__bfloat162float(B[i * ld + i]);
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
        partial[2 * blockIdx.x] = shl[0];
        partial[2 * blockIdx.x + 1] = shh[0];
    }
}

__global__ void dense_gershgorin_final_kernel(const double* partial, int nb, int64_t d, Params* prm,
                                              uint32_t* flags) {
    if (threadIdx.x != 0) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int b = 0; b < nb; ++b) {
        lo = fmin(lo, partial[2 * b]);
        hi = fmax(hi, partial[2 * b + 1]);
    }
    const int ok = finish_interval(lo, hi, d) ? 1 : 0;
    set_affine(prm, lo, hi);
    prm->interval_ok = ok;
    if (!ok) atomicOr(flags, 0x100u);
}

cudaError_t launch_dense_gershgorin(int64_t d, int64_t ld, const void* B, double* partial, int grid, Params* prm,
                                    uint32_t* flags, cudaStream_t s) {
    dense_gershgorin_kernel<<<grid, kThreads, 0, s>>>(d, ld, static_cast<const __nv_bfloat16*>(B), partial);
    dense_gershgorin_final_kernel<<<1, 32, 0, s>>>(partial, grid, d, prm, flags);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D BF16 map: inner extent `inner` (contiguous), `outer` rows `stride_elems`
// apart; box kDK x box_rows; 128-byte swizzle; out-of-range reads give 0.
static bool make_map(CUtensorMap* m, const void* ptr, int64_t inner, int64_t outer, int64_t stride_elems,
                     int box_rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)stride_elems * 2};
    cuuint32_t box[2] = {(cuuint32_t)kDK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Opts the dense kernel into its shared memory and the largest carveout
// (two CTAs need 210 KB at P = 32; the rest of a step needs little L1), once.
template <int P, int PREV>
static cudaError_t dense_opt_in() {
    static bool done = false;
    if (done) return cudaSuccess;
    const int smem = DenseSmem<P>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(dense_step_kernel<P, PREV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(dense_step_kernel<P, PREV>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess) done = true;
    return e;
}

int dense_threads_per_cta() { return kDThreads; }

// The stream-K schedule of a step: a persistent grid of as many CTAs as fit
// the GPU at once (at most one per unit), and the most pieces any tile is
// cut into (the slots of the partial-sum buffer).
cudaError_t dense_schedule(int P, int64_t d, int sms, int* grid, int* smax) {
    const int per_sm = P == 32 ? DenseSmem<32>::kPerSM : P == 64 ? DenseSmem<64>::kPerSM
                     : P == 128 ? DenseSmem<128>::kPerSM : 0;
    if (per_sm <= 0) return cudaErrorInvalidValue;
    const int64_t ntiles = (d + kDRows - 1) / kDRows, nk = (d + kDK - 1) / kDK, U = ntiles * nk;
    int64_t G = (int64_t)per_sm * (sms > 0 ? sms : 1);
    if (G > U) G = U;
    if (G < 1) G = 1;
    int64_t most = 1;
    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t np = dense_owner(U, G, (t + 1) * nk - 1) - dense_owner(U, G, t * nk) + 1;
        most = np > most ? np : most;
    }
    *grid = (int)G;
    *smax = (int)most;
    return cudaSuccess;
}

template <int P, int PREV>
static cudaError_t launch_dense_t(const CUtensorMap& a, const CUtensorMap& x, int grid, cudaStream_t s,
                                  const DenseArgs& args) {
    cudaError_t e = dense_opt_in<P, PREV>();
    if (e != cudaSuccess) return e;
    // programmatic stream serialization (see pdl_wait): a step's CTAs start
    // as the previous step's leave
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)kDThreads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)DenseSmem<P>::kBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, dense_step_kernel<P, PREV>, a, x, args);
}

// Host entry used by cld_api.cu.  B: d x d BF16 with leading dimension ld
// (elements); xt_in: the split of w_j ([3][P][dx]); prev: 0 first step,
// 1 second, 2 general; grid, part (ntiles x smax x 128 x P floats) and cnt
// (ntiles ints, zero before the first step) from dense_schedule.  Returns
// cudaErrorNotSupported when the tensor map cannot be encoded.
cudaError_t launch_dense_step(int P, int prev, int64_t d, int64_t ld, const void* B, const void* xt_in,
                              int64_t dx, const float* own, const float* wprev, float* out, void* xt_out,
                              const uint32_t* vbits, double* tpart, const Params* prm, int mreal, uint32_t* err,
                              float* part, int* cnt, int smax, int grid, cudaStream_t s) {
    CUtensorMap ma, mx;
    if (!make_map(&ma, B, d, d, ld, kDRows)) return cudaErrorNotSupported;
    // inner extent d: columns k >= d of the split (never written) read as 0
    if (!make_map(&mx, xt_in, d, (int64_t)kDSplit * P, dx, P)) return cudaErrorNotSupported;
    DenseArgs a{};
    a.d = d;
    a.own = own;
    a.wprev = wprev;
    a.out = out;
    a.xt_out = static_cast<__nv_bfloat16*>(xt_out);
    a.dx = dx;
    a.vbits = vbits;
    a.tpart = tpart;
    a.prm = prm;
    a.mreal = mreal;
    a.err = err;
    a.part = part;
    a.cnt = cnt;
    a.smax = smax;
#define CLD_DENSE_CASE(PP)                                                   \
    case PP:                                                                 \
        return prev == 0 ? launch_dense_t<PP, 0>(ma, mx, grid, s, a)         \
             : prev == 1 ? launch_dense_t<PP, 1>(ma, mx, grid, s, a)         \
                         : launch_dense_t<PP, 2>(ma, mx, grid, s, a);
    switch (P) {
        CLD_DENSE_CASE(32)
        CLD_DENSE_CASE(64)
        CLD_DENSE_CASE(128)
        default: return cudaErrorInvalidValue;
    }
#undef CLD_DENSE_CASE
}

cudaError_t launch_dense_sign_split(int64_t d, int64_t dx, int P, int mreal, const uint32_t* vbits, void* xt,
                                    int grid, cudaStream_t s) {
    dense_sign_split_kernel<<<grid, kThreads, 0, s>>>(d, dx, P, mreal, vbits, static_cast<__nv_bfloat16*>(xt));
    return cudaGetLastError();
}

}  // namespace cld
