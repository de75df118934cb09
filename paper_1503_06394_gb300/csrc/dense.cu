// Dense kernel-matrix path: the recurrence step w_{j+1} = 2 At w_j - w_{j-1}
// (Sec. 2.2) when B is a dense d x d matrix stored in BF16, as a tensor-core
// GEMM on sm_103a (tcgen05 + TMA + TMEM).
//
// Per CTA: 128 output rows (the MMA M), all P probes (the MMA N), the whole
// row of B as K.  B tiles (128 rows x 64 columns, 128-byte swizzled) and the
// matching W_j tiles are brought to shared memory by TMA through a ring of
// stages; one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in
// TMEM) and tcgen05.commit frees each stage; the four warps then read the
// 128 x P accumulator from TMEM and apply the recurrence epilogue.
//
// W_j enters the MMA as an exact three-way BF16 split, w = hi + mid + lo
// (hi = bf16(w), mid = bf16(w - hi), lo = bf16(w - hi - mid)): the MMA runs
// once per part, so B (w_hi + w_mid + w_lo) is accumulated in FP32 with about
// 24 significant bits of w, the accuracy of the FP32 recurrence.  The split is
// stored probe-major ([part][probe][row]), the K-major layout of the MMA's B
// operand, and double-buffered across steps.
//
// Every mbarrier wait is bounded; a wait that gives up sets *err, and the
// CTA still frees its TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "cld_internal.cuh"

namespace cld {

constexpr int kDRows = 128;     // MMA M: output rows per CTA
constexpr int kDK = 64;         // K per stage: 64 BF16 = 128 bytes, one swizzle atom
constexpr int kDSplit = 3;      // parts of the BF16 split of W
constexpr int kDThreads = 128;  // 4 warps: TMEM lane quarters 0..3

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
    // ring depth: 3 at P = 32 leaves room for two CTAs per SM (85 KB each),
    // so one CTA's epilogue overlaps another's main loop (4 stages, 113 KB,
    // measured 35 % slower); 4 at P = 64; 2 at 128
    static constexpr int kStages = P == 32 ? 3 : P == 64 ? 4 : 2;
    static constexpr int kA = kDRows * kDK * 2;        // 16 KB
    static constexpr int kX = kDSplit * P * kDK * 2;   // 3 parts x P rows x 128 B
    static constexpr int kStage = kA + kX;
    // the epilogue reuses the ring once every MMA has completed: the moment
    // transpose [128][P+1] and, per warp, a 32 x 33 tile for its rows of
    // w_j, w_{j-1} and w_{j+1} (coalesced loads and stores)
    // The i-th K block a CTA takes goes to TMEM accumulator i mod kAcc; the
    // kAcc accumulators are added in FP32 (round to nearest) in the epilogue.
    // The tensor cores' accumulation rounds each addition in a way that does
    // not average out: the error grows with the additions into one accumulator
    // that follow a large term (it showed as a probe-independent moment bias,
    // logdet -1.15 instead of about -0.02 for a near-identity d = 32768
    // matrix, -0.31 with 4 accumulators, -0.10 with 16).  So each CTA also
    // takes its K blocks starting after its diagonal block, which comes last:
    // the large diagonal products meet few later additions.  (16 accumulators
    // need 512 TMEM columns, one CTA per SM: 35 % slower.)
    static constexpr int kAcc = 4;
    static constexpr uint32_t kTmemCols = (uint32_t)(kAcc * P);  // 128, 256 or 512
    static constexpr int kTr = kDRows * (P + 1) * 4;
    static constexpr int kTile = 32 * 33 * 4;
    static_assert(kTr + 2 * (kDThreads / 32) * kTile <= kStage * kStages, "epilogue buffers must fit the ring");
    static constexpr int kBytes = kStage * kStages + 1024 /*align*/ + 256 /*barriers*/;
    static_assert(kBytes <= 232448, "shared memory");
};

template <int P, int PREV>
__global__ void __launch_bounds__(kDThreads, P == 32 ? 2 : 1)
    dense_step_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                      const DenseArgs args) {
    using S = DenseSmem<P>;
    constexpr int kDStages = S::kStages;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned ring (swizzle atoms)
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bars = base + S::kStage * kDStages;  // full[S], empty[S], accum
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + (2 * kDStages + 1) * 8 + S::kStage * kDStages);
    int* fail = reinterpret_cast<int*>(gbase + (2 * kDStages + 1) * 8 + 4 + S::kStage * kDStages);
    // epilogue buffers in the ring (valid once the accumulator is complete)
    float* tr = reinterpret_cast<float*>(gbase);  // [128][P+1]
    float* tile_own = reinterpret_cast<float*>(gbase + S::kTr + (threadIdx.x >> 5) * 2 * S::kTile);  // [32][33]
    float* tile_prev = tile_own + 32 * 33;
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (kDStages + s); };
    const uint32_t accum = bars + 8u * (2 * kDStages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * kDRows;
    const int nk = (int)((args.d + kDK - 1) / kDK);

    if (threadIdx.x == 0) {
        *fail = 0;
        for (int s = 0; s < kDStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // TMEM: P FP32 columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(S::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    int issued = 0;  // producer: stages loaded

    if (warp == 0 && lane == 0) {
        // producer: TMA into the ring; the i-th block taken is K block
        // (kfirst + i) mod nk, so that the diagonal blocks (columns row0 ..
        // row0 + 127) come last
        const int kfirst = (int)(((row0 + kDRows) / kDK) % nk);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kDStages;
            if (kb >= kDStages && !mbar_wait(empty(s), ((kb / kDStages) - 1) & 1)) {
                atomicExch(fail, 1);
                break;
            }
            mbar_expect_tx(full(s), S::kStage);
            const uint32_t sa = base + S::kStage * s;
            const int kx = (kfirst + kb) % nk;  // K block of this stage
            tma_load_2d(sa, &tmA, full(s), kx * kDK, (int)row0);
            for (int q = 0; q < kDSplit; ++q)
                tma_load_2d(sa + S::kA + q * P * kDK * 2, &tmX, full(s), kx * kDK, q * P);
            issued = kb + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(kDRows, P);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kDStages;
            if (!mbar_wait(full(s), (kb / kDStages) & 1)) {
                atomicExch(fail, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = base + S::kStage * s;
#pragma unroll
            for (int kk = 0; kk < kDK / 16; ++kk) {
                const uint64_t ad = smem_desc_sw128(sa + kk * 32);
#pragma unroll
                for (int q = 0; q < kDSplit; ++q) {
                    const uint64_t bd = smem_desc_sw128(sa + S::kA + q * P * kDK * 2 + kk * 32);
                    // accumulator kb mod kAcc; its first MMA overwrites
                    umma_bf16(tmem + (uint32_t)((kb % S::kAcc) * P), ad, bd, idesc,
                              (kb >= S::kAcc || kk != 0 || q != 0) ? 1u : 0u);
                }
            }
            umma_commit(empty(s));
        }
        umma_commit(accum);  // arrives once every MMA issued above has completed
    }
    // epilogue: row = row0 + threadIdx.x (TMEM lane = thread), P columns
    const bool got = mbar_wait(accum, 0);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool good = got && *fail == 0;
    const int64_t row = row0 + threadIdx.x;
    const bool live = row < args.d;
    if (good) {
        const float scale = args.prm->scale_hi, scale_lo = args.prm->scale_lo;
        const float shift = args.prm->shift_hi, shift_lo = args.prm->shift_lo;
        constexpr int NW = P <= 32 ? 1 : P / 32;
        // this warp's rows rw .. rw + nr - 1 (thread lane holds row rw + lane)
        const int64_t rw = row0 + warp * 32;
        const int nr = (int)(args.d - rw < 32 ? (args.d - rw > 0 ? args.d - rw : 0) : 32);
#pragma unroll 1
        for (int c0 = 0; c0 < P; c0 += 32) {
            float acc[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
            // the other accumulators, added in a fixed order (those that never
            // received an MMA, when nk < kAcc, are skipped)
#pragma unroll 1
            for (int a = 1; a < S::kAcc && a < nk; ++a) {
                float part[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * P + c0), part);
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[q] += part[q];
            }
            // columns c0 .. c0 + 31 of w_j and w_{j-1} for the warp's rows, one
            // 128-byte row at a time
            for (int r = 0; r < nr; ++r) {
                if (PREV != 0) tile_own[r * 33 + lane] = __ldg(args.own + (rw + r) * P + c0 + lane);
                if (PREV == 2) tile_prev[r * 33 + lane] = __ldg(args.wprev + (rw + r) * P + c0 + lane);
            }
            __syncwarp();
            if (live) {
                const uint32_t word = __ldg(args.vbits + row * NW + c0 / 32);
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int p = c0 + q;
                    const float vm = p < args.mreal ? 1.f : 0.f;
                    const float v = vm * __uint_as_float(0x3f800000u | (((word >> q) & 1u) << 31));
                    const float own = PREV == 0 ? v : tile_own[lane * 33 + q];
                    float y = fmaf(scale, acc[q], -shift * own) + fmaf(scale_lo, acc[q], -shift_lo * own);
                    float w;
                    if (PREV == 0) w = y;
                    else w = fmaf(2.f, y, -(PREV == 1 ? v : tile_prev[lane * 33 + q]));
                    tile_own[lane * 33 + q] = w;  // w_{j+1}, stored below by rows
                    const __nv_bfloat16 hi = __float2bfloat16_rn(w);
                    const float r1 = w - __bfloat162float(hi);
                    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
                    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
                    args.xt_out[(0 * P + p) * args.dx + row] = hi;
                    args.xt_out[(1 * P + p) * args.dx + row] = mid;
                    args.xt_out[(2 * P + p) * args.dx + row] = lo;
                    tr[threadIdx.x * (P + 1) + p] = v * w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) tr[threadIdx.x * (P + 1) + c0 + q] = 0.f;
            }
            __syncwarp();
            for (int r = 0; r < nr; ++r) args.out[(rw + r) * P + c0 + lane] = tile_own[r * 33 + lane];
            __syncwarp();
        }
    } else {
        if (threadIdx.x == 0) atomicOr(args.err, 1u);
        // a wait gave up: let copies and MMAs already issued finish (bounded)
        if (warp == 0 && lane == 0)
            for (int kb = issued > kDStages ? issued - kDStages : 0; kb < issued; ++kb)
                mbar_wait(full(kb % kDStages), (kb / kDStages) & 1);
        if (!got) mbar_wait(accum, 0);
    }
    __syncthreads();
    if (good) {
        for (int p = threadIdx.x; p < P; p += kDThreads) {
            double s = 0.0;
            for (int t = 0; t < kDRows; ++t) s += (double)tr[t * (P + 1) + p];
            args.tpart[(int64_t)blockIdx.x * P + p] = s;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
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

int dense_smem_bytes(int P) {
    switch (P) {
        case 32: return DenseSmem<32>::kBytes;
        case 64: return DenseSmem<64>::kBytes;
        case 128: return DenseSmem<128>::kBytes;
        default: return 0;
    }
}

template <int P, int PREV>
static cudaError_t launch_dense_t(const CUtensorMap& a, const CUtensorMap& x, int grid, cudaStream_t s,
                                  const DenseArgs& args) {
    const int smem = DenseSmem<P>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(dense_step_kernel<P, PREV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dense_step_kernel<P, PREV><<<grid, kDThreads, smem, s>>>(a, x, args);
    return cudaGetLastError();
}

// Host entry used by cld_api.cu.  B: d x d BF16 with leading dimension ld
// (elements); xt_in: the split of w_j ([3][P][dx]); prev: 0 first step,
// 1 second, 2 general.  Returns cudaErrorNotSupported when the tensor map
// cannot be encoded.
cudaError_t launch_dense_step(int P, int prev, int64_t d, int64_t ld, const void* B, const void* xt_in,
                              int64_t dx, const float* own, const float* wprev, float* out, void* xt_out,
                              const uint32_t* vbits, double* tpart, const Params* prm, int mreal, uint32_t* err,
                              cudaStream_t s) {
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
    const int grid = (int)((d + kDRows - 1) / kDRows);
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
