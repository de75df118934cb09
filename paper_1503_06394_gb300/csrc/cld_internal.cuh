// Internal declarations shared by the libcld translation units.
//
// Device-side pieces of the Chebyshev-Hutchinson estimator (Han, Malioutov,
// Shin, arXiv 1503.06394): the Rademacher probe stream, the parameter block
// the kernels read, the value loaders for FP32 / BF16 / FP64 storage, and the
// host-callable launchers implemented in step_*.cu and aux.cu.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

namespace cld {

constexpr int kThreads = 256;   // threads per CTA of every streaming kernel
constexpr int kMaxPanel = 128;  // probes per pass (counter word 2 = panel index)

// Parameter block in the workspace; written by the host (cudaMemcpyAsync) or
// by the interval kernels, read by every kernel of a run.  Keeping it on the
// device lets the captured graph of a run stay valid when [a, b] or the seed
// change.
// scale = 2/(b-a) and shift = (a+b)/(b-a) are kept as FP32 hi + lo pairs
// (hi = fl(x), lo = fl(x - hi)): a single FP32 constant would apply a
// systematically shifted matrix, an error of order 2^-24 d in every moment;
// the pair is exact to about 2^-48 and leaves only per-element rounding.
struct Params {
    double a, b;         // spectral interval [a, b]
    float scale_hi, scale_lo;
    float shift_hi, shift_lo;
    uint32_t key_lo;     // Philox key = probe seed
    uint32_t key_hi;
    int32_t interval_ok; // 1 once a and b are valid
    int32_t pad;
};

__host__ __device__ inline void split_f32(double x, float* hi, float* lo) {
    *hi = (float)x;
    *lo = (float)(x - (double)*hi);
}

__host__ __device__ inline void set_affine(Params* p, double a, double b) {
    p->a = a;
    p->b = b;
    split_f32(2.0 / (b - a), &p->scale_hi, &p->scale_lo);
    split_f32((a + b) / (b - a), &p->shift_hi, &p->shift_lo);
}

// Finishes a computed spectral enclosure [a, b] of a matrix (or batch block)
// of `rows` rows: an empty one gets [1, 2] (its estimate is 0 whatever the
// interval: t_0 = d = 0 and every other moment sums over no rows); a one-point
// spectrum (b - a <= 1e-12 b: a 1 x 1 matrix, equal diagonal entries and no
// off-diagonals) is widened by 0.1 % on each side, which keeps it an
// enclosure and gives the interpolation map 2/(b - a) a finite scale.
// Returns whether 0 < a < b with both finite.
__host__ __device__ inline bool finish_interval(double& a, double& b, int64_t rows) {
    if (rows == 0) {
        a = 1.0;
        b = 2.0;
    } else if (a > 0.0 && isfinite(a) && isfinite(b) && b - a <= 1e-12 * b) {
        a *= 1.0 - 1e-3;
        b *= 1.0 + 1e-3;
    }
    return a > 0.0 && a < b && isfinite(a) && isfinite(b);
}

// Result block in the workspace, written by the final kernel.
struct Result {
    double logdet;
    double stderr_;
    double max_ratio;    // max_{j,p} |t_{j,p}| / d
    int32_t spectrum_bad;
    int32_t pad;
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0..c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by the two Weyl constants after each round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
        uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// +-1 (or 0 for a padded probe) for the four probes whose sign bits sit at
// bits [sh, sh+4) of `word`.  bit = 1 -> -1.0f; mask_q = 0 -> 0.0f.
__device__ __forceinline__ float4 signs4(uint32_t word, int sh, float4 mask) {
    uint32_t b = word >> sh;
    float4 s;
    s.x = __uint_as_float(0x3f800000u | ((b & 1u) << 31)) * mask.x;
    s.y = __uint_as_float(0x3f800000u | (((b >> 1) & 1u) << 31)) * mask.y;
    s.z = __uint_as_float(0x3f800000u | (((b >> 2) & 1u) << 31)) * mask.z;
    s.w = __uint_as_float(0x3f800000u | (((b >> 3) & 1u) << 31)) * mask.w;
    return s;
}

// ------------------------------------------------------------------ PDL
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may become resident before its predecessor
// in the stream has finished.  pdl_wait() returns once the predecessor grid
// has completed and its memory writes are visible (at once when there is no
// programmatic predecessor); pdl_trigger() lets this kernel's own successor be
// scheduled.  Every read of data written by earlier kernels follows
// pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches kern<<<grid, kThreads, smem, s>>>(arg) with programmatic stream
// serialization (see pdl_wait): consecutive step launches overlap their
// launch latency with the predecessor's tail, in streams and in graphs.
template <typename Arg>
cudaError_t launch_pdl(void (*kern)(Arg), int grid, int smem, cudaStream_t s, const Arg& arg,
                       int threads = kThreads) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

// ------------------------------------------------------------------ values
struct bf16_t { uint16_t bits; };

__device__ __forceinline__ float load_val(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load_val(const double* p) { return (float)__ldg(p); }
__device__ __forceinline__ float load_val(const bf16_t* p) {
    uint16_t b = __ldg(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(((uint32_t)b) << 16);
}
__device__ __forceinline__ float load_val_cs(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float load_val_cs(const double* p) { return (float)__ldcs(p); }
__device__ __forceinline__ float load_val_cs(const bf16_t* p) {
    uint16_t b = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(((uint32_t)b) << 16);
}
// FP32 bits of stored value e, for the wide-lane loops (8 probes per lane,
// several gathers in flight).  A BF16 value is read as the aligned 4-byte word
// that holds it and the word's other half is dropped: with 16-bit loads the
// wide-lane step ran 13 % slower on BF16 values than on FP32 ones (the same
// requests and sectors, longer waits on the loads); with word loads it runs
// as fast.  (The narrower loops of variants 0-4 are the other way round: word
// loads made their BF16 steps 10-22 % slower, so they keep load_val.)  The
// other half lies outside the array only beside its first and its last entry,
// so a row that holds either (`edge`) reads its values 16 bits at a time.
__device__ __forceinline__ uint32_t load_bits(const float* v, int64_t e, bool) {
    return __float_as_uint(__ldg(v + e));
}
__device__ __forceinline__ uint32_t load_bits(const double* v, int64_t e, bool) {
    return __float_as_uint((float)__ldg(v + e));
}
__device__ __forceinline__ uint32_t load_bits(const bf16_t* v, int64_t e, bool edge) {
    const unsigned short* p = reinterpret_cast<const unsigned short*>(v + e);
    if (edge) return (uint32_t)__ldg(p) << 16;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(a & ~uintptr_t(3)));
    return (a & 2) ? (w & 0xffff0000u) : (w << 16);  // little-endian: the upper half is the later value
}
// One past the last stored position of a CSR array (rowptr[d]; its first is
// rowptr[0] = 0, checked when the workspace is attached), which decides the
// `edge` rows of load_bits: k0 == 0 or k1 == value_end.  Only BF16 values
// need it; other types get 0.
template <typename VT>
__device__ __forceinline__ int64_t value_end(const int64_t* rowptr, int64_t d) {
    return std::is_same<VT, bf16_t>::value ? __ldg(rowptr + d) : 0;
}

__device__ __forceinline__ double load_val_f64(const float* p) { return (double)__ldg(p); }
__device__ __forceinline__ double load_val_f64(const double* p) { return __ldg(p); }
__device__ __forceinline__ double load_val_f64(const bf16_t* p) {
    uint16_t b = __ldg(reinterpret_cast<const unsigned short*>(p));
    return (double)__uint_as_float(((uint32_t)b) << 16);
}

// ------------------------------------------------------------------ step launch
// One recurrence step over one probe panel.  The template modes are:
//   gather: 0 = gather rows of a float buffer `x`; 1 = gather probe signs
//   prev:   0 = first step (no w_{j-1}; own row is v), 1 = w_{j-1} is v,
//           2 = w_{j-1} is the float buffer `wprev`
//   epi:    0 = store the plain product y = X x;
//           1 = store w_{j+1} = f(scale, shift, X x, own, prev) and reduce
//               t_{j+1,p} = sum_i v[i,p] w_{j+1}[i,p] into per-CTA partials
struct StepArgs {
    int64_t d;
    const int64_t* rowptr;
    const int32_t* col;
    const void* val;
    const float* x;          // gather source (gather == 0)
    const float* own;        // w_j rows for the shift term (prev != 0)
    const float* wprev;      // w_{j-1} (prev == 2)
    float* out;              // w_{j+1} (epi 1) or y (epi 0)
    const uint32_t* vbits;   // d x nw sign words of the panel
    double* tpart;           // [grid][panel] partial moments (epi 1)
    const Params* prm;
    int mreal;               // real probes in this panel
    int impl;                // inner-loop variant (0..kNumStepImpls-1, see step_kernel.cuh)
    uint32_t* err;           // variant 6: set (bits) when a pipeline wait gave up
    int64_t withhold_tile;   // variant 6 testing aid: tile index + 1 never staged (0: none)
    const int32_t* lcol;     // variant 7: entries' window rows (null: no plan)
    const int32_t* wtab;     // variant 7: per-tile window ranges
};

constexpr int kNumStepImpls = 8;
constexpr int kNumBatchImpls = 7;  // variants with a batched (tile-queue) form

enum StepKind { kStepFirst = 0, kStepSecond = 1, kStepGeneral = 2, kProdBits = 3, kProdFloat = 4,
                kStepFirstFromFloat = 5 };

// Launches one step with `grid` CTAs on `stream`.  panel in {4,8,...,128}.
// grid 0 launches nothing and only sets the kernel's shared-memory attribute
// on the current device (done before a stream capture).
cudaError_t launch_step(int panel, int dtype, StepKind kind, int grid, cudaStream_t stream,
                        const StepArgs& a);
constexpr int kWinTabInts = 16;  // ints per tile in variant 7's plan table

// Variant 7's gather-window plan (window.cu): one table row per tile of
// 2048 / panel rows and each entry's window row; window_capx gives the rows a
// window holds for a panel and value type (0: no windows at that panel).
cudaError_t launch_window_plan(int panel, const int64_t* rowptr, const int32_t* col, int64_t d, int capx,
                               int32_t* tab, int32_t* lcol, int sms, cudaStream_t s);
int window_capx(int panel, int dtype);
// Resident CTAs per SM of the general step kernel (for grid sizing).
int step_ctas_per_sm(int panel, int dtype, int impl);
// Number of sign words per row for a panel width.
inline int sign_words(int panel) { return panel <= 32 ? 1 : panel / 32; }

// ------------------------------------------------------------------ aux launches (aux.cu)
cudaError_t launch_probe_bits(int64_t d, int nw, uint32_t panel_index, const Params* prm,
                              uint32_t* vbits, int grid, cudaStream_t s);
cudaError_t launch_reduce_moments(const double* tpart, int nsteps, int grid_blocks, int panel,
                                  int mreal, int M, int pbase, double* T, cudaStream_t s);
cudaError_t launch_finalize(int n, int M, int64_t d, int general, const Params* prm,
                            double* T, double* coeffs, double* coef_scratch, double* gamma_p,
                            Result* res, cudaStream_t s);
cudaError_t launch_validate_csr(int64_t d, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                                const void* val, int dtype, uint32_t* flags, int grid,
                                cudaStream_t s);
cudaError_t launch_gershgorin(int64_t d, const int64_t* rowptr, const int32_t* col,
                              const void* val, int dtype, double* partial, int grid,
                              Params* prm, uint32_t* flags, cudaStream_t s);
cudaError_t launch_set_params(Params* prm, double a, double b, cudaStream_t s);
cudaError_t launch_coeffs(int n, const Params* prm, double* coeffs, double* coef_scratch, cudaStream_t s);

// ------------------------------------------------------------------ batches (batch.cu)
// A row tile of one block of a batch: rows [lo, hi) of block blk.
struct Tile {
    int64_t lo, hi;
    int32_t blk;
    int32_t pad;
};

struct BatchStepArgs {
    StepArgs s;              // matrix, vectors, signs, panel (s.prm unused)
    const Tile* tiles;
    int64_t ntiles;
    const Params* bprm;      // per block
    double* tpart;           // [ntiles][panel] for this step
};

struct BatchAuxArgs {
    Params* bprm;
    const double* ab;        // interval pairs
    uint64_t seed;
    const Tile* tiles;
    int64_t ntiles;
    const int64_t* tile_start;
    const int64_t* blk_rows;
    int nw;
    uint32_t panel;          // panel index (probe bits)
    uint32_t* vbits;
    const double* tpart;
    int panel_width, mreal, n, M, pbase, nsteps;
    double* T;
    int dtype;
    const int64_t* rowptr;
    const int32_t* col;
    const void* val;
    const int64_t* rowptrT;
    const int32_t* colT;
    const void* valT;
    uint32_t* flags;
};

cudaError_t launch_batch_step(int panel, int dtype, StepKind kind, int grid, cudaStream_t s,
                              const BatchStepArgs& a);
// what: 0 set seeds, 1 set intervals, 2 probe bits, 3 reduce moments,
//       4 Gershgorin per block, 5 general bounds per block, 6 block check
cudaError_t launch_batch_aux(int what, int nb, int grid, cudaStream_t s, const BatchAuxArgs& a);
cudaError_t launch_finalize_batch(int nb, int n, int M, const int64_t* blk_rows, int general, const Params* prm,
                                  double* T, double* coeffs, double* coef_scratch, double* gamma_p, Result* res,
                                  cudaStream_t s);

// ------------------------------------------------------------------ dense (dense.cu)
cudaError_t launch_dense_step(int P, int prev, int64_t d, int64_t ld, const void* B, const void* xt_in,
                              int64_t dx, const float* own, const float* wprev, float* out, void* xt_out,
                              const uint32_t* vbits, double* tpart, const Params* prm, int mreal, uint32_t* err,
                              float* part, int* cnt, int smax, int grid, cudaStream_t s);
// The dense step's stream-K schedule: persistent grid and piece slots per
// 128-row tile (dense.cu).
cudaError_t dense_schedule(int P, int64_t d, int sms, int* grid, int* smax);
int dense_threads_per_cta();
cudaError_t launch_dense_sign_split(int64_t d, int64_t dx, int P, int mreal, const uint32_t* vbits, void* xt,
                                    int grid, cudaStream_t s);
cudaError_t launch_dense_gershgorin(int64_t d, int64_t ld, const void* B, double* partial, int grid, Params* prm,
                                    uint32_t* flags, cudaStream_t s);

// ------------------------------------------------------------------ adjoint (adjoint.cu)
// Arguments of one adjoint pass (see adjoint.cu).
struct AdjArgs {
    int64_t d;
    const int64_t* rowptr;
    const int32_t* col;
    const void* val;
    const float* lam_in;     // lambda_{i+1} (gathered)
    const float* lam_prev;   // lambda_{i+2}
    float* lam_out;          // lambda_i
    const float* w;          // w_i (own rows), MODE 1..2
    const uint32_t* vbits;
    float* H;                // nnz accumulators, by stored position
    const double* coeffs;    // c_0..c_n
    int ci;                  // i
    const Params* prm;
    int mreal;
    uint32_t* err;           // staged form: set when a pipeline wait gave up
    int64_t withhold_tile;   // staged form testing aid (as StepArgs::withhold_tile)
};
// form: 0 the per-lane reverse step; 1 the wide-lane one (8 probes per lane,
// panels of at least 8), used when the forward runs variant 5; 2 the staged
// tiles (variants 6 and 7; the wide one where it cannot run).
cudaError_t launch_adjoint(int panel, int dtype, int mode, int grid, cudaStream_t s, const AdjArgs& a, int form);
int adjoint_ctas_per_sm(int panel, int dtype, int form);
cudaError_t launch_adjoint_gather(int64_t d, const int64_t* rowptr, const int32_t* col, const float* H,
                                  double gscale, float* G, uint32_t* flags, int grid, cudaStream_t s);

}  // namespace cld
