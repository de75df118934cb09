/*
 * cld.h -- C ABI of libcld, a single-GPU (sm_103a) implementation of the
 * stochastic Chebyshev log-determinant estimator of Han, Malioutov and Shin,
 * "Large-scale Log-determinant Computation through Stochastic Chebyshev
 * Expansions" (arXiv 1503.06394).
 *
 * What is computed (Algorithm 1, restated on a general spectral interval):
 *   given a symmetric positive definite B with spectrum in [a, b], the shifted
 *   matrix At = (2B - (a+b) I) / (b - a) has spectrum in [-1, 1] (the affine
 *   map of Sec. 4.1).  With M Rademacher probes v_p (Sec. 2.2), the
 *   three-term recurrence w_0 = v, w_1 = At v, w_{j+1} = 2 At w_j - w_{j-1}
 *   (Sec. 2.2, Eq. chebreq) yields moments t_{j,p} = v_p^T w_j, and
 *     logdet B ~= Gamma = (1/M) sum_p sum_{j=0..n} c_j t_{j,p},
 *   where c_j are the degree-n Chebyshev interpolation coefficients of log on
 *   [a, b] at the first-kind nodes (Sec. 2.1).  For a general non-singular C
 *   (Algorithm 2, Sec. 3.2) the same runs on C^T C, applied as C then C^T, and
 *   the result is halved: log|det C| = 1/2 logdet(C^T C).
 *
 * Conventions
 *   - Every call returns a cld_status; no C++ exception crosses the ABI.
 *     cld_last_error() returns a thread-local message for the last failure.
 *   - Matrix arrays are BORROWED device pointers: the caller keeps them alive
 *     and unchanged until cld_destroy.  CSR rows need not be sorted; repeated
 *     (row, col) entries are added.
 *   - All device scratch memory comes from a caller-supplied workspace
 *     (cld_workspace_size / cld_set_workspace).  The library allocates no
 *     device memory of its own except where an entry point says so.
 *   - Work is enqueued on the stream given at creation.  cld_estimate
 *     synchronises that stream once to return host doubles.
 *   - Probe vectors are never stored: entry v[i,p] in {+1,-1} is regenerated
 *     from Philox4x32-10 (Salmon et al., SC'11) with key = seed (low word,
 *     high word) and counter = (i low word, i high word, p / 128, 0):
 *     v = 1 - 2 * bit (p mod 32) of output word ((p / 32) mod 4).
 *   - Recurrence vectors are FP32; stored matrix values are FP32, BF16 or
 *     FP64; coefficients, moments and the final reduction are FP64.
 */
#ifndef CLD_H
#define CLD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CLD_API __attribute__((visibility("default")))
#else
#define CLD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cld_ctx* cld_handle;

typedef enum {
    CLD_OK = 0,
    CLD_ERR_INVALID = 1,     /* bad argument, malformed CSR, NULL pointer       */
    CLD_ERR_INTERVAL = 2,    /* a <= 0, a >= b, or interval not set / not finite */
    CLD_ERR_SPECTRUM = 3,    /* some |t_{j,p}| > d (1 + 1e-3) or not finite:    */
                             /* the spectrum is not inside [a, b]                */
    CLD_ERR_NOMEM = 4,       /* workspace missing or smaller than required      */
    CLD_ERR_CUDA = 5,        /* a CUDA runtime call failed                      */
    CLD_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                   */
    CLD_ERR_UNSUPPORTED = 7  /* valid request this build does not implement     */
} cld_status;

typedef enum { CLD_F32 = 0, CLD_BF16 = 1, CLD_F64 = 2 } cld_dtype;

/* CLD_SPD: the matrix B itself is symmetric positive definite (Algorithm 1).
 * CLD_GENERAL: the matrix C is a general non-singular matrix; the estimate is
 * of log|det C| = 1/2 logdet(C^T C) and the interval bounds the spectrum of
 * C^T C, i.e. [sigma_min^2, sigma_max^2] (Algorithm 2). */
typedef enum { CLD_SPD = 0, CLD_GENERAL = 1 } cld_kind;

/* Largest probe count handled by one pass; larger M runs in panels of 128. */
#define CLD_PROBE_PANEL 128

/* Creates a handle for a d x d CSR matrix on the device: the input B of
 * Algorithm 1 (Sec. 3.1) or C of Algorithm 2 (Sec. 3.2), which the paper
 * takes as a sparse matrix accessed only through products (Sec. 3.1: cost
 * O(mn ||B||_0)); the storage format itself has no paper counterpart.
 *   rowptr: d+1 int64 (device), rowptr[0] = 0, non-decreasing, rowptr[d] = nnz
 *   col:    nnz int32 (device), 0 <= col < d
 *   val:    nnz values (device) of type val_dtype
 *   stream: cudaStream_t to enqueue on (NULL = legacy default stream)
 * Each array must be aligned to its element size (torch allocations are).
 * Only host-side checks run here (sizes, NULLs, alignment, d < 2^31); the
 * arrays are checked on the device by cld_set_workspace.
 * Errors: CLD_ERR_INVALID. */
CLD_API cld_status cld_create_csr(cld_handle* out, int64_t d, int64_t nnz, const int64_t* rowptr,
                          const int32_t* col, const void* val, cld_dtype val_dtype,
                          cld_kind kind, void* stream);

/* Creates a handle for a DENSE d x d symmetric positive definite matrix B on
 * the device (a kernel matrix, say), stored row-major in BF16 with leading
 * dimension ld (elements; ld >= d, ld a multiple of 8, base 16-byte
 * aligned).  Each recurrence step is then the product B W_j (d x d by d x P)
 * on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation, W_j split
 * into three BF16 parts so the product keeps FP32 accuracy), followed by the
 * same recurrence epilogue.  The cost per step is one pass over B, O(d^2)
 * instead of O(nnz) (Sec. 3.1: O(mn ||B||_0)).  cld_workspace_size,
 * cld_set_workspace, cld_set_interval, cld_auto_interval (Gershgorin, no
 * Lanczos), cld_estimate and cld_set_graph apply.  Errors: CLD_ERR_INVALID,
 * CLD_ERR_UNSUPPORTED (dtype other than CLD_BF16, kind other than CLD_SPD);
 * cld_estimate returns CLD_ERR_TIMEOUT if a pipeline wait on the device gave
 * up (results invalid). */
CLD_API cld_status cld_create_dense(cld_handle* out, int64_t d, int64_t ld, const void* val_dev,
                                    cld_dtype val_dtype, cld_kind kind, void* stream);

/* Bytes of device workspace an estimate of degree n with M probes needs
 * (with_grad != 0: also enough for cld_grad).  No paper counterpart
 * (memory infrastructure): the three recurrence blocks w_{j-1}, w_j, w_{j+1}
 * of Algorithm 1 are the dominant term, d x panel x 4 bytes each; CLD_SPD
 * single-matrix handles add variant 7's gather-window plan (nnz x 4 bytes and
 * 4 bytes per row).
 * Errors: CLD_ERR_INVALID. */
CLD_API cld_status cld_workspace_size(cld_handle h, int n, int M, int with_grad, size_t* bytes);

/* No paper counterpart (memory infrastructure).
 * Attaches caller-owned device workspace (at least 256-byte aligned) and
 * validates the CSR arrays on the device (monotone rowptr, column range,
 * finite values).  The workspace must stay alive until cld_destroy or the
 * next cld_set_workspace.  Errors: CLD_ERR_INVALID (malformed CSR or
 * unaligned pointer), CLD_ERR_CUDA. */
CLD_API cld_status cld_set_workspace(cld_handle h, void* dev_ptr, size_t bytes);

/* Sets the spectral interval [a, b] that must contain the spectrum of B
 * (CLD_SPD) or of C^T C (CLD_GENERAL); by Sec. 3 the bounds may be loose
 * (a wider interval costs accuracy at a given degree, not correctness).  Errors: CLD_ERR_INTERVAL if !(0 < a < b) or not finite. */
CLD_API cld_status cld_set_interval(cld_handle h, double a, double b);

/* Computes an interval on the device and stores it on the handle (Sec. 3.2).
 * CLD_SPD: a = min_i (B_ii - R_i), b = max_i (B_ii + R_i) (Gershgorin,
 * R_i = sum_{k != i} |B_ik|); a must come out positive, else
 * CLD_ERR_INTERVAL.  If lanczos_iters > 0, b is tightened to
 * min(b, theta_max + r), theta_max the largest Ritz value of a Lanczos run of
 * that many steps from a Philox start vector and r its residual norm; a is
 * never taken from Lanczos.
 * CLD_GENERAL: b = ||C||_1 ||C||_inf (the square of the paper's sigma_max
 * bound); a = alpha * beta with alpha = min_i (|C_ii| - R_i) and
 * beta = min_i (|C_ii| - S_i) (R_i, S_i the off-diagonal absolute row and
 * column sums) when both are positive: Varah's bounds ||C^-1||_inf <= 1/alpha
 * and ||C^-1||_1 <= 1/beta give sigma_min^2 >= alpha beta, the diagonal-
 * dominance route of Sec. 3.2.  Otherwise CLD_ERR_INTERVAL.
 * Either pointer may be NULL.  Needs the workspace.  Errors:
 * CLD_ERR_INTERVAL, CLD_ERR_NOMEM, CLD_ERR_CUDA. */
CLD_API cld_status cld_auto_interval(cld_handle h, int lanczos_iters, double* a, double* b);

/* Runs the estimator of Algorithm 1 (Sec. 3.1; CLD_SPD) or Algorithm 2
 * (Sec. 3.2; CLD_GENERAL): Rademacher probes and the Hutchinson trace
 * estimate of Sec. 2.2, the Chebyshev recurrence of Eq. (chebreq) applied to
 * the probes, and the coefficients of the degree-n interpolant of log at the
 * first-kind nodes of Sec. 2.1, on the interval set on the handle.
 * Degree n >= 0, M >= 1 probes, probe seed `seed`.
 *   logdet_out: Gamma (CLD_SPD: logdet B; CLD_GENERAL: log|det C|)
 *   stderr_out: std over probes of Gamma_p divided by sqrt(M) (NULL ok;
 *               NaN when M = 1); for CLD_GENERAL it is halved as well
 *   moments_out: NULL or host array of (n+1) x M doubles, t[j*M + p]
 * Needs an interval and a workspace of cld_workspace_size(h, n, M, 0).
 * Errors: CLD_ERR_INVALID (n < 0, M < 1), CLD_ERR_INTERVAL, CLD_ERR_NOMEM,
 * CLD_ERR_SPECTRUM (outputs are still written), CLD_ERR_CUDA. */
CLD_API cld_status cld_estimate(cld_handle h, int n, int M, uint64_t seed, double* logdet_out,
                        double* stderr_out, double* moments_out);

/* After a successful cld_estimate: copies the n+1 coefficients c_j used
 * (Sec. 2.1) and the M per-probe estimates Gamma_p (the summands of the
 * Hutchinson average of Algorithm 1) to host arrays (either may be NULL). */
CLD_API cld_status cld_last_details(cld_handle h, double* coeffs_out, double* gamma_p_out);

/* Gradient of the estimate (same n, M, seed and interval, interval held fixed)
 * with respect to every stored value: dvalues_dev[k] = dGamma / d val[k], an
 * FP32 device array of nnz entries, each stored entry treated as an
 * independent variable.  Reverse-mode differentiation of the recurrence of
 * Sec. 2.2 (an extension; the paper has no gradient).  CLD_SPD only.
 * Needs cld_workspace_size(h, n, M, 1) (which follows the checkpoint
 * interval below).  Errors as cld_estimate, plus CLD_ERR_UNSUPPORTED for
 * CLD_GENERAL. */
CLD_API cld_status cld_grad(cld_handle h, int n, int M, uint64_t seed, double* logdet_out,
                    float* dvalues_dev);

/* Memory of cld_grad (an extension; no paper counterpart).  interval 0 (default): the forward keeps every w_1..w_n
 * (n blocks of d x panel floats).  interval K >= 2: the forward keeps only the
 * pairs (w_{sK-1}, w_{sK}); the reverse pass recomputes w_{sK+1} .. w_{(s+1)K}
 * from them, segment by segment from the last, before taking those reverse
 * steps - about 2n/K + K blocks (K near sqrt(2n) is smallest) for one extra
 * forward pass.  The gradient and the estimate are bit-identical to
 * interval 0's (the recomputation repeats the same kernels on the same data).
 * Errors: CLD_ERR_INVALID for 1, a negative value or more than 100000. */
CLD_API cld_status cld_set_grad_checkpoint(cld_handle h, int interval);

/* One-shot estimate from HOST arrays (Algorithm 1 or 2 as cld_estimate; the
 * copies are infrastructure without a paper counterpart): copies the CSR (rowptr, col, val as
 * above but in host memory, ideally pinned) into the front of the device
 * workspace, runs cld_estimate on [a, b] and returns Gamma and its stderr.
 * Workspace size: cld_host_workspace_size.  Nothing is kept after return.
 * Errors: as cld_create_csr, cld_set_workspace and cld_estimate. */
CLD_API cld_status cld_host_workspace_size(int64_t d, int64_t nnz, cld_dtype val_dtype, int n, int M,
                                   size_t* bytes);
CLD_API cld_status cld_logdet_csr_host(int64_t d, int64_t nnz, const int64_t* rowptr_host,
                               const int32_t* col_host, const void* val_host, cld_dtype val_dtype,
                               cld_kind kind, double a, double b, int n, int M, uint64_t seed,
                               void* workspace_dev, size_t workspace_bytes, void* stream,
                               double* logdet_out, double* stderr_out);

/* Size of the library's built-in device scratch array used by
 * cld_estimate_static (32 MiB). */
#define CLD_STATIC_SCRATCH_BYTES (32u << 20)

/* Estimate without any device allocation, for callers that cannot allocate
 * device memory: code whose device memory is entirely owned by another
 * allocator (a framework's caching pool that must not be bypassed), code that
 * runs under a fixed device-memory budget, and latency-critical loops that
 * must never block in cudaMalloc/cudaFree.  The paper has no counterpart: this
 * is the same estimate as cld_create_csr + cld_set_interval + cld_estimate
 * (CLD_SPD only; it runs inner-loop variant 0, so the moments' last bits can
 * differ from a handle's by summation order), but its scratch lives in one
 * file-scope __device__ array of CLD_STATIC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits.
 *   rowptr, col, val: the CSR matrix on the device, as in cld_create_csr
 *   a, b, n, M, seed: as in cld_set_interval / cld_estimate
 *   stream: cudaStream_t to enqueue on (NULL = legacy default stream)
 *   logdet_out, stderr_out: host doubles (stderr_out may be NULL)
 * The needed scratch is d x P x 12 bytes for the three recurrence blocks
 * (P = M rounded up to a power of two >= 4, at most 128) plus small terms;
 * requests that do not fit are rejected with CLD_ERR_NOMEM and a message that
 * gives both sizes.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  The first call on each device looks up the array's device address
 * on that device (cudaGetSymbolAddress, with that device current) and keeps
 * it for the life of the process; make that first call before any stream
 * capture, and do not use the entry point across a cudaDeviceReset (or any
 * other re-creation of the device's primary context), after which the kept
 * address is stale.  Each CSR array must be aligned to its element size; a
 * pointer that is not is refused with CLD_ERR_INVALID before any CUDA call.  All calls share the one array and it
 * keeps the last call's contents (the call clears what must start at zero):
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it.  Synchronises `stream` to return.  Errors: as cld_create_csr,
 * cld_set_interval, cld_set_workspace (CSR checks) and cld_estimate, plus
 * CLD_ERR_NOMEM when the request exceeds the array. */
CLD_API cld_status cld_estimate_static(int64_t d, int64_t nnz, const int64_t* rowptr,
                                       const int32_t* col, const void* val, cld_dtype val_dtype,
                                       double a, double b, int n, int M, uint64_t seed,
                                       void* stream, double* logdet_out, double* stderr_out);

/* ------------------------------------------------------------------------ */
/* Batches: many independent matrices of uneven size estimated together, one */
/* pass over all of them per degree step (each block is a separate problem   */
/* of Algorithm 1, or of Algorithm 2 for CLD_GENERAL).                        */
/* ------------------------------------------------------------------------ */

/* Creates a batch handle (no paper counterpart: each block is an
 * independent problem of Algorithm 1 or 2).  The nb matrices are given as one block-diagonal
 * CSR with GLOBAL row and column indices: block b holds rows (and columns)
 * [blk_rows[b], blk_rows[b+1]); blk_rows is a HOST array of nb+1 offsets,
 * copied.  rowptr/col/val/val_dtype/kind/stream as in cld_create_csr (all
 * blocks share the kind).  Block b's probes use the seed seed + b with the
 * block's local row index, so its estimate equals a single-matrix
 * cld_estimate of that block with seed + b.  cld_workspace_size and
 * cld_set_workspace apply (the latter also checks that every column lies in
 * its row's block).  Errors: CLD_ERR_INVALID. */
CLD_API cld_status cld_create_batch(cld_handle* out, int nb, const int64_t* blk_rows, int64_t nnz,
                                    const int64_t* rowptr, const int32_t* col, const void* val,
                                    cld_dtype val_dtype, cld_kind kind, void* stream);

/* Tuning control, no paper counterpart.  Rows per work tile of the batched step kernel (>= 256; default 1024): a
 * tile never spans two blocks; CTAs take tiles from a static queue.
 * cld_autotune on a batch handle also picks it (256 ... 4096). */
CLD_API cld_status cld_batch_set_tile_rows(cld_handle h, int rows);

/* The current rows per tile of a batch handle (no paper counterpart).  Errors: CLD_ERR_INVALID. */
CLD_API cld_status cld_batch_get_tile_rows(cld_handle h, int* rows);

/* Per-block intervals (host arrays of nb doubles), as cld_set_interval (Sec. 3). */
CLD_API cld_status cld_batch_set_intervals(cld_handle h, const double* a, const double* b);

/* Per-block intervals computed on the device as cld_auto_interval (Sec. 3.2; without
 * Lanczos); written to the host arrays a_out, b_out (nb each, may be NULL). */
CLD_API cld_status cld_batch_auto_intervals(cld_handle h, double* a_out, double* b_out);

/* Runs all blocks, each as cld_estimate (Algorithm 1 or 2): logdet_out[b] and stderr_out[b] (host arrays of nb; the
 * latter may be NULL).  Errors as cld_estimate (CLD_ERR_SPECTRUM names the
 * first failing block; all outputs are still written). */
CLD_API cld_status cld_batch_estimate(cld_handle h, int n, int M, uint64_t seed, double* logdet_out,
                                      double* stderr_out);

/* Execution control, no paper counterpart.  When on, cld_estimate /
 * cld_batch_estimate replay one CUDA graph of the
 * whole estimate (captured on first use per (n, M, variant, workspace, tile
 * size) on a stream of the handle; the seed is set by a launch before it).
 * Profiling events are not recorded in graph mode. */
CLD_API cld_status cld_set_graph(cld_handle h, int on);

/* Selects the inner loop of the recurrence-step kernel (the matrix-block
 * product of the recurrence in Algorithm 1; a tuning control with no paper
 * counterpart; all
 * variants compute the same sums in the same order):
 *   0: each lane loads 4 (column, value) pairs itself, 4 row gathers in flight;
 *   1: the lanes of a row load 8 pairs cooperatively and issue 8 row gathers
 *      back to back, the next chunk's pairs loaded ahead;
 *   2: as 1 with chunks of 4 pairs (fewer registers, more resident CTAs);
 *   3: a shared-memory ring: the rows of w_j gathered by a row's first 5
 *      entries, its own row and its row of w_{j-1} are copied into shared
 *      memory with cp.async while the group consumes the previous row (for
 *      short rows, e.g. stencils, where dependent loads otherwise serialise);
 *      entries past the 5th are gathered directly;
 *   4: as 3 with the first 8 entries staged (more shared memory, 2 CTAs/SM);
 *   5: wide lanes: each lane owns 8 consecutive probes of a row (256-bit
 *      gathers) and keeps 4 stored entries in flight, paying the per-entry
 *      index, value and address work once per 8 probes (panels of at least 8
 *      probes, else variant 0; batch handles have a wide-lane tile kernel
 *      too).  BF16 values are read as the aligned 4-byte words that hold them
 *      (16-bit loads in the rows that hold the array's first or last entry);
 *   6: staged tiles: a CTA takes tiles of 2048 / P consecutive rows, one
 *      producer warp copies each tile's row pointers, stored indices and
 *      values, own rows of w_j, rows of w_{j-1} and sign words into a ring of
 *      shared-memory stages with bulk asynchronous copies (TMA), and eight
 *      consumer warps compute with the wide lanes of variant 5, so only the
 *      gathers stay on a row's chain of dependent loads (for matrices whose
 *      gathers hit the caches: stencils, point clouds numbered by cell).
 *      Panels of at least 8 probes and CSR arrays on 16-byte boundaries, else
 *      variant 5 runs; tiles with more than 16 stored entries per row on
 *      average read their indices and values from global memory.  Its waits
 *      are bounded: cld_estimate / cld_grad return CLD_ERR_TIMEOUT if one
 *      gave up (results invalid).  Batch handles have a staged tile-queue
 *      form (queue tiles cut into sub-tiles of 2048 / P rows), and
 *      cld_batch_estimate returns CLD_ERR_TIMEOUT the same way;
 *   7: gather windows, for CLD_SPD single-matrix handles whose tiles of rows
 *      reach few compact index ranges (stencils, points numbered by cell):
 *      a plan, computed on the device once per workspace and panel width,
 *      gives each tile of 2048 / P rows up to 4 ranges of rows (gaps of up to
 *      16 rows merged) and each stored entry its row in them; the staged
 *      tiles of variant 6 then also copy those ranges of w_j, and every
 *      gather reads shared memory.  Tiles whose columns need more ranges or
 *      more rows than a stage holds gather from global memory; steps 0, the
 *      products of CLD_GENERAL handles, panels of fewer than 16 probes and
 *      FP64 values at 16 probes run variant 6.  Needs the plan's workspace
 *      (cld_workspace_size counts it for CLD_SPD handles: nnz x 4 bytes and
 *      4 bytes per row); batch handles do not take it.
 * The default at creation is 6 from d = 1e5 up; below, 3 when the matrix
 * holds at most 6 stored entries per row on average, else 4 (batches: 0).
 * The variant also sets the grid size, so the last bits of the moments (their
 * summation order) can change with it.
 * Errors: CLD_ERR_INVALID for an unknown variant. */
CLD_API cld_status cld_set_kernel_variant(cld_handle h, int variant);

/* Autotuner (no paper counterpart): times three blocks of `reps` launches of
 * the general recurrence step of every variant on this matrix with M probes
 * (for CLD_GENERAL both kernels of a step: y = C w_j and the step on C^T y),
 * each candidate scored by its fastest block (workspace and interval must be set;
 * the workspace contents are overwritten) and keeps the fastest on the handle
 * (the current choice stays unless another is at least 2 % faster).  On a
 * batch handle every variant is timed at every tile size of 256, 512, 1024,
 * 2048 and 4096 rows and the fastest pair is kept (read the tile size back
 * with cld_batch_get_tile_rows).
 * Returns the chosen variant and its step time in ms (either may be NULL).
 * Errors: CLD_ERR_INVALID, CLD_ERR_NOMEM, CLD_ERR_INTERVAL, CLD_ERR_CUDA. */
CLD_API cld_status cld_autotune(cld_handle h, int M, int reps, int* variant_out, float* ms_out);

/* Testing aid for the bounded waits of variant 6 (no paper counterpart):
 * with tile > 0, the staged step kernel withholds the copies and arrivals of
 * row tile tile - 1 (rows (tile-1) T .. tile T - 1, T = 2048 / panel), so the
 * consumers' waits for that tile run out after about 2 s and cld_estimate
 * returns CLD_ERR_TIMEOUT; the CUDA context stays usable.  0 (the default)
 * turns it off.  Errors: CLD_ERR_INVALID for a negative tile. */
CLD_API cld_status cld_debug_withhold_tile(cld_handle h, int64_t tile);

/* Timing of the dominant kernel (no paper counterpart).  When on, every
 * cld_estimate, and every cld_batch_estimate outside graph mode, records CUDA
 * events on its stream around the general recurrence steps (j >= 2) and
 * cld_last_timing returns their elapsed time and the number of such degree
 * steps in the last estimate (for CLD_GENERAL a degree step is two launches,
 * C w_j then C^T y).  Off by default. */
CLD_API cld_status cld_set_profiling(cld_handle h, int on);
CLD_API cld_status cld_last_timing(cld_handle h, float* step_ms, int* step_launches, int* total_launches);

/* Kernel configuration of the recurrence step, for reports (no paper
 * counterpart): probe panel width
 * (padded M), lanes per row, CTAs per launch, threads per CTA (dense
 * handles: the stream-K step's persistent grid, one epilogue thread per row
 * of a tile). */
CLD_API cld_status cld_launch_config(cld_handle h, int M, int* panel, int* lanes_per_row, int* ctas,
                             int* threads);

/* Handle and error infrastructure (no paper counterpart): cld_destroy frees
 * the handle's host state and CUDA graph (never the borrowed arrays or the
 * workspace); cld_last_error returns the calling thread's message for its
 * last failed call; cld_version names the build. */
CLD_API void cld_destroy(cld_handle h);
CLD_API const char* cld_last_error(void);
CLD_API const char* cld_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CLD_H */
