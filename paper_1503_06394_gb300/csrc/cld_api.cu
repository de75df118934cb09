// C ABI of libcld (declared in include/cld.h): handle management, workspace
// layout, and the driver that enqueues one estimate of the Chebyshev-Hutchinson
// log-determinant (Algorithm 1; Algorithm 2 for general C) on a CUDA stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/cld.h"
#include "cld_internal.cuh"

namespace cld {
cudaError_t launch_set_seed(Params* prm, uint64_t seed, cudaStream_t s);
cudaError_t launch_transpose(int64_t d, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                             const void* val, int vsize, int64_t* rowptrT, int32_t* colT, void* valT,
                             int64_t* scratch, int grid, cudaStream_t s);
cudaError_t launch_general_bounds(int64_t d, const int64_t* rowptr, const int32_t* col,
                                  const void* val, const int64_t* rowptrT, const int32_t* colT,
                                  const void* valT, int dtype, double* partial, int grid,
                                  Params* prm, uint32_t* flags, cudaStream_t s);
cudaError_t launch_lanczos(int64_t d, const int64_t* rowptr, const int32_t* col, const void* val,
                           int dtype, int iters, double* vecs, double* scal, int grid,
                           Params* prm, uint32_t* flags, cudaStream_t s);
}  // namespace cld

using namespace cld;

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

static cld_status fail(cld_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

namespace cld {
// Lets other translation units report through cld_last_error().
void set_error_message(const char* msg) { g_err = msg; }
}  // namespace cld

#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(CLD_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));   \
    } while (0)

static inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

static int value_size(cld_dtype t) { return t == CLD_F32 ? 4 : t == CLD_BF16 ? 2 : 8; }

// ---------------------------------------------------------------- handle
struct cld_ctx {
    int64_t d = 0, nnz = 0;
    const int64_t* rowptr = nullptr;
    const int32_t* col = nullptr;
    const void* val = nullptr;
    cld_dtype dtype = CLD_F32;
    cld_kind kind = CLD_SPD;
    cudaStream_t stream = nullptr;
    int device = 0, sms = 1;

    char* ws = nullptr;
    size_t ws_bytes = 0;
    bool ready = false;  // workspace attached and CSR validated (and transposed)

    double a = 0.0, b = 0.0;
    bool have_interval = false;

    int impl = 1;  // recurrence-step inner loop (see step_kernel.cuh)
    int ckpt = 0;  // gradient checkpoint interval K (0: keep every w_j)
    int64_t withhold_tile = 0;  // testing aid of variant 6 (cld_debug_withhold_tile)
    int plan_panel = 0;         // panel width of variant 7's plan in the workspace (0: none)

    // batch (nb > 0): block-diagonal super matrix, blocks [blk_rows[b], blk_rows[b+1])
    int nb = 0;
    std::vector<int64_t> blk_rows;
    int tile_rows = 1024;
    int64_t max_tiles = 0;
    std::vector<Tile> tiles;
    std::vector<int64_t> tile_start;
    std::vector<double> ba, bb;  // per-block intervals
    bool have_bintervals = false;

    // dense matrix (tensor-core path): d x d, leading dimension ld, values in val
    bool dense = false;
    int64_t ld = 0;

    // CUDA graph of one estimate (set-seed stays outside the graph)
    bool use_graph = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long gkey[6] = {0, 0, 0, 0, 0, 0};

    int last_n = -1, last_M = -1;
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    float last_step_ms = 0.f;
    int last_step_launches = 0, last_total_launches = 0;
};

// Workspace layout.  Front: fixed header (parameters, result, flags), then
// (general C only) the transposed CSR of C, then the per-run region.
struct Layout {
    size_t params, result, flags, rowptrT, colT, valT, tscratch, run;  // fixed part
    size_t coeffs, coef_scratch, T, gamma_p, tpart, gpart, vbits, W[3], Y, lanczos, total;
    size_t Wall, lam[3], H;  // gradient: w_1..w_n (or checkpoints + a segment), the adjoint ring, per-entry sums
    int nseg, ckK;           // checkpointed gradient: segments of w_1..w_{n-1}, their length K (0: every w_j kept)
    size_t blk_rows, tile_start, tiles, bprm, ab, bres;  // batches
    size_t xt[2];            // dense: BF16 splits of w_j, [3][panel][dx], double-buffered
    size_t wtab, lcol;       // variant 7's gather-window plan (single-matrix SPD handles)
    bool plan;
    size_t dpart, dcnt;      // dense: stream-K partial sums [ntiles][dsmax][128][panel], tile counters
    int dgrid, dsmax;
    int64_t dx;
    int panel, nw, grid, ggrid;
};

// Inner-loop variant at creation: from d = 1e5 up, where throughput counts,
// the staged tiles (6; measured fastest on GB300 for the random SPD matrix
// of 11 entries per row, the 5-point grid and the Wendland matrix); below,
// where a step is one short burst of rows and latency counts, the
// shared-memory ring staging the first 5 entries of a row (3) for short rows,
// else the ring staging 8 (4).
static int default_impl(int64_t d, int64_t nnz) { return d >= 100000 ? 6 : nnz <= 6 * d ? 3 : 4; }

static int panel_for_dense(int M) { return M <= 32 ? 32 : M <= 64 ? 64 : 128; }

static int panel_for(int M) {
    if (M >= kMaxPanel) return kMaxPanel;
    int p = 4;
    while (p < M) p <<= 1;
    return p;
}

static int step_grid(const cld_ctx* h, int panel) {
    // rows a CTA covers in one pass: 4 probes per lane (the staged tiles of
    // variant 6: tiles of 2048 / panel rows)
    const int rows_per_cta = (h->impl >= 6 && panel >= 8) ? 2048 / panel : (kThreads / 32) * (128 / panel);
    const int64_t need = (h->d + rows_per_cta - 1) / rows_per_cta;
    const int64_t full = (int64_t)step_ctas_per_sm(panel, (int)h->dtype, h->impl) * h->sms;
    int64_t g = need < full ? need : full;
    return (int)(g > 0 ? g : 1);
}

static int stream_grid(const cld_ctx* h) {
    const int64_t need = (h->d + kThreads - 1) / kThreads;
    const int64_t full = (int64_t)h->sms * 8;
    int64_t g = need < full ? need : full;
    return (int)(g > 0 ? g : 1);
}

static Layout make_layout(const cld_ctx* h, int n, int M, int with_grad) {
    Layout L{};
    size_t o = 0;
    L.params = o; o += align_up(sizeof(Params));
    L.result = o; o += align_up(sizeof(Result));
    L.flags = o; o += 256;
    if (h->kind == CLD_GENERAL) {
        L.rowptrT = o; o += align_up((size_t)(h->d + 1) * 8);
        L.colT = o; o += align_up((size_t)h->nnz * 4);
        L.valT = o; o += align_up((size_t)h->nnz * value_size(h->dtype));
        L.tscratch = o; o += align_up((size_t)(h->d + 1) * 8);
    }
    // variant 7's plan: a table row per tile (tiles of 16 or more rows) and
    // each entry's window row
    L.plan = h->kind == CLD_SPD && h->nb == 0 && !h->dense;
    if (L.plan) {
        L.wtab = o; o += align_up((size_t)((h->d + 15) / 16 + 1) * kWinTabInts * 4);
        L.lcol = o; o += align_up((size_t)h->nnz * 4);
    }
    const int nprob = h->nb > 0 ? h->nb : 1;
    if (h->nb > 0) {
        L.blk_rows = o; o += align_up((size_t)(h->nb + 1) * 8);
        L.tile_start = o; o += align_up((size_t)(h->nb + 1) * 8);
        L.tiles = o; o += align_up((size_t)h->max_tiles * sizeof(Tile));
        L.bprm = o; o += align_up((size_t)h->nb * sizeof(Params));
        L.ab = o; o += align_up((size_t)h->nb * 2 * 8);
    }
    L.run = o;
    const int nn = n > 0 ? n : 0;
    const int MM = M > 0 ? M : 1;
    L.panel = h->dense ? panel_for_dense(MM) : panel_for(MM);
    L.nw = sign_words(L.panel);
    L.grid = h->dense ? (int)((h->d + 127) / 128) : step_grid(h, L.panel);
    L.ggrid = stream_grid(h);
    L.coeffs = o; o += align_up((size_t)nprob * (nn + 1) * 8);
    L.coef_scratch = o; o += align_up((size_t)nprob * 5 * (nn + 1) * 8);
    L.T = o; o += align_up((size_t)nprob * (nn + 1) * MM * 8);
    L.gamma_p = o; o += align_up((size_t)nprob * MM * 8);
    L.bres = o; o += align_up((size_t)nprob * sizeof(Result));
    const int64_t tslots = h->nb > 0 ? h->max_tiles : L.grid;
    L.tpart = o; o += align_up((size_t)(nn > 0 ? nn : 1) * tslots * L.panel * 8);
    L.gpart = o; o += align_up((size_t)4 * L.ggrid * 8 + 64);  // 4 doubles per CTA (general bounds)
    L.vbits = o; o += align_up((size_t)h->d * L.nw * 4);
    const size_t wb = align_up((size_t)h->d * L.panel * 4);
    for (int i = 0; i < 3; ++i) { L.W[i] = o; o += wb; }
    if (h->kind == CLD_GENERAL) { L.Y = o; o += wb; }
    if (h->dense) {
        L.dx = (h->d + 63) / 64 * 64;
        for (int i = 0; i < 2; ++i) { L.xt[i] = o; o += align_up((size_t)3 * L.panel * L.dx * 2); }
        L.dgrid = 1;
        L.dsmax = 1;
        if (h->d > 0 && dense_schedule(L.panel, h->d, h->sms, &L.dgrid, &L.dsmax) != cudaSuccess) L.dgrid = 0;
        const int64_t ntiles = (h->d + 127) / 128;
        L.dpart = o; o += align_up((size_t)ntiles * L.dsmax * 128 * L.panel * 4);
        L.dcnt = o; o += align_up((size_t)ntiles * 4);
    }
    // Lanczos scratch (5 FP64 vectors + scalars) reuses the W buffers when they are
    // large enough, else gets its own region.
    const size_t lz = align_up((size_t)5 * h->d * 8) + align_up((size_t)(8000 + L.ggrid + 64) * 8);
    if (lz > 3 * wb) { L.lanczos = o; o += lz; } else { L.lanczos = L.W[0]; }
    if (with_grad) {
        if (h->ckpt >= 2 && nn >= 2) {
            // checkpoint pairs (w_{sK-1}, w_{sK}) for 1 <= s < nseg, then K segment buffers
            L.ckK = h->ckpt;
            L.nseg = (nn - 1 + L.ckK - 1) / L.ckK;
            const int seglen = L.ckK < nn - 1 ? L.ckK : nn - 1;  // longest segment
            L.Wall = o; o += (size_t)(2 * (L.nseg - 1) + seglen) * wb;
        } else {
            L.ckK = 0;
            L.nseg = 0;
            L.Wall = o; o += (size_t)(nn > 0 ? nn : 1) * wb;
        }
        for (int i = 0; i < 3; ++i) { L.lam[i] = o; o += wb; }
        L.H = o; o += align_up((size_t)h->nnz * 4);
    }
    L.total = o;
    return L;
}

template <typename T>
static T* at(cld_ctx* h, size_t off) { return reinterpret_cast<T*>(h->ws + off); }

static cld_status check_handle(cld_handle h) {
    if (!h) return fail(CLD_ERR_INVALID, "NULL handle");
    return CLD_OK;
}

// Where w_m (m >= 1) lives during a run.
//   kMapRing: the 3-buffer ring W[m % 3];
//   kMapAll:  buffer m-1 of Wall (gradient keeping every w_j);
//   kMapCkpt: the ring, except w_{sK-1} and w_{sK} (1 <= s < nseg), which go
//             to checkpoint pair s-1 at the start of Wall (checkpointed gradient);
//   kMapSeg:  w_lo .. w_hi of a recomputed segment in the K buffers after the
//             checkpoint pairs; its inputs w_{lo-2}, w_{lo-1} in their pair.
enum { kMapRing = 0, kMapAll = 1, kMapCkpt = 2, kMapSeg = 3 };
struct WMap {
    int mode;
    int lo;  // kMapSeg: first index of the segment
};

static float* wbuf(cld_ctx* h, const Layout& L, int m, const WMap& wm) {
    const size_t wb = L.W[1] - L.W[0];
    auto blk = [&](size_t i) { return reinterpret_cast<float*>(h->ws + L.Wall + i * wb); };
    if (wm.mode == kMapAll) return blk((size_t)(m - 1));
    if (wm.mode == kMapSeg && m >= wm.lo) return blk((size_t)(2 * (L.nseg - 1) + (m - wm.lo)));
    if (wm.mode == kMapSeg || wm.mode == kMapCkpt) {
        const int K = L.ckK;
        const int r = m % K, sidx = (m + 1) / K;
        if (m >= K - 1 && (r == K - 1 || r == 0) && sidx >= 1 && sidx <= L.nseg - 1)
            return blk((size_t)(2 * (sidx - 1) + (r == 0 ? 1 : 0)));
    }
    return at<float>(h, L.W[m % 3]);
}

// Enqueues recurrence steps j0 <= j < j1 of panel pk (step j writes w_{j+1}
// from w_j and w_{j-1}; w_0 = v, the panel's signs, already in place) with
// the buffers of `wm`.  Counts launches; `events` records the profiling
// events around the general steps.
static cld_status enqueue_steps(cld_ctx* h, const Layout& L, int n, int M, int pk, int j0, int j1, const WMap& wm,
                                bool events, int* launches, int* step_launches) {
    Params* prm = at<Params>(h, L.params);
    double* tpart = at<double>(h, L.tpart);
    uint32_t* vbits = at<uint32_t>(h, L.vbits);
    float* Y = h->kind == CLD_GENERAL ? at<float>(h, L.Y) : nullptr;
    const bool general = h->kind == CLD_GENERAL;
    const int64_t* rpT = general ? at<int64_t>(h, L.rowptrT) : h->rowptr;
    const int32_t* colT = general ? at<int32_t>(h, L.colT) : h->col;
    const void* valT = general ? at<void>(h, L.valT) : h->val;
    const int pbase = pk * kMaxPanel;
    const int mreal = (M - pbase) < L.panel ? (M - pbase) : L.panel;
    StepArgs a{};
    a.d = h->d;
    a.vbits = vbits;
    a.prm = prm;
    a.mreal = mreal;
    a.impl = h->impl;
    a.err = at<uint32_t>(h, L.flags) + 1;
    a.withhold_tile = h->withhold_tile;
    if (h->impl == 7 && L.plan && h->plan_panel == L.panel) {
        a.lcol = at<int32_t>(h, L.lcol);
        a.wtab = at<int32_t>(h, L.wtab);
    }
    for (int j = j0; j < j1; ++j) {
        // w_{j+1} <- step j; w_j and w_{j-1} from the previous steps (w_0 = v).
        if (events && h->profiling && j == 2) CUDA_TRY(cudaEventRecord(h->ev[2 * pk], h->stream));
        const float* wj = j >= 1 ? wbuf(h, L, j, wm) : nullptr;
        const float* wjm = j >= 2 ? wbuf(h, L, j - 1, wm) : nullptr;
        float* wout = wbuf(h, L, j + 1, wm);
        a.tpart = tpart + (size_t)j * L.grid * L.panel;
        StepKind kind;
        if (general) {
            // y = C w_j, then w_{j+1} from C^T y
            StepArgs p = a;
            p.rowptr = h->rowptr; p.col = h->col; p.val = h->val;
            p.x = wj; p.out = Y;
            CUDA_TRY(launch_step(L.panel, (int)h->dtype, j == 0 ? kProdBits : kProdFloat, L.grid,
                                 h->stream, p));
            ++*launches;
            a.rowptr = rpT; a.col = colT; a.val = valT;
            a.x = Y; a.own = wj; a.wprev = wjm; a.out = wout;
            kind = j == 0 ? kStepFirstFromFloat : j == 1 ? kStepSecond : kStepGeneral;
        } else {
            a.rowptr = h->rowptr; a.col = h->col; a.val = h->val;
            a.x = wj; a.own = wj; a.wprev = wjm; a.out = wout;
            kind = j == 0 ? kStepFirst : j == 1 ? kStepSecond : kStepGeneral;
        }
        CUDA_TRY(launch_step(L.panel, (int)h->dtype, kind, L.grid, h->stream, a));
        ++*launches;
        if (j >= 2) ++*step_launches;
    }
    if (events && h->profiling && n >= 3 && j1 == n) CUDA_TRY(cudaEventRecord(h->ev[2 * pk + 1], h->stream));
    return CLD_OK;
}

// Enqueues the probe signs and the n recurrence steps of panel pk, then the
// moment reduction of that panel.  Counts launches.
static cld_status enqueue_panel_forward(cld_ctx* h, const Layout& L, int n, int M, int pk, const WMap& wm,
                                        int* launches, int* step_launches) {
    const int pbase = pk * kMaxPanel;
    const int mreal = (M - pbase) < L.panel ? (M - pbase) : L.panel;
    CUDA_TRY(launch_probe_bits(h->d, L.nw, (uint32_t)pk, at<Params>(h, L.params), at<uint32_t>(h, L.vbits),
                               L.ggrid, h->stream));
    ++*launches;
    cld_status st = enqueue_steps(h, L, n, M, pk, 0, n, wm, true, launches, step_launches);
    if (st != CLD_OK) return st;
    if (n > 0) {
        CUDA_TRY(launch_reduce_moments(at<double>(h, L.tpart), n, L.grid, L.panel, mreal, M, pbase,
                                       at<double>(h, L.T), h->stream));
        ++*launches;
    }
    return CLD_OK;
}

// Dense tensor-core path: per panel, the split of the signs, n GEMM steps,
// the moment reduction; then the final sums.
static cld_status enqueue_dense(cld_ctx* h, const Layout& L, int n, int M, uint64_t seed, bool with_seed) {
    Params* prm = at<Params>(h, L.params);
    uint32_t* vbits = at<uint32_t>(h, L.vbits);
    double* tpart = at<double>(h, L.tpart);
    uint32_t* err = at<uint32_t>(h, L.flags) + 1;
    float* W[3] = {at<float>(h, L.W[0]), at<float>(h, L.W[1]), at<float>(h, L.W[2])};
    void* xt[2] = {h->ws + L.xt[0], h->ws + L.xt[1]};
    int launches = 0;
    if (with_seed) {
        CUDA_TRY(launch_set_seed(prm, seed, h->stream));
        ++launches;
    }
    if (L.dgrid <= 0) return fail(CLD_ERR_CUDA, "dense step: no launch configuration");
    // stream-K tile counters start at 0; each step's finishing CTAs reset them
    CUDA_TRY(cudaMemsetAsync(at<int>(h, L.dcnt), 0, (size_t)((h->d + 127) / 128) * 4, h->stream));
    const int npanels = (M + kMaxPanel - 1) / kMaxPanel;
    for (int pk = 0; pk < npanels; ++pk) {
        const int pbase = pk * kMaxPanel;
        const int mreal = (M - pbase) < L.panel ? (M - pbase) : L.panel;
        CUDA_TRY(launch_probe_bits(h->d, L.nw, (uint32_t)pk, prm, vbits, L.ggrid, h->stream));
        CUDA_TRY(launch_dense_sign_split(h->d, L.dx, L.panel, mreal, vbits, xt[0], L.ggrid, h->stream));
        launches += 2;
        for (int j = 0; j < n; ++j) {
            const int prev = j == 0 ? 0 : j == 1 ? 1 : 2;
            cudaError_t e = launch_dense_step(L.panel, prev, h->d, h->ld, h->val, xt[j % 2], L.dx,
                                              j >= 1 ? W[j % 3] : nullptr, j >= 2 ? W[(j - 1) % 3] : nullptr,
                                              W[(j + 1) % 3], xt[(j + 1) % 2], vbits,
                                              tpart + (size_t)j * L.grid * L.panel, prm, mreal, err,
                                              at<float>(h, L.dpart), at<int>(h, L.dcnt), L.dsmax, L.dgrid,
                                              h->stream);
            if (e == cudaErrorNotSupported) return fail(CLD_ERR_UNSUPPORTED, "TMA tensor map encoding unavailable");
            if (e != cudaSuccess) return fail(CLD_ERR_CUDA, "dense step launch: %s", cudaGetErrorString(e));
            ++launches;
        }
        if (n > 0) {
            CUDA_TRY(launch_reduce_moments(tpart, n, L.grid, L.panel, mreal, M, pbase, at<double>(h, L.T),
                                           h->stream));
            ++launches;
        }
    }
    CUDA_TRY(launch_finalize(n, M, h->d, 0, prm, at<double>(h, L.T), at<double>(h, L.coeffs),
                             at<double>(h, L.coef_scratch), at<double>(h, L.gamma_p), at<Result>(h, L.result),
                             h->stream));
    ++launches;
    h->last_total_launches = launches;
    h->last_step_launches = 0;
    return CLD_OK;
}

static cld_status ensure_events(cld_ctx* h, int M) {
    const int npanels = (M + kMaxPanel - 1) / kMaxPanel;
    while (h->profiling && (int)h->ev.size() < 2 * npanels) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        h->ev.push_back(e);
    }
    return CLD_OK;
}

static cld_status enqueue_estimate(cld_ctx* h, const Layout& L, int n, int M, uint64_t seed, bool with_seed) {
    Params* prm = at<Params>(h, L.params);
    int launches = 0, step_launches = 0;
    const int npanels = (M + kMaxPanel - 1) / kMaxPanel;
    cld_status st = ensure_events(h, M);
    if (st != CLD_OK) return st;
    if (with_seed) {
        CUDA_TRY(launch_set_seed(prm, seed, h->stream));
        ++launches;
    }
    for (int pk = 0; pk < npanels; ++pk) {
        st = enqueue_panel_forward(h, L, n, M, pk, WMap{kMapRing, 0}, &launches, &step_launches);
        if (st != CLD_OK) return st;
    }
    CUDA_TRY(launch_finalize(n, M, h->d, h->kind == CLD_GENERAL ? 1 : 0, prm, at<double>(h, L.T),
                             at<double>(h, L.coeffs), at<double>(h, L.coef_scratch), at<double>(h, L.gamma_p),
                             at<Result>(h, L.result), h->stream));
    ++launches;
    h->last_total_launches = launches;
    h->last_step_launches = step_launches;
    return CLD_OK;
}


// ---------------------------------------------------------------- batches
static void build_tiles(cld_ctx* h) {
    h->tiles.clear();
    h->tile_start.assign((size_t)h->nb + 1, 0);
    for (int b = 0; b < h->nb; ++b) {
        h->tile_start[b] = (int64_t)h->tiles.size();
        for (int64_t r = h->blk_rows[b]; r < h->blk_rows[b + 1]; r += h->tile_rows) {
            Tile t;
            t.lo = r;
            t.hi = r + h->tile_rows < h->blk_rows[b + 1] ? r + h->tile_rows : h->blk_rows[b + 1];
            t.blk = b;
            t.pad = 0;
            h->tiles.push_back(t);
        }
    }
    h->tile_start[h->nb] = (int64_t)h->tiles.size();
}

static cld_status upload_batch_tables(cld_ctx* h, const Layout& L) {
    CUDA_TRY(cudaMemcpyAsync(at<int64_t>(h, L.blk_rows), h->blk_rows.data(), sizeof(int64_t) * (h->nb + 1),
                             cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(at<int64_t>(h, L.tile_start), h->tile_start.data(), sizeof(int64_t) * (h->nb + 1),
                             cudaMemcpyHostToDevice, h->stream));
    if (!h->tiles.empty())
        CUDA_TRY(cudaMemcpyAsync(at<Tile>(h, L.tiles), h->tiles.data(), sizeof(Tile) * h->tiles.size(),
                                 cudaMemcpyHostToDevice, h->stream));
    return CLD_OK;
}

static BatchAuxArgs batch_aux_args(cld_ctx* h, const Layout& L) {
    BatchAuxArgs x{};
    x.bprm = at<Params>(h, L.bprm);
    x.ab = at<double>(h, L.ab);
    x.tiles = at<Tile>(h, L.tiles);
    x.ntiles = (int64_t)h->tiles.size();
    x.tile_start = at<int64_t>(h, L.tile_start);
    x.blk_rows = at<int64_t>(h, L.blk_rows);
    x.nw = L.nw;
    x.vbits = at<uint32_t>(h, L.vbits);
    x.dtype = (int)h->dtype;
    x.rowptr = h->rowptr;
    x.col = h->col;
    x.val = h->val;
    if (h->kind == CLD_GENERAL) {
        x.rowptrT = at<int64_t>(h, L.rowptrT);
        x.colT = at<int32_t>(h, L.colT);
        x.valT = at<void>(h, L.valT);
    }
    x.flags = at<uint32_t>(h, L.flags);
    return x;
}

static cld_status enqueue_batch(cld_ctx* h, const Layout& L, int n, int M, uint64_t seed, bool with_seed) {
    BatchAuxArgs x = batch_aux_args(h, L);
    const int nb = h->nb;
    int launches = 0, step_launches = 0;
    // profiling events around the general steps (plain launches only)
    const bool events = with_seed && h->profiling;
    if (events) {
        cld_status est = ensure_events(h, M);
        if (est != CLD_OK) return est;
    }
    if (with_seed) {
        x.seed = seed;
        CUDA_TRY(launch_batch_aux(0, nb, 1, h->stream, x));
        ++launches;
    }
    const bool general = h->kind == CLD_GENERAL;
    const int64_t ntiles = (int64_t)h->tiles.size();
    const int grid = (int)(ntiles < L.grid ? (ntiles > 0 ? ntiles : 1) : L.grid);
    double* tpart = at<double>(h, L.tpart);
    float* W[3] = {at<float>(h, L.W[0]), at<float>(h, L.W[1]), at<float>(h, L.W[2])};
    float* Y = general ? at<float>(h, L.Y) : nullptr;
    const int npanels = (M + kMaxPanel - 1) / kMaxPanel;
    for (int pk = 0; pk < npanels; ++pk) {
        const int pbase = pk * kMaxPanel;
        const int mreal = (M - pbase) < L.panel ? (M - pbase) : L.panel;
        x.panel = (uint32_t)pk;
        CUDA_TRY(launch_batch_aux(2, nb, L.ggrid, h->stream, x));
        ++launches;
        BatchStepArgs bs{};
        bs.tiles = x.tiles;
        bs.ntiles = ntiles;
        bs.bprm = x.bprm;
        bs.s.d = h->d;
        bs.s.vbits = x.vbits;
        bs.s.mreal = mreal;
        bs.s.impl = h->impl;
        bs.s.err = x.flags + 1;  // the staged tiles' pipeline error word
        for (int j = 0; j < n; ++j) {
            if (events && j == 2) CUDA_TRY(cudaEventRecord(h->ev[2 * pk], h->stream));
            const float* wj = j >= 1 ? W[j % 3] : nullptr;
            const float* wjm = j >= 2 ? W[(j - 1) % 3] : nullptr;
            float* wout = W[(j + 1) % 3];
            bs.tpart = tpart + (size_t)j * ntiles * L.panel;
            StepKind kind;
            if (general) {
                StepArgs p{};
                p.d = h->d;
                p.rowptr = h->rowptr; p.col = h->col; p.val = h->val;
                p.vbits = x.vbits; p.mreal = mreal; p.impl = h->impl;
                p.err = bs.s.err;  // the staged form's error word, as the C^T step's
                p.x = wj; p.out = Y;
                CUDA_TRY(launch_step(L.panel, (int)h->dtype, j == 0 ? kProdBits : kProdFloat, L.grid, h->stream, p));
                ++launches;
                bs.s.rowptr = x.rowptrT; bs.s.col = x.colT; bs.s.val = x.valT;
                bs.s.x = Y; bs.s.own = wj; bs.s.wprev = wjm; bs.s.out = wout;
                kind = j == 0 ? kStepFirstFromFloat : j == 1 ? kStepSecond : kStepGeneral;
            } else {
                bs.s.rowptr = h->rowptr; bs.s.col = h->col; bs.s.val = h->val;
                bs.s.x = wj; bs.s.own = wj; bs.s.wprev = wjm; bs.s.out = wout;
                kind = j == 0 ? kStepFirst : j == 1 ? kStepSecond : kStepGeneral;
            }
            CUDA_TRY(launch_batch_step(L.panel, (int)h->dtype, kind, grid, h->stream, bs));
            ++launches;
            if (j >= 2) ++step_launches;
        }
        if (events && n >= 3) CUDA_TRY(cudaEventRecord(h->ev[2 * pk + 1], h->stream));
        if (n > 0) {
            x.tpart = tpart;
            x.panel_width = L.panel;
            x.mreal = mreal;
            x.n = n;
            x.M = M;
            x.pbase = pbase;
            x.nsteps = n;
            x.T = at<double>(h, L.T);
            CUDA_TRY(launch_batch_aux(3, nb, 1, h->stream, x));
            ++launches;
        }
    }
    CUDA_TRY(launch_finalize_batch(nb, n, M, x.blk_rows, general ? 1 : 0, x.bprm, at<double>(h, L.T),
                                   at<double>(h, L.coeffs), at<double>(h, L.coef_scratch), at<double>(h, L.gamma_p),
                                   at<Result>(h, L.bres), h->stream));
    ++launches;
    h->last_total_launches = launches;
    h->last_step_launches = events ? step_launches : 0;
    return CLD_OK;
}

// Uploads the per-block intervals (a_b, b_b pairs) and sets each block's
// parameters on the device.
static cld_status apply_bintervals(cld_ctx* h, const Layout& L) {
    std::vector<double> ab((size_t)2 * h->nb);
    for (int b = 0; b < h->nb; ++b) {
        ab[2 * b] = h->ba[b];
        ab[2 * b + 1] = h->bb[b];
    }
    CUDA_TRY(cudaMemcpyAsync(at<double>(h, L.ab), ab.data(), sizeof(double) * ab.size(), cudaMemcpyHostToDevice,
                             h->stream));
    BatchAuxArgs x = batch_aux_args(h, L);
    CUDA_TRY(launch_batch_aux(1, h->nb, 1, h->stream, x));
    return CLD_OK;
}

// Variant 7's gather-window plan for the layout's panel width, computed on
// the handle's stream before the steps that read it (once per workspace and
// panel width; an estimate at another width recomputes it, so a graph
// captured at this width never reads another width's plan).
static cld_status ensure_plan(cld_ctx* h, const Layout& L) {
    if (h->impl != 7 || !L.plan || h->d == 0 || h->plan_panel == L.panel) return CLD_OK;
    const int capx = window_capx(L.panel, (int)h->dtype);
    if (capx <= 0) return CLD_OK;  // no windows at this panel width: variant 6 runs
    CUDA_TRY(launch_window_plan(L.panel, h->rowptr, h->col, h->d, capx, at<int32_t>(h, L.wtab),
                                at<int32_t>(h, L.lcol), h->sms, h->stream));
    h->plan_panel = L.panel;
    return CLD_OK;
}

// Runs enqueue(with_seed = false) through a CUDA graph captured once per
// (call kind, n, M, variant, workspace, tile size); the seed is set by a
// separate launch before the graph.
template <typename F>
static cld_status run_graph(cld_ctx* h, long long kind, int n, int M, F&& enqueue) {
    const long long key[6] = {kind, n, M, h->impl, (long long)(uintptr_t)h->ws, h->tile_rows};
    if (!h->gexec || memcmp(key, h->gkey, sizeof(key)) != 0) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        if (!h->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        // kernel attributes (shared-memory opt-in of the ring variants) are set
        // outside the capture
        if (!h->dense) {
            StepArgs a{};
            a.impl = h->impl;
            BatchStepArgs b{};
            b.s.impl = h->impl;
            for (int k = kStepFirst; k <= kStepFirstFromFloat; ++k) {
                CUDA_TRY(launch_step(panel_for(M), (int)h->dtype, (StepKind)k, 0, h->stream, a));
                if (h->nb > 0 && k != kProdBits && k != kProdFloat)
                    CUDA_TRY(launch_batch_step(panel_for(M), (int)h->dtype, (StepKind)k, 0, h->stream, b));
            }
        }
        // order the capture after work already queued on the user's stream
        cudaStream_t user = h->stream;
        const bool prof = h->profiling;
        h->profiling = false;
        h->stream = h->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        cld_status st = e == cudaSuccess ? enqueue() : fail(CLD_ERR_CUDA, "cudaStreamBeginCapture: %s",
                                                            cudaGetErrorString(e));
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
        h->stream = user;
        h->profiling = prof;
        if (st != CLD_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e2 != cudaSuccess) return fail(CLD_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
        e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->gexec = nullptr;
            return fail(CLD_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        memcpy(h->gkey, key, sizeof(key));
    }
    CUDA_TRY(cudaGraphLaunch(h->gexec, h->stream));
    return CLD_OK;
}

static cld_status read_result(cld_ctx* h, const Layout& L, int n, int M, double* logdet_out, double* stderr_out,
                              double* moments_out, Result* r) {
    CUDA_TRY(cudaMemcpyAsync(r, at<Result>(h, L.result), sizeof(Result), cudaMemcpyDeviceToHost, h->stream));
    if (moments_out)
        CUDA_TRY(cudaMemcpyAsync(moments_out, at<double>(h, L.T), sizeof(double) * (size_t)(n + 1) * M,
                                 cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (h->profiling && n >= 3) {
        float total = 0.f;
        const int npanels = (M + kMaxPanel - 1) / kMaxPanel;
        for (int pk = 0; pk < npanels; ++pk) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, h->ev[2 * pk], h->ev[2 * pk + 1]));
            total += ms;
        }
        h->last_step_ms = total;
    } else {
        h->last_step_ms = 0.f;
    }
    *logdet_out = r->logdet;
    if (stderr_out) *stderr_out = r->stderr_;
    h->last_n = n;
    h->last_M = M;
    return CLD_OK;
}

extern "C" {

const char* cld_last_error(void) { return g_err.c_str(); }
const char* cld_version(void) { return "libcld 0.1 (sm_103a)"; }

cld_status cld_create_csr(cld_handle* out, int64_t d, int64_t nnz, const int64_t* rowptr,
                          const int32_t* col, const void* val, cld_dtype val_dtype,
                          cld_kind kind, void* stream) {
    if (!out) return fail(CLD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (d < 0 || nnz < 0) return fail(CLD_ERR_INVALID, "negative size (d=%lld, nnz=%lld)",
                                      (long long)d, (long long)nnz);
    if (d >= (int64_t)INT32_MAX) return fail(CLD_ERR_INVALID, "d must be < 2^31 (int32 columns)");
    if (!rowptr || (nnz > 0 && (!col || !val)))
        return fail(CLD_ERR_INVALID, "NULL CSR array");
    if (val_dtype != CLD_F32 && val_dtype != CLD_BF16 && val_dtype != CLD_F64)
        return fail(CLD_ERR_INVALID, "unknown value dtype %d", (int)val_dtype);
    if (kind != CLD_SPD && kind != CLD_GENERAL) return fail(CLD_ERR_INVALID, "unknown kind %d", (int)kind);
    if (((uintptr_t)rowptr) % 8 || ((uintptr_t)col) % 4 || ((uintptr_t)val) % value_size(val_dtype))
        return fail(CLD_ERR_INVALID, "CSR arrays must be aligned to their element size");
    cld_ctx* h = new (std::nothrow) cld_ctx;
    if (!h) return fail(CLD_ERR_NOMEM, "host allocation failed");
    h->d = d; h->nnz = nnz; h->rowptr = rowptr; h->col = col; h->val = val;
    h->dtype = val_dtype; h->kind = kind; h->stream = (cudaStream_t)stream;
    // Default inner loop: cooperative 4-entry chunks pay off once rows hold
    // about 8 or more stored entries (measured on GB300: random SPD with 11
    // entries per row 3.22 vs 3.27 ms per step; 5-point grid 0.32 vs 0.22 ms).
    h->impl = default_impl(d, nnz);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return fail(CLD_ERR_CUDA, "no CUDA device");
    }
    *out = h;
    return CLD_OK;
}

void cld_destroy(cld_handle h) {
    if (!h) return;
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

cld_status cld_workspace_size(cld_handle h, int n, int M, int with_grad, size_t* bytes) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (!bytes || n < 0 || M < 1) return fail(CLD_ERR_INVALID, "bad arguments (n=%d, M=%d)", n, M);
    *bytes = make_layout(h, n, M, with_grad).total;
    return CLD_OK;
}

cld_status cld_set_workspace(cld_handle h, void* dev_ptr, size_t bytes) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (!dev_ptr) return fail(CLD_ERR_INVALID, "NULL workspace");
    if (((uintptr_t)dev_ptr) % 256) return fail(CLD_ERR_INVALID, "workspace not 256-byte aligned");
    const Layout L = make_layout(h, 0, 1, 0);
    if (bytes < L.run) return fail(CLD_ERR_NOMEM, "workspace smaller than the fixed header");
    h->ws = static_cast<char*>(dev_ptr);
    h->ws_bytes = bytes;
    h->ready = false;
    h->plan_panel = 0;
    uint32_t* flags = at<uint32_t>(h, L.flags);
    CUDA_TRY(cudaMemsetAsync(flags, 0, 256, h->stream));
    if (h->d > 0 && !h->dense)
        CUDA_TRY(launch_validate_csr(h->d, h->nnz, h->rowptr, h->col, h->val, (int)h->dtype, flags,
                                     stream_grid(h), h->stream));
    uint32_t f = 0;
    CUDA_TRY(cudaMemcpyAsync(&f, flags, 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (f & 1u) return fail(CLD_ERR_INVALID, "row pointers must start at 0, end at nnz and not decrease");
    if (f & 2u) return fail(CLD_ERR_INVALID, "column index out of range [0, d)");
    if (f & 4u) return fail(CLD_ERR_INVALID, "non-finite stored value");
    if (h->nb > 0) {
        cld_status st = upload_batch_tables(h, L);
        if (st != CLD_OK) return st;
        BatchAuxArgs x = batch_aux_args(h, L);
        if (h->d > 0) CUDA_TRY(launch_batch_aux(6, h->nb, stream_grid(h), h->stream, x));
        CUDA_TRY(cudaMemcpyAsync(&f, flags, 4, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (f & 8u) return fail(CLD_ERR_INVALID, "batch matrix is not block diagonal (column outside its block)");
        if (h->have_bintervals) {
            st = apply_bintervals(h, L);
            if (st != CLD_OK) return st;
        }
    }
    if (h->kind == CLD_GENERAL && h->d > 0) {
        CUDA_TRY(launch_transpose(h->d, h->nnz, h->rowptr, h->col, h->val, value_size(h->dtype),
                                  at<int64_t>(h, L.rowptrT), at<int32_t>(h, L.colT), at<void>(h, L.valT),
                                  at<int64_t>(h, L.tscratch), stream_grid(h), h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    if (h->have_interval)
        CUDA_TRY(launch_set_params(at<Params>(h, L.params), h->a, h->b, h->stream));
    h->ready = true;
    return CLD_OK;
}

cld_status cld_set_interval(cld_handle h, double a, double b) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (!(a > 0.0) || !(a < b) || !isfinite(a) || !isfinite(b))
        return fail(CLD_ERR_INTERVAL, "interval must satisfy 0 < a < b (got [%g, %g])", a, b);
    h->a = a;
    h->b = b;
    h->have_interval = true;
    if (h->ws) {
        const Layout L = make_layout(h, 0, 1, 0);
        CUDA_TRY(launch_set_params(at<Params>(h, L.params), a, b, h->stream));
    }
    return CLD_OK;
}

cld_status cld_auto_interval(cld_handle h, int lanczos_iters, double* a_out, double* b_out) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (!h->ready) return fail(CLD_ERR_NOMEM, "workspace not set");
    if (h->nb > 0) return fail(CLD_ERR_INVALID, "batch handle: use cld_batch_auto_intervals");
    if (h->d == 0) return fail(CLD_ERR_INTERVAL, "empty matrix has no spectrum");
    if (lanczos_iters < 0 || lanczos_iters > 4000) return fail(CLD_ERR_INVALID, "lanczos_iters in [0, 4000]");
    const Layout L = make_layout(h, 0, 1, 0);
    if (lanczos_iters > 0 && h->ws_bytes < make_layout(h, 0, 1, 0).total)
        return fail(CLD_ERR_NOMEM, "workspace too small for the Lanczos pass");
    Params* prm = at<Params>(h, L.params);
    uint32_t* flags = at<uint32_t>(h, L.flags);
    CUDA_TRY(cudaMemsetAsync(flags, 0, 4, h->stream));
    if (h->dense) {
        if (lanczos_iters > 0) return fail(CLD_ERR_UNSUPPORTED, "Lanczos is available for CSR matrices");
        CUDA_TRY(launch_dense_gershgorin(h->d, h->ld, h->val, at<double>(h, L.gpart), L.ggrid, prm, flags,
                                         h->stream));
    } else if (h->kind == CLD_SPD) {
        CUDA_TRY(launch_gershgorin(h->d, h->rowptr, h->col, h->val, (int)h->dtype, at<double>(h, L.gpart),
                                   L.ggrid, prm, flags, h->stream));
        if (lanczos_iters > 0)
            CUDA_TRY(launch_lanczos(h->d, h->rowptr, h->col, h->val, (int)h->dtype, lanczos_iters,
                                    at<double>(h, L.lanczos), at<double>(h, L.lanczos) + 5 * h->d,
                                    L.ggrid, prm, flags, h->stream));
    } else {
        CUDA_TRY(launch_general_bounds(h->d, h->rowptr, h->col, h->val, at<int64_t>(h, L.rowptrT),
                                       at<int32_t>(h, L.colT), at<void>(h, L.valT), (int)h->dtype,
                                       at<double>(h, L.gpart), L.ggrid, prm, flags, h->stream));
    }
    Params p{};
    uint32_t f = 0;
    CUDA_TRY(cudaMemcpyAsync(&p, prm, sizeof(Params), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(&f, flags, 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (a_out) *a_out = p.a;
    if (b_out) *b_out = p.b;
    if ((f & 0x100u) || !p.interval_ok) {
        h->have_interval = false;
        return fail(CLD_ERR_INTERVAL, "computed interval [%g, %g] is not a valid 0 < a < b", p.a, p.b);
    }
    h->a = p.a;
    h->b = p.b;
    h->have_interval = true;
    return CLD_OK;
}

cld_status cld_estimate(cld_handle h, int n, int M, uint64_t seed, double* logdet_out,
                        double* stderr_out, double* moments_out) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (n < 0 || M < 1) return fail(CLD_ERR_INVALID, "need n >= 0 and M >= 1 (n=%d, M=%d)", n, M);
    if (n > 100000) return fail(CLD_ERR_INVALID, "degree n > 100000 is not supported");
    if (!logdet_out) return fail(CLD_ERR_INVALID, "logdet_out is NULL");
    if (h->nb > 0) return fail(CLD_ERR_INVALID, "batch handle: use cld_batch_estimate");
    if (!h->have_interval) return fail(CLD_ERR_INTERVAL, "no spectral interval set");
    if (!h->ready) return fail(CLD_ERR_NOMEM, "workspace not set");
    const Layout L = make_layout(h, n, M, 0);
    if (h->ws_bytes < L.total)
        return fail(CLD_ERR_NOMEM, "workspace has %zu bytes, %zu needed", h->ws_bytes, L.total);
    h->last_n = -1;
    if (h->d == 0) {
        *logdet_out = 0.0;
        if (stderr_out) *stderr_out = 0.0;
        if (moments_out) memset(moments_out, 0, sizeof(double) * (size_t)(n + 1) * M);
        h->last_total_launches = h->last_step_launches = 0;
        return CLD_OK;
    }
    cld_status st = ensure_plan(h, L);
    if (st != CLD_OK) return st;
    uint32_t* err = at<uint32_t>(h, L.flags) + 1;
    const bool pipelined = h->dense || h->impl >= 6;  // kernels with bounded pipeline waits
    if (pipelined) CUDA_TRY(cudaMemsetAsync(err, 0, 4, h->stream));
    auto body = [&](bool with_seed) {
        return h->dense ? enqueue_dense(h, L, n, M, seed, with_seed) : enqueue_estimate(h, L, n, M, seed, with_seed);
    };
    if (h->use_graph) {
        CUDA_TRY(launch_set_seed(at<Params>(h, L.params), seed, h->stream));
        st = run_graph(h, h->dense ? 3 : 1, n, M, [&]() { return body(false); });
        ++h->last_total_launches;
    } else {
        st = body(true);
    }
    if (st != CLD_OK) return st;
    uint32_t derr = 0;
    if (pipelined) CUDA_TRY(cudaMemcpyAsync(&derr, err, 4, cudaMemcpyDeviceToHost, h->stream));
    Result r{};
    st = read_result(h, L, n, M, logdet_out, stderr_out, moments_out, &r);
    if (st != CLD_OK) return st;
    if (derr)
        return fail(CLD_ERR_TIMEOUT, "a %s pipeline wait gave up (results invalid)",
                    h->dense ? "dense-step" : "staged-step");
    if (r.spectrum_bad)
        return fail(CLD_ERR_SPECTRUM,
                    "max |t_jp|/d = %g exceeds 1: the spectrum is not inside [%g, %g]", r.max_ratio,
                    h->a, h->b);
    return CLD_OK;
}

cld_status cld_last_details(cld_handle h, double* coeffs_out, double* gamma_p_out) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (h->last_n < 0) return fail(CLD_ERR_INVALID, "no completed estimate");
    const Layout L = make_layout(h, h->last_n, h->last_M, 0);
    if (coeffs_out)
        CUDA_TRY(cudaMemcpyAsync(coeffs_out, at<double>(h, L.coeffs), sizeof(double) * (h->last_n + 1),
                                 cudaMemcpyDeviceToHost, h->stream));
    if (gamma_p_out)
        CUDA_TRY(cudaMemcpyAsync(gamma_p_out, at<double>(h, L.gamma_p), sizeof(double) * h->last_M,
                                 cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return CLD_OK;
}

cld_status cld_grad(cld_handle h, int n, int M, uint64_t seed, double* logdet_out, float* dvalues_dev) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (h->kind != CLD_SPD || h->nb > 0 || h->dense)
        return fail(CLD_ERR_UNSUPPORTED, "cld_grad supports single sparse CLD_SPD matrices only");
    if (n < 0 || M < 1 || n > 100000) return fail(CLD_ERR_INVALID, "need 0 <= n <= 100000 and M >= 1");
    if (!logdet_out) return fail(CLD_ERR_INVALID, "logdet_out is NULL");
    if (!dvalues_dev && h->nnz > 0) return fail(CLD_ERR_INVALID, "dvalues_dev is NULL");
    if (!h->have_interval) return fail(CLD_ERR_INTERVAL, "no spectral interval set");
    if (!h->ready) return fail(CLD_ERR_NOMEM, "workspace not set");
    const Layout L = make_layout(h, n, M, 1);
    if (h->ws_bytes < L.total)
        return fail(CLD_ERR_NOMEM, "gradient workspace has %zu bytes, %zu needed", h->ws_bytes, L.total);
    h->last_n = -1;
    if (h->d == 0) {
        *logdet_out = 0.0;
        return CLD_OK;
    }
    Params* prm = at<Params>(h, L.params);
    uint32_t* flags = at<uint32_t>(h, L.flags);
    float* H = at<float>(h, L.H);
    int launches = 0, step_launches = 0;
    cld_status st = ensure_events(h, M);
    if (st != CLD_OK) return st;
    st = ensure_plan(h, L);
    if (st != CLD_OK) return st;
    CUDA_TRY(cudaMemsetAsync(flags, 0, 8, h->stream));  // flags and the pipeline error word
    CUDA_TRY(cudaMemsetAsync(H, 0, (size_t)h->nnz * 4, h->stream));
    CUDA_TRY(launch_set_seed(prm, seed, h->stream));
    CUDA_TRY(launch_coeffs(n, prm, at<double>(h, L.coeffs), at<double>(h, L.coef_scratch), h->stream));
    launches += 2;
    const int npanels = (M + kMaxPanel - 1) / kMaxPanel;
    float* lam[3] = {at<float>(h, L.lam[0]), at<float>(h, L.lam[1]), at<float>(h, L.lam[2])};
    for (int pk = 0; pk < npanels; ++pk) {
        const WMap fwd{L.ckK > 0 ? kMapCkpt : kMapAll, 0};
        st = enqueue_panel_forward(h, L, n, M, pk, fwd, &launches, &step_launches);
        if (st != CLD_OK) return st;
        if (n == 0) continue;
        const int mreal = (M - pk * kMaxPanel) < L.panel ? (M - pk * kMaxPanel) : L.panel;
        AdjArgs a{};
        a.d = h->d;
        a.rowptr = h->rowptr;
        a.col = h->col;
        a.val = h->val;
        a.vbits = at<uint32_t>(h, L.vbits);
        a.H = H;
        a.coeffs = at<double>(h, L.coeffs);
        a.prm = prm;
        a.mreal = mreal;
        a.err = flags + 1;
        a.withhold_tile = h->withhold_tile;
        // the reverse step follows the forward's form: per-lane, wide lanes
        // (variant 5) or staged tiles (variants 6 and 7; a windowed reverse
        // step measured slower than the staged one: its per-entry SDDMM term
        // keeps it issue bound, not latency bound; both forms cover 2048 /
        // panel rows per CTA pass)
        const int form = L.panel < 8 ? 0 : h->impl >= 6 ? 2 : h->impl == 5 ? 1 : 0;
        const int rows_per_cta = (kThreads / 32) * ((form > 0 ? 256 : 128) / L.panel);
        const int64_t need = (h->d + rows_per_cta - 1) / rows_per_cta;
        const int64_t full = (int64_t)adjoint_ctas_per_sm(L.panel, (int)h->dtype, form) * h->sms;
        const int agrid = (int)(need < full ? (need > 0 ? need : 1) : full);
        // lambda_i lives in lam[i % 3]; reverse steps i = n, n-1, ..., 1, step
        // i < n reading w_i
        auto reverse_step = [&](int i, const WMap& wm) -> cld_status {
            a.ci = i;
            a.lam_out = lam[i % 3];
            a.lam_in = lam[(i + 1) % 3];
            a.lam_prev = lam[(i + 2) % 3];
            a.w = i <= n - 1 ? wbuf(h, L, i, wm) : nullptr;
            const int mode = i == n ? 0 : i == n - 1 ? 1 : 2;
            CUDA_TRY(launch_adjoint(L.panel, (int)h->dtype, mode, agrid, h->stream, a, form));
            ++launches;
            return CLD_OK;
        };
        if (L.ckK == 0) {
            for (int i = n; i >= 1; --i) {
                st = reverse_step(i, WMap{kMapAll, 0});
                if (st != CLD_OK) return st;
            }
        } else {
            // checkpointed: segment s holds w_{sK+1} .. w_{min((s+1)K, n-1)}; from
            // the last segment down, recompute it from its checkpoint pair (or
            // from v for s = 0), then take its reverse steps
            st = reverse_step(n, WMap{kMapSeg, 0});
            if (st != CLD_OK) return st;
            for (int sg = L.nseg - 1; sg >= 0; --sg) {
                const int lo = sg * L.ckK + 1;
                const int hi = (sg + 1) * L.ckK < n - 1 ? (sg + 1) * L.ckK : n - 1;
                const WMap seg{kMapSeg, lo};
                st = enqueue_steps(h, L, n, M, pk, lo - 1, hi, seg, false, &launches, &step_launches);
                if (st != CLD_OK) return st;
                for (int i = hi; i >= lo; --i) {
                    st = reverse_step(i, seg);
                    if (st != CLD_OK) return st;
                }
            }
        }
        a.lam_in = lam[1 % 3];  // lambda_1
        a.lam_out = nullptr;
        a.w = nullptr;
        CUDA_TRY(launch_adjoint(L.panel, (int)h->dtype, 3, agrid, h->stream, a, form));
        ++launches;
    }
    CUDA_TRY(launch_finalize(n, M, h->d, 0, prm, at<double>(h, L.T), at<double>(h, L.coeffs),
                             at<double>(h, L.coef_scratch), at<double>(h, L.gamma_p), at<Result>(h, L.result),
                             h->stream));
    ++launches;
    if (h->nnz > 0) {
        CUDA_TRY(launch_adjoint_gather(h->d, h->rowptr, h->col, H, 2.0 / (h->b - h->a) / M, dvalues_dev, flags,
                                       L.ggrid, h->stream));
        ++launches;
    }
    h->last_total_launches = launches;
    h->last_step_launches = step_launches;
    uint32_t f[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(f, flags, 8, cudaMemcpyDeviceToHost, h->stream));
    Result r{};
    st = read_result(h, L, n, M, logdet_out, nullptr, nullptr, &r);
    if (st != CLD_OK) return st;
    if (f[0] & 0x10000u) return fail(CLD_ERR_INVALID, "cld_grad needs a structurally symmetric sparsity pattern");
    if (f[1]) return fail(CLD_ERR_TIMEOUT, "a staged-step pipeline wait gave up (results invalid)");
    if (r.spectrum_bad)
        return fail(CLD_ERR_SPECTRUM, "max |t_jp|/d = %g exceeds 1: the spectrum is not inside [%g, %g]",
                    r.max_ratio, h->a, h->b);
    return CLD_OK;
}

cld_status cld_set_grad_checkpoint(cld_handle h, int interval) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (interval < 0 || interval == 1 || interval > 100000)
        return fail(CLD_ERR_INVALID, "checkpoint interval must be 0 (keep every w_j) or in [2, 100000]");
    h->ckpt = interval;
    return CLD_OK;
}

cld_status cld_host_workspace_size(int64_t d, int64_t nnz, cld_dtype val_dtype, int n, int M,
                                   size_t* bytes) {
    if (!bytes || d < 0 || nnz < 0 || n < 0 || M < 1) return fail(CLD_ERR_INVALID, "bad arguments");
    if (val_dtype != CLD_F32 && val_dtype != CLD_BF16 && val_dtype != CLD_F64)
        return fail(CLD_ERR_INVALID, "unknown value dtype");
    cld_ctx tmp;
    tmp.d = d; tmp.nnz = nnz; tmp.dtype = val_dtype; tmp.kind = CLD_GENERAL;  // largest layout
    tmp.impl = default_impl(d, nnz);
    if (cudaGetDevice(&tmp.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&tmp.sms, cudaDevAttrMultiProcessorCount, tmp.device) != cudaSuccess)
        return fail(CLD_ERR_CUDA, "no CUDA device");
    const size_t csr = align_up((size_t)(d + 1) * 8) + align_up((size_t)nnz * 4) +
                       align_up((size_t)nnz * value_size(val_dtype));
    *bytes = csr + make_layout(&tmp, n, M, 0).total;
    return CLD_OK;
}

cld_status cld_logdet_csr_host(int64_t d, int64_t nnz, const int64_t* rowptr_host,
                               const int32_t* col_host, const void* val_host, cld_dtype val_dtype,
                               cld_kind kind, double a, double b, int n, int M, uint64_t seed,
                               void* workspace_dev, size_t workspace_bytes, void* stream,
                               double* logdet_out, double* stderr_out) {
    size_t need = 0;
    cld_status st = cld_host_workspace_size(d, nnz, val_dtype, n, M, &need);
    if (st) return st;
    if (!workspace_dev || workspace_bytes < need)
        return fail(CLD_ERR_NOMEM, "host-input workspace needs %zu bytes", need);
    if (((uintptr_t)workspace_dev) % 256) return fail(CLD_ERR_INVALID, "workspace not 256-byte aligned");
    if (!rowptr_host || (nnz > 0 && (!col_host || !val_host))) return fail(CLD_ERR_INVALID, "NULL CSR array");
    cudaStream_t s = (cudaStream_t)stream;
    char* w = static_cast<char*>(workspace_dev);
    const size_t o_col = align_up((size_t)(d + 1) * 8);
    const size_t o_val = o_col + align_up((size_t)nnz * 4);
    const size_t o_ws = o_val + align_up((size_t)nnz * value_size(val_dtype));
    CUDA_TRY(cudaMemcpyAsync(w, rowptr_host, (size_t)(d + 1) * 8, cudaMemcpyHostToDevice, s));
    if (nnz > 0) {
        CUDA_TRY(cudaMemcpyAsync(w + o_col, col_host, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(w + o_val, val_host, (size_t)nnz * value_size(val_dtype),
                                 cudaMemcpyHostToDevice, s));
    }
    cld_handle h = nullptr;
    st = cld_create_csr(&h, d, nnz, reinterpret_cast<int64_t*>(w), reinterpret_cast<int32_t*>(w + o_col),
                        w + o_val, val_dtype, kind, stream);
    if (st) return st;
    st = cld_set_interval(h, a, b);
    if (!st) st = cld_set_workspace(h, w + o_ws, workspace_bytes - o_ws);
    if (!st) st = cld_estimate(h, n, M, seed, logdet_out, stderr_out, nullptr);
    cld_destroy(h);
    return st;
}


cld_status cld_create_dense(cld_handle* out, int64_t d, int64_t ld, const void* val_dev, cld_dtype val_dtype,
                            cld_kind kind, void* stream) {
    if (!out) return fail(CLD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (d < 1 || ld < d) return fail(CLD_ERR_INVALID, "need d >= 1 and ld >= d");
    if (!val_dev) return fail(CLD_ERR_INVALID, "NULL matrix");
    if (val_dtype != CLD_BF16)
        return fail(CLD_ERR_UNSUPPORTED, "the dense tensor-core path takes BF16 values");
    if (kind != CLD_SPD) return fail(CLD_ERR_UNSUPPORTED, "the dense path takes symmetric positive definite B");
    if (ld % 8 != 0 || ((uintptr_t)val_dev) % 16 != 0)
        return fail(CLD_ERR_INVALID, "dense rows must start 16-byte aligned (ld multiple of 8, aligned base)");
    cld_ctx* h = new (std::nothrow) cld_ctx;
    if (!h) return fail(CLD_ERR_NOMEM, "host allocation failed");
    h->d = d;
    h->nnz = 0;
    h->val = val_dev;
    h->dtype = val_dtype;
    h->kind = kind;
    h->stream = (cudaStream_t)stream;
    h->dense = true;
    h->ld = ld;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return fail(CLD_ERR_CUDA, "no CUDA device");
    }
    *out = h;
    return CLD_OK;
}

cld_status cld_create_batch(cld_handle* out, int nb, const int64_t* blk_rows, int64_t nnz, const int64_t* rowptr,
                            const int32_t* col, const void* val, cld_dtype val_dtype, cld_kind kind, void* stream) {
    if (!out) return fail(CLD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (nb < 1 || !blk_rows) return fail(CLD_ERR_INVALID, "need nb >= 1 and block row offsets");
    if (blk_rows[0] != 0) return fail(CLD_ERR_INVALID, "blk_rows[0] must be 0");
    for (int b = 0; b < nb; ++b)
        if (blk_rows[b + 1] < blk_rows[b]) return fail(CLD_ERR_INVALID, "blk_rows must not decrease");
    cld_handle h = nullptr;
    cld_status st = cld_create_csr(&h, blk_rows[nb], nnz, rowptr, col, val, val_dtype, kind, stream);
    if (st != CLD_OK) return st;
    h->nb = nb;
    h->blk_rows.assign(blk_rows, blk_rows + nb + 1);
    h->max_tiles = 0;
    for (int b = 0; b < nb; ++b) h->max_tiles += (blk_rows[b + 1] - blk_rows[b] + 255) / 256;
    h->impl = 0;  // small blocks: per-lane loads
    build_tiles(h);
    *out = h;
    return CLD_OK;
}

cld_status cld_batch_get_tile_rows(cld_handle h, int* rows) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (h->nb == 0) return fail(CLD_ERR_INVALID, "not a batch handle");
    if (!rows) return fail(CLD_ERR_INVALID, "rows is NULL");
    *rows = h->tile_rows;
    return CLD_OK;
}

cld_status cld_batch_set_tile_rows(cld_handle h, int rows) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (h->nb == 0) return fail(CLD_ERR_INVALID, "not a batch handle");
    if (rows < 256 || rows > (1 << 20)) return fail(CLD_ERR_INVALID, "tile rows must be in [256, 2^20]");
    h->tile_rows = rows;
    build_tiles(h);
    if (h->ws) {
        const Layout L = make_layout(h, 0, 1, 0);
        cld_status st = upload_batch_tables(h, L);
        if (st != CLD_OK) return st;
    }
    return CLD_OK;
}

cld_status cld_batch_set_intervals(cld_handle h, const double* a, const double* b) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (h->nb == 0) return fail(CLD_ERR_INVALID, "not a batch handle");
    if (!a || !b) return fail(CLD_ERR_INVALID, "NULL interval arrays");
    for (int k = 0; k < h->nb; ++k)
        if (!(a[k] > 0.0) || !(a[k] < b[k]) || !isfinite(a[k]) || !isfinite(b[k]))
            return fail(CLD_ERR_INTERVAL, "block %d: interval must satisfy 0 < a < b (got [%g, %g])", k, a[k], b[k]);
    h->ba.assign(a, a + h->nb);
    h->bb.assign(b, b + h->nb);
    h->have_bintervals = true;
    if (h->ws) return apply_bintervals(h, make_layout(h, 0, 1, 0));
    return CLD_OK;
}

cld_status cld_batch_auto_intervals(cld_handle h, double* a_out, double* b_out) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (h->nb == 0) return fail(CLD_ERR_INVALID, "not a batch handle");
    if (!h->ready) return fail(CLD_ERR_NOMEM, "workspace not set");
    const Layout L = make_layout(h, 0, 1, 0);
    BatchAuxArgs x = batch_aux_args(h, L);
    CUDA_TRY(cudaMemsetAsync(x.flags, 0, 4, h->stream));
    CUDA_TRY(launch_batch_aux(h->kind == CLD_GENERAL ? 5 : 4, h->nb, 1, h->stream, x));
    std::vector<Params> p((size_t)h->nb);
    CUDA_TRY(cudaMemcpyAsync(p.data(), x.bprm, sizeof(Params) * h->nb, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->ba.resize(h->nb);
    h->bb.resize(h->nb);
    int bad = -1;
    for (int k = 0; k < h->nb; ++k) {
        h->ba[k] = p[k].a;
        h->bb[k] = p[k].b;
        if (a_out) a_out[k] = p[k].a;
        if (b_out) b_out[k] = p[k].b;
        if (!p[k].interval_ok && bad < 0) bad = k;
    }
    if (bad >= 0) {
        h->have_bintervals = false;
        return fail(CLD_ERR_INTERVAL, "block %d: computed interval [%g, %g] is not a valid 0 < a < b", bad,
                    p[bad].a, p[bad].b);
    }
    h->have_bintervals = true;
    return CLD_OK;
}

cld_status cld_batch_estimate(cld_handle h, int n, int M, uint64_t seed, double* logdet_out, double* stderr_out) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (h->nb == 0) return fail(CLD_ERR_INVALID, "not a batch handle");
    if (n < 0 || M < 1 || n > 100000) return fail(CLD_ERR_INVALID, "need 0 <= n <= 100000 and M >= 1");
    if (!logdet_out) return fail(CLD_ERR_INVALID, "logdet_out is NULL");
    if (!h->have_bintervals) return fail(CLD_ERR_INTERVAL, "no block intervals set");
    if (!h->ready) return fail(CLD_ERR_NOMEM, "workspace not set");
    const Layout L = make_layout(h, n, M, 0);
    if (h->ws_bytes < L.total)
        return fail(CLD_ERR_NOMEM, "workspace has %zu bytes, %zu needed", h->ws_bytes, L.total);
    cld_status st;
    uint32_t* perr = at<uint32_t>(h, L.flags) + 1;
    if (h->impl == 6) CUDA_TRY(cudaMemsetAsync(perr, 0, 4, h->stream));
    if (h->use_graph) {
        BatchAuxArgs x = batch_aux_args(h, L);
        x.seed = seed;
        CUDA_TRY(launch_batch_aux(0, h->nb, 1, h->stream, x));
        st = run_graph(h, 2, n, M, [&]() { return enqueue_batch(h, L, n, M, seed, false); });
        ++h->last_total_launches;
    } else {
        st = enqueue_batch(h, L, n, M, seed, true);
    }
    if (st != CLD_OK) return st;
    std::vector<Result> r((size_t)h->nb);
    uint32_t perr_h = 0;
    if (h->impl == 6) CUDA_TRY(cudaMemcpyAsync(&perr_h, perr, 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(r.data(), at<Result>(h, L.bres), sizeof(Result) * h->nb, cudaMemcpyDeviceToHost,
                             h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->last_step_ms = 0.f;
    if (h->profiling && !h->use_graph && n >= 3) {
        const int npanels = (M + kMaxPanel - 1) / kMaxPanel;
        for (int pk = 0; pk < npanels; ++pk) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, h->ev[2 * pk], h->ev[2 * pk + 1]));
            h->last_step_ms += ms;
        }
    }
    if (perr_h) return fail(CLD_ERR_TIMEOUT, "a staged-step pipeline wait gave up (results invalid)");
    int bad = -1;
    for (int k = 0; k < h->nb; ++k) {
        logdet_out[k] = r[k].logdet;
        if (stderr_out) stderr_out[k] = r[k].stderr_;
        if (r[k].spectrum_bad && bad < 0) bad = k;
    }
    if (bad >= 0)
        return fail(CLD_ERR_SPECTRUM, "block %d: max |t_jp|/d = %g exceeds 1: spectrum not inside [%g, %g]", bad,
                    r[bad].max_ratio, h->ba[bad], h->bb[bad]);
    return CLD_OK;
}

cld_status cld_set_graph(cld_handle h, int on) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    h->use_graph = on != 0;
    return CLD_OK;
}

cld_status cld_set_kernel_variant(cld_handle h, int variant) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (variant < 0 || variant >= kNumStepImpls)
        return fail(CLD_ERR_INVALID, "variant must be in [0, %d)", kNumStepImpls);
    if (h->nb > 0 && variant >= kNumBatchImpls)
        return fail(CLD_ERR_INVALID, "batch handles take variants 0 .. %d", kNumBatchImpls - 1);
    h->impl = variant;
    return CLD_OK;
}

cld_status cld_autotune(cld_handle h, int M, int reps, int* variant_out, float* ms_out) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (M < 1 || reps < 1 || reps > 1000) return fail(CLD_ERR_INVALID, "need M >= 1 and 1 <= reps <= 1000");
    if (!h->ready) return fail(CLD_ERR_NOMEM, "workspace not set");
    if (!(h->nb > 0 ? h->have_bintervals : h->have_interval))
        return fail(CLD_ERR_INTERVAL, "no spectral interval set");
    if (h->d == 0) return fail(CLD_ERR_INVALID, "empty matrix");
    if (h->dense) return fail(CLD_ERR_UNSUPPORTED, "the dense path has a single kernel");
    const int saved = h->impl;
    const int saved_tiles = h->tile_rows;
    int best = -1, best_tiles = saved_tiles;
    float best_ms = 0.f, saved_ms = -1.f;
    uint32_t* perr = at<uint32_t>(h, make_layout(h, 0, 1, 0).flags) + 1;  // pipeline error word (variant 6)
    CUDA_TRY(cudaMemsetAsync(perr, 0, 4, h->stream));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // batches: every variant at every tile size; single matrices: variants only
    static const int kTileRows[] = {256, 512, 1024, 2048, 4096};
    const int ntiles_cand = h->nb > 0 ? (int)(sizeof(kTileRows) / sizeof(kTileRows[0])) : 1;
    for (int ti = 0; ti < ntiles_cand; ++ti) {
        if (h->nb > 0) {
            h->tile_rows = kTileRows[ti];
            build_tiles(h);
            const cld_status ust = upload_batch_tables(h, make_layout(h, 0, 1, 0));
            if (ust != CLD_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return ust;
            }
        }
        for (int v = 0; v < (h->nb > 0 ? kNumBatchImpls : kNumStepImpls); ++v) {
            h->impl = v;
            const Layout L = make_layout(h, 2, M, 0);
            if (L.total > h->ws_bytes) continue;
            // Timing runs of the general step on the current workspace contents
            // (whatever they hold: the cost does not depend on the values).
            StepArgs a{};
            a.d = h->d;
            a.vbits = at<uint32_t>(h, L.vbits);
            a.prm = at<Params>(h, L.params);
            a.mreal = M < L.panel ? M : L.panel;
            a.impl = v;
            a.err = at<uint32_t>(h, L.flags) + 1;
            if (v == 7 && L.plan) {
                const cld_status pst = ensure_plan(h, L);
                if (pst != CLD_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return pst;
                }
                if (h->plan_panel == L.panel) {
                    a.lcol = at<int32_t>(h, L.lcol);
                    a.wtab = at<int32_t>(h, L.wtab);
                }
            }
            const bool general = h->kind == CLD_GENERAL;
            a.rowptr = general ? at<int64_t>(h, L.rowptrT) : h->rowptr;
            a.col = general ? at<int32_t>(h, L.colT) : h->col;
            a.val = general ? at<void>(h, L.valT) : h->val;
            a.x = at<float>(h, L.W[1]);
            a.own = at<float>(h, L.W[1]);
            a.wprev = at<float>(h, L.W[0]);
            a.out = at<float>(h, L.W[2]);
            a.tpart = at<double>(h, L.tpart);
            CUDA_TRY(cudaMemsetAsync(at<float>(h, L.W[0]), 0, 3 * ((size_t)h->d * L.panel * 4), h->stream));
            BatchStepArgs ba{};
            int bgrid = L.grid;
            if (h->nb > 0) {  // batches: time the tile-queue kernel
                ba.s = a;
                ba.tiles = at<Tile>(h, L.tiles);
                ba.ntiles = (int64_t)h->tiles.size();
                ba.bprm = at<Params>(h, L.bprm);
                ba.tpart = at<double>(h, L.tpart);
                bgrid = (int)(ba.ntiles < L.grid ? (ba.ntiles > 0 ? ba.ntiles : 1) : L.grid);
            }
            // general C: a degree step is y = C w_j and then the step on C^T y,
            // both with the variant under test, so both are timed
            StepArgs pa = a;
            if (general) {
                CUDA_TRY(cudaMemsetAsync(at<float>(h, L.Y), 0, (size_t)h->d * L.panel * 4, h->stream));
                pa.rowptr = h->rowptr; pa.col = h->col; pa.val = h->val;
                pa.x = at<float>(h, L.W[1]); pa.out = at<float>(h, L.Y);
                a.x = pa.out;
                ba.s.x = pa.out;
            }
            auto one = [&]() {
                if (general) {
                    const cudaError_t pe = launch_step(L.panel, (int)h->dtype, kProdFloat, L.grid, h->stream, pa);
                    if (pe != cudaSuccess) return pe;
                }
                return h->nb > 0 ? launch_batch_step(L.panel, (int)h->dtype, kStepGeneral, bgrid, h->stream, ba)
                                 : launch_step(L.panel, (int)h->dtype, kStepGeneral, L.grid, h->stream, a);
            };
            CUDA_TRY(one());  // warm-up
            // the best of three timed blocks of `reps` launches: a block that
            // another process or a clock change disturbed does not decide
            float ms = 0.f;
            for (int blk = 0; blk < 3; ++blk) {
                CUDA_TRY(cudaEventRecord(e0, h->stream));
                for (int r = 0; r < reps; ++r) CUDA_TRY(one());
                CUDA_TRY(cudaEventRecord(e1, h->stream));
                CUDA_TRY(cudaEventSynchronize(e1));
                float bms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&bms, e0, e1));
                bms /= reps;
                if (blk == 0 || bms < ms) ms = bms;
            }
            if (v == saved && h->tile_rows == saved_tiles) saved_ms = ms;
            if (best < 0 || ms < best_ms) {
                best = v;
                best_ms = ms;
                best_tiles = h->tile_rows;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    uint32_t perr_h = 0;
    CUDA_TRY(cudaMemcpyAsync(&perr_h, perr, 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (perr_h) {
        h->impl = saved;
        return fail(CLD_ERR_TIMEOUT, "a staged-step pipeline wait gave up while timing the variants");
    }
    if (best < 0) {
        h->impl = saved;
        best_tiles = saved_tiles;
    }
    // keep the current choice unless another is at least 2 % faster, so that
    // timing noise does not flip it (and the summation order) run to run
    if (best >= 0 && saved_ms > 0.f && saved_ms <= 1.02f * best_ms) {
        best = saved;
        best_ms = saved_ms;
        best_tiles = saved_tiles;
    }
    if (h->nb > 0 && h->tile_rows != best_tiles) {
        h->tile_rows = best_tiles;
        build_tiles(h);
        const cld_status ust = upload_batch_tables(h, make_layout(h, 0, 1, 0));
        if (ust != CLD_OK) return ust;
    }
    if (best < 0) return fail(CLD_ERR_NOMEM, "workspace too small to time any variant");
    h->impl = best;
    if (variant_out) *variant_out = best;
    if (ms_out) *ms_out = best_ms;
    return CLD_OK;
}

cld_status cld_debug_withhold_tile(cld_handle h, int64_t tile) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (tile < 0) return fail(CLD_ERR_INVALID, "tile must be >= 0");
    h->withhold_tile = tile;
    return CLD_OK;
}

cld_status cld_set_profiling(cld_handle h, int on) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    h->profiling = on != 0;
    return CLD_OK;
}

cld_status cld_last_timing(cld_handle h, float* step_ms, int* step_launches, int* total_launches) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (step_ms) *step_ms = h->last_step_ms;
    if (step_launches) *step_launches = h->last_step_launches;
    if (total_launches) *total_launches = h->last_total_launches;
    return CLD_OK;
}

cld_status cld_launch_config(cld_handle h, int M, int* panel, int* lanes_per_row, int* ctas,
                             int* threads) {
    if (check_handle(h)) return CLD_ERR_INVALID;
    if (M < 1) return fail(CLD_ERR_INVALID, "M >= 1");
    const Layout L = make_layout(h, 1, M, 0);
    if (panel) *panel = L.panel;
    if (h->dense) {
        // the stream-K tensor-core step: one thread (TMEM lane) per row of a
        // tile in the epilogue, a persistent grid
        if (lanes_per_row) *lanes_per_row = 1;
        if (ctas) *ctas = L.dgrid;
        if (threads) *threads = dense_threads_per_cta();
        return CLD_OK;
    }
    // 4 probes per lane; 8 with the wide lanes (variant 5, panels of 8 or more)
    const bool wide = h->impl >= 5 && h->nb == 0 && L.panel >= 8;
    if (lanes_per_row) *lanes_per_row = wide ? L.panel / 8 : L.panel / 4;
    if (ctas) *ctas = L.grid;
    // variants 6 and 7: 8 consumer warps and one producer warp
    if (threads) *threads = (h->impl >= 6 && h->nb == 0 && L.panel >= 8) ? 288 : kThreads;
    return CLD_OK;
}

}  // extern "C"
