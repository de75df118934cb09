// cld_estimate_static: the estimate of cld_estimate (CLD_SPD) with all of its
// scratch in one file-scope device array instead of a caller workspace, for
// callers that cannot allocate device memory.  The kernels are the library's
// own (probe signs, recurrence steps, moment reduction, final sum); only where
// their scratch lives differs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/cld.h"
#include "cld_internal.cuh"

namespace cld {
void set_error_message(const char* msg);
cudaError_t launch_set_seed(Params* prm, uint64_t seed, cudaStream_t s);
}  // namespace cld

using namespace cld;

// The scratch array.  In host code `g_static_scratch` is only a host-side
// stand-in for the symbol: its device address is looked up per device with
// cudaGetSymbolAddress and passed to the kernels.
static __device__ __align__(256) unsigned char g_static_scratch[CLD_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_addr[kMaxDevices] = {};

cld_status err(cld_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_error_message(buf);
    return st;
}

#define STATIC_TRY(expr)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return err(CLD_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));    \
    } while (0)

size_t up(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the array on the current device (set-up on first use).
cld_status scratch_address(void** out) {
    int dev = 0;
    STATIC_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return err(CLD_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return err(CLD_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                       cudaGetErrorString(e));
        g_dev_addr[dev] = p;
    }
    *out = g_dev_addr[dev];
    return CLD_OK;
}

}  // namespace

extern "C" cld_status cld_estimate_static(int64_t d, int64_t nnz, const int64_t* rowptr,
                                          const int32_t* col, const void* val, cld_dtype val_dtype,
                                          double a, double b, int n, int M, uint64_t seed,
                                          void* stream, double* logdet_out, double* stderr_out) {
    if (!logdet_out) return err(CLD_ERR_INVALID, "logdet_out is NULL");
    if (d < 0 || nnz < 0) return err(CLD_ERR_INVALID, "negative size");
    if (d >= (int64_t)INT32_MAX) return err(CLD_ERR_INVALID, "d must be < 2^31");
    if (!rowptr || (nnz > 0 && (!col || !val))) return err(CLD_ERR_INVALID, "NULL CSR array");
    if (val_dtype != CLD_F32 && val_dtype != CLD_BF16 && val_dtype != CLD_F64)
        return err(CLD_ERR_INVALID, "unknown value dtype %d", (int)val_dtype);
    // The kernels load each array at its element width: a pointer that is not
    // aligned to it would fault on the device, so it is refused here, before
    // any CUDA call.
    const uintptr_t vsize = val_dtype == CLD_F32 ? 4 : val_dtype == CLD_BF16 ? 2 : 8;
    if (((uintptr_t)rowptr) % 8 || ((uintptr_t)col) % 4 || ((uintptr_t)val) % vsize)
        return err(CLD_ERR_INVALID, "CSR arrays must be aligned to their element size");
    if (n < 0 || M < 1 || n > 100000) return err(CLD_ERR_INVALID, "need 0 <= n <= 100000 and M >= 1");
    if (!(a > 0.0) || !(a < b) || !isfinite(a) || !isfinite(b))
        return err(CLD_ERR_INTERVAL, "interval must satisfy 0 < a < b (got [%g, %g])", a, b);
    if (d == 0) {
        *logdet_out = 0.0;
        if (stderr_out) *stderr_out = 0.0;
        return CLD_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    STATIC_TRY(cudaGetDevice(&dev));
    STATIC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    // sizes: the per-lane inner loop (variant 0) with its cld_estimate launch shape
    int panel = 4;
    if (M >= kMaxPanel) panel = kMaxPanel;
    else while (panel < M) panel <<= 1;
    const int nw = sign_words(panel);
    const int rows_per_cta = (kThreads / 32) * (128 / panel);
    int64_t g = (d + rows_per_cta - 1) / rows_per_cta;
    const int64_t gfull = (int64_t)step_ctas_per_sm(panel, (int)val_dtype, 0) * sms;
    const int grid = (int)(g < gfull ? (g > 0 ? g : 1) : gfull);
    int64_t sg = (d + kThreads - 1) / kThreads;
    const int sgrid = (int)(sg < (int64_t)sms * 8 ? (sg > 0 ? sg : 1) : (int64_t)sms * 8);
    const int nn = n > 0 ? n : 1;
    size_t o = 0;
    const size_t o_params = o; o += up(sizeof(Params));
    const size_t o_result = o; o += up(sizeof(Result));
    const size_t o_flags = o; o += 256;
    const size_t o_coeffs = o; o += up((size_t)(n + 1) * 8);
    const size_t o_cscr = o; o += up((size_t)5 * (n + 1) * 8);
    const size_t o_T = o; o += up((size_t)(n + 1) * M * 8);
    const size_t o_gp = o; o += up((size_t)M * 8);
    const size_t o_tpart = o; o += up((size_t)nn * grid * panel * 8);
    const size_t o_vbits = o; o += up((size_t)d * nw * 4);
    const size_t wb = up((size_t)d * panel * 4);
    const size_t o_W = o; o += 3 * wb;
    if (o > (size_t)CLD_STATIC_SCRATCH_BYTES)
        return err(CLD_ERR_NOMEM,
                   "cld_estimate_static needs %zu bytes of scratch for d=%lld, n=%d, M=%d; the built-in "
                   "array holds %zu bytes (use cld_estimate with a workspace)",
                   o, (long long)d, n, M, (size_t)CLD_STATIC_SCRATCH_BYTES);

    void* base = nullptr;
    cld_status st = scratch_address(&base);
    if (st != CLD_OK) return st;
    char* w = static_cast<char*>(base);
    Params* prm = reinterpret_cast<Params*>(w + o_params);
    Result* res = reinterpret_cast<Result*>(w + o_result);
    uint32_t* flags = reinterpret_cast<uint32_t*>(w + o_flags);
    double* T = reinterpret_cast<double*>(w + o_T);
    double* tpart = reinterpret_cast<double*>(w + o_tpart);
    uint32_t* vbits = reinterpret_cast<uint32_t*>(w + o_vbits);
    float* W[3] = {reinterpret_cast<float*>(w + o_W), reinterpret_cast<float*>(w + o_W + wb),
                   reinterpret_cast<float*>(w + o_W + 2 * wb)};

    // The array keeps the previous call's contents: clear the check flags.
    STATIC_TRY(cudaMemsetAsync(flags, 0, 256, s));
    STATIC_TRY(launch_validate_csr(d, nnz, rowptr, col, val, (int)val_dtype, flags, sgrid, s));
    uint32_t f = 0;
    STATIC_TRY(cudaMemcpyAsync(&f, flags, 4, cudaMemcpyDeviceToHost, s));
    STATIC_TRY(cudaStreamSynchronize(s));
    if (f & 1u) return err(CLD_ERR_INVALID, "row pointers must start at 0, end at nnz and not decrease");
    if (f & 2u) return err(CLD_ERR_INVALID, "column index out of range [0, d)");
    if (f & 4u) return err(CLD_ERR_INVALID, "non-finite stored value");

    STATIC_TRY(launch_set_params(prm, a, b, s));
    STATIC_TRY(launch_set_seed(prm, seed, s));
    const int npanels = (M + kMaxPanel - 1) / kMaxPanel;
    for (int pk = 0; pk < npanels; ++pk) {
        const int pbase = pk * kMaxPanel;
        const int mreal = (M - pbase) < panel ? (M - pbase) : panel;
        STATIC_TRY(launch_probe_bits(d, nw, (uint32_t)pk, prm, vbits, sgrid, s));
        StepArgs sa{};
        sa.d = d;
        sa.rowptr = rowptr;
        sa.col = col;
        sa.val = val;
        sa.vbits = vbits;
        sa.prm = prm;
        sa.mreal = mreal;
        for (int j = 0; j < n; ++j) {
            const float* wj = j >= 1 ? W[j % 3] : nullptr;
            sa.x = wj;
            sa.own = wj;
            sa.wprev = j >= 2 ? W[(j - 1) % 3] : nullptr;
            sa.out = W[(j + 1) % 3];
            sa.tpart = tpart + (size_t)j * grid * panel;
            const StepKind kind = j == 0 ? kStepFirst : j == 1 ? kStepSecond : kStepGeneral;
            STATIC_TRY(launch_step(panel, (int)val_dtype, kind, grid, s, sa));
        }
        if (n > 0) STATIC_TRY(launch_reduce_moments(tpart, n, grid, panel, mreal, M, pbase, T, s));
    }
    STATIC_TRY(launch_finalize(n, M, d, 0, prm, T, reinterpret_cast<double*>(w + o_coeffs),
                               reinterpret_cast<double*>(w + o_cscr), reinterpret_cast<double*>(w + o_gp),
                               res, s));
    Result r{};
    STATIC_TRY(cudaMemcpyAsync(&r, res, sizeof(Result), cudaMemcpyDeviceToHost, s));
    STATIC_TRY(cudaStreamSynchronize(s));
    *logdet_out = r.logdet;
    if (stderr_out) *stderr_out = r.stderr_;
    if (r.spectrum_bad)
        return err(CLD_ERR_SPECTRUM, "max |t_jp|/d = %g exceeds 1: the spectrum is not inside [%g, %g]",
                   r.max_ratio, a, b);
    return CLD_OK;
}
