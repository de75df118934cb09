// Kernels around the recurrence: probe signs (Sec. 2.2), moment reduction and
// the final Chebyshev-weighted sum (Algorithm 1), Chebyshev coefficients at
// first-kind nodes (Sec. 2.1), CSR validation and Gershgorin bounds (Sec. 3.2).
#include <math.h>

#include "cld_internal.cuh"

namespace cld {

cudaError_t launch_step_f32(int panel, StepKind kind, int grid, cudaStream_t s, const StepArgs& a);
cudaError_t launch_step_bf16(int panel, StepKind kind, int grid, cudaStream_t s, const StepArgs& a);
cudaError_t launch_step_f64(int panel, StepKind kind, int grid, cudaStream_t s, const StepArgs& a);
int step_ctas_per_sm_f32(int panel, int impl);
int step_ctas_per_sm_bf16(int panel, int impl);
int step_ctas_per_sm_f64(int panel, int impl);

cudaError_t launch_step(int panel, int dtype, StepKind kind, int grid, cudaStream_t stream,
                        const StepArgs& a) {
    switch (dtype) {
        case 0: return launch_step_f32(panel, kind, grid, stream, a);
        case 1: return launch_step_bf16(panel, kind, grid, stream, a);
        case 2: return launch_step_f64(panel, kind, grid, stream, a);
        default: return cudaErrorInvalidValue;
    }
}

int step_ctas_per_sm(int panel, int dtype, int impl) {
    switch (dtype) {
        case 0: return step_ctas_per_sm_f32(panel, impl);
        case 1: return step_ctas_per_sm_bf16(panel, impl);
        case 2: return step_ctas_per_sm_f64(panel, impl);
        default: return 1;
    }
}

// ------------------------------------------------------------------ parameters
__global__ void set_interval_kernel(Params* prm, double a, double b) {
    set_affine(prm, a, b);
    prm->interval_ok = (a > 0.0 && a < b && isfinite(a) && isfinite(b)) ? 1 : 0;
}

__global__ void set_seed_kernel(Params* prm, uint32_t lo, uint32_t hi) {
    prm->key_lo = lo;
    prm->key_hi = hi;
}

cudaError_t launch_set_params(Params* prm, double a, double b, cudaStream_t s) {
    set_interval_kernel<<<1, 1, 0, s>>>(prm, a, b);
    return cudaGetLastError();
}

cudaError_t launch_set_seed(Params* prm, uint64_t seed, cudaStream_t s) {
    set_seed_kernel<<<1, 1, 0, s>>>(prm, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ probe signs
// vbits[i * nw + w] = output word w of Philox4x32-10 at counter
// (i_lo, i_hi, panel_index, 0) with key = seed: bit b of word w is the sign
// of probe panel_index * 128 + 32 w + b (1 means -1).
__global__ void probe_bits_kernel(int64_t d, int nw, uint32_t panel_index, const Params* prm,
                                  uint32_t* __restrict__ vbits) {
    const uint32_t k0 = prm->key_lo, k1 = prm->key_hi;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t u = (uint64_t)i;
        uint4 r = philox4x32_10(make_uint4((uint32_t)u, (uint32_t)(u >> 32), panel_index, 0u), k0, k1);
        uint32_t w[4] = {r.x, r.y, r.z, r.w};
        for (int q = 0; q < nw; ++q) vbits[i * nw + q] = w[q];
    }
}

cudaError_t launch_probe_bits(int64_t d, int nw, uint32_t panel_index, const Params* prm,
                              uint32_t* vbits, int grid, cudaStream_t s) {
    probe_bits_kernel<<<grid, kThreads, 0, s>>>(d, nw, panel_index, prm, vbits);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ moments
// T[(s+1) * M + pbase + p] = sum over CTAs b (ascending) of tpart[s][b][p].
// One CTA per step; thread (p, q) sums every (kThreads/panel)-th CTA starting
// at q, then the q-partials are added in ascending q.
__global__ void reduce_moments_kernel(const double* __restrict__ tpart, int grid_blocks, int panel,
                                      int mreal, int M, int pbase, double* __restrict__ T) {
    const int s = blockIdx.x;
    const int p = threadIdx.x % panel;
    const int q = threadIdx.x / panel;
    const int nq = kThreads / panel;
    __shared__ double part[kThreads];
    double acc = 0.0;
    const double* base = tpart + (int64_t)s * grid_blocks * panel;
    for (int b = q; b < grid_blocks; b += nq) acc += base[(int64_t)b * panel + p];
    part[threadIdx.x] = acc;
    __syncthreads();
    if (q == 0 && p < mreal) {
        double sum = 0.0;
        for (int r = 0; r < nq; ++r) sum += part[r * panel + p];
        T[(int64_t)(s + 1) * M + pbase + p] = sum;
    }
}

cudaError_t launch_reduce_moments(const double* tpart, int nsteps, int grid_blocks, int panel,
                                  int mreal, int M, int pbase, double* T, cudaStream_t s) {
    if (nsteps <= 0) return cudaSuccess;
    reduce_moments_kernel<<<nsteps, kThreads, 0, s>>>(tpart, grid_blocks, panel, mreal, M, pbase, T);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ final sum
// Chebyshev coefficients of log on [a, b] at the N = n+1 first-kind nodes
// (Sec. 2.1):  c_j = (2 - [j=0]) / N * sum_k f(x_k) cos(j pi (k + 1/2) / N),
// f(x) = log(((b - a) x + a + b) / 2), x_k = cos(pi (k + 1/2) / N).
// cos(j pi (2k+1) / (2N)) is read from a table of cospi(m / (2N)),
// m = j (2k+1) mod 4N.
// Then t_{0,p} = v_p^T v_p = d, Gamma_p = sum_j c_j t_{j,p},
// Gamma = mean_p Gamma_p, stderr = std_p(Gamma_p) / sqrt(M), and the spectrum
// check max |t_{j,p}| / d <= 1 + 1e-3.  One CTA, fixed reduction order.
__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// c_0..c_n into coeffs, by one CTA (scratch: 5 (n+1) doubles).
__device__ void chebyshev_coefficients(int n, double a, double b, double* __restrict__ coeffs,
                                       double* __restrict__ scratch) {
    const int N = n + 1;
    double* tab = scratch;          // 4N
    double* f = scratch + 4 * N;    // N
    for (int m = threadIdx.x; m < 4 * N; m += blockDim.x) tab[m] = cospi((double)m / (2.0 * N));
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x)
        f[k] = log(((b - a) * tab[2 * k + 1] + a + b) / 2.0);
    __syncthreads();
    for (int j = threadIdx.x; j <= n; j += blockDim.x) {
        double s = 0.0;
        int idx = j % (4 * N);
        const int step = (2 * j) % (4 * N);
        for (int k = 0; k < N; ++k) {
            s += f[k] * tab[idx];
            idx += step;
            if (idx >= 4 * N) idx -= 4 * N;
        }
        coeffs[j] = (j == 0 ? 1.0 : 2.0) * s / N;
    }
}

__global__ void coeffs_kernel(int n, const Params* prm, double* __restrict__ coeffs,
                              double* __restrict__ scratch) {
    chebyshev_coefficients(n, prm->a, prm->b, coeffs, scratch);
}

cudaError_t launch_coeffs(int n, const Params* prm, double* coeffs, double* coef_scratch, cudaStream_t s) {
    coeffs_kernel<<<1, kThreads, 0, s>>>(n, prm, coeffs, coef_scratch);
    return cudaGetLastError();
}

// One problem's final sums (one CTA): coefficients, t_0 = d, Gamma_p, Gamma,
// stderr and the spectrum check into *res.
__device__ void finalize_one(int n, int M, int64_t d, int general, const Params* prm,
                             double* __restrict__ T, double* __restrict__ coeffs,
                             double* __restrict__ scratch, double* __restrict__ gamma_p, Result* res) {
    __shared__ double sh[kThreads];
    chebyshev_coefficients(n, prm->a, prm->b, coeffs, scratch);
    for (int p = threadIdx.x; p < M; p += blockDim.x) T[p] = (double)d;
    __syncthreads();

    double gsum = 0.0, ratio = 0.0;
    int bad = 0;
    const double dd = d > 0 ? (double)d : 1.0;
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
        double g = 0.0;
        for (int j = 0; j <= n; ++j) {
            const double t = T[(int64_t)j * M + p];
            g += coeffs[j] * t;
            const double r = fabs(t) / dd;
            if (!isfinite(t)) bad = 1;
            ratio = fmax(ratio, r);
        }
        gamma_p[p] = g;
        gsum += g;
    }
    const double total = block_sum(gsum, sh);
    const double rmax = block_max(ratio, sh);
    const double nbad = block_sum((double)bad, sh);
    const double mean = total / M;
    double var = 0.0;
    for (int p = threadIdx.x; p < M; p += blockDim.x) var += (gamma_p[p] - mean) * (gamma_p[p] - mean);
    const double vs = block_sum(var, sh);
    if (threadIdx.x == 0) {
        const double half = general ? 0.5 : 1.0;
        res->logdet = half * mean;
        res->stderr_ = M > 1 ? half * sqrt(vs / (M - 1)) / sqrt((double)M) : nan("");
        res->max_ratio = rmax;
        res->spectrum_bad = (nbad > 0.0 || !(rmax <= 1.0 + 1e-3)) ? 1 : 0;
    }
}

__global__ void finalize_kernel(int n, int M, int64_t d, int general, const Params* prm,
                                double* __restrict__ T, double* __restrict__ coeffs,
                                double* __restrict__ scratch, double* __restrict__ gamma_p,
                                Result* res) {
    finalize_one(n, M, d, general, prm, T, coeffs, scratch, gamma_p, res);
}

// Batched final sums: CTA b finalises block b (its own interval, d_b rows).
__global__ void finalize_batch_kernel(int n, int M, const int64_t* __restrict__ blk_rows, int general,
                                      const Params* prm, double* __restrict__ T, double* __restrict__ coeffs,
                                      double* __restrict__ scratch, double* __restrict__ gamma_p, Result* res) {
    const int b = blockIdx.x;
    const int64_t db = blk_rows[b + 1] - blk_rows[b];
    finalize_one(n, M, db, general, prm + b, T + (size_t)b * (n + 1) * M, coeffs + (size_t)b * (n + 1),
                 scratch + (size_t)b * 5 * (n + 1), gamma_p + (size_t)b * M, res + b);
}

cudaError_t launch_finalize_batch(int nb, int n, int M, const int64_t* blk_rows, int general, const Params* prm,
                                  double* T, double* coeffs, double* coef_scratch, double* gamma_p, Result* res,
                                  cudaStream_t s) {
    finalize_batch_kernel<<<nb, kThreads, 0, s>>>(n, M, blk_rows, general, prm, T, coeffs, coef_scratch, gamma_p, res);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int n, int M, int64_t d, int general, const Params* prm, double* T,
                            double* coeffs, double* coef_scratch, double* gamma_p, Result* res,
                            cudaStream_t s) {
    finalize_kernel<<<1, kThreads, 0, s>>>(n, M, d, general, prm, T, coeffs, coef_scratch, gamma_p, res);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ CSR checks
// flags bit 0: row pointers not monotone / wrong ends; bit 1: column out of
// range; bit 2: non-finite value.
template <typename VT>
__global__ void validate_csr_kernel(int64_t d, int64_t nnz, const int64_t* __restrict__ rowptr,
                                    const int32_t* __restrict__ col, const VT* __restrict__ val,
                                    uint32_t* flags) {
    uint32_t f = 0;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0 && (rowptr[0] != 0 || rowptr[d] != nnz)) f |= 1u;
    for (int64_t i = tid; i < d; i += nt)
        if (rowptr[i] > rowptr[i + 1]) f |= 1u;
    for (int64_t k = tid; k < nnz; k += nt) {
        const int32_t c = col[k];
        if (c < 0 || (int64_t)c >= d) f |= 2u;
        if (!isfinite(load_val_f64(val + k))) f |= 4u;
    }
    if (f) atomicOr(flags, f);
}

cudaError_t launch_validate_csr(int64_t d, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                                const void* val, int dtype, uint32_t* flags, int grid,
                                cudaStream_t s) {
    switch (dtype) {
        case 0:
            validate_csr_kernel<float><<<grid, kThreads, 0, s>>>(d, nnz, rowptr, col,
                                                                 static_cast<const float*>(val), flags);
            break;
        case 1:
            validate_csr_kernel<bf16_t><<<grid, kThreads, 0, s>>>(d, nnz, rowptr, col,
                                                                  static_cast<const bf16_t*>(val), flags);
            break;
        case 2:
            validate_csr_kernel<double><<<grid, kThreads, 0, s>>>(d, nnz, rowptr, col,
                                                                  static_cast<const double*>(val), flags);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Gershgorin
// Every eigenvalue of symmetric B lies in [min_i (B_ii - R_i), max_i (B_ii + R_i)],
// R_i = sum_{k != i} |B_ik| (Sec. 3.2: Gershgorin).  Pass 1: per-CTA min/max
// into partial[2 b], partial[2 b + 1]; pass 2: one CTA reduces and sets the
// interval in the parameter block (flags bit 8 if the lower end is not > 0).
template <typename VT>
__global__ void gershgorin_kernel(int64_t d, const int64_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ col, const VT* __restrict__ val,
                                  double* partial) {
    __shared__ double shl[kThreads], shh[kThreads];
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        double diag = 0.0, r = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const double v = load_val_f64(val + k);
            if (col[k] == i) diag += v;
            else r += fabs(v);
        }
        lo = fmin(lo, diag - r);
        hi = fmax(hi, diag + r);
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

__global__ void gershgorin_final_kernel(const double* partial, int nblocks, int64_t d, Params* prm,
                                        uint32_t* flags) {
    __shared__ double shl[kThreads], shh[kThreads];
    double lo = INFINITY, hi = -INFINITY;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        lo = fmin(lo, partial[2 * b]);
        hi = fmax(hi, partial[2 * b + 1]);
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
        double a = shl[0], b = shh[0];
        const int ok = finish_interval(a, b, d) ? 1 : 0;
        set_affine(prm, a, b);
        prm->interval_ok = ok;
        if (!ok) atomicOr(flags, 0x100u);
    }
}

cudaError_t launch_gershgorin(int64_t d, const int64_t* rowptr, const int32_t* col,
                              const void* val, int dtype, double* partial, int grid, Params* prm,
                              uint32_t* flags, cudaStream_t s) {
    switch (dtype) {
        case 0:
            gershgorin_kernel<float><<<grid, kThreads, 0, s>>>(d, rowptr, col,
                                                               static_cast<const float*>(val), partial);
            break;
        case 1:
            gershgorin_kernel<bf16_t><<<grid, kThreads, 0, s>>>(d, rowptr, col,
                                                                static_cast<const bf16_t*>(val), partial);
            break;
        case 2:
            gershgorin_kernel<double><<<grid, kThreads, 0, s>>>(d, rowptr, col,
                                                                static_cast<const double*>(val), partial);
            break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gershgorin_final_kernel<<<1, kThreads, 0, s>>>(partial, grid, d, prm, flags);
    return cudaGetLastError();
}

}  // namespace cld
