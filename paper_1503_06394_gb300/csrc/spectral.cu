// Spectral bounds for the interval [a, b] (Sec. 3.2) and the transposed CSR
// that Algorithm 2 needs to apply C^T without forming C^T C.
//
//  - transpose: counting pass, exclusive scan, scatter, then each row of C^T
//    sorted by column so that every later product is deterministic;
//  - general bounds: b = ||C||_1 ||C||_inf >= sigma_max^2 (the paper's norm
//    bound, squared); a = alpha * beta from row / column diagonal-dominance
//    margins (Varah's bound), a lower bound on sigma_min^2;
//  - Lanczos: k steps of the symmetric Lanczos process in FP64 from a Philox
//    start vector; the largest Ritz value plus its residual norm tightens b.
#include <math.h>

#include "cld_internal.cuh"

namespace cld {

// ---------------------------------------------------------------- transpose
__global__ void count_cols_kernel(int64_t nnz, const int32_t* __restrict__ col,
                                  unsigned long long* __restrict__ cnt) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[k], 1ull);
}

// Exclusive scan of n int64 values in place, one CTA (n up to a few million
// takes a few ms; only used once per matrix).
__global__ void scan_single_block_kernel(int64_t* __restrict__ x, int64_t n) {
    __shared__ int64_t sh[kThreads];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * per;
    const int64_t hi = lo + per < n ? lo + per : n;
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += x[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            int64_t v = sh[t];
            sh[t] = run;
            run += v;
        }
    }
    __syncthreads();
    int64_t run = sh[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) {
        int64_t v = x[i];
        x[i] = run;
        run += v;
    }
}

__global__ void copy_i64_kernel(int64_t n, const int64_t* __restrict__ a, int64_t* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void scatter_transpose_kernel(int64_t d, const int64_t* __restrict__ rowptr,
                                         const int32_t* __restrict__ col, const char* __restrict__ val,
                                         int vsize, unsigned long long* __restrict__ cursor,
                                         int32_t* __restrict__ colT, char* __restrict__ valT) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int64_t pos = (int64_t)atomicAdd(cursor + col[k], 1ull);
            colT[pos] = (int32_t)i;
            for (int q = 0; q < vsize; ++q) valT[pos * vsize + q] = val[k * vsize + q];
        }
    }
}

// Insertion sort of each row of C^T by column (rows of sparse matrices are short).
__global__ void sort_rows_kernel(int64_t d, const int64_t* __restrict__ rowptr,
                                 int32_t* __restrict__ colT, char* __restrict__ valT, int vsize) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = rowptr[i], hi = rowptr[i + 1];
        for (int64_t k = lo + 1; k < hi; ++k) {
            const int32_t c = colT[k];
            char v[8];
            for (int q = 0; q < vsize; ++q) v[q] = valT[k * vsize + q];
            int64_t m = k - 1;
            while (m >= lo && colT[m] > c) {
                colT[m + 1] = colT[m];
                for (int q = 0; q < vsize; ++q) valT[(m + 1) * vsize + q] = valT[m * vsize + q];
                --m;
            }
            colT[m + 1] = c;
            for (int q = 0; q < vsize; ++q) valT[(m + 1) * vsize + q] = v[q];
        }
    }
}

cudaError_t launch_transpose(int64_t d, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                             const void* val, int vsize, int64_t* rowptrT, int32_t* colT, void* valT,
                             int64_t* scratch, int grid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(rowptrT, 0, sizeof(int64_t) * (size_t)(d + 1), s);
    if (e != cudaSuccess) return e;
    if (nnz > 0) count_cols_kernel<<<grid, kThreads, 0, s>>>(nnz, col, reinterpret_cast<unsigned long long*>(rowptrT));
    scan_single_block_kernel<<<1, kThreads, 0, s>>>(rowptrT, d + 1);
    copy_i64_kernel<<<grid, kThreads, 0, s>>>(d + 1, rowptrT, scratch);
    if (nnz > 0) {
        scatter_transpose_kernel<<<grid, kThreads, 0, s>>>(d, rowptr, col, static_cast<const char*>(val), vsize,
                                                           reinterpret_cast<unsigned long long*>(scratch),
                                                           colT, static_cast<char*>(valT));
        sort_rows_kernel<<<grid, kThreads, 0, s>>>(d, rowptrT, colT, static_cast<char*>(valT), vsize);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- general C bounds
// partial[4 b + 0..3] = (min_i |C_ii| - R_i, max_i rowabs_i, min_i |C_ii| - S_i, max_i colabs_i)
template <typename VT>
__global__ void general_bounds_kernel(int64_t d, const int64_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ col, const VT* __restrict__ val,
                                      const int64_t* __restrict__ rowptrT, const int32_t* __restrict__ colT,
                                      const VT* __restrict__ valT, double* partial) {
    __shared__ double sh[4][kThreads];
    double amin = INFINITY, rmax = 0.0, bmin = INFINITY, cmax = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
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
    if (threadIdx.x < 4) partial[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void general_bounds_final_kernel(const double* partial, int nb, int64_t d, Params* prm, uint32_t* flags) {
    if (threadIdx.x != 0) return;
    double amin = INFINITY, rmax = 0.0, bmin = INFINITY, cmax = 0.0;
    for (int b = 0; b < nb; ++b) {
        amin = fmin(amin, partial[4 * b]);
        rmax = fmax(rmax, partial[4 * b + 1]);
        bmin = fmin(bmin, partial[4 * b + 2]);
        cmax = fmax(cmax, partial[4 * b + 3]);
    }
    double a = (amin > 0.0 && bmin > 0.0) ? amin * bmin : 0.0;
    double b = rmax * cmax;
    const int ok = finish_interval(a, b, d) ? 1 : 0;
    set_affine(prm, a, b);
    prm->interval_ok = ok;
    if (!ok) atomicOr(flags, 0x100u);
}

cudaError_t launch_general_bounds(int64_t d, const int64_t* rowptr, const int32_t* col,
                                  const void* val, const int64_t* rowptrT, const int32_t* colT,
                                  const void* valT, int dtype, double* partial, int grid,
                                  Params* prm, uint32_t* flags, cudaStream_t s) {
    switch (dtype) {
        case 0:
            general_bounds_kernel<float><<<grid, kThreads, 0, s>>>(
                d, rowptr, col, static_cast<const float*>(val), rowptrT, colT,
                static_cast<const float*>(valT), partial);
            break;
        case 1:
            general_bounds_kernel<bf16_t><<<grid, kThreads, 0, s>>>(
                d, rowptr, col, static_cast<const bf16_t*>(val), rowptrT, colT,
                static_cast<const bf16_t*>(valT), partial);
            break;
        case 2:
            general_bounds_kernel<double><<<grid, kThreads, 0, s>>>(
                d, rowptr, col, static_cast<const double*>(val), rowptrT, colT,
                static_cast<const double*>(valT), partial);
            break;
        default: return cudaErrorInvalidValue;
    }
    general_bounds_final_kernel<<<1, 32, 0, s>>>(partial, grid, d, prm, flags);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Lanczos
// Vectors (FP64, d each): q_prev, q, u.  Scalars: alpha[k], beta[k], partial[grid].
template <typename VT>
__global__ void lz_matvec_kernel(int64_t d, const int64_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col, const VT* __restrict__ val,
                                 const double* __restrict__ q, const double* __restrict__ qprev,
                                 const double* beta_prev, double* __restrict__ u) {
    const double bp = beta_prev ? *beta_prev : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += load_val_f64(val + k) * q[col[k]];
        u[i] = s - bp * qprev[i];
    }
}

__global__ void lz_dot_kernel(int64_t d, const double* __restrict__ x, const double* __restrict__ y,
                              double* partial) {
    __shared__ double sh[kThreads];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x)
        s += x[i] * y[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// out = sqrt_flag ? sqrt(sum partial) : sum partial
__global__ void lz_sum_kernel(const double* partial, int nb, double* out, int take_sqrt) {
    __shared__ double sh[kThreads];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = take_sqrt ? sqrt(sh[0]) : sh[0];
}

// u -= alpha q
__global__ void lz_axpy_kernel(int64_t d, const double* alpha, const double* __restrict__ q,
                               double* __restrict__ u) {
    const double a = *alpha;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x)
        u[i] -= a * q[i];
}

// q_prev <- q ; q <- u / beta  (beta == 0: q <- 0, the Krylov space is exhausted)
__global__ void lz_shift_kernel(int64_t d, const double* beta, double* __restrict__ qprev,
                                double* __restrict__ q, const double* __restrict__ u) {
    const double b = *beta;
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        qprev[i] = q[i];
        q[i] = u[i] * inv;
    }
}

// Start vector: Philox signs (key 0x4c414e43, counter (i, 0, 0, 1)) scaled to unit norm.
__global__ void lz_start_kernel(int64_t d, double* __restrict__ q, double* __restrict__ qprev) {
    const double inv = 1.0 / sqrt((double)d);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t u = (uint64_t)i;
        uint4 r = philox4x32_10(make_uint4((uint32_t)u, (uint32_t)(u >> 32), 0u, 1u), 0x4c414e43u, 0u);
        q[i] = (r.x & 1u) ? -inv : inv;
        qprev[i] = 0.0;
    }
}

// Largest eigenvalue of the k x k tridiagonal (alpha, beta) by bisection on the
// Sturm count, its eigenvector's last component by the three-term recurrence,
// and b <- min(b, theta + max(r, 1e-4 |theta|)) with r = beta_k |s_k|.
__global__ void lz_finish_kernel(int k, const double* alpha, const double* beta, Params* prm,
                                 uint32_t* flags) {
    if (threadIdx.x != 0) return;
    // Gershgorin range of the tridiagonal
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < k ? fabs(beta[i]) : 0.0);
        lo = fmin(lo, alpha[i] - r);
        hi = fmax(hi, alpha[i] + r);
    }
    // count of eigenvalues < x
    auto count_below = [&](double x) {
        int c = 0;
        double q = alpha[0] - x;
        if (q < 0) ++c;
        for (int i = 1; i < k; ++i) {
            if (q == 0.0) q = 1e-300;
            q = (alpha[i] - x) - beta[i - 1] * beta[i - 1] / q;
            if (q < 0) ++c;
        }
        return c;
    };
    double l = lo, h = hi;
    for (int it = 0; it < 200 && h - l > 1e-15 * fmax(1.0, fabs(h)); ++it) {
        const double m = 0.5 * (l + h);
        if (count_below(m) >= k) h = m; else l = m;  // all k eigenvalues below m -> theta_max < m
    }
    const double theta = h;
    // eigenvector recurrence with rescaling
    double s_prev = 0.0, s = 1.0, nrm2 = 1.0;
    bool broke = false;
    for (int i = 0; i + 1 < k; ++i) {
        if (fabs(beta[i]) < 1e-300) { broke = true; break; }
        const double nx = ((theta - alpha[i]) * s - (i > 0 ? beta[i - 1] * s_prev : 0.0)) / beta[i];
        s_prev = s;
        s = nx;
        nrm2 += s * s;
        if (fabs(s) > 1e100) { s *= 1e-100; s_prev *= 1e-100; nrm2 *= 1e-200; }
    }
    const double last = broke ? 0.0 : fabs(s) / sqrt(nrm2);
    const double r = fabs(beta[k - 1]) * last;
    const double bnew = theta + fmax(r, 1e-4 * fabs(theta));
    if (isfinite(bnew) && bnew < prm->b && bnew > prm->a) {
        set_affine(prm, prm->a, bnew);
    }
    (void)flags;
}

template <typename VT>
static cudaError_t lanczos_t(int64_t d, const int64_t* rowptr, const int32_t* col, const VT* val,
                             int iters, double* vecs, double* scal, int grid, Params* prm,
                             uint32_t* flags, cudaStream_t s) {
    double* qprev = vecs;
    double* q = vecs + d;
    double* u = vecs + 2 * d;
    double* alpha = scal;
    double* beta = scal + iters;
    double* partial = scal + 2 * iters;
    lz_start_kernel<<<grid, kThreads, 0, s>>>(d, q, qprev);
    for (int i = 0; i < iters; ++i) {
        lz_matvec_kernel<VT><<<grid, kThreads, 0, s>>>(d, rowptr, col, val, q, qprev,
                                                       i > 0 ? beta + i - 1 : nullptr, u);
        lz_dot_kernel<<<grid, kThreads, 0, s>>>(d, q, u, partial);
        lz_sum_kernel<<<1, kThreads, 0, s>>>(partial, grid, alpha + i, 0);
        lz_axpy_kernel<<<grid, kThreads, 0, s>>>(d, alpha + i, q, u);
        lz_dot_kernel<<<grid, kThreads, 0, s>>>(d, u, u, partial);
        lz_sum_kernel<<<1, kThreads, 0, s>>>(partial, grid, beta + i, 1);
        lz_shift_kernel<<<grid, kThreads, 0, s>>>(d, beta + i, qprev, q, u);
    }
    lz_finish_kernel<<<1, 32, 0, s>>>(iters, alpha, beta, prm, flags);
    return cudaGetLastError();
}

cudaError_t launch_lanczos(int64_t d, const int64_t* rowptr, const int32_t* col, const void* val,
                           int dtype, int iters, double* vecs, double* scal, int grid,
                           Params* prm, uint32_t* flags, cudaStream_t s) {
    switch (dtype) {
        case 0: return lanczos_t(d, rowptr, col, static_cast<const float*>(val), iters, vecs, scal, grid, prm, flags, s);
        case 1: return lanczos_t(d, rowptr, col, static_cast<const bf16_t*>(val), iters, vecs, scal, grid, prm, flags, s);
        case 2: return lanczos_t(d, rowptr, col, static_cast<const double*>(val), iters, vecs, scal, grid, prm, flags, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cld
