// Launchers of the recurrence-step kernels: every (panel, value type,
// variant, step kind) instantiation behind run-time switches, the dynamic
// shared-memory opt-in of the ring variants, programmatic dependent launch,
// and the occupancy that sizes the persistent grids.
#pragma once

#include "step_kernel.cuh"
#include "step_staged.cuh"
#include "step_window.cuh"
#include "step_wide.cuh"

namespace cld {

template <int MP, typename VT, int GATHER, int PREV, int EPI, int IMPL>
cudaError_t launch_one_step(int grid, cudaStream_t s, const StepArgs& a) {
    constexpr auto kern = step_kernel<MP, VT, GATHER, PREV, EPI, IMPL>;
    constexpr int smem = step_smem<IMPL, GATHER>();
    cudaError_t e = smem_opt_in<kern>(smem);
    if (e != cudaSuccess || grid == 0) return e;  // grid 0: opt in only
    return launch_pdl(kern, grid, smem, s, a);
}

// Variant 5 runs step_kernel_wide (panels of at least 8 probes; a 4-probe
// panel runs variant 0).
template <int MP, typename VT, int GATHER, int PREV, int EPI>
cudaError_t launch_one_wide(int grid, cudaStream_t s, const StepArgs& a) {
    if constexpr (MP >= 8) {
        if (grid == 0) return cudaSuccess;
        return launch_pdl(step_kernel_wide<MP, VT, GATHER, PREV, EPI>, grid, 0, s, a);
    } else {
        return launch_one_step<MP, VT, GATHER, PREV, EPI, 0>(grid, s, a);
    }
}

// Variant 6 runs step_kernel_staged (panels of at least 8 probes and CSR
// arrays on 16-byte boundaries, which its bulk copies need; otherwise the
// wide lanes of variant 5, whose grid-stride loop covers the same grid).
// Shape of the staged kernel (variant 6): 4 entries in flight per lane, 8
// consumer warps, 3 CTAs per SM.  Measured on GB300 against 8 or 6 entries
// in flight at 2 CTAs per SM and 16 consumer warps at 1 CTA per SM (grid
// GMRF and Wendland steps): this one is as fast or faster, and four CTAs per
// SM are slower (the ring's shared memory takes L1 from the gathers).
template <int I> struct StagedShape;
template <> struct StagedShape<0> { using C = StagedCfg<4, 8, 3>; };

template <int MP, typename VT, int GATHER, int PREV, int EPI, int I>
cudaError_t launch_one_staged(int grid, cudaStream_t s, const StepArgs& a) {
    if constexpr (MP >= 8) {
        using C = typename StagedShape<I>::C;
        const bool aligned = (reinterpret_cast<uintptr_t>(a.rowptr) % 16 == 0) &&
                             (reinterpret_cast<uintptr_t>(a.col) % 16 == 0) &&
                             (reinterpret_cast<uintptr_t>(a.val) % 16 == 0);
        if (!aligned || a.err == nullptr) return launch_one_wide<MP, VT, GATHER, PREV, EPI>(grid, s, a);
        constexpr auto kern = step_kernel_staged<MP, VT, GATHER, PREV, EPI, C>;
        constexpr int smem = StagedLayout<MP, VT, PREV, EPI, C>::bytes;
        cudaError_t e = smem_opt_in<kern>(smem, C::MINB);
        if (e != cudaSuccess || grid == 0) return e;
        return launch_pdl(kern, grid, smem, s, a, C::threads);
    } else {
        return launch_one_step<MP, VT, GATHER, PREV, EPI, 0>(grid, s, a);
    }
}

// Variant 7's step j >= 1 of an SPD matrix (x = w_j): the windowed kernel
// when the handle's plan for this panel is attached and the arrays are
// 16-byte aligned, else the staged tiles.  grid 0 opts both kernels in.
template <int MP, typename VT, int PREV>
cudaError_t launch_one_window(int grid, cudaStream_t s, const StepArgs& a) {
    if constexpr (window_ok<MP, VT>()) {
        using C = WindowShape;
        constexpr auto kern = step_kernel_window<MP, VT, PREV, C>;
        constexpr int smem = WindowLayout<MP, VT, PREV, C>::bytes;
        if (grid == 0) {
            const cudaError_t e = smem_opt_in<kern>(smem, C::MINB);
            if (e != cudaSuccess) return e;
        } else {
            const bool aligned = (reinterpret_cast<uintptr_t>(a.rowptr) % 16 == 0) &&
                                 (reinterpret_cast<uintptr_t>(a.lcol) % 16 == 0) &&
                                 (reinterpret_cast<uintptr_t>(a.col) % 16 == 0) &&
                                 (reinterpret_cast<uintptr_t>(a.val) % 16 == 0);
            if (a.lcol != nullptr && a.wtab != nullptr && a.err != nullptr && a.x == a.own && aligned) {
                const cudaError_t e = smem_opt_in<kern>(smem, C::MINB);
                if (e != cudaSuccess) return e;
                return launch_pdl(kern, grid, smem, s, a, C::threads);
            }
        }
    }
    return launch_one_staged<MP, VT, 0, PREV, 1, 0>(grid, s, a);
}

template <int MP, typename VT, int IMPL>
cudaError_t launch_step_impl(StepKind kind, int grid, cudaStream_t s, const StepArgs& a) {
    if constexpr (IMPL == 7) {
        switch (kind) {
            case kStepSecond: return launch_one_window<MP, VT, 1>(grid, s, a);
            case kStepGeneral: return launch_one_window<MP, VT, 2>(grid, s, a);
            default: return launch_step_impl<MP, VT, 6>(kind, grid, s, a);
        }
    }
    if constexpr (IMPL == 6) {
        constexpr int I = IMPL - 6;
        switch (kind) {
            case kStepFirst: return launch_one_staged<MP, VT, 1, 0, 1, I>(grid, s, a);
            case kStepSecond: return launch_one_staged<MP, VT, 0, 1, 1, I>(grid, s, a);
            case kStepGeneral: return launch_one_staged<MP, VT, 0, 2, 1, I>(grid, s, a);
            case kProdBits: return launch_one_staged<MP, VT, 1, 0, 0, I>(grid, s, a);
            case kProdFloat: return launch_one_staged<MP, VT, 0, 0, 0, I>(grid, s, a);
            case kStepFirstFromFloat: return launch_one_staged<MP, VT, 0, 0, 1, I>(grid, s, a);
            default: return cudaErrorInvalidValue;
        }
    }
    if constexpr (IMPL == 5) {
        switch (kind) {
            case kStepFirst: return launch_one_wide<MP, VT, 1, 0, 1>(grid, s, a);
            case kStepSecond: return launch_one_wide<MP, VT, 0, 1, 1>(grid, s, a);
            case kStepGeneral: return launch_one_wide<MP, VT, 0, 2, 1>(grid, s, a);
            case kProdBits: return launch_one_wide<MP, VT, 1, 0, 0>(grid, s, a);
            case kProdFloat: return launch_one_wide<MP, VT, 0, 0, 0>(grid, s, a);
            case kStepFirstFromFloat: return launch_one_wide<MP, VT, 0, 0, 1>(grid, s, a);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (kind) {
        case kStepFirst: return launch_one_step<MP, VT, 1, 0, 1, IMPL>(grid, s, a);
        case kStepSecond: return launch_one_step<MP, VT, 0, 1, 1, IMPL>(grid, s, a);
        case kStepGeneral: return launch_one_step<MP, VT, 0, 2, 1, IMPL>(grid, s, a);
        case kProdBits: return launch_one_step<MP, VT, 1, 0, 0, IMPL>(grid, s, a);
        case kProdFloat: return launch_one_step<MP, VT, 0, 0, 0, IMPL>(grid, s, a);
        case kStepFirstFromFloat: return launch_one_step<MP, VT, 0, 0, 1, IMPL>(grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int MP, typename VT>
cudaError_t launch_step_mp(StepKind kind, int grid, cudaStream_t s, const StepArgs& a) {
    switch (a.impl) {
        case 0: return launch_step_impl<MP, VT, 0>(kind, grid, s, a);
        case 1: return launch_step_impl<MP, VT, 1>(kind, grid, s, a);
        case 2: return launch_step_impl<MP, VT, 2>(kind, grid, s, a);
        case 3: return launch_step_impl<MP, VT, 3>(kind, grid, s, a);
        case 4: return launch_step_impl<MP, VT, 4>(kind, grid, s, a);
        case 5: return launch_step_impl<MP, VT, 5>(kind, grid, s, a);
        case 6: return launch_step_impl<MP, VT, 6>(kind, grid, s, a);
        case 7: return launch_step_impl<MP, VT, 7>(kind, grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <typename VT>
cudaError_t launch_step_vt(int panel, StepKind kind, int grid, cudaStream_t s, const StepArgs& a) {
    switch (panel) {
        case 4: return launch_step_mp<4, VT>(kind, grid, s, a);
        case 8: return launch_step_mp<8, VT>(kind, grid, s, a);
        case 16: return launch_step_mp<16, VT>(kind, grid, s, a);
        case 32: return launch_step_mp<32, VT>(kind, grid, s, a);
        case 64: return launch_step_mp<64, VT>(kind, grid, s, a);
        case 128: return launch_step_mp<128, VT>(kind, grid, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int MP, typename VT, int IMPL>
int ctas_per_sm_impl() {
    constexpr auto kern = step_kernel<MP, VT, 0, 2, 1, IMPL>;
    constexpr int smem = step_smem<IMPL, 0>();
    int n = 0;
    if (smem_opt_in<kern>(smem) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

template <int MP, typename VT>
int ctas_per_sm_wide() {
    int n = 0;
    if constexpr (MP >= 8) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_wide<MP, VT, 0, 2, 1>, kThreads, 0) !=
            cudaSuccess)
            return 1;
        return n > 0 ? n : 1;
    } else {
        return ctas_per_sm_impl<MP, VT, 0>();
    }
}

template <int MP, typename VT, int I>
int ctas_per_sm_staged() {
    int n = 0;
    if constexpr (MP >= 8) {
        using C = typename StagedShape<I>::C;
        constexpr auto kern = step_kernel_staged<MP, VT, 0, 2, 1, C>;
        constexpr int smem = StagedLayout<MP, VT, 2, 1, C>::bytes;
        if (smem_opt_in<kern>(smem, C::MINB) != cudaSuccess) return 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, C::threads, smem) != cudaSuccess) return 1;
        return n > 0 ? n : 1;
    } else {
        return ctas_per_sm_impl<MP, VT, 0>();
    }
}

template <int MP, typename VT>
int ctas_per_sm_window() {
    if constexpr (window_ok<MP, VT>()) {
        using C = WindowShape;
        constexpr auto kern = step_kernel_window<MP, VT, 2, C>;
        constexpr int smem = WindowLayout<MP, VT, 2, C>::bytes;
        int n = 0;
        if (smem_opt_in<kern>(smem, C::MINB) != cudaSuccess) return 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, C::threads, smem) != cudaSuccess) return 1;
        return n > 0 ? n : 1;
    } else {
        return ctas_per_sm_staged<MP, VT, 0>();
    }
}

template <int MP, typename VT>
int ctas_per_sm_mp(int impl) {
    switch (impl) {
        case 0: return ctas_per_sm_impl<MP, VT, 0>();
        case 1: return ctas_per_sm_impl<MP, VT, 1>();
        case 2: return ctas_per_sm_impl<MP, VT, 2>();
        case 3: return ctas_per_sm_impl<MP, VT, 3>();
        case 4: return ctas_per_sm_impl<MP, VT, 4>();
        case 5: return ctas_per_sm_wide<MP, VT>();
        case 6: return ctas_per_sm_staged<MP, VT, 0>();
        case 7: return ctas_per_sm_window<MP, VT>();
        default: return 1;
    }
}

template <typename VT>
int ctas_per_sm_vt(int panel, int impl) {
    switch (panel) {
        case 4: return ctas_per_sm_mp<4, VT>(impl);
        case 8: return ctas_per_sm_mp<8, VT>(impl);
        case 16: return ctas_per_sm_mp<16, VT>(impl);
        case 32: return ctas_per_sm_mp<32, VT>(impl);
        case 64: return ctas_per_sm_mp<64, VT>(impl);
        case 128: return ctas_per_sm_mp<128, VT>(impl);
        default: return 1;
    }
}

}  // namespace cld
