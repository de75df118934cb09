// Recurrence-step kernels for bf16 stored values (one translation unit per
// value type so the instantiations compile in parallel).
#include "step_launch.cuh"

namespace cld {

cudaError_t launch_step_bf16(int panel, StepKind kind, int grid, cudaStream_t s, const StepArgs& a) {
    return launch_step_vt<bf16_t>(panel, kind, grid, s, a);
}

int step_ctas_per_sm_bf16(int panel, int impl) { return ctas_per_sm_vt<bf16_t>(panel, impl); }

}  // namespace cld
