// Recurrence-step kernels for f32 stored values (one translation unit per
// value type so the instantiations compile in parallel).
#include "step_launch.cuh"

namespace cld {

cudaError_t launch_step_f32(int panel, StepKind kind, int grid, cudaStream_t s, const StepArgs& a) {
    return launch_step_vt<float>(panel, kind, grid, s, a);
}

int step_ctas_per_sm_f32(int panel, int impl) { return ctas_per_sm_vt<float>(panel, impl); }

}  // namespace cld
