// mixed-precision (GLEMUR_MIXED: FP32 storage and stencils, float-float determinants, FP64 reductions) instantiations of the mimetic-current stage kernels.
#include "stage_kernels.cuh"

namespace glemur {

cudaError_t launch_f32_mimetic(const StageArgs<float>& a, int stage, dim3 grid, cudaStream_t s) {
  return launch_stage_t<float, float, 0, 3>(a, stage, grid, s);
}

cudaError_t prepare_f32_mimetic() { return prepare_stage_t<float, float, 0, 3>(); }

int ctas_per_sm_f32_mimetic() { return stage_ctas_per_sm_t<float, float, 0, 3>(); }

}  // namespace glemur
