// FP64 (GLEMUR_FP64) instantiations of the mimetic-current stage kernels.
#include "stage_kernels.cuh"

namespace glemur {

cudaError_t launch_f64_mimetic(const StageArgs<double>& a, int stage, dim3 grid, cudaStream_t s) {
  return launch_stage_t<double, double, 0, 1>(a, stage, grid, s);
}

cudaError_t prepare_f64_mimetic() { return prepare_stage_t<double, double, 0, 1>(); }

int ctas_per_sm_f64_mimetic() { return stage_ctas_per_sm_t<double, double, 0, 1>(); }

}  // namespace glemur
