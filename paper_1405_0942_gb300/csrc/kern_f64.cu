// FP64 instantiations of the stage kernels (precision GLEMUR_FP64).
#include "stage_kernels.cuh"

namespace glemur {

cudaError_t prepare_stage_f64() {
  cudaError_t e;
  const size_t sm = stage_smem_bytes(0, sizeof(double));
  const size_t sd = stage_smem_bytes(1, sizeof(double));
  if ((e = cudaFuncSetAttribute(k_stage_mimetic<double, double, false, 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
    return e;
  if ((e = cudaFuncSetAttribute(k_stage_mimetic<double, double, true, 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
    return e;
  if ((e = cudaFuncSetAttribute(k_stage_direct<double, double, false, 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sd)))
    return e;
  return cudaFuncSetAttribute(k_stage_direct<double, double, true, 2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sd);
}

int stage_ctas_per_sm_f64(int curl) {
  int n = 0;
  const size_t s = stage_smem_bytes(curl, sizeof(double));
  if (curl == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_mimetic<double, double, false, 2>,
                                                  NT, s);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_direct<double, double, false, 2>,
                                                  NT, s);
  return n;
}

cudaError_t launch_stage_f64(const StageArgs<double>& a, int curl, bool final_stage,
                             dim3 grid, cudaStream_t s) {
  const size_t smem = stage_smem_bytes(curl, sizeof(double));
  if (curl == 0) {
    if (final_stage)
      k_stage_mimetic<double, double, true, 2><<<grid, NT, smem, s>>>(a);
    else
      k_stage_mimetic<double, double, false, 2><<<grid, NT, smem, s>>>(a);
  } else {
    if (final_stage)
      k_stage_direct<double, double, true, 2><<<grid, NT, smem, s>>>(a);
    else
      k_stage_direct<double, double, false, 2><<<grid, NT, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace glemur
