// Mixed-precision instantiations of the stage kernels (GLEMUR_MIXED): FP32
// storage of the displacement, B0 and stage fields, FP32 stencil arithmetic,
// float-float determinants, FP64 reductions.
#include "stage_kernels.cuh"

namespace glemur {

cudaError_t prepare_stage_f32() {
  cudaError_t e;
  const size_t sm = stage_smem_bytes(0, sizeof(float));
  const size_t sd = stage_smem_bytes(1, sizeof(float));
  if ((e = cudaFuncSetAttribute(k_stage_mimetic<float, float, false, 3>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
    return e;
  if ((e = cudaFuncSetAttribute(k_stage_mimetic<float, float, true, 3>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
    return e;
  if ((e = cudaFuncSetAttribute(k_stage_direct<float, float, false, 3>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sd)))
    return e;
  return cudaFuncSetAttribute(k_stage_direct<float, float, true, 3>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sd);
}

int stage_ctas_per_sm_f32(int curl) {
  int n = 0;
  const size_t s = stage_smem_bytes(curl, sizeof(float));
  if (curl == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_mimetic<float, float, false, 3>,
                                                  NT, s);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_direct<float, float, false, 3>,
                                                  NT, s);
  return n;
}

cudaError_t launch_stage_f32(const StageArgs<float>& a, int curl, bool final_stage,
                             dim3 grid, cudaStream_t s) {
  const size_t smem = stage_smem_bytes(curl, sizeof(float));
  if (curl == 0) {
    if (final_stage)
      k_stage_mimetic<float, float, true, 3><<<grid, NT, smem, s>>>(a);
    else
      k_stage_mimetic<float, float, false, 3><<<grid, NT, smem, s>>>(a);
  } else {
    if (final_stage)
      k_stage_direct<float, float, true, 3><<<grid, NT, smem, s>>>(a);
    else
      k_stage_direct<float, float, false, 3><<<grid, NT, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace glemur
