// mixed-precision (GLEMUR_MIXED: FP32 storage and stencils, float-float determinants, FP64 reductions) instantiations of the mimetic-current stage kernels.
#include "stage_tma.cuh"

namespace glemur {

cudaError_t launch_f32_mimetic(const StageArgs<float>& a, int stage, dim3 grid, cudaStream_t s) {
  return launch_stage_t<float, float, 0, 3>(a, stage, grid, s);
}

cudaError_t prepare_f32_mimetic() { return prepare_stage_t<float, float, 0, 3>(); }

int ctas_per_sm_f32_mimetic() { return stage_ctas_per_sm_t<float, float, 0, 3>(); }

// The same stages with the stage input and B0 loaded as TMA tiles (nx a
// multiple of 4): 8 warps, one output row per thread (32 x 8 tile), 3 CTAs
// per SM.  (Two rows per thread, 32 x 14 tiles of 7 warps or 32 x 16 of 8,
// 2 CTAs per SM, measured 9-10 % slower on the 384^3 workload.)
using TmaGeo0 = TmaGeo<8, 1>;

cudaError_t launch_f32_mimetic_tma(const StageArgs<float>& a, const TmaMaps& maps, int stage,
                                   dim3 grid, cudaStream_t s) {
  return launch_stage_tma_t<8, 1, 3>(a, maps, stage, grid, s);
}

cudaError_t prepare_f32_mimetic_tma() { return prepare_stage_tma_t<8, 1, 3>(); }

int ctas_per_sm_f32_mimetic_tma() { return stage_tma_ctas_per_sm_t<8, 1, 3>(); }

// Tile height (nodes); the stage-input box is 4 rows higher, the B0 box 2.
int tile_rows_f32_mimetic_tma() { return TmaGeo0::TH; }

}  // namespace glemur
