// dg_stage_f32.cu -- FP32 instantiations of the fused stage kernel.
#include "dg_stage.cuh"

namespace dg {
cudaError_t launch_stage_f32(int p, const float *u, const float *u0, float *out,
                             const Geometry &geo, long long stride, int m,
                             const Gll &g, const StageCoef<float> &c, cudaStream_t s,
                             const ChunkSel &sel, const StageCopies &cp) {
  return launch_stage_any<float>(p, u, u0, out, geo, stride, m, g, c, s, sel, cp);
}
}  // namespace dg
