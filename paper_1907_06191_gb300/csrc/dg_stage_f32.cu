// dg_stage_f32.cu -- FP32 instantiations of the fused stage kernel.
#include "dg_stage.cuh"

namespace dg {
cudaError_t launch_stage_f32(int p, const float *u, const float *u0, float *out,
                             const Geometry &geo, long long stride, int m,
                             const Gll &g, const StageCoef<float> &c, cudaStream_t s,
                             const ChunkSel &sel, const StageCopies &cp) {
  if (p == 5 && cp.tensor_core) {
    const cudaError_t e = launch_stage_tc_f32(u, u0, out, geo, stride, m, g, c, s, sel, cp);
    if (e != cudaErrorNotSupported) return e;
  }
  return launch_stage_any<float>(p, u, u0, out, geo, stride, m, g, c, s, sel, cp);
}

int stage_pipe_max_blocks(int precision, int p, const Geometry &geo) {
  return precision == DG_FP32 ? stage_pipe_max_blocks_any<float>(p, geo) : 0;
}
}  // namespace dg
