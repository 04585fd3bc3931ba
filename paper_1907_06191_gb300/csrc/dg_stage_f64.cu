// dg_stage_f64.cu -- FP64 instantiations of the fused stage kernel.
#include "dg_stage.cuh"

namespace dg {
cudaError_t launch_stage_f64(int p, const double *u, const double *u0, double *out,
                             const Geometry &geo, long long stride, int m,
                             const Gll &g, const StageCoef<double> &c, cudaStream_t s,
                             const ChunkSel &sel, const StageCopies &cp) {
  return launch_stage_any<double>(p, u, u0, out, geo, stride, m, g, c, s, sel, cp);
}
}  // namespace dg
