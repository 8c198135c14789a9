// The N = 5 tensor-core stage's launchers for curved tiles and its operator
// tables (the kernel: stage_tc5_kernel.cuh; the planar-element
// instantiations: stage_tc5_planar.cu).
#include "stage_tc5_kernel.cuh"

namespace wadg {

cudaError_t launch_stage_tc5(const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream) {
  return launch_stage_tc5_n<false>(P, mode, fmt, grid, stream);
}

bool pack_tc5_ops(const RefOps& o, int fmt, std::vector<uint8_t>& out) {
  if (!face_nodes_match<5>(o)) return false;
  if (o.Nq == 216) {
    pack_dims<TcDims5<216>>(o, fmt, out);
    return true;
  }
  if (o.Nq == fewer_point_nq(5)) {
    pack_dims<TcDims5<fewer_point_nq(5)>>(o, fmt, out);
    return true;
  }
  return false;
}

}  // namespace wadg
