// The N = 5 tensor-core stage over tiles of affine elements: the kernel of
// stage_tc5_kernel.cuh with PLANAR = true, which reads each element's
// constant geometric factors and face normals once instead of at every
// quadrature point (Sec. 6: separate kernels for planar and curvilinear
// elements).
#include "stage_tc5_kernel.cuh"

namespace wadg {

cudaError_t launch_stage_tc5_planar(const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream) {
  return launch_stage_tc5_n<true>(P, mode, fmt, grid, stream);
}

}  // namespace wadg
