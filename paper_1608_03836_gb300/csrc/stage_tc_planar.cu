// The tensor-core stage over tiles of affine elements (N <= 4): the kernel of
// stage_tc_kernel.cuh with PLANAR = true, which reads each element's constant
// geometric factors and face normals once instead of at every quadrature
// point (Sec. 6: separate kernels for planar and curvilinear elements).
#include "stage_tc_kernel.cuh"

namespace wadg {

cudaError_t launch_stage_tc_planar(int N, const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream) {
  switch (N) {
    case 1: return launch_stage_tc_n<1, true>(P, mode, fmt, grid, stream);
    case 2: return launch_stage_tc_n<2, true>(P, mode, fmt, grid, stream);
    case 3: return launch_stage_tc_n<3, true>(P, mode, fmt, grid, stream);
    case 4: return launch_stage_tc_n<4, true>(P, mode, fmt, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wadg
