// Instantiations of the fused stage kernel and the adjoint update: float, N in {1 2 3}.
#include "adjoint_simt.cuh"

namespace wadg {
template cudaError_t launch_stage_n<float, 1>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<float, 1>(const AdjUpdateParams<float>&, int, cudaStream_t);
template cudaError_t launch_stage_n<float, 2>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<float, 2>(const AdjUpdateParams<float>&, int, cudaStream_t);
template cudaError_t launch_stage_n<float, 3>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<float, 3>(const AdjUpdateParams<float>&, int, cudaStream_t);
}  // namespace wadg
