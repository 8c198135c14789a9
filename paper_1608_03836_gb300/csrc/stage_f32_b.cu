// Instantiations of the fused stage kernel and the adjoint update: float, N in {4 5 6}.
#include "adjoint_simt.cuh"

namespace wadg {
template cudaError_t launch_stage_n<float, 4>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<float, 4>(const AdjUpdateParams<float>&, int, cudaStream_t);
template cudaError_t launch_stage_n<float, 5>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<float, 5>(const AdjUpdateParams<float>&, int, cudaStream_t);
template cudaError_t launch_stage_n<float, 6>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<float, 6>(const AdjUpdateParams<float>&, int, cudaStream_t);
}  // namespace wadg
