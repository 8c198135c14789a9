// Instantiations of the fused stage kernel and the adjoint update: double, N in {1 2 3}.
#include "adjoint_simt.cuh"

namespace wadg {
template cudaError_t launch_stage_n<double, 1>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<double, 1>(const AdjUpdateParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_n<double, 2>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<double, 2>(const AdjUpdateParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_n<double, 3>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<double, 3>(const AdjUpdateParams<double>&, int, cudaStream_t);
}  // namespace wadg
