// Instantiations of the fused stage kernel and the adjoint update: double, N in {4 5 6}.
#include "adjoint_simt.cuh"

namespace wadg {
template cudaError_t launch_stage_n<double, 4>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<double, 4>(const AdjUpdateParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_n<double, 5>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<double, 5>(const AdjUpdateParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_n<double, 6>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_adj_update_n<double, 6>(const AdjUpdateParams<double>&, int, cudaStream_t);
}  // namespace wadg
