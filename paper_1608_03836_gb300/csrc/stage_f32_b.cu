// Instantiations of the fused stage kernel: float, N in {4 5 6}.
#include "stage_simt.cuh"

namespace wadg {
template cudaError_t launch_stage_n<float, 4>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_stage_n<float, 5>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_stage_n<float, 6>(const StageParams<float>&, int, cudaStream_t);
}  // namespace wadg
