// Instantiations of the fused stage kernel: float, N in {1 2 3}.
#include "stage_simt.cuh"

namespace wadg {
template cudaError_t launch_stage_n<float, 1>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_stage_n<float, 2>(const StageParams<float>&, int, cudaStream_t);
template cudaError_t launch_stage_n<float, 3>(const StageParams<float>&, int, cudaStream_t);
}  // namespace wadg
