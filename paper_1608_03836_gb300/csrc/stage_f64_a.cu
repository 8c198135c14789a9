// Instantiations of the fused stage kernel: double, N in {1 2 3}.
#include "stage_simt.cuh"

namespace wadg {
template cudaError_t launch_stage_n<double, 1>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_n<double, 2>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_n<double, 3>(const StageParams<double>&, int, cudaStream_t);
}  // namespace wadg
