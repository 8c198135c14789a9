// Instantiations of the fused stage kernel: double, N in {4 5 6}.
#include "stage_simt.cuh"

namespace wadg {
template cudaError_t launch_stage_n<double, 4>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_n<double, 5>(const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_n<double, 6>(const StageParams<double>&, int, cudaStream_t);
}  // namespace wadg
