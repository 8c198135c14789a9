// Batches of meshes of uneven size and degree, stepped together: one
// persistent launch per LSRK stage walks a work list of (mesh, tile) items,
// each block dispatching on the item's degree to the CUDA-core stage tile
// (stage_simt.cuh), so that 12 meshes cost 5 launches per step instead of 60.
// Items are ordered heaviest degree first; an autotuner picks the number of
// persistent blocks.  FP32 fields (WADG_FP32 meshes).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "stage_simt.cuh"

namespace wadg {

template <int MODE>
__global__ void __launch_bounds__(kStageThreads) batch_stage_kernel(const StageParams<float>* __restrict__ params,
                                                                    const int* __restrict__ item_mesh,
                                                                    const int* __restrict__ item_blk,
                                                                    const int* __restrict__ mesh_N, int nitems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int mi = item_mesh[it];
    const StageParams<float>& p = params[mi];
    const int64_t blk = item_blk[it];
    switch (mesh_N[mi]) {
      case 1: stage_tile<float, 1, cols_per_block<float, 1>(), MODE>(p, blk, smem_raw); break;
      case 2: stage_tile<float, 2, cols_per_block<float, 2>(), MODE>(p, blk, smem_raw); break;
      case 3: stage_tile<float, 3, cols_per_block<float, 3>(), MODE>(p, blk, smem_raw); break;
      case 4: stage_tile<float, 4, cols_per_block<float, 4>(), MODE>(p, blk, smem_raw); break;
      case 5: stage_tile<float, 5, cols_per_block<float, 5>(), MODE>(p, blk, smem_raw); break;
      case 6: stage_tile<float, 6, cols_per_block<float, 6>(), MODE>(p, blk, smem_raw); break;
      default: break;
    }
    __syncthreads();
  }
}

int batch_cols_per_block(int N) {
  switch (N) {
    case 1: return cols_per_block<float, 1>();
    case 2: return cols_per_block<float, 2>();
    case 3: return cols_per_block<float, 3>();
    case 4: return cols_per_block<float, 4>();
    case 5: return cols_per_block<float, 5>();
    case 6: return cols_per_block<float, 6>();
    default: return 0;
  }
}

size_t batch_smem_bytes(int N) {
  switch (N) {
    case 1: return (size_t)Dims<1>::PER_COL * cols_per_block<float, 1>() * 4;
    case 2: return (size_t)Dims<2>::PER_COL * cols_per_block<float, 2>() * 4;
    case 3: return (size_t)Dims<3>::PER_COL * cols_per_block<float, 3>() * 4;
    case 4: return (size_t)Dims<4>::PER_COL * cols_per_block<float, 4>() * 4;
    case 5: return (size_t)Dims<5>::PER_COL * cols_per_block<float, 5>() * 4;
    case 6: return (size_t)Dims<6>::PER_COL * cols_per_block<float, 6>() * 4;
    default: return 0;
  }
}

cudaError_t launch_batch_stage(int mode, const StageParams<float>* params, const int* item_mesh, const int* item_blk,
                               const int* mesh_N, int nitems, int grid, size_t smem, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  if (mode == kRhs) {
    cudaError_t e = cudaFuncSetAttribute(batch_stage_kernel<kRhs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    batch_stage_kernel<kRhs><<<grid, kStageThreads, smem, st>>>(params, item_mesh, item_blk, mesh_N, nitems);
  } else {
    cudaError_t e = cudaFuncSetAttribute(batch_stage_kernel<kLsrk>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    batch_stage_kernel<kLsrk><<<grid, kStageThreads, smem, st>>>(params, item_mesh, item_blk, mesh_N, nitems);
  }
  return cudaGetLastError();
}

int batch_max_blocks_per_sm(size_t smem) {
  int n = 0;
  if (cudaFuncSetAttribute(batch_stage_kernel<kLsrk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_kernel<kLsrk>, kStageThreads, smem) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace wadg
