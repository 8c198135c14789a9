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

// Tile rules: rule 0 is the single-mesh rule (cols_per_block); rule 1 caps
// every degree to ~76 KB of shared memory so that a mixed batch keeps three
// blocks per SM, taking the widest of the single-mesh width, 8 and 4 columns
// that fits (degree 5 then takes 8 columns per tile, degree 6 takes 4).
template <int N, int RULE>
constexpr int batch_cols() {
  constexpr int per = Dims<N>::PER_COL * 4;
  constexpr int e0 = cols_per_block<float, N>();
  return RULE == 0 ? e0 : (per * e0 <= 77824 ? e0 : (per * 8 <= 77824 ? 8 : 4));
}

template <int MODE, int RULE>
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
      case 1: stage_tile<float, 1, batch_cols<1, RULE>(), MODE>(p, blk, smem_raw); break;
      case 2: stage_tile<float, 2, batch_cols<2, RULE>(), MODE>(p, blk, smem_raw); break;
      case 3: stage_tile<float, 3, batch_cols<3, RULE>(), MODE>(p, blk, smem_raw); break;
      case 4: stage_tile<float, 4, batch_cols<4, RULE>(), MODE>(p, blk, smem_raw); break;
      case 5: stage_tile<float, 5, batch_cols<5, RULE>(), MODE>(p, blk, smem_raw); break;
      case 6: stage_tile<float, 6, batch_cols<6, RULE>(), MODE>(p, blk, smem_raw); break;
      default: break;
    }
    __syncthreads();
  }
}

template <int RULE>
int cols_rule(int N) {
  switch (N) {
    case 1: return batch_cols<1, RULE>();
    case 2: return batch_cols<2, RULE>();
    case 3: return batch_cols<3, RULE>();
    case 4: return batch_cols<4, RULE>();
    case 5: return batch_cols<5, RULE>();
    case 6: return batch_cols<6, RULE>();
    default: return 0;
  }
}

static size_t per_col_bytes(int N) {
  switch (N) {
    case 1: return (size_t)Dims<1>::PER_COL * 4;
    case 2: return (size_t)Dims<2>::PER_COL * 4;
    case 3: return (size_t)Dims<3>::PER_COL * 4;
    case 4: return (size_t)Dims<4>::PER_COL * 4;
    case 5: return (size_t)Dims<5>::PER_COL * 4;
    case 6: return (size_t)Dims<6>::PER_COL * 4;
    default: return 0;
  }
}

int batch_cols_per_block(int N, int rule) { return rule == 0 ? cols_rule<0>(N) : cols_rule<1>(N); }

size_t batch_smem_bytes(int N, int rule) { return per_col_bytes(N) * batch_cols_per_block(N, rule); }

template <int MODE, int RULE>
static cudaError_t launch_rule(const StageParams<float>* params, const int* item_mesh, const int* item_blk,
                               const int* mesh_N, int nitems, int grid, size_t smem, cudaStream_t st) {
  auto kern = batch_stage_kernel<MODE, RULE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kStageThreads, smem, st>>>(params, item_mesh, item_blk, mesh_N, nitems);
  return cudaGetLastError();
}

cudaError_t launch_batch_stage(int mode, int rule, const StageParams<float>* params, const int* item_mesh,
                               const int* item_blk, const int* mesh_N, int nitems, int grid, size_t smem,
                               cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  if (mode == kRhs)
    return rule == 0 ? launch_rule<kRhs, 0>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st)
                     : launch_rule<kRhs, 1>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st);
  return rule == 0 ? launch_rule<kLsrk, 0>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st)
                   : launch_rule<kLsrk, 1>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st);
}

int batch_max_blocks_per_sm(int rule, size_t smem) {
  int n = 0;
  auto kern = rule == 0 ? batch_stage_kernel<kLsrk, 0> : batch_stage_kernel<kLsrk, 1>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kStageThreads, smem) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace wadg
