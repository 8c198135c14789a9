// Batches of meshes of uneven size and degree, stepped together: one
// persistent launch per LSRK stage walks a work list of (mesh, tile) items,
// each block dispatching on the item's degree to the CUDA-core stage tile
// (stage_simt.cuh), so that 12 meshes cost 5 launches per step instead of 60.
// Items are ordered heaviest degree first; an autotuner picks the tile rule
// and the number of persistent blocks.  FP32 fields (WADG_FP32 meshes).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "stage_simt.cuh"

namespace wadg {

// Tile rules.  One kernel holds every degree's tile, so its register count is
// the largest over the degrees and its shared memory the largest tile's.
//   rule 0: tiles of at most 76 KB (28, 20, 12, 8 or 4 columns, the widest
//           that fits), registers capped for two blocks per SM (128);
//   rule 1: the same widths, registers capped for three blocks per SM (80);
//   rule 2: tiles of at most 56 KB and registers capped for four blocks per
//           SM (64), the occupancy that degree 6 reaches on its own.
// The cap trades per-tile speed (registers, spills) for resident blocks: a
// batch of many tiles gains from occupancy, a batch of few tiles from per-tile
// latency, which is why the autotuner times all three (kBatchRules).

template <int N, int RULE>
constexpr int batch_cols() {
  return cols_for_budget<float, N, Dims<N>::PER_COL, RULE < 2 ? 77824 : 57344>();
}

template <int RULE>
constexpr int batch_min_blocks() { return RULE + 2; }

template <int MODE, int RULE>
__global__ void __launch_bounds__(kStageThreads, batch_min_blocks<RULE>()) batch_stage_kernel(const StageParams<float>* __restrict__ params,
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

int batch_cols_per_block(int N, int rule) {
  return rule == 0 ? cols_rule<0>(N) : (rule == 1 ? cols_rule<1>(N) : cols_rule<2>(N));
}

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
  if (mode == kRhs) {
    if (rule == 0) return launch_rule<kRhs, 0>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st);
    if (rule == 1) return launch_rule<kRhs, 1>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st);
    return launch_rule<kRhs, 2>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st);
  }
  if (rule == 0) return launch_rule<kLsrk, 0>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st);
  if (rule == 1) return launch_rule<kLsrk, 1>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st);
  return launch_rule<kLsrk, 2>(params, item_mesh, item_blk, mesh_N, nitems, grid, smem, st);
}

int batch_max_blocks_per_sm(int rule, size_t smem) {
  int n = 0;
  auto kern = rule == 0 ? batch_stage_kernel<kLsrk, 0>
                        : (rule == 1 ? batch_stage_kernel<kLsrk, 1> : batch_stage_kernel<kLsrk, 2>);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kStageThreads, smem) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace wadg
