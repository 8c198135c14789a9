// Launchers of the tensor-core stage for N <= 4 (the kernel is in
// stage_tc_kernel.cuh; the planar-element instantiations in stage_tc_planar.cu)
// and the host packing of its operators.
#include "stage_tc_kernel.cuh"

namespace wadg {

// Failure path of the bounded waits: one block waits, with the same loop the
// stage kernel uses, on an mbarrier that nothing arrives at; the expired wait
// sets the error flag exactly as in the stage kernel.
__global__ void bounded_wait_selftest_kernel(int* err, uint32_t max_iters) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) tc::mbar_init(tc::smem_addr(&mbar), 1);
  __syncthreads();
  const bool ok = tc::mbar_wait(tc::smem_addr(&mbar), 0, max_iters);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

cudaError_t launch_bounded_wait_selftest(int* err, uint32_t max_iters, cudaStream_t stream) {
  bounded_wait_selftest_kernel<<<1, 32, 0, stream>>>(err, max_iters);
  return cudaGetLastError();
}

cudaError_t launch_stage_tc(int N, const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream) {
  switch (N) {
    case 1: return launch_stage_tc_n<1, false>(P, mode, fmt, grid, stream);
    case 2: return launch_stage_tc_n<2, false>(P, mode, fmt, grid, stream);
    case 3: return launch_stage_tc_n<3, false>(P, mode, fmt, grid, stream);
    case 4: return launch_stage_tc_n<4, false>(P, mode, fmt, grid, stream);
    case 5: return launch_stage_tc5(P, mode, fmt, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Host: pack the operators of the tensor-core stage, split into bf16 hi + lo,
// in the K-major no-swizzle layout, chunk by chunk in the order the kernel
// stages them.
// ---------------------------------------------------------------------------

template <int N>
bool pack_q(const RefOps& o, int fmt, std::vector<uint8_t>& out) {
  if (!face_nodes_match<N>(o)) return false;
  if (o.Nq == Dims<N>::NQ) {
    pack_dims<TcDims<N, Dims<N>::NQ>>(o, fmt, out);
    return true;
  }
  if constexpr (fewer_point_nq(N) > 0)
    if (o.Nq == fewer_point_nq(N)) {
      pack_dims<TcDims<N, fewer_point_nq(N)>>(o, fmt, out);
      return true;
    }
  return false;
}

bool pack_tc_ops(int N, const RefOps& o, int fmt, std::vector<uint8_t>& out) {
  switch (N) {
    case 1: return pack_q<1>(o, fmt, out);
    case 2: return pack_q<2>(o, fmt, out);
    case 3: return pack_q<3>(o, fmt, out);
    case 4: return pack_q<4>(o, fmt, out);
    case 5: return pack_tc5_ops(o, fmt, out);
    default: return false;
  }
}

}  // namespace wadg
