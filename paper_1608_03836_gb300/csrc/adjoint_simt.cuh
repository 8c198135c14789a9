// Transpose of the weight-adjusted update, beta = U^T mu = (V_q M^^{-1})^T
// diag(W) P_q^T mu (Sec. 6.2, Eq. (matfree) transposed; W = c^2/J for p, 1/J
// for u), one block per E columns, on CUDA cores.
//
// LSRK mode is the reverse of one 2N-storage stage res = a res + dt L Q,
// Q += b res with L = U A:  mu = lambda_res + b lambda_Q, beta = U^T mu,
// lambda_res = a mu; the caller then adds dt A^T beta to lambda_Q (stage
// kernel, adjoint mode).  When a recorded forward factor y_q = (V_q M^^{-1}
// b_p)_q / J_q is given, the gradient of the misfit with respect to c^2 at the
// volume points gains dt (P_q^T mu_p)_q y_q, since dr_p/dc^2_q = P_q e_q y_q.
#pragma once

#include "stage_simt.cuh"

namespace wadg {

template <typename T, int N, int E, int LSRK>
__global__ void __launch_bounds__(kStageThreads) adj_update_kernel(const AdjUpdateParams<T> p) {
  using Dm = Dims<N>;
  constexpr int NP = Dm::NP, NQ = Dm::NQ, NQP = Dm::NQP, NPP = Dm::NPP;
  constexpr int NG = E / 4;
  constexpr int NT = kStageThreads;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sM = reinterpret_cast<T*>(smem_raw);  // [4][NP][E] mu
  T* sZ = sM + 4 * NP * E;                 // [4][NQ][E] W P_q^T mu

  const int tid = threadIdx.x;
  const int64_t col0 = (int64_t)blockIdx.x * E;
  const int64_t ncols = p.ncols;
  const int64_t fs = ncols * NP;
  const int S = p.S;

  for (int it = tid; it < 4 * E * NP; it += NT) {
    const int n = it % NP;
    const int e = (it / NP) % E;
    const int f = it / (NP * E);
    int64_t c = col0 + e;
    c = c < ncols ? c : ncols - 1;
    const int64_t idx = f * fs + c * NP + n;
    sM[(f * NP + n) * E + e] = LSRK ? p.lamR[idx] + p.rk_b * p.lamQ[idx] : p.lam[idx];
  }
  __syncthreads();

  // z = W (P_q^T mu), and the c^2 gradient from the pressure row
  {
    constexpr int RG = NQP / 4;
    for (int it = tid; it < 4 * RG * NG; it += NT) {
      const int g = it % NG;
      const int m0 = ((it / NG) % RG) * 4;
      const int fld = it / (RG * NG);
      T acc[4][4];
      tile_dot<T, E, 4, NQP, NP>(p.ops.PqTT, sM + fld * NP * E + g * 4, m0, acc);
      const int wc = fld == 0 ? 9 : 10;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t cc = col0 + g * 4 + e;
        const int64_t c = cc < ncols ? cc : ncols - 1;
        const int64_t k = c / S;
        const T* w = p.vgeo + (k * 11 + wc) * NQ;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int q = m0 + r;
          if (q >= NQ) continue;
          if (fld == 0 && p.dc2 != nullptr && cc < ncols)
            atomicAdd(p.dc2 + k * NQ + q, (double)p.dt * (double)acc[r][e] * (double)p.yrec[c * NQ + q]);
          sZ[(fld * NQ + q) * E + g * 4 + e] = acc[r][e] * __ldg(w + q);
        }
      }
    }
  }
  __syncthreads();

  // beta = (V_q M^^{-1})^T z; LSRK: lambda_res = a mu
  {
    constexpr int RG = NPP / 2;
    for (int it = tid; it < 4 * RG * NG; it += NT) {
      const int g = it % NG;
      const int m0 = ((it / NG) % RG) * 2;
      const int fld = it / (RG * NG);
      T acc[2][4];
      tile_dot<T, E, 2, NPP, NQ>(p.ops.VtTT, sZ + fld * NQ * E + g * 4, m0, acc);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t c = col0 + g * 4 + e;
        if (c >= ncols) continue;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int m = m0 + r;
          if (m >= NP) continue;
          const int64_t idx = fld * fs + c * NP + m;
          p.beta[idx] = acc[r][e];
          if (LSRK) p.lamR[idx] = p.rk_a * sM[(fld * NP + m) * E + g * 4 + e];
        }
      }
    }
  }
}

template <typename T, int N>
cudaError_t launch_adj_update_n(const AdjUpdateParams<T>& p, int lsrk, cudaStream_t stream) {
  constexpr int E = 12;
  const size_t smem = (size_t)(4 * Dims<N>::NP + 4 * Dims<N>::NQ) * E * sizeof(T);
  const int64_t blocks = (p.ncols + E - 1) / E;
  if (blocks == 0) return cudaSuccess;
  if (lsrk) {
    auto kern = adj_update_kernel<T, N, E, 1>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)blocks, kStageThreads, smem, stream>>>(p);
  } else {
    auto kern = adj_update_kernel<T, N, E, 0>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)blocks, kStageThreads, smem, stream>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace wadg
