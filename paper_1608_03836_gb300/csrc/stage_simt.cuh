// Fused WADG stage kernel on CUDA cores (FP64 or FP32).
//
// One block owns E consecutive columns (element, shot) of the field arrays and
// computes, entirely in shared memory and registers:
//   1. volume terms of the strong-weak form (Sec. 6.4, volume kernel):
//        u_q = V_q u_i, (dp/dx^_a)_q = V_q^a p,
//        U^a = sum_i G_ai u_i,  (J grad p)_i = sum_a G_ai dp/dx^_a,
//        b_p = sum_a (V_q^a)^T diag(w) U^a,  b_ui = -V_q^T diag(w) (J grad p)_i;
//   2. surface terms (Sec. 6.4, surface kernels 1 and 2, fused): the jump of p,
//      the average and jump of u at the face nodes (own values from shared
//      memory, neighbour values gathered from global memory in the owner's
//      node order), interpolated to the owner's face points (V_tri), the
//      strong-weak flux with n J^f, and the lift V_tri^T diag(w_f) scattered to
//      the volume nodes;
//   3. the weight-adjusted update (Sec. 6.2, Eq. (matfree); Sec. 7):
//        r = P_q diag(W) (V_q M^^{-1}) b,  W = c^2/J (p) or 1/J (u);
//   4. RHS mode: dQ/dt = r.  LSRK mode (Sec. 5.2): res = a res + dt r,
//      Q_out = Q + b res.
// Every phase is a set of small matrix products "A (rows x k) times a block of
// E columns" in which a thread owns one output row for EG columns; the
// reference operators are read through the read-only data path (they are
// shared by all blocks and stay resident in L1/L2).
#pragma once

#include "wadg_internal.h"

namespace wadg {

template <int N>
struct Dims {
  static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int NQ = (N + 1) * (N + 1) * (N + 1);
  static constexpr int NFP = (N + 1) * (N + 2) / 2;
  static constexpr int NFQ = (N + 1) * (N + 1);
  static constexpr int XV = 6 * NQ;                    // volume quadrature arrays
  static constexpr int XF = 7 * 4 * NFP + 7 * 4 * NFQ; // face node + face point arrays
  static constexpr int XS = XV > XF ? XV : XF;
  static constexpr int PER_COL = 8 * NP + XS;          // shared values per column
};

// Columns per block: about 96 KB of shared memory, a multiple of 4.
template <typename T, int N>
constexpr int cols_per_block() {
  constexpr int per = Dims<N>::PER_COL * (int)sizeof(T);
  constexpr int e = (98304 / per) / 4 * 4;
  return e < 4 ? 4 : (e > 32 ? 32 : e);
}

constexpr int kStageThreads = 256;

// acc[e] = sum_k A[k*M + m] * in[k*E + e], e < EG
template <typename T, int E, int EG, int M, int KK>
__device__ __forceinline__ void rowdot(const T* __restrict__ A, const T* in, int m, T (&acc)[EG]) {
#pragma unroll
  for (int e = 0; e < EG; ++e) acc[e] = T(0);
#pragma unroll 4
  for (int k = 0; k < KK; ++k) {
    const T a = __ldg(A + k * M + m);
#pragma unroll
    for (int e = 0; e < EG; ++e) acc[e] = fma(a, in[k * E + e], acc[e]);
  }
}

template <typename T, int N, int E, int MODE>
__global__ void __launch_bounds__(kStageThreads) stage_kernel(const StageParams<T> p) {
  using Dm = Dims<N>;
  constexpr int NP = Dm::NP, NQ = Dm::NQ, NFP = Dm::NFP, NFQ = Dm::NFQ;
  constexpr int EG = 4, NG = E / EG;
  constexpr int NT = kStageThreads;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);  // [4][NP][E]
  T* sR = sQ + 4 * NP * E;                 // [4][NP][E]  load vector b (un-inverted)
  T* sX = sR + 4 * NP * E;                 // [XS][E]     scratch
  T* sFN = sX;                             // [7][4 NFP][E] face-node combos
  T* sFQ = sX + 7 * 4 * NFP * E;           // [7][4 NFQ][E] face-point values

  const int tid = threadIdx.x;
  const int64_t col0 = (int64_t)blockIdx.x * E;
  const int64_t ncols = p.ncols;
  const int64_t fs = ncols * NP;  // field stride
  const int S = p.S;
  const DevOps<T>& ops = p.ops;

  // ---- load Q (columns past the end are clamped to the last one) ----
  for (int it = tid; it < 4 * E * NP; it += NT) {
    const int n = it % NP;
    const int e = (it / NP) % E;
    const int f = it / (NP * E);
    int64_t c = col0 + e;
    c = c < ncols ? c : ncols - 1;
    sQ[(f * NP + n) * E + e] = p.Qin[f * fs + c * NP + n];
  }
  __syncthreads();

  // ---- 1a. volume: values at quadrature points ----
  for (int it = tid; it < 6 * NQ * NG; it += NT) {
    const int m = it % NQ;
    const int g = (it / NQ) % NG;
    const int job = it / (NQ * NG);
    const T* A = job < 3 ? ops.VqT : ops.VaT + (job - 3) * NP * NQ;
    const T* in = (job < 3 ? sQ + (1 + job) * NP * E : sQ) + g * EG;
    T acc[EG];
    rowdot<T, E, EG, NQ, NP>(A, in, m, acc);
#pragma unroll
    for (int e = 0; e < EG; ++e) sX[(job * NQ + m) * E + g * EG + e] = acc[e];
  }
  __syncthreads();

  // ---- 1b. geometric factors: U^a and J grad p ----
  for (int it = tid; it < NQ * E; it += NT) {
    const int q = it % NQ;
    const int e = it / NQ;
    int64_t c = col0 + e;
    c = c < ncols ? c : ncols - 1;
    const int64_t k = c / S;
    const T* gk = p.vgeo + k * 11 * NQ + q;
    T G[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) G[i] = __ldg(gk + i * NQ);
    T u[3], d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      u[i] = sX[(i * NQ + q) * E + e];
      d[i] = sX[((3 + i) * NQ + q) * E + e];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
      sX[(a * NQ + q) * E + e] = G[a * 3 + 0] * u[0] + G[a * 3 + 1] * u[1] + G[a * 3 + 2] * u[2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      sX[((3 + i) * NQ + q) * E + e] = G[0 * 3 + i] * d[0] + G[1 * 3 + i] * d[1] + G[2 * 3 + i] * d[2];
  }
  __syncthreads();

  // ---- 1c. volume: test against the basis ----
  for (int it = tid; it < 4 * NP * NG; it += NT) {
    const int m = it % NP;
    const int g = (it / NP) % NG;
    const int job = it / (NP * NG);
    T acc[EG];
    if (job == 0) {
      rowdot<T, E, EG, NP, 3 * NQ>(ops.DwT, sX + g * EG, m, acc);
    } else {
      rowdot<T, E, EG, NP, NQ>(ops.VwT, sX + (3 + job - 1) * NQ * E + g * EG, m, acc);
#pragma unroll
      for (int e = 0; e < EG; ++e) acc[e] = -acc[e];
    }
#pragma unroll
    for (int e = 0; e < EG; ++e) sR[(job * NP + m) * E + g * EG + e] = acc[e];
  }
  __syncthreads();

  // ---- 2a. face nodes: [p], {u}, [u] in the owner's node order ----
  for (int it = tid; it < 4 * NFP * E; it += NT) {
    const int j = it % NFP;
    const int f = (it / NFP) % 4;
    const int e = it / (4 * NFP);
    int64_t c = col0 + e;
    c = c < ncols ? c : ncols - 1;
    const int64_t k = c / S;
    const int sh = (int)(c - k * S);
    const int code = p.fcode[k * 4 + f];
    const int pio = code % 6, pin = (code / 6) % 6, fn = code / 36;
    const int nown = ops.gidx[(f * 6 + pio) * NFP + j];
    const T pm = sQ[(0 * NP + nown) * E + e];
    const T u1m = sQ[(1 * NP + nown) * E + e];
    const T u2m = sQ[(2 * NP + nown) * E + e];
    const T u3m = sQ[(3 * NP + nown) * E + e];
    const int64_t kn = p.EToE[k * 4 + f];
    T pp, u1p, u2p, u3p;
    if (kn >= 0) {
      const int nn = ops.gidx[(fn * 6 + pin) * NFP + j];
      const int64_t b = (kn * S + sh) * NP + nn;
      pp = __ldg(p.Qin + b);
      u1p = __ldg(p.Qin + fs + b);
      u2p = __ldg(p.Qin + 2 * fs + b);
      u3p = __ldg(p.Qin + 3 * fs + b);
    } else {  // Dirichlet ghost state (Sec. 4.1): p+ = -p-, u+ = u-
      pp = -pm;
      u1p = u1m;
      u2p = u2m;
      u3p = u3m;
    }
    const int row = f * NFP + j;
    sFN[(0 * 4 * NFP + row) * E + e] = pp - pm;
    sFN[(1 * 4 * NFP + row) * E + e] = T(0.5) * (u1p + u1m);
    sFN[(2 * 4 * NFP + row) * E + e] = T(0.5) * (u2p + u2m);
    sFN[(3 * 4 * NFP + row) * E + e] = T(0.5) * (u3p + u3m);
    sFN[(4 * 4 * NFP + row) * E + e] = u1p - u1m;
    sFN[(5 * 4 * NFP + row) * E + e] = u2p - u2m;
    sFN[(6 * 4 * NFP + row) * E + e] = u3p - u3m;
  }
  __syncthreads();

  // ---- 2b. interpolate the 7 combinations to the face points ----
  for (int it = tid; it < 28 * NFQ * NG; it += NT) {
    const int m = it % NFQ;
    const int g = (it / NFQ) % NG;
    const int job = it / (NFQ * NG);  // combo * 4 + face
    T acc[EG];
    rowdot<T, E, EG, NFQ, NFP>(ops.VtriT, sFN + job * NFP * E + g * EG, m, acc);
#pragma unroll
    for (int e = 0; e < EG; ++e) sFQ[(job * NFQ + m) * E + g * EG + e] = acc[e];
  }
  __syncthreads();

  // ---- 2c. strong-weak flux (Sec. 4.1) ----
  for (int it = tid; it < 4 * NFQ * E; it += NT) {
    const int qf = it % (4 * NFQ);
    const int e = it / (4 * NFQ);
    int64_t c = col0 + e;
    c = c < ncols ? c : ncols - 1;
    const int64_t k = c / S;
    const T* fg = p.fgeo + k * 3 * 4 * NFQ + qf;
    const T nx = __ldg(fg), ny = __ldg(fg + 4 * NFQ), nz = __ldg(fg + 8 * NFQ);
    const T Jf = sqrt(nx * nx + ny * ny + nz * nz);
    const T jp = sFQ[(0 * 4 * NFQ + qf) * E + e];
    const T a1 = sFQ[(1 * 4 * NFQ + qf) * E + e];
    const T a2 = sFQ[(2 * 4 * NFQ + qf) * E + e];
    const T a3 = sFQ[(3 * 4 * NFQ + qf) * E + e];
    const T j1 = sFQ[(4 * 4 * NFQ + qf) * E + e];
    const T j2 = sFQ[(5 * 4 * NFQ + qf) * E + e];
    const T j3 = sFQ[(6 * 4 * NFQ + qf) * E + e];
    const T aun = a1 * nx + a2 * ny + a3 * nz;
    const T jun = (j1 * nx + j2 * ny + j3 * nz) / Jf;
    const T Fp = -aun + T(0.5) * p.tau_p * jp * Jf;
    const T s = T(-0.5) * (jp - p.tau_u * jun);
    sFQ[(0 * 4 * NFQ + qf) * E + e] = Fp;
    sFQ[(1 * 4 * NFQ + qf) * E + e] = s * nx;
    sFQ[(2 * 4 * NFQ + qf) * E + e] = s * ny;
    sFQ[(3 * 4 * NFQ + qf) * E + e] = s * nz;
  }
  __syncthreads();

  // ---- 2d. V_tri^T diag(w_f): back to face nodes ----
  for (int it = tid; it < 16 * NFP * NG; it += NT) {
    const int m = it % NFP;
    const int g = (it / NFP) % NG;
    const int job = it / (NFP * NG);  // field * 4 + face
    T acc[EG];
    rowdot<T, E, EG, NFP, NFQ>(ops.VtriTwT, sFQ + job * NFQ * E + g * EG, m, acc);
#pragma unroll
    for (int e = 0; e < EG; ++e) sFN[(job * NFP + m) * E + g * EG + e] = acc[e];
  }
  __syncthreads();

  // ---- 2e. scatter to volume nodes (+ point source) ----
  for (int it = tid; it < 4 * NP * E; it += NT) {
    const int n = it % NP;
    const int e = (it / NP) % E;
    const int fld = it / (NP * E);
    int64_t c = col0 + e;
    c = c < ncols ? c : ncols - 1;
    const int64_t k = c / S;
    T acc = sR[(fld * NP + n) * E + e];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int pio = p.fcode[k * 4 + f] % 6;
      const int jo = ops.ginv[(f * 6 + pio) * NP + n];
      if (jo >= 0) acc += sFN[((fld * 4 + f) * NFP + jo) * E + e];
    }
    if (fld == 0 && p.src_elem != nullptr) {
      const int sh = (int)(c - k * S);
      if (p.src_elem[sh] == (int32_t)k) acc += p.src_amp * p.src_vec[sh * NP + n];
    }
    sR[(fld * NP + n) * E + e] = acc;
  }
  __syncthreads();

  // ---- 3a. update: W (V_q M^^{-1}) b at quadrature points ----
  for (int it = tid; it < 4 * NQ * NG; it += NT) {
    const int m = it % NQ;
    const int g = (it / NQ) % NG;
    const int fld = it / (NQ * NG);
    T acc[EG];
    rowdot<T, E, EG, NQ, NP>(ops.VtT, sR + fld * NP * E + g * EG, m, acc);
    const int wc = fld == 0 ? 9 : 10;
#pragma unroll
    for (int e = 0; e < EG; ++e) {
      int64_t c = col0 + g * EG + e;
      c = c < ncols ? c : ncols - 1;
      const int64_t k = c / S;
      sX[(fld * NQ + m) * E + g * EG + e] = acc[e] * __ldg(p.vgeo + (k * 11 + wc) * NQ + m);
    }
  }
  __syncthreads();

  // ---- 3b. update: P_q back to nodes, then the epilogue ----
  for (int it = tid; it < 4 * NP * NG; it += NT) {
    const int m = it % NP;
    const int g = (it / NP) % NG;
    const int fld = it / (NP * NG);
    T acc[EG];
    rowdot<T, E, EG, NP, NQ>(ops.PqT, sX + fld * NQ * E + g * EG, m, acc);
#pragma unroll
    for (int e = 0; e < EG; ++e) {
      const int64_t c = col0 + g * EG + e;
      if (c >= ncols) continue;
      const int64_t idx = fld * fs + c * NP + m;
      if (MODE == 0) {
        p.out[idx] = acc[e];
      } else {
        const T r = p.rk_a * p.res[idx] + p.dt * acc[e];
        p.res[idx] = r;
        p.Qout[idx] = sQ[(fld * NP + m) * E + g * EG + e] + p.rk_b * r;
      }
    }
  }
}

template <typename T, int N>
cudaError_t launch_stage_n(const StageParams<T>& p, int mode, cudaStream_t stream) {
  constexpr int E = cols_per_block<T, N>();
  const size_t smem = (size_t)Dims<N>::PER_COL * E * sizeof(T);
  const int64_t blocks = (p.ncols + E - 1) / E;
  if (blocks == 0) return cudaSuccess;
  if (mode == 0) {
    auto kern = stage_kernel<T, N, E, 0>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)blocks, kStageThreads, smem, stream>>>(p);
  } else {
    auto kern = stage_kernel<T, N, E, 1>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)blocks, kStageThreads, smem, stream>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace wadg
