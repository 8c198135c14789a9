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
//      Q_out = Q + b res (the first stage, a = 0, reads no res).  Record
//      mode: LSRK, and also stores y_q = (V_q M^^{-1} b_p)_q / J_q, the factor
//      of dr_p/dc^2_q.
// Strong modes (Sec. 4.1, Sec. 6.3) replace step 1 by the strong form's volume
// terms -V^T diag(w) (J div u, J grad p) on their own rule (the energy-stable
// degree 4N-3 rule, or the 2N+1 rule), walked in chunks of points, and carry
// only [p] and [u] through step 2.  The volume rule of steps 1 and 3 has NQX
// points (the collapsed (N+1)^3 rule or a fewer-point symmetric rule).
// Adjoint modes apply A^T (the transpose of steps 1-2) to an input beta and
// skip step 3: the strong-weak volume operator is skew, so its transpose is
// its negative; the transpose of the surface operator is the same pipeline
// with the central flux terms negated and the penalty terms unchanged.  Mode
// ADJ_LSRK adds dt A^T beta to lambda_Q in place; mode ADJ_RHS writes it.
// Every phase is a set of small matrix products "A (rows x k) times a block of
// E columns" in which a thread owns a register tile of 4 (or 2) output rows by
// 4 columns, loading 4 rows of A with one 128-bit read-only load and 4 columns
// of the input with one 128-bit shared-memory load per k; the reference
// operators are shared by all blocks and stay resident in L1/L2.
#pragma once

#include "wadg_internal.h"

namespace wadg {

// Sizes for degree N and a volume rule of NQX points (default: the collapsed
// (N+1)^3 rule; fewer_point_nq(N) for the symmetric rules).
template <int N, int NQX = (N + 1) * (N + 1) * (N + 1)>
struct Dims {
  static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int NQ = NQX;
  static constexpr int NFP = (N + 1) * (N + 2) / 2;
  static constexpr int NFQ = (N + 1) * (N + 1);
  static constexpr int XV = 6 * NQ;                    // volume quadrature arrays
  static constexpr int XF = 7 * 4 * NFP + 7 * 4 * NFQ; // face node + face point arrays
  static constexpr int XS = XV > XF ? XV : XF;
  static constexpr int PER_COL = 10 * NP + XS;         // shared values per column
  // operator row counts padded to a multiple of 4 (k-major tables)
  static constexpr int NQP = (NQ + 3) / 4 * 4;
  static constexpr int NPP = (NP + 3) / 4 * 4;
  static constexpr int NFQP = (NFQ + 3) / 4 * 4;
  static constexpr int NFPP = (NFP + 3) / 4 * 4;
};

// Columns per block E.  E = 4 (mod 8) makes the row stride of the [row][E]
// shared arrays 16 words modulo 32 banks, so that the 4x4 register tiles of a
// warp (column group fastest) store without bank conflicts; E = 8 is taken
// where 12 columns do not fit.  FP32 budget (BUDGET bytes of shared memory
// per block): 56 KB, four blocks per SM at 256 threads and at most 64
// registers, for every degree but N = 5, which keeps 76 KB (three blocks).
// The stage waits on its operator loads, so resident warps count for more
// than wide tiles; measured per LSRK step (FP32): N = 2 -15 %, N = 3 -6 %,
// N = 4 -8 % (-24 % in the strong form) against 76 KB, N = 5 +4 % (8 columns
// in 69 KB beat 4 in 35 KB, and 12 columns in 103 KB by 18 %).
// FP64 is bound by the FP64 pipe, not by shared memory: it keeps ~96 KB
// blocks with E a multiple of 4.
template <typename T, int N, int PER, int BUDGET>
constexpr int cols_for_budget() {
  constexpr int per = PER * (int)sizeof(T);
  if (sizeof(T) == 8) {
    constexpr int e8 = (98304 / per) / 4 * 4;
    return e8 < 4 ? 4 : (e8 > 32 ? 32 : e8);
  }
  constexpr int fit = BUDGET / per;
  constexpr int e = fit >= 28 ? 28 : (fit >= 20 ? 20 : (fit >= 12 ? 12 : (fit >= 8 ? 8 : 4)));
  return e;
}
template <typename T, int N, int PER>
constexpr int cols_for() {
  return cols_for_budget<T, N, PER, N == 5 ? 77824 : 57344>();
}
template <typename T, int N>
constexpr int cols_per_block() {
  return cols_for<T, N, Dims<N>::PER_COL>();
}

constexpr bool strong_mode(int mode) {
  return mode == kRhsStrong || mode == kLsrkStrong || mode == kRhsStrongU || mode == kLsrkStrongU;
}
// Shared values per column of a mode: the strong modes use their own layout.
template <int N, int MODE, int NQX>
constexpr int mode_per_col() {
  if constexpr (MODE == kRhsStrong || MODE == kLsrkStrong) return StrongDims<N, 1>::PER_COL;
  if constexpr (MODE == kRhsStrongU || MODE == kLsrkStrongU) return StrongDims<N, 2>::PER_COL;
  return Dims<N, NQX>::PER_COL;
}

constexpr int kStageThreads = 256;

// (StageMode: see wadg_internal.h)

// Vector loads: R consecutive operator rows through the read-only path, and
// 4 consecutive columns from shared memory.
__device__ __forceinline__ void ldg_rows(const float* p, float (&v)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ldg_rows(const float* p, float (&v)[2]) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ldg_rows(const double* p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ldg_rows(const double* p, double (&v)[2]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ void lds_cols(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void lds_cols(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ void sts_cols(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void sts_cols(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// Register tile: acc[r][e] = sum_k A[k*MP + m0 + r] * in[k*E + e] for R rows and
// 4 columns.  A is a k-major operator table with MP (a multiple of 4) rows.
template <typename T, int E, int R, int MP, int KK>
__device__ __forceinline__ void tile_dot(const T* __restrict__ A, const T* in, int m0, T (&acc)[R][4]) {
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[r][e] = T(0);
#pragma unroll 8
  for (int k = 0; k < KK; ++k) {
    T a[R], b[4];
    ldg_rows(A + k * MP + m0, a);
    lds_cols(in + k * E, b);
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[r][e] = fma(a[r], b[e], acc[r][e]);
  }
}

// One block's tile: columns [blk*E, blk*E + E) of the mesh described by p,
// whose volume rule has NQX points.
template <typename T, int N, int E, int MODE, int NQX = (N + 1) * (N + 1) * (N + 1)>
__device__ __forceinline__ void stage_tile(const StageParams<T>& p, int64_t blk, unsigned char* smem_raw) {
  using Dm = Dims<N, NQX>;
  constexpr int NP = Dm::NP, NQ = Dm::NQ, NFP = Dm::NFP, NFQ = Dm::NFQ;
  constexpr int NQP = Dm::NQP, NPP = Dm::NPP, NFQP = Dm::NFQP, NFPP = Dm::NFPP;
  constexpr int NG = E / 4;
  constexpr int NT = kStageThreads;
  constexpr bool ADJ = MODE == kAdjLsrk || MODE == kAdjRhs;
  constexpr bool STRONG = strong_mode(MODE);
  constexpr bool SFULL = MODE == kRhsStrong || MODE == kLsrkStrong;
  constexpr bool RHS_OUT = MODE == kRhs || MODE == kRhsStrong || MODE == kRhsStrongU;
  using SD = StrongDims<N, SFULL ? 1 : 2>;
  // face phase: jump/average combinations at the face nodes and points
  constexpr int NCMB = STRONG ? 4 : 7;
  constexpr int FQ = STRONG ? SD::NFQS : NFQ;
  constexpr int FQP = STRONG ? SD::NFQSP : NFQP;

  T* sQ = reinterpret_cast<T*>(smem_raw);  // [4][NP][E]
  T* sR = sQ + 4 * NP * E;                 // [4][NP][E]  load vector b (un-inverted)
  T* sP = sR + 4 * NP * E;                 // [2][NP][E]  partial pressure volume terms (strong-weak)
  T* sX = STRONG ? sP : sP + 2 * NP * E;   // [XS][E]     scratch
  T* sFN = sX;                             // [NCMB][4 NFP][E] face-node combos
  T* sFQ = sX + NCMB * 4 * NFP * E;        // [NCMB][4 FQ][E]  face-point values

  const int tid = threadIdx.x;
  const int64_t col0 = blk * E;
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

  if constexpr (!STRONG) {
  // ---- 1a. volume: values at quadrature points (6 products, 4 rows x 4 cols) ----
  {
    constexpr int RG = NQP / 4;
    for (int it = tid; it < 6 * RG * NG; it += NT) {
      const int g = it % NG;
      const int m0 = ((it / NG) % RG) * 4;
      const int job = it / (RG * NG);
      const T* A = job < 3 ? ops.VqT : ops.VaT + (job - 3) * NP * NQP;
      const T* in = (job < 3 ? sQ + (1 + job) * NP * E : sQ) + g * 4;
      T acc[4][4];
      tile_dot<T, E, 4, NQP, NP>(A, in, m0, acc);
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (m0 + r < NQ) sts_cols(sX + (job * NQ + m0 + r) * E + g * 4, acc[r]);
    }
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

  // ---- 1c. volume: test against the basis (6 equal products, 2 rows x 4 cols) ----
  // jobs 0..2: (V_q^a)^T diag(w) U^a  -> pressure partials; jobs 3..5: -V_q^T diag(w) (J grad p)_i
  {
    constexpr int RG = NPP / 2;
    for (int it = tid; it < 6 * RG * NG; it += NT) {
      const int g = it % NG;
      const int m0 = ((it / NG) % RG) * 2;
      const int job = it / (RG * NG);
      const T* A = job < 3 ? ops.DwT + job * NQ * NPP : ops.VwT;
      T acc[2][4];
      tile_dot<T, E, 2, NPP, NQ>(A, sX + job * NQ * E + g * 4, m0, acc);
      T* out = job == 0 ? sR : (job < 3 ? sP + (job - 1) * NP * E : sR + (job - 2) * NP * E);
      T sgn = job < 3 ? T(1) : T(-1);
      if (ADJ) sgn = -sgn;  // the volume operator is skew
#pragma unroll
      for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[r][e] *= sgn;
        if (m0 + r < NP) sts_cols(out + (m0 + r) * E + g * 4, acc[r]);
      }
    }
  }
  __syncthreads();
  } else {
    // ---- 1 (strong form, Sec. 6.3): at the rule's NQS volume points, QC at
    // a time, the 12 reference derivatives d(p, u_i)/dx^_a; then pointwise
    // J div u = sum_{a,i} G_ai du_i/dx^_a and J grad p = sum_a G_ai dp/dx^_a;
    // then b_p = -V_q^T diag(w) (J div u), b_ui = -V_q^T diag(w) (J grad p)_i,
    // accumulated over the chunks by the thread that owns each output ----
    constexpr int NQS = SD::NQS, QC = SD::QC, NQSC = SD::NQSC;
    static_assert(12 * QC <= SD::XS && 4 * NQ <= SD::XS, "strong-form scratch");
    const T* sg = SFULL ? p.sgeo : p.vgeo;
    constexpr int64_t GST = SFULL ? 9 * NQS : 11 * NQ;  // element stride of G_ai
    for (int q0 = 0; q0 < NQSC; q0 += QC) {
      {
        constexpr int RG = QC / 4;
        for (int it = tid; it < 12 * RG * NG; it += NT) {
          const int g = it % NG;
          const int m0 = ((it / NG) % RG) * 4;
          const int job = it / (RG * NG);  // 3 field + a
          const int fld = job / 3, a = job % 3;
          T acc[4][4];
          tile_dot<T, E, 4, NQSC, NP>(p.sops.VaT + a * NP * NQSC + q0, sQ + fld * NP * E + g * 4, m0, acc);
#pragma unroll
          for (int r = 0; r < 4; ++r) sts_cols(sX + (job * QC + m0 + r) * E + g * 4, acc[r]);
        }
      }
      __syncthreads();
      for (int it = tid; it < QC * E; it += NT) {
        const int q = it % QC;
        const int e = it / QC;
        T v[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) v[j] = sX[(j * QC + q) * E + e];
        T jdiv = T(0), gp[3] = {T(0), T(0), T(0)};
        if (q0 + q < NQS) {  // padded points carry no geometry
          int64_t c = col0 + e;
          c = c < ncols ? c : ncols - 1;
          const T* gk = sg + (c / S) * GST + q0 + q;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const T G = __ldg(gk + (a * 3 + i) * NQS);
              jdiv += G * v[3 * (1 + i) + a];
              gp[i] += G * v[a];
            }
        }
        sX[q * E + e] = jdiv;
#pragma unroll
        for (int i = 0; i < 3; ++i) sX[((1 + i) * QC + q) * E + e] = gp[i];
      }
      __syncthreads();
      {
        constexpr int RG = NPP / 2;
        for (int it = tid; it < 4 * RG * NG; it += NT) {
          const int g = it % NG;
          const int m0 = ((it / NG) % RG) * 2;
          const int job = it / (RG * NG);
          T acc[2][4];
          tile_dot<T, E, 2, NPP, QC>(p.sops.VwT + q0 * NPP, sX + job * QC * E + g * 4, m0, acc);
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            if (m0 + r >= NP) continue;
            T* o = sR + (job * NP + m0 + r) * E + g * 4;
            T cur[4];
            if (q0 == 0) {
#pragma unroll
              for (int e = 0; e < 4; ++e) cur[e] = -acc[r][e];
            } else {
              lds_cols(o, cur);
#pragma unroll
              for (int e = 0; e < 4; ++e) cur[e] -= acc[r][e];
            }
            sts_cols(o, cur);
          }
        }
      }
      __syncthreads();
    }
  }

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
    if constexpr (STRONG) {  // [p], [u]
      sFN[(1 * 4 * NFP + row) * E + e] = u1p - u1m;
      sFN[(2 * 4 * NFP + row) * E + e] = u2p - u2m;
      sFN[(3 * 4 * NFP + row) * E + e] = u3p - u3m;
    } else {  // [p], {u}, [u]
      sFN[(1 * 4 * NFP + row) * E + e] = T(0.5) * (u1p + u1m);
      sFN[(2 * 4 * NFP + row) * E + e] = T(0.5) * (u2p + u2m);
      sFN[(3 * 4 * NFP + row) * E + e] = T(0.5) * (u3p + u3m);
      sFN[(4 * 4 * NFP + row) * E + e] = u1p - u1m;
      sFN[(5 * 4 * NFP + row) * E + e] = u2p - u2m;
      sFN[(6 * 4 * NFP + row) * E + e] = u3p - u3m;
    }
  }
  __syncthreads();

  // ---- 2b. interpolate the combinations to the face points ----
  {
    constexpr int RG = FQP / 4;
    const T* Vtri = STRONG ? p.sops.VtriT : ops.VtriT;
    for (int it = tid; it < NCMB * 4 * RG * NG; it += NT) {
      const int g = it % NG;
      const int m0 = ((it / NG) % RG) * 4;
      const int job = it / (RG * NG);  // combo * 4 + face
      T acc[4][4];
      tile_dot<T, E, 4, FQP, NFP>(Vtri, sFN + job * NFP * E + g * 4, m0, acc);
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (m0 + r < FQ) sts_cols(sFQ + (job * FQ + m0 + r) * E + g * 4, acc[r]);
    }
  }
  __syncthreads();

  // ---- 2c. fluxes (Sec. 4.1) ----
  for (int it = tid; it < 4 * FQ * E; it += NT) {
    const int qf = it % (4 * FQ);
    const int e = it / (4 * FQ);
    int64_t c = col0 + e;
    c = c < ncols ? c : ncols - 1;
    const int64_t k = c / S;
    const T* fg = (SFULL ? p.sfgeo : p.fgeo) + k * 3 * 4 * FQ + qf;
    const T nx = __ldg(fg), ny = __ldg(fg + 4 * FQ), nz = __ldg(fg + 8 * FQ);
    const T Jf = sqrt(nx * nx + ny * ny + nz * nz);
    const T jp = sFQ[(0 * 4 * FQ + qf) * E + e];
    if constexpr (STRONG) {
      // F_p = -1/2 ([u].n J^f - tau_p [p] J^f), F_u = -1/2 ([p] - tau_u [u].n) n J^f
      const T j1 = sFQ[(1 * 4 * FQ + qf) * E + e];
      const T j2 = sFQ[(2 * 4 * FQ + qf) * E + e];
      const T j3 = sFQ[(3 * 4 * FQ + qf) * E + e];
      const T junJ = j1 * nx + j2 * ny + j3 * nz;
      const T s = T(0.5) * (-jp + p.tau_u * junJ / Jf);
      sFQ[(0 * 4 * FQ + qf) * E + e] = T(-0.5) * junJ + T(0.5) * p.tau_p * jp * Jf;
      sFQ[(1 * 4 * FQ + qf) * E + e] = s * nx;
      sFQ[(2 * 4 * FQ + qf) * E + e] = s * ny;
      sFQ[(3 * 4 * FQ + qf) * E + e] = s * nz;
    } else {
      // F_p = -1/2 (2 {u}.n J^f - tau_p [p] J^f), F_u = -1/2 ([p] - tau_u [u].n) n J^f
      const T a1 = sFQ[(1 * 4 * FQ + qf) * E + e];
      const T a2 = sFQ[(2 * 4 * FQ + qf) * E + e];
      const T a3 = sFQ[(3 * 4 * FQ + qf) * E + e];
      const T j1 = sFQ[(4 * 4 * FQ + qf) * E + e];
      const T j2 = sFQ[(5 * 4 * FQ + qf) * E + e];
      const T j3 = sFQ[(6 * 4 * FQ + qf) * E + e];
      const T aun = a1 * nx + a2 * ny + a3 * nz;
      const T jun = (j1 * nx + j2 * ny + j3 * nz) / Jf;
      // central terms change sign in the transpose; penalty terms do not
      const T cs = ADJ ? T(1) : T(-1);
      const T s = T(0.5) * (cs * jp + p.tau_u * jun);
      sFQ[(0 * 4 * FQ + qf) * E + e] = cs * aun + T(0.5) * p.tau_p * jp * Jf;
      sFQ[(1 * 4 * FQ + qf) * E + e] = s * nx;
      sFQ[(2 * 4 * FQ + qf) * E + e] = s * ny;
      sFQ[(3 * 4 * FQ + qf) * E + e] = s * nz;
    }
  }
  __syncthreads();

  // ---- 2d. V_tri^T diag(w_f): back to face nodes ----
  {
    constexpr int RG = NFPP / 2;
    for (int it = tid; it < 16 * RG * NG; it += NT) {
      const int g = it % NG;
      const int m0 = ((it / NG) % RG) * 2;
      const int job = it / (RG * NG);  // field * 4 + face
      T acc[2][4];
      tile_dot<T, E, 2, NFPP, FQ>(STRONG ? p.sops.VtriTwT : ops.VtriTwT, sFQ + job * FQ * E + g * 4, m0, acc);
#pragma unroll
      for (int r = 0; r < 2; ++r)
        if (m0 + r < NFP) sts_cols(sFN + (job * NFP + m0 + r) * E + g * 4, acc[r]);
    }
  }
  __syncthreads();

  // ---- 2e. scatter to volume nodes, pressure partials, point source ----
  for (int it = tid; it < 4 * NP * E; it += NT) {
    const int n = it % NP;
    const int e = (it / NP) % E;
    const int fld = it / (NP * E);
    int64_t c = col0 + e;
    c = c < ncols ? c : ncols - 1;
    const int64_t k = c / S;
    T acc = sR[(fld * NP + n) * E + e];
    if (!STRONG && fld == 0) acc += sP[n * E + e] + sP[(NP + n) * E + e];
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
  if (ADJ) {
    // ---- adjoint epilogue: A^T beta is complete in sR ----
    __syncthreads();
    for (int it = tid; it < 4 * NP * E; it += NT) {
      const int n = it % NP;
      const int e = (it / NP) % E;
      const int fld = it / (NP * E);
      const int64_t c = col0 + e;
      if (c >= ncols) continue;
      const int64_t idx = fld * fs + c * NP + n;
      const T a = sR[(fld * NP + n) * E + e];
      if (MODE == kAdjLsrk) p.Qout[idx] += p.dt * a;
      else p.out[idx] = a;
    }
    return;
  }
  __syncthreads();

  // ---- 3a. update: W (V_q M^^{-1}) b at quadrature points ----
  {
    constexpr int RG = NQP / 4;
    for (int it = tid; it < 4 * RG * NG; it += NT) {
      const int g = it % NG;
      const int m0 = ((it / NG) % RG) * 4;
      const int fld = it / (RG * NG);
      T acc[4][4];
      tile_dot<T, E, 4, NQP, NP>(ops.VtT, sR + fld * NP * E + g * 4, m0, acc);
      const int wc = fld == 0 ? 9 : 10;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int64_t c = col0 + g * 4 + e;
        c = c < ncols ? c : ncols - 1;
        const T* w = p.vgeo + ((c / S) * 11 + wc) * NQ;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (m0 + r < NQ) sX[(fld * NQ + m0 + r) * E + g * 4 + e] = acc[r][e] * __ldg(w + m0 + r);
        if (MODE == kRecord && fld == 0 && col0 + g * 4 + e < ncols) {
          const T* wj = p.vgeo + ((c / S) * 11 + 10) * NQ;  // 1/J
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (m0 + r < NQ) p.yrec[c * NQ + m0 + r] = acc[r][e] * __ldg(wj + m0 + r);
        }
      }
    }
  }
  __syncthreads();

  // ---- 3b. update: P_q back to nodes, then the epilogue ----
  {
    constexpr int RG = NPP / 2;
    for (int it = tid; it < 4 * RG * NG; it += NT) {
      const int g = it % NG;
      const int m0 = ((it / NG) % RG) * 2;
      const int fld = it / (RG * NG);
      T acc[2][4];
      tile_dot<T, E, 2, NPP, NQ>(ops.PqT, sX + fld * NQ * E + g * 4, m0, acc);
      if (RHS_OUT) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t c = col0 + g * 4 + e;
          if (c >= ncols) continue;
#pragma unroll
          for (int r = 0; r < 2; ++r)
            if (m0 + r < NP) p.out[fld * fs + c * NP + m0 + r] = acc[r][e];
        }
      } else {
        // The first stage (a_1 = 0) does not read the incoming residual.  Each
        // res element is read once and then written by this thread only: its
        // eight values are loaded (read-only path) before any store.
        const bool rd = p.rk_a != T(0);
        T rs[2][4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int64_t c = col0 + g * 4 + e;
            rs[r][e] = rd && c < ncols && m0 + r < NP ? __ldg(p.res + fld * fs + c * NP + m0 + r) : T(0);
          }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t c = col0 + g * 4 + e;
          if (c >= ncols) continue;
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int m = m0 + r;
            if (m >= NP) continue;
            const int64_t idx = fld * fs + c * NP + m;
            const T rr = rd ? p.rk_a * rs[r][e] + p.dt * acc[r][e] : p.dt * acc[r][e];
            p.res[idx] = rr;
            const T qi = sQ[(fld * NP + m) * E + g * 4 + e];
            if (p.qlo) {  // compensated sum (Fast2Sum, |Q| >= |b res + carried error|)
              const T y = p.rk_b * rr + p.qlo[idx];
              const T q = qi + y;
              p.qlo[idx] = (qi - q) + y;
              p.Qout[idx] = q;
            } else {
              p.Qout[idx] = qi + p.rk_b * rr;
            }
          }
        }
      }
    }
  }
}

template <typename T, int N, int E, int MODE, int NQX>
__global__ void __launch_bounds__(kStageThreads) stage_kernel(const StageParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_tile<T, N, E, MODE, NQX>(p, blockIdx.x, smem_raw);
}

template <typename T, int N, int MODE, int NQX = (N + 1) * (N + 1) * (N + 1)>
cudaError_t launch_stage_mode(const StageParams<T>& p, cudaStream_t stream) {
  constexpr int PER = mode_per_col<N, MODE, NQX>();
  constexpr int E = cols_for<T, N, PER>();
  const size_t smem = (size_t)PER * E * sizeof(T);
  const int64_t blocks = (p.ncols + E - 1) / E;
  if (blocks == 0) return cudaSuccess;
  auto kern = stage_kernel<T, N, E, MODE, NQX>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<(unsigned)blocks, kStageThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t launch_stage_n(const StageParams<T>& p, int mode, cudaStream_t stream) {
  if (p.nq != Dims<N>::NQ) {
    // a fewer-point volume rule: the RHS and LSRK stages
    if constexpr (fewer_point_nq(N) > 0) {
      if (p.nq == fewer_point_nq(N)) {
        if (mode == kRhs) return launch_stage_mode<T, N, kRhs, fewer_point_nq(N)>(p, stream);
        if (mode == kLsrk) return launch_stage_mode<T, N, kLsrk, fewer_point_nq(N)>(p, stream);
      }
    }
    return cudaErrorInvalidValue;
  }
  switch (mode) {
    case kRhs: return launch_stage_mode<T, N, kRhs>(p, stream);
    case kLsrk: return launch_stage_mode<T, N, kLsrk>(p, stream);
    case kRecord: return launch_stage_mode<T, N, kRecord>(p, stream);
    case kAdjLsrk: return launch_stage_mode<T, N, kAdjLsrk>(p, stream);
    case kAdjRhs: return launch_stage_mode<T, N, kAdjRhs>(p, stream);
    case kRhsStrong:
      if constexpr (N <= 5) return launch_stage_mode<T, N, kRhsStrong>(p, stream);
      return cudaErrorInvalidValue;
    case kLsrkStrong:
      if constexpr (N <= 5) return launch_stage_mode<T, N, kLsrkStrong>(p, stream);
      return cudaErrorInvalidValue;
    case kRhsStrongU:
      if constexpr (N <= 5) return launch_stage_mode<T, N, kRhsStrongU>(p, stream);
      return cudaErrorInvalidValue;
    case kLsrkStrongU:
      if constexpr (N <= 5) return launch_stage_mode<T, N, kLsrkStrongU>(p, stream);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wadg
