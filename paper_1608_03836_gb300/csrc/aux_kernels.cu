// FP64 set-up and diagnostic kernels: geometric factors of the isoparametric
// map, the weight-adjusted pseudo-projection, the energy and L2 error
// reductions, and the receiver samples.
#include <cstdint>

#include "aux_kernels.h"

namespace wadg {

// ---------------------------------------------------------------------------
// Volume geometric factors (Sec. 4.1): with A_a = dx/dx^_a,
//   J = A_0 . (A_1 x A_2),  G_a = A_b x A_c for cyclic (a,b,c),
// so that G_ai = J dx^_a/dx_i; G and J are polynomial for an isoparametric
// map.  One block per element, threads over quadrature points.
// ---------------------------------------------------------------------------
__global__ void geo_volume_kernel(int64_t K, int Np, int Nq, const double* __restrict__ X,
                                  const double* __restrict__ Vq, const double* __restrict__ Vqa,
                                  double* __restrict__ J, double* __restrict__ G, double* __restrict__ xq,
                                  int* __restrict__ nbad) {
  extern __shared__ double sXk[];  // [Np][3]
  const int64_t k = blockIdx.x;
  for (int i = threadIdx.x; i < 3 * Np; i += blockDim.x) sXk[i] = X[k * 3 * Np + i];
  __syncthreads();
  for (int q = threadIdx.x; q < Nq; q += blockDim.x) {
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // A[a][i]
    double x[3] = {0, 0, 0};
    for (int n = 0; n < Np; ++n) {
      const double v = Vq[q * Np + n];
      const double d0 = Vqa[(0 * Nq + q) * Np + n];
      const double d1 = Vqa[(1 * Nq + q) * Np + n];
      const double d2 = Vqa[(2 * Nq + q) * Np + n];
      for (int i = 0; i < 3; ++i) {
        const double xi = sXk[n * 3 + i];
        x[i] += v * xi;
        A[0][i] += d0 * xi;
        A[1][i] += d1 * xi;
        A[2][i] += d2 * xi;
      }
    }
    double Gm[3][3];
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, c = (a + 2) % 3;
      Gm[a][0] = A[b][1] * A[c][2] - A[b][2] * A[c][1];
      Gm[a][1] = A[b][2] * A[c][0] - A[b][0] * A[c][2];
      Gm[a][2] = A[b][0] * A[c][1] - A[b][1] * A[c][0];
    }
    const double Jq = A[0][0] * Gm[0][0] + A[0][1] * Gm[0][1] + A[0][2] * Gm[0][2];
    J[k * Nq + q] = Jq;
    if (!(Jq > 0.0)) atomicAdd(nbad, 1);
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < 3; ++i) G[(k * 9 + a * 3 + i) * Nq + q] = Gm[a][i];
    for (int i = 0; i < 3; ++i) xq[(k * Nq + q) * 3 + i] = x[i];
  }
}

// Face normals times surface Jacobian at the owner's face points, by
// Nanson's formula n J^f = sum_a G_ai (n^ |f^|)_a.  Owner faces only.
__global__ void geo_face_owner_kernel(int64_t K, int Np, int Nfq, const double* __restrict__ X,
                                      const double* __restrict__ Vfa, const uint8_t* __restrict__ owner,
                                      double* __restrict__ nJ) {
  extern __shared__ double sXk[];
  const int64_t k = blockIdx.x;
  for (int i = threadIdx.x; i < 3 * Np; i += blockDim.x) sXk[i] = X[k * 3 * Np + i];
  __syncthreads();
  const double nref[4][3] = {{0, 0, -1}, {0, -1, 0}, {1, 1, 1}, {-1, 0, 0}};
  for (int it = threadIdx.x; it < 4 * Nfq; it += blockDim.x) {
    const int f = it / Nfq, q = it % Nfq;
    if (!owner[k * 4 + f]) continue;
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int n = 0; n < Np; ++n)
      for (int a = 0; a < 3; ++a) {
        const double d = Vfa[((f * 3 + a) * Nfq + q) * Np + n];
        for (int i = 0; i < 3; ++i) A[a][i] += d * sXk[n * 3 + i];
      }
    double out[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, c = (a + 2) % 3;
      const double g0 = A[b][1] * A[c][2] - A[b][2] * A[c][1];
      const double g1 = A[b][2] * A[c][0] - A[b][0] * A[c][2];
      const double g2 = A[b][0] * A[c][1] - A[b][1] * A[c][0];
      out[0] += g0 * nref[f][a];
      out[1] += g1 * nref[f][a];
      out[2] += g2 * nref[f][a];
    }
    for (int i = 0; i < 3; ++i) nJ[(k * 3 + i) * 4 * Nfq + f * Nfq + q] = out[i];
  }
}

// Non-owner faces take the owner's values with the sign flipped: both sides
// use the same physical points in the same (owner) order.
__global__ void geo_face_copy_kernel(int64_t K, int Nfq, const int32_t* __restrict__ EToE,
                                     const int32_t* __restrict__ EToF, const uint8_t* __restrict__ owner,
                                     double* __restrict__ nJ) {
  const int64_t total = K * 4 * Nfq;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(it % Nfq);
    const int f = (int)((it / Nfq) % 4);
    const int64_t k = it / (4 * Nfq);
    if (owner[k * 4 + f]) continue;
    const int64_t ko = EToE[k * 4 + f];
    const int fo = EToF[k * 4 + f];
    for (int i = 0; i < 3; ++i) nJ[(k * 3 + i) * 4 * Nfq + f * Nfq + q] = -nJ[(ko * 3 + i) * 4 * Nfq + fo * Nfq + q];
  }
}

template <typename T>
__global__ void geo_pack_kernel(int64_t K, int Nq, int Nfq, const double* __restrict__ J, const double* __restrict__ G,
                                const double* __restrict__ c2, const double* __restrict__ Wpu, const double* __restrict__ nJ,
                                T* __restrict__ vgeo, T* __restrict__ fgeo) {
  const int64_t nv = K * Nq, nf = K * 3 * 4 * Nfq;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nv + nf; it += (int64_t)gridDim.x * blockDim.x) {
    if (it < nv) {
      const int64_t k = it / Nq;
      const int q = (int)(it % Nq);
      const double Jq = J[it];
      for (int c = 0; c < 9; ++c) vgeo[(k * 11 + c) * Nq + q] = (T)G[(k * 9 + c) * Nq + q];
      vgeo[(k * 11 + 9) * Nq + q] = (T)(Wpu ? Wpu[(k * 2) * Nq + q] : (c2 ? c2[it] : 1.0) / Jq);
      vgeo[(k * 11 + 10) * Nq + q] = (T)(Wpu ? Wpu[(k * 2 + 1) * Nq + q] : 1.0 / Jq);
    } else {
      const int64_t j = it - nv;
      fgeo[j] = (T)nJ[j];
    }
  }
}

// Column-interleaved FP32 copies for the tensor-core stage, where one thread
// owns one element, a warp owns 32 consecutive elements and a thread reads
// four consecutive points at once (one 16-byte load):
//   vgeo_il[k/128][c][q/4][k % 128][q % 4]           (c < 11, q < 4 ceil(Nq/4)),
//   fgeo_il[k/128][d * 4 + face][q/4][k % 128][q % 4] (q < 4 ceil(Nfq/4)),
// zero in the padding (points beyond Nq or Nfq, elements beyond K).
__global__ void geo_pack_il_kernel(int64_t K, int Nq, int Nfq, const double* __restrict__ J, const double* __restrict__ G,
                                   const double* __restrict__ c2, const double* __restrict__ Wpu,
                                   const double* __restrict__ nJ, float* __restrict__ vgeo, float* __restrict__ fgeo) {
  const int nq4 = (Nq + 3) / 4, nf4 = (Nfq + 3) / 4;
  const int64_t Kt = (K + 127) / 128;
  const int64_t nv = Kt * 11 * nq4 * 512, nf = Kt * 12 * nf4 * 512;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nv + nf; it += (int64_t)gridDim.x * blockDim.x) {
    // it = (((kt * rows + row) * groups + g) * 128 + kl) * 4 + e
    const bool vol = it < nv;
    const int64_t j = vol ? it : it - nv;
    const int e = (int)(j & 3), kl = (int)((j >> 2) & 127);
    const int64_t rest = j >> 9;
    const int groups = vol ? nq4 : nf4, rows = vol ? 11 : 12;
    const int g = (int)(rest % groups);
    const int row = (int)((rest / groups) % rows);
    const int64_t kt = rest / groups / rows;
    const int64_t k = kt * 128 + kl;
    const int q = 4 * g + e;
    float v = 0.f;  // padding: elements beyond K, points beyond Nq / Nfq
    if (vol) {
      if (k < K && q < Nq) {
        const double Jq = J[k * Nq + q];
        if (row < 9) v = (float)G[(k * 9 + row) * Nq + q];
        else if (Wpu) v = (float)Wpu[(k * 2 + (row - 9)) * Nq + q];
        else if (row == 9) v = (float)((c2 ? c2[k * Nq + q] : 1.0) / Jq);
        else v = (float)(1.0 / Jq);
      }
      vgeo[j] = v;
    } else {
      // row = d * 4 + face
      if (k < K && q < Nfq) v = (float)nJ[k * 12 * Nfq + row * Nfq + q];
      fgeo[j] = v;
    }
  }
}

template <typename T>
__global__ void to_precision_kernel(int64_t n, const double* __restrict__ in, T* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)in[i];
}

template <typename T>
cudaError_t launch_to_precision(int64_t n, const double* in, T* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  to_precision_kernel<T><<<2048, 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}
template cudaError_t launch_to_precision<float>(int64_t, const double*, float*, cudaStream_t);
template cudaError_t launch_to_precision<double>(int64_t, const double*, double*, cudaStream_t);

// Compact geometry of affine elements (constant G and n J^f): the values at
// the first volume and face point, interleaved over 128 elements,
// gP[(k >> 7) * 9 + a i][k & 127], nP[(k >> 7) * 12 + d * 4 + f][k & 127].
__global__ void geo_planar_pack_kernel(int64_t K, int Nq, int Nfq, const double* __restrict__ G,
                                       const double* __restrict__ nJ, float* __restrict__ gP, float* __restrict__ nP) {
  const int64_t Kt = (K + 127) / 128;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < Kt * 128 * 21;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int kl = (int)(it & 127);
    const int64_t rest = it >> 7;
    const int row = (int)(rest % 21);
    const int64_t k = (rest / 21) * 128 + kl;
    if (row < 9) gP[((k >> 7) * 9 + row) * 128 + kl] = k < K ? (float)G[(k * 9 + row) * Nq] : 0.f;
    else nP[((k >> 7) * 12 + row - 9) * 128 + kl] = k < K ? (float)nJ[k * 12 * Nfq + (row - 9) * Nfq] : 0.f;
  }
}

cudaError_t launch_geo_planar_pack(int64_t K, int Nq, int Nfq, const double* G, const double* nJ, float* gP, float* nP,
                                   cudaStream_t st) {
  geo_planar_pack_kernel<<<1024, 256, 0, st>>>(K, Nq, Nfq, G, nJ, gP, nP);
  return cudaGetLastError();
}

__global__ void fill_kernel(int64_t n, double v, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}

cudaError_t launch_fill(int64_t n, double v, double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  fill_kernel<<<2048, 256, 0, st>>>(n, v, out);
  return cudaGetLastError();
}

cudaError_t launch_geo_pack_il(int64_t K, int Nq, int Nfq, const double* J, const double* G, const double* c2,
                               const double* Wpu, const double* nJ, float* vgeo_il, float* fgeo_il, cudaStream_t st) {
  geo_pack_il_kernel<<<2048, 256, 0, st>>>(K, Nq, Nfq, J, G, c2, Wpu, nJ, vgeo_il, fgeo_il);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pseudo-projection P_N u = Pi_N(J^{-1} Pi_N(u J)) (Sec. 3, Theorem), with
// Pi_N g = P_q g_q.  One block per column, FP64 arithmetic.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void project_kernel(int64_t ncols, int S, int Np, int Nq, const double* __restrict__ fq,
                               const double* __restrict__ J, const double* __restrict__ Vq, const double* __restrict__ Pq,
                               T* __restrict__ Q) {
  extern __shared__ double sm[];
  double* g = sm;        // [Nq]
  double* c1 = sm + Nq;  // [Np]
  const int64_t c = blockIdx.x;
  const int fld = blockIdx.y;
  const int64_t k = c / S;
  const double* Jk = J + k * Nq;
  for (int q = threadIdx.x; q < Nq; q += blockDim.x) g[q] = fq[(fld * ncols + c) * Nq + q] * Jk[q];
  __syncthreads();
  for (int n = threadIdx.x; n < Np; n += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < Nq; ++q) acc += Pq[n * Nq + q] * g[q];
    c1[n] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < Nq; q += blockDim.x) {
    double acc = 0.0;
    for (int n = 0; n < Np; ++n) acc += Vq[q * Np + n] * c1[n];
    g[q] = acc / Jk[q];
  }
  __syncthreads();
  for (int n = threadIdx.x; n < Np; n += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < Nq; ++q) acc += Pq[n * Nq + q] * g[q];
    Q[(fld * ncols + c) * Np + n] = (T)acc;
  }
}

// ---------------------------------------------------------------------------
// Reductions.  mode 0: energy 1/2 sum w (p^2 J/c^2 + |u|^2 J);
// mode 1: squared L2 error of the fields in mask against exact values.
// One block per column; block partial sums, then a second pass on the host.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void reduce_kernel(int mode, int64_t ncols, int S, int Np, int Nq, const T* __restrict__ Q,
                              const double* __restrict__ Vq, const double* __restrict__ wq, const double* __restrict__ J,
                              const double* __restrict__ c2, const double* __restrict__ exact, int mask,
                              double* __restrict__ partial) {
  extern __shared__ double sm[];
  double* qv = sm;            // [4][Np]
  double* red = sm + 4 * Np;  // [blockDim]
  const int64_t c = blockIdx.x;
  const int64_t k = c / S;
  for (int i = threadIdx.x; i < 4 * Np; i += blockDim.x) {
    const int f = i / Np, n = i % Np;
    qv[i] = (double)Q[(f * ncols + c) * Np + n];
  }
  __syncthreads();
  double acc = 0.0;
  for (int q = threadIdx.x; q < Nq; q += blockDim.x) {
    double v[4];
    for (int f = 0; f < 4; ++f) {
      double s = 0.0;
      for (int n = 0; n < Np; ++n) s += Vq[q * Np + n] * qv[f * Np + n];
      v[f] = s;
    }
    const double wJ = wq[q] * J[k * Nq + q];
    if (mode == 0) {
      const double cc = c2 ? c2[k * Nq + q] : 1.0;
      acc += 0.5 * wJ * (v[0] * v[0] / cc + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
    } else {
      for (int f = 0; f < 4; ++f)
        if (mask & (1 << f)) {
          const double d = v[f] - exact[(f * ncols + c) * Nq + q];
          acc += wJ * d * d;
        }
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[c] = red[0];
}

__global__ void sum_kernel(int64_t n, const double* __restrict__ in, double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += in[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// Receivers: trace[s][r] = sum_n l_n(x^_r) p_n of the receiver's column.
template <typename T>
__global__ void receiver_kernel(int64_t ncols, int S, int R, int Np, const T* __restrict__ Q,
                                const int32_t* __restrict__ rec_col, const T* __restrict__ rec_vec, T* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S * R) return;
  const int64_t c = rec_col[i];
  T acc = 0;
  for (int n = 0; n < Np; ++n) acc += rec_vec[(int64_t)i * Np + n] * Q[c * Np + n];
  out[i] = acc;
}

// Transpose of the receiver samples: lambda_Q[p][col_r][n] += w_r l_n(x^_r).
template <typename T>
__global__ void receiver_adjoint_kernel(int S, int R, int Np, const T* __restrict__ w, const int32_t* __restrict__ rec_col,
                                        const T* __restrict__ rec_vec, T* __restrict__ lamQ) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)S * R * Np) return;
  const int r = (int)(i / Np), n = (int)(i % Np);
  atomicAdd(lamQ + (int64_t)rec_col[r] * Np + n, w[r] * rec_vec[(int64_t)r * Np + n]);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_geo_volume(int64_t K, int Np, int Nq, const double* X, const double* Vq, const double* Vqa, double* J,
                              double* G, double* xq, int* nbad, cudaStream_t st) {
  geo_volume_kernel<<<(unsigned)K, 128, 3 * Np * sizeof(double), st>>>(K, Np, Nq, X, Vq, Vqa, J, G, xq, nbad);
  return cudaGetLastError();
}

cudaError_t launch_geo_face(int64_t K, int Np, int Nfq, const double* X, const double* Vfa, const uint8_t* owner,
                            const int32_t* EToE, const int32_t* EToF, double* nJ, cudaStream_t st) {
  geo_face_owner_kernel<<<(unsigned)K, 128, 3 * Np * sizeof(double), st>>>(K, Np, Nfq, X, Vfa, owner, nJ);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  geo_face_copy_kernel<<<1024, 256, 0, st>>>(K, Nfq, EToE, EToF, owner, nJ);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_geo_pack(int64_t K, int Nq, int Nfq, const double* J, const double* G, const double* c2,
                            const double* Wpu, const double* nJ, T* vgeo, T* fgeo, cudaStream_t st) {
  geo_pack_kernel<T><<<2048, 256, 0, st>>>(K, Nq, Nfq, J, G, c2, Wpu, nJ, vgeo, fgeo);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Locally conservative weights (Sec. 3, the remark after the moment estimate):
// the mass weights w_p = J/c^2 and w_u = J are replaced by their projections
// onto P^N within the weight-adjusted inner product, Pi_N w = V_q P_q w_q, and
// the update uses W = 1 / Pi_N w at the volume points.  Wpu [K][2][Nq]
// (pressure, velocity).  One block per element, FP64.
// ---------------------------------------------------------------------------
__global__ void geo_conservative_kernel(int64_t K, int Np, int Nq, const double* __restrict__ J,
                                        const double* __restrict__ c2, const double* __restrict__ Vq,
                                        const double* __restrict__ Pq, double* __restrict__ Wpu,
                                        int* __restrict__ nbad) {
  extern __shared__ double sw[];
  double* f = sw;            // [Nq]
  double* coef = sw + Nq;    // [Np]
  const int64_t k = blockIdx.x;
  for (int kind = 0; kind < 2; ++kind) {
    for (int q = threadIdx.x; q < Nq; q += blockDim.x)
      f[q] = J[k * Nq + q] / (kind == 0 && c2 ? c2[k * Nq + q] : 1.0);
    __syncthreads();
    for (int n = threadIdx.x; n < Np; n += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < Nq; ++q) acc += Pq[n * Nq + q] * f[q];
      coef[n] = acc;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < Nq; q += blockDim.x) {
      double g = 0.0;
      for (int n = 0; n < Np; ++n) g += Vq[q * Np + n] * coef[n];
      if (!(g > 0.0)) atomicAdd(nbad, 1);
      Wpu[(k * 2 + kind) * Nq + q] = 1.0 / g;
    }
    __syncthreads();
  }
}

cudaError_t launch_geo_conservative(int64_t K, int Np, int Nq, const double* J, const double* c2, const double* Vq,
                                    const double* Pq, double* Wpu, int* nbad, cudaStream_t st) {
  geo_conservative_kernel<<<(unsigned)K, 128, (Nq + Np) * sizeof(double), st>>>(K, Np, Nq, J, c2, Vq, Pq, Wpu, nbad);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project(int64_t ncols, int S, int Np, int Nq, const double* fq, const double* J, const double* Vq,
                           const double* Pq, T* Q, cudaStream_t st) {
  if (ncols == 0) return cudaSuccess;
  dim3 grid((unsigned)ncols, 4);
  project_kernel<T><<<grid, 128, (Nq + Np) * sizeof(double), st>>>(ncols, S, Np, Nq, fq, J, Vq, Pq, Q);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce(int mode, int64_t ncols, int S, int Np, int Nq, const T* Q, const double* Vq, const double* wq,
                          const double* J, const double* c2, const double* exact, int mask, double* partial, double* out,
                          cudaStream_t st) {
  if (ncols == 0) return cudaMemsetAsync(out, 0, sizeof(double), st);
  reduce_kernel<T><<<(unsigned)ncols, 128, (4 * Np + 128) * sizeof(double), st>>>(mode, ncols, S, Np, Nq, Q, Vq, wq, J,
                                                                                   c2, exact, mask, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_kernel<<<1, 256, 0, st>>>(ncols, partial, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_receivers(int64_t ncols, int S, int R, int Np, const T* Q, const int32_t* rec_col, const T* rec_vec,
                             T* out, cudaStream_t st) {
  const int n = S * R;
  if (n == 0) return cudaSuccess;
  receiver_kernel<T><<<(n + 127) / 128, 128, 0, st>>>(ncols, S, R, Np, Q, rec_col, rec_vec, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_receivers_adjoint(int S, int R, int Np, const T* w, const int32_t* rec_col, const T* rec_vec, T* lamQ,
                                     cudaStream_t st) {
  const int64_t n = (int64_t)S * R * Np;
  if (n == 0) return cudaSuccess;
  receiver_adjoint_kernel<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(S, R, Np, w, rec_col, rec_vec, lamQ);
  return cudaGetLastError();
}

template cudaError_t launch_receivers_adjoint<double>(int, int, int, const double*, const int32_t*, const double*,
                                                      double*, cudaStream_t);
template cudaError_t launch_receivers_adjoint<float>(int, int, int, const float*, const int32_t*, const float*, float*,
                                                     cudaStream_t);
template cudaError_t launch_geo_pack<double>(int64_t, int, int, const double*, const double*, const double*,
                                             const double*, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_geo_pack<float>(int64_t, int, int, const double*, const double*, const double*,
                                            const double*, const double*, float*, float*, cudaStream_t);
template cudaError_t launch_project<double>(int64_t, int, int, int, const double*, const double*, const double*,
                                            const double*, double*, cudaStream_t);
template cudaError_t launch_project<float>(int64_t, int, int, int, const double*, const double*, const double*,
                                           const double*, float*, cudaStream_t);
template cudaError_t launch_reduce<double>(int, int64_t, int, int, int, const double*, const double*, const double*,
                                           const double*, const double*, const double*, int, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_reduce<float>(int, int64_t, int, int, int, const float*, const double*, const double*,
                                          const double*, const double*, const double*, int, double*, double*,
                                          cudaStream_t);
template cudaError_t launch_receivers<double>(int64_t, int, int, int, const double*, const int32_t*, const double*,
                                              double*, cudaStream_t);
template cudaError_t launch_receivers<float>(int64_t, int, int, int, const float*, const int32_t*, const float*, float*,
                                             cudaStream_t);

}  // namespace wadg
