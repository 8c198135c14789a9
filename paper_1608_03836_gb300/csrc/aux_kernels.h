// Launchers of the FP64 set-up and diagnostic kernels (aux_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wadg {

cudaError_t launch_geo_volume(int64_t K, int Np, int Nq, const double* X, const double* Vq, const double* Vqa, double* J,
                              double* G, double* xq, int* nbad, cudaStream_t st);
cudaError_t launch_geo_face(int64_t K, int Np, int Nfq, const double* X, const double* Vfa, const uint8_t* owner,
                            const int32_t* EToE, const int32_t* EToF, double* nJ, cudaStream_t st);
// Wpu (nullable): update weights [K][2][Nq] (pressure, velocity) replacing
// c^2/J and 1/J (the locally conservative weights of launch_geo_conservative).
template <typename T>
cudaError_t launch_geo_pack(int64_t K, int Nq, int Nfq, const double* J, const double* G, const double* c2,
                            const double* Wpu, const double* nJ, T* vgeo, T* fgeo, cudaStream_t st);
cudaError_t launch_geo_pack_il(int64_t K, int Nq, int Nfq, const double* J, const double* G, const double* c2,
                               const double* Wpu, const double* nJ, float* vgeo_il, float* fgeo_il, cudaStream_t st);
// Wpu [K][2][Nq] = 1 / Pi_N(J/c^2), 1 / Pi_N(J) at the volume points; nbad
// counts points where a projected weight is not positive.
cudaError_t launch_geo_conservative(int64_t K, int Np, int Nq, const double* J, const double* c2, const double* Vq,
                                    const double* Pq, double* Wpu, int* nbad, cudaStream_t st);
// out[i] = (T) in[i], i < n.
template <typename T>
cudaError_t launch_to_precision(int64_t n, const double* in, T* out, cudaStream_t st);
// out[i] = v, i < n.
cudaError_t launch_fill(int64_t n, double v, double* out, cudaStream_t st);
// Constant G [K][9][Nq] and n J^f [K][12][Nfq] of affine elements, compact and
// interleaved over 128 elements: gP [Kt][9][128], nP [Kt][12][128].
cudaError_t launch_geo_planar_pack(int64_t K, int Nq, int Nfq, const double* G, const double* nJ, float* gP, float* nP,
                                   cudaStream_t st);
template <typename T>
cudaError_t launch_project(int64_t ncols, int S, int Np, int Nq, const double* fq, const double* J, const double* Vq,
                           const double* Pq, T* Q, cudaStream_t st);
// mode 0: energy, mode 1: squared L2 error; partial has ncols doubles, out one.
template <typename T>
cudaError_t launch_reduce(int mode, int64_t ncols, int S, int Np, int Nq, const T* Q, const double* Vq, const double* wq,
                          const double* J, const double* c2, const double* exact, int mask, double* partial, double* out,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_receivers(int64_t ncols, int S, int R, int Np, const T* Q, const int32_t* rec_col, const T* rec_vec,
                             T* out, cudaStream_t st);

template <typename T>
cudaError_t launch_receivers_adjoint(int S, int R, int Np, const T* w, const int32_t* rec_col, const T* rec_vec, T* lamQ,
                                     cudaStream_t st);

}  // namespace wadg
