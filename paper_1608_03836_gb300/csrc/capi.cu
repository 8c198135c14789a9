// C ABI of the WADG library (see include/wadg.h).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "aux_kernels.h"
#include "wadg_internal.h"

namespace wadg {

template <typename T, int N>
cudaError_t launch_stage_n(const StageParams<T>& p, int mode, cudaStream_t stream);

template <typename T>
cudaError_t launch_stage(int N, const StageParams<T>& p, int mode, cudaStream_t stream) {
  switch (N) {
    case 1: return launch_stage_n<T, 1>(p, mode, stream);
    case 2: return launch_stage_n<T, 2>(p, mode, stream);
    case 3: return launch_stage_n<T, 3>(p, mode, stream);
    case 4: return launch_stage_n<T, 4>(p, mode, stream);
    case 5: return launch_stage_n<T, 5>(p, mode, stream);
    case 6: return launch_stage_n<T, 6>(p, mode, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int N>
cudaError_t launch_adj_update_n(const AdjUpdateParams<T>& p, int lsrk, cudaStream_t stream);

template <typename T>
cudaError_t launch_adj_update(int N, const AdjUpdateParams<T>& p, int lsrk, cudaStream_t stream) {
  switch (N) {
    case 1: return launch_adj_update_n<T, 1>(p, lsrk, stream);
    case 2: return launch_adj_update_n<T, 2>(p, lsrk, stream);
    case 3: return launch_adj_update_n<T, 3>(p, lsrk, stream);
    case 4: return launch_adj_update_n<T, 4>(p, lsrk, stream);
    case 5: return launch_adj_update_n<T, 5>(p, lsrk, stream);
    case 6: return launch_adj_update_n<T, 6>(p, lsrk, stream);
    default: return cudaErrorInvalidValue;
  }
}

static const int kFaceV[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

}  // namespace wadg

using namespace wadg;

namespace {

int fail(wadg_mesh* m, int status, const char* fmt, ...) {
  if (m) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    m->last_error = buf;
  }
  return status;
}

int cuda_fail(wadg_mesh* m, cudaError_t e, const char* where) {
  return fail(m, e == cudaErrorMemoryAllocation ? WADG_ENOMEM : WADG_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define WADG_CUDA(m, call)                                  \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return cuda_fail((m), _e, #call); \
  } while (0)

// Runs a body with the mesh's device current, restoring the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = (cudaSetDevice(dev) == cudaSuccess);
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

size_t tsize(int precision) { return precision == WADG_FP64 ? sizeof(double) : sizeof(float); }

// Upload the k-major operator tables in precision T.
template <typename T>
int upload_ops(wadg_mesh* m, DevOps<T>& ops) {
  const RefOps& o = m->ref;
  const int Np = o.Np, Nq = o.Nq, Nfp = o.Nfp, Nfq = o.Nfq;
  std::vector<T> h;
  auto push = [&](size_t n) {
    size_t off = h.size();
    h.resize(off + ((n + 31) / 32) * 32, T(0));
    return off;
  };
  // Row counts padded to a multiple of 4 so that 4 rows load as one vector.
  auto pad4 = [](int n) { return (n + 3) / 4 * 4; };
  const int NQP = pad4(Nq), NPP = pad4(Np), NFQP = pad4(Nfq), NFPP = pad4(Nfp);
  size_t oVq = push((size_t)Np * NQP), oVa = push(3 * (size_t)Np * NQP), oDw = push(3 * (size_t)Nq * NPP),
         oVw = push((size_t)Nq * NPP), oVt = push((size_t)Np * NQP), oPq = push((size_t)Nq * NPP),
         oVtri = push((size_t)Nfp * NFQP), oVtriTw = push((size_t)Nfq * NFPP), oPqTT = push((size_t)Np * NQP),
         oVtTT = push((size_t)Nq * NPP);
  for (int n = 0; n < Np; ++n)
    for (int q = 0; q < Nq; ++q) {
      h[oVq + n * NQP + q] = (T)o.Vq[q * Np + n];
      for (int a = 0; a < 3; ++a) h[oVa + (a * Np + n) * NQP + q] = (T)o.Vqa[(a * Nq + q) * Np + n];
      for (int a = 0; a < 3; ++a) h[oDw + (a * Nq + q) * NPP + n] = (T)o.Dw[(a * Np + n) * Nq + q];
      h[oVw + q * NPP + n] = (T)o.Vw[n * Nq + q];
      h[oVt + n * NQP + q] = (T)o.Vtilde[q * Np + n];
      h[oPq + q * NPP + n] = (T)o.Pq[n * Nq + q];
      h[oPqTT + n * NQP + q] = (T)o.Pq[n * Nq + q];      // P_q^T: rows q, k = n
      h[oVtTT + q * NPP + n] = (T)o.Vtilde[q * Np + n];  // (V_q M^-1)^T: rows n, k = q
    }
  for (int j = 0; j < Nfp; ++j)
    for (int q = 0; q < Nfq; ++q) {
      h[oVtri + j * NFQP + q] = (T)o.Vtri[q * Nfp + j];
      h[oVtriTw + q * NFPP + j] = (T)o.VtriTw[j * Nfq + q];
    }
  std::vector<int16_t> hi(4 * 6 * Nfp + 4 * 6 * Np);
  for (int i = 0; i < 4 * 6 * Nfp; ++i) hi[i] = (int16_t)o.gidx[i];
  for (int i = 0; i < 4 * 6 * Np; ++i) hi[4 * 6 * Nfp + i] = (int16_t)o.ginv[i];
  size_t bytes_t = h.size() * sizeof(T);
  size_t bytes = bytes_t + hi.size() * sizeof(int16_t);
  void* base = nullptr;
  WADG_CUDA(m, cudaMalloc(&base, bytes));
  WADG_CUDA(m, cudaMemcpy(base, h.data(), bytes_t, cudaMemcpyHostToDevice));
  WADG_CUDA(m, cudaMemcpy((char*)base + bytes_t, hi.data(), hi.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
  T* b = (T*)base;
  ops.base = base;
  ops.VqT = b + oVq;
  ops.VaT = b + oVa;
  ops.DwT = b + oDw;
  ops.VwT = b + oVw;
  ops.VtT = b + oVt;
  ops.PqT = b + oPq;
  ops.VtriT = b + oVtri;
  ops.VtriTwT = b + oVtriTw;
  ops.PqTT = b + oPqTT;
  ops.VtTT = b + oVtTT;
  ops.gidx = (const int16_t*)((char*)base + bytes_t);
  ops.ginv = ops.gidx + 4 * 6 * Nfp;
  return WADG_OK;
}

// The update weights of the locally conservative variant (m->d_Wpu), or
// nothing for the pointwise weights; depends on J and c^2.
int conservative_weights(wadg_mesh* m) {
  if (!m->conservative) {
    dfree(m->d_Wpu);
    return WADG_OK;
  }
  const RefOps& o = m->ref;
  const int64_t K = m->K;
  if (!m->d_Wpu) WADG_CUDA(m, cudaMalloc((void**)&m->d_Wpu, (size_t)K * 2 * o.Nq * 8));
  int* d_nbad = nullptr;
  WADG_CUDA(m, cudaMalloc((void**)&d_nbad, sizeof(int)));
  int nbad = 0;
  const double* dVq = m->d_ref64;
  const double* dPq = dVq + 4 * (size_t)o.Nq * o.Np;  // after Vq and the three Vqa
  cudaError_t e = cudaMemset(d_nbad, 0, sizeof(int));
  if (e == cudaSuccess) e = launch_geo_conservative(K, o.Np, o.Nq, m->d_J, m->d_c2, dVq, dPq, m->d_Wpu, d_nbad, 0);
  if (e == cudaSuccess) e = cudaMemcpy(&nbad, d_nbad, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_nbad);
  if (e != cudaSuccess) return cuda_fail(m, e, "conservative weights");
  if (nbad > 0) {
    dfree(m->d_Wpu);
    return fail(m, WADG_EGEOM, "the projection of J or J/c^2 onto P^N is not positive at %d volume points", nbad);
  }
  return WADG_OK;
}

// The mesh uses the collapsed (N+1)^3 volume rule (or another rule of that
// size); the strong forms, the adjoint and batches are built for it only.
bool collapsed_size(const wadg_mesh* m) { return m->ref.Nq == (m->N + 1) * (m->N + 1) * (m->N + 1); }

// Sizes of the strong-form stage tables for a runtime (N, form).
struct StrongSizes {
  int nqs = 0, nfqs = 0, nqsc = 0, nfqsp = 0;
};
template <int N, int F>
StrongSizes strong_sizes_t() {
  using D = StrongDims<N, F>;
  return {D::NQS, D::NFQS, D::NQSC, D::NFQSP};
}
template <int F>
StrongSizes strong_sizes_f(int N) {
  switch (N) {
    case 1: return strong_sizes_t<1, F>();
    case 2: return strong_sizes_t<2, F>();
    case 3: return strong_sizes_t<3, F>();
    case 4: return strong_sizes_t<4, F>();
    case 5: return strong_sizes_t<5, F>();
    default: return StrongSizes();
  }
}
StrongSizes strong_sizes(int N, int form) { return form == 1 ? strong_sizes_f<1>(N) : strong_sizes_f<2>(N); }

void free_strong(wadg_mesh* m) {
  dfree(m->d_sgeo);
  dfree(m->d_sfgeo);
  if (m->sops64.base) cudaFree(m->sops64.base);
  if (m->sops32.base) cudaFree(m->sops32.base);
  m->sops64 = StrongOps<double>();
  m->sops32 = StrongOps<float>();
  m->strong_form = 0;
  m->strong_precision = -1;
}

// Tables of the rules R in precision T, k-major and zero padded to the row
// counts of the strong-form stage (StrongDims).
template <typename T>
int upload_strong_ops(wadg_mesh* m, const RuleOps& R, const StrongSizes& z, StrongOps<T>& so) {
  const int Np = m->ref.Np, Nfp = m->ref.Nfp;
  const int NPP = (Np + 3) / 4 * 4, NFPP = (Nfp + 3) / 4 * 4;
  if (R.Nq != z.nqs || R.Nfq != z.nfqs) return fail(m, WADG_EUNSUPPORTED, "strong-form rule sizes");
  std::vector<T> h;
  auto push = [&](size_t n) {
    size_t off = h.size();
    h.resize(off + ((n + 31) / 32) * 32, T(0));
    return off;
  };
  const size_t oVa = push((size_t)3 * Np * z.nqsc), oVw = push((size_t)z.nqsc * NPP),
               oVtri = push((size_t)Nfp * z.nfqsp), oVtriTw = push((size_t)z.nfqs * NFPP);
  for (int n = 0; n < Np; ++n)
    for (int q = 0; q < R.Nq; ++q) {
      for (int a = 0; a < 3; ++a)
        h[oVa + ((size_t)a * Np + n) * z.nqsc + q] = (T)R.Vqa[((size_t)a * R.Nq + q) * Np + n];
      h[oVw + (size_t)q * NPP + n] = (T)(R.Vq[(size_t)q * Np + n] * R.wq[q]);
    }
  for (int j = 0; j < Nfp; ++j)
    for (int q = 0; q < R.Nfq; ++q) {
      h[oVtri + (size_t)j * z.nfqsp + q] = (T)R.Vtri[(size_t)q * Nfp + j];
      h[oVtriTw + (size_t)q * NFPP + j] = (T)R.VtriTw[(size_t)j * R.Nfq + q];
    }
  void* base = nullptr;
  WADG_CUDA(m, cudaMalloc(&base, h.size() * sizeof(T)));
  cudaError_t e = cudaMemcpy(base, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(base);
    return cuda_fail(m, e, "strong-form tables");
  }
  T* b = (T*)base;
  so.base = base;
  so.VaT = b + oVa;
  so.VwT = b + oVw;
  so.VtriT = b + oVtri;
  so.VtriTwT = b + oVtriTw;
  return WADG_OK;
}

// Geometric factors G_ai at the volume points and n J^f at the (owner) face
// points of the rules R, by the same FP64 kernels as the mesh's own rules,
// stored in precision T as d_sgeo [K][9][Nq_R] and d_sfgeo [K][3][4 Nfq_R].
template <typename T>
int strong_geometry(wadg_mesh* m, const RuleOps& R) {
  const int64_t K = m->K;
  const int Np = m->ref.Np;
  const size_t nVq = R.Vq.size(), nVqa = R.Vqa.size(), nVfa = R.Vfa.size();
  const size_t nG = (size_t)K * 9 * R.Nq, nF = (size_t)K * 12 * R.Nfq;
  std::vector<double> tab(nVq + nVqa + nVfa);
  std::copy(R.Vq.begin(), R.Vq.end(), tab.begin());
  std::copy(R.Vqa.begin(), R.Vqa.end(), tab.begin() + nVq);
  std::copy(R.Vfa.begin(), R.Vfa.end(), tab.begin() + nVq + nVqa);
  std::vector<int32_t> EToF32(m->EToF.begin(), m->EToF.end());
  double *dTab = nullptr, *dJ = nullptr, *dG = nullptr, *dxq = nullptr, *dnJ = nullptr;
  int32_t* dEToF = nullptr;
  int* dbad = nullptr;
  int nbad = 0;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc((void**)&dTab, tab.size() * 8)) != cudaSuccess) break;
    if ((e = cudaMalloc((void**)&dJ, (size_t)K * R.Nq * 8)) != cudaSuccess) break;
    if ((e = cudaMalloc((void**)&dG, nG * 8)) != cudaSuccess) break;
    if ((e = cudaMalloc((void**)&dxq, (size_t)K * R.Nq * 3 * 8)) != cudaSuccess) break;
    if ((e = cudaMalloc((void**)&dnJ, nF * 8)) != cudaSuccess) break;
    if ((e = cudaMalloc((void**)&dEToF, (size_t)K * 4 * 4)) != cudaSuccess) break;
    if ((e = cudaMalloc((void**)&dbad, sizeof(int))) != cudaSuccess) break;
    if ((e = cudaMemcpy(dTab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess) break;
    if ((e = cudaMemcpy(dEToF, EToF32.data(), (size_t)K * 16, cudaMemcpyHostToDevice)) != cudaSuccess) break;
    if ((e = cudaMemset(dbad, 0, sizeof(int))) != cudaSuccess) break;
    if ((e = launch_geo_volume(K, Np, R.Nq, m->d_X, dTab, dTab + nVq, dJ, dG, dxq, dbad, 0)) != cudaSuccess) break;
    if ((e = launch_geo_face(K, Np, R.Nfq, m->d_X, dTab + nVq + nVqa, m->d_owner, m->d_EToE, dEToF, dnJ, 0)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemcpy(&nbad, dbad, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
    if (nbad == 0) {
      if (sizeof(T) == sizeof(double)) {
        m->d_sgeo = dG;
        m->d_sfgeo = dnJ;
        dG = dnJ = nullptr;
      } else {
        if ((e = cudaMalloc(&m->d_sgeo, nG * sizeof(T))) != cudaSuccess) break;
        if ((e = cudaMalloc(&m->d_sfgeo, nF * sizeof(T))) != cudaSuccess) break;
        if ((e = launch_to_precision<T>((int64_t)nG, dG, (T*)m->d_sgeo, 0)) != cudaSuccess) break;
        if ((e = launch_to_precision<T>((int64_t)nF, dnJ, (T*)m->d_sfgeo, 0)) != cudaSuccess) break;
        e = cudaDeviceSynchronize();
      }
    }
  } while (0);
  cudaFree(dTab);
  cudaFree(dJ);
  cudaFree(dG);
  cudaFree(dxq);
  cudaFree(dnJ);
  cudaFree(dEToF);
  cudaFree(dbad);
  if (e != cudaSuccess) return cuda_fail(m, e, "strong-form geometry");
  if (nbad > 0)
    return fail(m, WADG_EGEOM, "J <= 0 at %d points of the strong form's volume rule (%d points per direction)", nbad,
                R.nv);
  return WADG_OK;
}

// Brings the strong-form state to the mesh's formulation and precision: the
// tables of its rules and, for form 1, the geometric factors at their points.
int prepare_strong(wadg_mesh* m) {
  if (m->form == 0 || m->precision < 0) {
    free_strong(m);
    return WADG_OK;
  }
  if (m->strong_form == m->form && m->strong_precision == m->precision) return WADG_OK;
  free_strong(m);
  int nv = 0, nf = 0;
  strong_rule_points(m->N, m->form, &nv, &nf);
  RuleOps R;
  char err[256];
  if (!build_rule_ops(m->ref, nv, nf, R, err, sizeof(err))) return fail(m, WADG_EUNSUPPORTED, "%s", err);
  const StrongSizes z = strong_sizes(m->N, m->form);
  const bool f64 = m->precision == WADG_FP64;
  int st = f64 ? upload_strong_ops<double>(m, R, z, m->sops64) : upload_strong_ops<float>(m, R, z, m->sops32);
  if (st == WADG_OK && m->form == 1) st = f64 ? strong_geometry<double>(m, R) : strong_geometry<float>(m, R);
  if (st != WADG_OK) {
    free_strong(m);
    return st;
  }
  m->strong_form = m->form;
  m->strong_precision = m->precision;
  return WADG_OK;
}

// Locate a physical point: element index and reference coordinates.  Among
// the elements whose node bounding box holds the point, Newton's method on
// x_h(x^) = x; the element where the point is most interior wins.
bool locate(const wadg_mesh* m, const double* x, int64_t& kout, double* rst) {
  const RefOps& o = m->ref;
  const int Np = o.Np;
  double best = -1e300;
  std::vector<double> vals(Np), grads(3 * Np);
  for (int64_t k = 0; k < m->K; ++k) {
    const double* X = &m->geom[(size_t)k * Np * 3];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int n = 0; n < Np; ++n)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], X[n * 3 + d]);
        hi[d] = std::max(hi[d], X[n * 3 + d]);
      }
    bool in = true;
    for (int d = 0; d < 3; ++d) {
      double pad = 0.05 * (hi[d] - lo[d]) + 1e-12;
      if (x[d] < lo[d] - pad || x[d] > hi[d] + pad) in = false;
    }
    if (!in) continue;
    double r[3] = {-0.5, -0.5, -0.5};
    bool ok = false;
    for (int it = 0; it < 50; ++it) {
      lattice_basis(o, 1, &r[0], &r[1], &r[2], vals.data(), grads.data());
      double F[3] = {-x[0], -x[1], -x[2]}, A[3][3] = {{0}};
      for (int n = 0; n < Np; ++n)
        for (int i = 0; i < 3; ++i) {
          F[i] += vals[n] * X[n * 3 + i];
          for (int a = 0; a < 3; ++a) A[i][a] += grads[a * Np + n] * X[n * 3 + i];
        }
      double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                   A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
      if (std::fabs(det) < 1e-300) break;
      double inv[3][3];
      inv[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
      inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
      inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
      inv[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
      inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
      inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
      inv[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
      inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
      inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
      double step = 0.0;
      for (int a = 0; a < 3; ++a) {
        double d = inv[a][0] * F[0] + inv[a][1] * F[1] + inv[a][2] * F[2];
        r[a] -= d;
        step = std::max(step, std::fabs(d));
      }
      if (std::fabs(r[0]) > 10 || std::fabs(r[1]) > 10 || std::fabs(r[2]) > 10) break;
      if (step < 1e-14) {
        ok = true;
        break;
      }
    }
    if (!ok) continue;
    // interior measure: smallest barycentric coordinate
    double lam = std::min(std::min((1 + r[0]) / 2, (1 + r[1]) / 2), std::min((1 + r[2]) / 2, -(1 + r[0] + r[1] + r[2]) / 2));
    if (lam > best && lam > -1e-10) {
      best = lam;
      kout = k;
      rst[0] = r[0];
      rst[1] = r[1];
      rst[2] = r[2];
    }
  }
  return best > -1e-10;
}

template <typename T>
int set_points(wadg_mesh* m, int count, const double* xyz, int64_t* elem_out, std::vector<T>& vec) {
  const int Np = m->ref.Np;
  vec.assign((size_t)count * Np, T(0));
  std::vector<double> vals(Np);
  for (int i = 0; i < count; ++i) {
    int64_t k = -1;
    double rst[3];
    if (!locate(m, xyz + 3 * i, k, rst))
      return fail(m, WADG_EINVAL, "point %d (%g, %g, %g) is not inside the mesh", i, xyz[3 * i], xyz[3 * i + 1],
                  xyz[3 * i + 2]);
    lattice_basis(m->ref, 1, &rst[0], &rst[1], &rst[2], vals.data(), nullptr);
    for (int n = 0; n < Np; ++n) vec[(size_t)i * Np + n] = (T)vals[n];
    elem_out[i] = k;
  }
  return WADG_OK;
}

// The tensor-core stage's mean correction and its tile lists of affine
// elements (defined with the stage launch helpers below).
int mean_correction(wadg_mesh* m);
int planar_tiles(wadg_mesh* m, int shots);

}  // namespace

extern "C" {

int wadg_version(void) { return 100; }

const char* wadg_status_string(int status) {
  switch (status) {
    case WADG_OK: return "ok";
    case WADG_EINVAL: return "invalid argument";
    case WADG_ENOMEM: return "out of memory";
    case WADG_ECUDA: return "CUDA error";
    case WADG_EGEOM: return "invalid geometry";
    case WADG_ESTATE: return "invalid call order";
    case WADG_ETIMEOUT: return "device wait timed out";
    case WADG_EUNSTABLE: return "non-finite energy";
    case WADG_EUNSUPPORTED: return "unsupported order or precision";
    default: return "unknown status";
  }
}

const char* wadg_last_error(const wadg_mesh* m) { return m ? m->last_error.c_str() : ""; }

int wadg_reference_rules(int N, double* rst_q, double* w_q, double* rs_f, double* w_f) {
  RefOps o;
  char err[256];
  if (!build_refops(N, o, err, sizeof(err))) return WADG_EUNSUPPORTED;
  for (int q = 0; q < o.Nq; ++q) {
    if (rst_q) {
      rst_q[3 * q] = o.rq[q];
      rst_q[3 * q + 1] = o.sq[q];
      rst_q[3 * q + 2] = o.tq[q];
    }
    if (w_q) w_q[q] = o.wq[q];
  }
  for (int q = 0; q < o.Nfq; ++q) {
    if (rs_f) {
      rs_f[2 * q] = o.rf[q];
      rs_f[2 * q + 1] = o.sf[q];
    }
    if (w_f) w_f[q] = o.wf[q];
  }
  return WADG_OK;
}

void wadg_mesh_destroy(wadg_mesh* m) {
  if (!m) return;
  DeviceGuard g(m->device);
  dfree(m->d_X);
  dfree(m->d_J);
  dfree(m->d_G);
  dfree(m->d_nJ);
  dfree(m->d_xq);
  dfree(m->d_c2);
  dfree(m->d_EToE);
  dfree(m->d_fcode);
  dfree(m->d_owner);
  dfree(m->d_ref64);
  dfree(m->d_vgeo);
  dfree(m->d_fgeo);
  if (m->ops64.base) cudaFree(m->ops64.base);
  if (m->ops32.base) cudaFree(m->ops32.base);
  free_strong(m);
  dfree(m->d_Wpu);
  dfree(m->d_Qtmp);
  dfree(m->d_red);
  dfree(m->d_tcops);
  dfree(m->d_vgeo_il);
  dfree(m->d_meanc);
  dfree(m->d_Qlo);
  dfree(m->d_tlist);
  dfree(m->d_gP);
  dfree(m->d_nP);
  dfree(m->d_hostQ);
  dfree(m->d_hostR);
  dfree(m->d_fgeo_il);
  dfree(m->d_err);
  dfree(m->d_src_elem);
  dfree(m->d_src_vec);
  dfree(m->d_rec_col);
  dfree(m->d_rec_vec);
  if (m->solve_exec) cudaGraphExecDestroy(m->solve_exec);
  if (m->ev_in) cudaEventDestroy(m->ev_in);
  if (m->ev_out) cudaEventDestroy(m->ev_out);
  if (m->solve_stream) cudaStreamDestroy(m->solve_stream);
  delete m;
}

int wadg_mesh_create(int N, int64_t Nv, const double* VXYZ, int64_t K, const int64_t* EToV, const double* geom_xyz,
                     wadg_mesh** out) {
  return wadg_mesh_create_rule(N, Nv, VXYZ, K, EToV, geom_xyz, 0, nullptr, out);
}

int wadg_mesh_create_rule(int N, int64_t Nv, const double* VXYZ, int64_t K, const int64_t* EToV,
                          const double* geom_xyz, int nq, const double* rule, wadg_mesh** out) {
  if (!out) return WADG_EINVAL;
  *out = nullptr;
  if (N < 1 || N > 6) return WADG_EUNSUPPORTED;
  if (Nv < 4 || K < 1 || K > (int64_t)1 << 30 || !VXYZ || !EToV) return WADG_EINVAL;
  if (rule && nq != (N + 1) * (N + 1) * (N + 1) && nq != fewer_point_nq(N)) return WADG_EUNSUPPORTED;
  wadg_mesh* m = new (std::nothrow) wadg_mesh();
  if (!m) return WADG_ENOMEM;
  char err[256];
  if (!build_refops(N, m->ref, err, sizeof(err), rule ? nq : 0, rule)) {
    delete m;
    return WADG_EUNSUPPORTED;
  }
  cudaGetDevice(&m->device);
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  if (m->num_sms <= 0) m->num_sms = 1;
  m->N = N;
  m->K = K;
  const RefOps& o = m->ref;
  const int Np = o.Np, Nq = o.Nq, Nfq = o.Nfq;

  auto bail = [&](int st) {
    // keep the message for the caller: copy into a static buffer is not
    // possible without a mesh, so the mesh is returned only on success.
    wadg_mesh_destroy(m);
    return st;
  };

  // vertex indices and orientation
  for (int64_t k = 0; k < K; ++k) {
    const int64_t* v = EToV + 4 * k;
    for (int i = 0; i < 4; ++i)
      if (v[i] < 0 || v[i] >= Nv) return bail(WADG_EINVAL);
    double a[3][3];
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) a[i][d] = VXYZ[3 * v[i + 1] + d] - VXYZ[3 * v[0] + d];
    double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                 a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    if (!(det > 0)) return bail(WADG_EGEOM);
  }

  // connectivity: sort faces by their vertex triple
  struct FaceRec {
    int64_t a, b, c;
    int64_t k;
    int f;
  };
  std::vector<FaceRec> faces((size_t)K * 4);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      int64_t v[3] = {EToV[4 * k + kFaceV[f][0]], EToV[4 * k + kFaceV[f][1]], EToV[4 * k + kFaceV[f][2]]};
      std::sort(v, v + 3);
      faces[k * 4 + f] = {v[0], v[1], v[2], k, f};
    }
  std::sort(faces.begin(), faces.end(), [](const FaceRec& x, const FaceRec& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    if (x.c != y.c) return x.c < y.c;
    return x.k < y.k;
  });
  m->EToE.assign(K * 4, -1);
  m->EToF.assign(K * 4, -1);
  for (size_t i = 0; i < faces.size();) {
    size_t j = i + 1;
    while (j < faces.size() && faces[j].a == faces[i].a && faces[j].b == faces[i].b && faces[j].c == faces[i].c) ++j;
    if (j - i > 2) return bail(WADG_EGEOM);
    if (j - i == 2) {
      const FaceRec &x = faces[i], &y = faces[i + 1];
      if (x.k == y.k) return bail(WADG_EGEOM);
      m->EToE[x.k * 4 + x.f] = (int32_t)y.k;
      m->EToF[x.k * 4 + x.f] = y.f;
      m->EToE[y.k * 4 + y.f] = (int32_t)x.k;
      m->EToF[y.k * 4 + y.f] = x.f;
    }
    i = j;
  }
  // owners and permutation codes
  m->fcode.assign(K * 4, 0);
  m->owner.assign(K * 4, 0);
  auto perm_of = [&](int64_t k, int f, int64_t ko, int fo) {
    int64_t mine[3], theirs[3];
    for (int s = 0; s < 3; ++s) {
      mine[s] = EToV[4 * k + kFaceV[f][s]];
      theirs[s] = EToV[4 * ko + kFaceV[fo][s]];
    }
    int sig[3];
    for (int s = 0; s < 3; ++s)
      for (int t = 0; t < 3; ++t)
        if (theirs[t] == mine[s]) sig[s] = t;
    for (int pi = 0; pi < 6; ++pi)
      if (kPerm[pi][0] == sig[0] && kPerm[pi][1] == sig[1] && kPerm[pi][2] == sig[2]) return pi;
    return -1;
  };
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      const int64_t kn = m->EToE[k * 4 + f];
      const int fn = m->EToF[k * 4 + f];
      if (kn < 0) {
        m->owner[k * 4 + f] = 1;
        m->fcode[k * 4 + f] = 0;
        continue;
      }
      const bool own = k < kn;
      m->owner[k * 4 + f] = own ? 1 : 0;
      const int64_t ko = own ? k : kn;
      const int fo = own ? f : fn;
      int pio = perm_of(k, f, ko, fo), pin = perm_of(kn, fn, ko, fo);
      if (pio < 0 || pin < 0) return bail(WADG_EGEOM);
      m->fcode[k * 4 + f] = (uint8_t)(pio + 6 * (pin + 6 * fn));
    }

  // geometry nodes (affine lattice map when none are given)
  m->geom.resize((size_t)K * Np * 3);
  if (geom_xyz) {
    std::memcpy(m->geom.data(), geom_xyz, m->geom.size() * sizeof(double));
  } else {
    for (int64_t k = 0; k < K; ++k)
      for (int n = 0; n < Np; ++n) {
        double l[4] = {-(1 + o.r[n] + o.s[n] + o.t[n]) / 2, (1 + o.r[n]) / 2, (1 + o.s[n]) / 2, (1 + o.t[n]) / 2};
        for (int d = 0; d < 3; ++d) {
          double x = 0;
          for (int v = 0; v < 4; ++v) x += l[v] * VXYZ[3 * EToV[4 * k + v] + d];
          m->geom[((size_t)k * Np + n) * 3 + d] = x;
        }
      }
  }

  // affine elements: geometry nodes equal to the vertices' affine lattice map
  // (to 1e-13 of the element's extent); all of them when no nodes are given
  m->affine.assign((size_t)K, 1);
  m->n_affine = K;
  if (geom_xyz) {
    m->n_affine = 0;
    for (int64_t k = 0; k < K; ++k) {
      double ext = 0, dev = 0;
      for (int d = 0; d < 3; ++d)
        for (int v = 1; v < 4; ++v)
          ext = std::max(ext, std::fabs(VXYZ[3 * EToV[4 * k + v] + d] - VXYZ[3 * EToV[4 * k] + d]));
      for (int n = 0; n < Np; ++n) {
        const double l[4] = {-(1 + o.r[n] + o.s[n] + o.t[n]) / 2, (1 + o.r[n]) / 2, (1 + o.s[n]) / 2, (1 + o.t[n]) / 2};
        for (int d = 0; d < 3; ++d) {
          double x = 0;
          for (int v = 0; v < 4; ++v) x += l[v] * VXYZ[3 * EToV[4 * k + v] + d];
          dev = std::max(dev, std::fabs(x - m->geom[((size_t)k * Np + n) * 3 + d]));
        }
      }
      m->affine[k] = dev <= 1e-13 * ext ? 1 : 0;
      m->n_affine += m->affine[k];
    }
  }

  // device uploads
  auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes); };
  cudaError_t e;
  if ((e = alloc((void**)&m->d_X, m->geom.size() * 8)) != cudaSuccess ||
      (e = alloc((void**)&m->d_J, (size_t)K * Nq * 8)) != cudaSuccess ||
      (e = alloc((void**)&m->d_G, (size_t)K * 9 * Nq * 8)) != cudaSuccess ||
      (e = alloc((void**)&m->d_nJ, (size_t)K * 12 * Nfq * 8)) != cudaSuccess ||
      (e = alloc((void**)&m->d_xq, (size_t)K * Nq * 3 * 8)) != cudaSuccess ||
      (e = alloc((void**)&m->d_EToE, (size_t)K * 4 * 4)) != cudaSuccess ||
      (e = alloc((void**)&m->d_fcode, (size_t)K * 4)) != cudaSuccess ||
      (e = alloc((void**)&m->d_owner, (size_t)K * 4)) != cudaSuccess) {
    return bail(e == cudaErrorMemoryAllocation ? WADG_ENOMEM : WADG_ECUDA);
  }
  // FP64 tables: Vq, Vqa, Pq, Vfa, wq
  const size_t nVq = (size_t)Nq * Np, nVqa = 3 * nVq, nPq = nVq, nVfa = (size_t)4 * 3 * Nfq * Np;
  std::vector<double> ref64(nVq + nVqa + nPq + nVfa + Nq);
  std::copy(o.Vq.begin(), o.Vq.end(), ref64.begin());
  std::copy(o.Vqa.begin(), o.Vqa.end(), ref64.begin() + nVq);
  std::copy(o.Pq.begin(), o.Pq.end(), ref64.begin() + nVq + nVqa);
  std::copy(o.Vfa.begin(), o.Vfa.end(), ref64.begin() + nVq + nVqa + nPq);
  std::copy(o.wq.begin(), o.wq.end(), ref64.begin() + nVq + nVqa + nPq + nVfa);
  if ((e = alloc((void**)&m->d_ref64, ref64.size() * 8)) != cudaSuccess) return bail(WADG_ENOMEM);
  std::vector<int32_t> EToF32(m->EToF.begin(), m->EToF.end());
  int32_t* d_EToF = nullptr;
  int* d_nbad = nullptr;
  if ((e = alloc((void**)&d_EToF, (size_t)K * 4 * 4)) != cudaSuccess) return bail(WADG_ENOMEM);
  if ((e = alloc((void**)&d_nbad, sizeof(int))) != cudaSuccess) {
    cudaFree(d_EToF);
    return bail(WADG_ENOMEM);
  }
  int nbad = 0;
  bool okc = cudaMemcpy(m->d_X, m->geom.data(), m->geom.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(m->d_ref64, ref64.data(), ref64.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(m->d_EToE, m->EToE.data(), (size_t)K * 16, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(d_EToF, EToF32.data(), (size_t)K * 16, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(m->d_fcode, m->fcode.data(), (size_t)K * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(m->d_owner, m->owner.data(), (size_t)K * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(d_nbad, 0, sizeof(int)) == cudaSuccess;
  const double* dVq = m->d_ref64;
  const double* dVqa = dVq + nVq;
  const double* dVfa = dVq + nVq + nVqa + nPq;
  okc = okc && launch_geo_volume(K, Np, Nq, m->d_X, dVq, dVqa, m->d_J, m->d_G, m->d_xq, d_nbad, 0) == cudaSuccess &&
        launch_geo_face(K, Np, Nfq, m->d_X, dVfa, m->d_owner, m->d_EToE, d_EToF, m->d_nJ, 0) == cudaSuccess &&
        cudaMemcpy(&nbad, d_nbad, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d_EToF);
  cudaFree(d_nbad);
  if (!okc) return bail(WADG_ECUDA);
  if (nbad > 0) return bail(WADG_EGEOM);
  *out = m;
  return WADG_OK;
}

int wadg_mesh_info(const wadg_mesh* m, int64_t info[8]) {
  if (!m || !info) return WADG_EINVAL;
  info[0] = m->N;
  info[1] = m->K;
  info[2] = m->ref.Np;
  info[3] = m->ref.Nq;
  info[4] = m->ref.Nfp;
  info[5] = m->ref.Nfq;
  info[6] = m->S;
  info[7] = m->precision;
  return WADG_OK;
}

int wadg_volume_points(const wadg_mesh* m, double* xyz) {
  if (!m || !xyz) return WADG_EINVAL;
  DeviceGuard g(m->device);
  cudaError_t e = cudaMemcpy(xyz, m->d_xq, (size_t)m->K * m->ref.Nq * 3 * 8, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? WADG_OK : WADG_ECUDA;
}

int wadg_set_operators(wadg_mesh* m, int precision, int shots, double tau_p, double tau_u, const double* c2q) {
  if (!m) return WADG_EINVAL;
  if (precision != WADG_FP64 && precision != WADG_FP32 && precision != WADG_FP32_TF32 &&
      precision != WADG_FP32_3XBF16)
    return fail(m, WADG_EUNSUPPORTED, "precision %d is not built", precision);
  const bool tensor = precision == WADG_FP32_3XBF16 || precision == WADG_FP32_TF32;
  if (tensor && m->N > 5) return fail(m, WADG_EUNSUPPORTED, "the tensor-core stage is built for N <= 5");
  if (tensor && m->N == 5 && m->ref.Nq != 216 && m->ref.Nq != fewer_point_nq(5))
    return fail(m, WADG_EUNSUPPORTED,
                "the tensor-core stage at N = 5 is built for the 216-point collapsed rule and the fewer-point rule");
  if (tensor && m->form != 0)
    return fail(m, WADG_EUNSUPPORTED, "the tensor-core stage is built for the strong-weak formulation");
  if (shots < 1 || shots > (1 << 20)) return fail(m, WADG_EINVAL, "shots=%d", shots);
  if (tensor && (int64_t)m->K * shots * m->ref.Np >= ((int64_t)1 << 31))
    return fail(m, WADG_EUNSUPPORTED, "the tensor-core stage needs K * shots * Np < 2^31 (31-bit gather offsets)");
  if (!(tau_p >= 0) || !(tau_u >= 0)) return fail(m, WADG_EINVAL, "penalties must be >= 0");
  DeviceGuard g(m->device);
  const int64_t K = m->K;
  const int Nq = m->ref.Nq, Nfq = m->ref.Nfq, Np = m->ref.Np;
  if (c2q) {
    for (int64_t i = 0; i < K * Nq; ++i)
      if (!(c2q[i] > 0) || !std::isfinite(c2q[i])) return fail(m, WADG_EINVAL, "c2q[%lld] = %g", (long long)i, c2q[i]);
    if (!m->d_c2) WADG_CUDA(m, cudaMalloc(&m->d_c2, (size_t)K * Nq * 8));
    WADG_CUDA(m, cudaMemcpy(m->d_c2, c2q, (size_t)K * Nq * 8, cudaMemcpyHostToDevice));
  } else {
    dfree(m->d_c2);
  }
  if (precision != m->precision) {
    dfree(m->d_vgeo);
    dfree(m->d_fgeo);
  }
  {
    const int st = conservative_weights(m);
    if (st != WADG_OK) return st;
  }
  const double* Wpu = m->conservative ? m->d_Wpu : nullptr;
  const size_t ts = tsize(precision);
  m->n_planar_tiles = m->n_curved_tiles = m->n_planar_launch = 0;  // rebuilt for the tensor-core precisions
  if (!m->d_vgeo) WADG_CUDA(m, cudaMalloc(&m->d_vgeo, (size_t)K * 11 * Nq * ts));
  if (!m->d_fgeo) WADG_CUDA(m, cudaMalloc(&m->d_fgeo, (size_t)K * 12 * Nfq * ts));
  if (precision == WADG_FP64) {
    WADG_CUDA(m, launch_geo_pack<double>(K, Nq, Nfq, m->d_J, m->d_G, m->d_c2, Wpu, m->d_nJ, (double*)m->d_vgeo,
                                         (double*)m->d_fgeo, 0));
    if (!m->ops64.base) {
      int st = upload_ops<double>(m, m->ops64);
      if (st != WADG_OK) return st;
    }
  } else {
    WADG_CUDA(m, launch_geo_pack<float>(K, Nq, Nfq, m->d_J, m->d_G, m->d_c2, Wpu, m->d_nJ, (float*)m->d_vgeo,
                                        (float*)m->d_fgeo, 0));
    if (!m->ops32.base) {
      int st = upload_ops<float>(m, m->ops32);
      if (st != WADG_OK) return st;
    }
    if (tensor) {
      const int fmt = precision == WADG_FP32_3XBF16 ? 0 : 1;
      if (!m->d_tcops || m->tc_fmt != fmt) {
        std::vector<uint8_t> packed;
        if (!pack_tc_ops(m->N, m->ref, fmt, packed)) return fail(m, WADG_EUNSUPPORTED, "tensor-core tables");
        if (!m->d_tcops) WADG_CUDA(m, cudaMalloc((void**)&m->d_tcops, packed.size()));
        WADG_CUDA(m, cudaMemcpy(m->d_tcops, packed.data(), packed.size(), cudaMemcpyHostToDevice));
        m->tc_fmt = fmt;
      }
      const int64_t Kt = (K + 127) / 128;
      const int64_t nq4 = (Nq + 3) / 4, nf4 = (Nfq + 3) / 4;
      if (!m->d_vgeo_il) WADG_CUDA(m, cudaMalloc((void**)&m->d_vgeo_il, (size_t)Kt * 128 * 11 * nq4 * 4 * sizeof(float)));
      if (!m->d_fgeo_il) WADG_CUDA(m, cudaMalloc((void**)&m->d_fgeo_il, (size_t)Kt * 128 * 12 * nf4 * 4 * sizeof(float)));
      WADG_CUDA(m, launch_geo_pack_il(K, Nq, Nfq, m->d_J, m->d_G, m->d_c2, Wpu, m->d_nJ, m->d_vgeo_il, m->d_fgeo_il, 0));
      int st = mean_correction(m);
      if (st != WADG_OK) return st;
      st = planar_tiles(m, shots);
      if (st != WADG_OK) return st;
    }
  }
  if (!m->d_err) {
    WADG_CUDA(m, cudaMalloc((void**)&m->d_err, sizeof(int)));
    WADG_CUDA(m, cudaMemset(m->d_err, 0, sizeof(int)));
  }
  const size_t qbytes = (size_t)4 * K * shots * Np * ts;
  if (qbytes != m->qtmp_bytes) {
    dfree(m->d_Qtmp);
    dfree(m->d_red);
    WADG_CUDA(m, cudaMalloc(&m->d_Qtmp, qbytes));
    WADG_CUDA(m, cudaMalloc((void**)&m->d_red, ((size_t)K * shots + 1) * 8));
    m->qtmp_bytes = qbytes;
    dfree(m->d_Qlo);
  }
  if (precision == WADG_FP64) {
    m->compensate = 0;
    dfree(m->d_Qlo);
  } else if (m->compensate && !m->d_Qlo) {
    WADG_CUDA(m, cudaMalloc(&m->d_Qlo, qbytes));
    WADG_CUDA(m, cudaMemset(m->d_Qlo, 0, qbytes));
  }
  if (shots != m->S || precision != m->precision) {
    // sources and receivers depend on the shot count and precision
    m->nsrc = 0;
    m->R = 0;
    dfree(m->d_src_elem);
    dfree(m->d_src_vec);
    dfree(m->d_rec_col);
    dfree(m->d_rec_vec);
  }
  m->precision = precision;
  m->S = shots;
  m->tau_p = tau_p;
  m->tau_u = tau_u;
  ++m->generation;
  WADG_CUDA(m, cudaDeviceSynchronize());
  return prepare_strong(m);
}

}  // extern "C"

namespace {

inline const DevOps<double>& ops_of(const wadg_mesh* m, double) { return m->ops64; }
inline const DevOps<float>& ops_of(const wadg_mesh* m, float) { return m->ops32; }
inline const StrongOps<double>& sops_of(const wadg_mesh* m, double) { return m->sops64; }
inline const StrongOps<float>& sops_of(const wadg_mesh* m, float) { return m->sops32; }

template <typename T>
StageParams<T> base_params(const wadg_mesh* m) {
  StageParams<T> p;
  p.vgeo = (const T*)m->d_vgeo;
  p.fgeo = (const T*)m->d_fgeo;
  p.EToE = m->d_EToE;
  p.fcode = m->d_fcode;
  p.ops = ops_of(m, T());
  p.sgeo = (const T*)m->d_sgeo;
  p.sfgeo = (const T*)m->d_sfgeo;
  p.sops = sops_of(m, T());
  p.nq = m->ref.Nq;
  p.ncols = m->K * m->S;
  p.S = m->S;
  p.tau_p = (T)m->tau_p;
  p.tau_u = (T)m->tau_u;
  return p;
}

// The tensor-core stage forms its products from each column's fields less
// their element means (the derivatives of smooth fields and the nearly
// cancelling volume and face terms of the p equation are then products of
// small operands, so the rounding of the split operands stays small beside
// the result) and adds back in FP32 the term of the element-constant
// velocity: with p = 0 and u = e_i on every element, {u} = e_i on every face
// and every jump vanishes, so r_p of that state is element k's own term D_i,
// and r_p(Q) = r_p(Q - Qbar) + sum_i ubar_i D_i (the mean of p drops out:
// p enters only through derivatives and jumps).  The FP64 CUDA-core stage
// evaluates D_1..3 whenever the operators or update weights change.
int mean_correction(wadg_mesh* m) {
  const int64_t K = m->K;
  const int Np = m->ref.Np, Nq = m->ref.Nq, Nfq = m->ref.Nfq;
  const int64_t stride = (K + 3) / 4 * 4 * Np;
  if (!m->d_meanc) {
    WADG_CUDA(m, cudaMalloc((void**)&m->d_meanc, (size_t)3 * stride * sizeof(float)));
    WADG_CUDA(m, cudaMemset(m->d_meanc, 0, (size_t)3 * stride * sizeof(float)));
  }
  m->meanc_stride = stride;
  if (!m->ops64.base) {
    const int st = upload_ops<double>(m, m->ops64);
    if (st != WADG_OK) return st;
  }
  double *vg = nullptr, *fg = nullptr, *Q = nullptr, *out = nullptr;
  const int64_t nf = K * Np;
  cudaError_t e = cudaMalloc((void**)&vg, (size_t)K * 11 * Nq * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&fg, (size_t)K * 12 * Nfq * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&Q, (size_t)4 * nf * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&out, (size_t)4 * nf * sizeof(double));
  const double* Wpu = m->conservative ? m->d_Wpu : nullptr;
  if (e == cudaSuccess) e = launch_geo_pack<double>(K, Nq, Nfq, m->d_J, m->d_G, m->d_c2, Wpu, m->d_nJ, vg, fg, 0);
  StageParams<double> p = base_params<double>(m);
  p.vgeo = vg;
  p.fgeo = fg;
  p.ncols = K;
  p.S = 1;
  p.Qin = Q;
  p.out = out;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = cudaMemset(Q, 0, (size_t)4 * nf * sizeof(double));
    if (e == cudaSuccess) e = launch_fill(nf, 1.0, Q + (1 + i) * nf, 0);
    if (e == cudaSuccess) e = launch_stage<double>(m->N, p, kRhs, 0);
    if (e == cudaSuccess) e = launch_to_precision<float>(nf, out, m->d_meanc + i * stride, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(vg);
  cudaFree(fg);
  cudaFree(Q);
  cudaFree(out);
  return e == cudaSuccess ? WADG_OK : cuda_fail(m, e, "the tensor-core stage's mean correction");
}

// How many of the all-affine tiles the planar kernel runs; the rest join the
// curved launch (the curved kernel takes any tile).  Each launch's CTAs (one
// per SM) walk its tiles in rounds, so a launch costs ceil(tiles / SMs)
// rounds of its kernel; a planar tile takes a fraction of a curved one and a
// second launch in the stage adds a ramp, both measured in curved rounds:
// N = 4 (196,608 tets, 1,536 tiles, 52 us rounds): planar 0.86 (0.499 ms per
// stage all planar, 0.578 all curved), second launch 0.7 (0.577 ms with 760
// planar tiles after 776 curved ones against 0.542 from the rounds alone);
// N = 5 (82,944 tets, 648 tiles, 118 us rounds): planar 0.91 (0.534 vs
// 0.589 ms), second launch 0.2 (0.568 ms with 567 planar tiles after 81
// curved ones against 0.545); N = 2, 3 (196,608 and 82,944 tets, 29 and
// 44 us rounds): planar 0.96 (0.307 vs 0.319 and 0.212 vs 0.222 ms), second
// launch 0.35 (0.318 ms with 1,232 planar tiles after 304 curved ones at
// N = 2; 0.229 ms with 567 after 81 at N = 3).  N = 1 takes the N = 2
// values.  The cheapest
// split wins, ties going to the larger curved launch (a single launch when
// nothing is saved).  Mode 2 runs every all-affine tile on the planar kernel.
void plan_planar_launch(wadg_mesh* m) {
  const int64_t np = m->n_planar_tiles, nc = m->n_curved_tiles, G = std::max(1, m->num_sms);
  m->n_planar_launch = 0;
  if (np == 0 || m->planar_split == 0) return;
  if (m->planar_split == 2) {
    m->n_planar_launch = np;
    return;
  }
  const double planar_cost = m->N == 5 ? 0.91 : m->N == 4 ? 0.86 : 0.96;
  const double second_launch = m->N == 5 ? 0.2 : m->N == 4 ? 0.7 : 0.35;
  auto rounds = [&](int64_t n) { return (double)((n + G - 1) / G); };
  double best = 1e300;
  for (int64_t mv = np; mv >= 0; --mv) {
    const int64_t c = nc + mv, q = np - mv;
    const double t = (c > 0 ? rounds(c) : 0.0) + (q > 0 ? planar_cost * rounds(q) : 0.0) +
                     (c > 0 && q > 0 ? second_launch : 0.0);
    if (t < best - 1e-9) {
      best = t;
      m->n_planar_launch = q;
    }
  }
}

// The tiles of 128 columns (element, shot) whose elements are all affine run
// the planar tensor-core kernel, which reads each element's constant G and
// n J^f once (Sec. 6: separate kernels for planar and curvilinear elements);
// the others the curved one.  Lists: the planar tiles, then the others.
int planar_tiles(wadg_mesh* m, int shots) {
  dfree(m->d_tlist);
  dfree(m->d_gP);
  dfree(m->d_nP);
  m->n_planar_tiles = m->n_curved_tiles = m->n_planar_launch = 0;
  if (m->N > 5 || m->n_affine == 0) return WADG_OK;
  const int64_t ncols = m->K * shots, ntiles = (ncols + 127) / 128;
  std::vector<int32_t> planar, curved;
  for (int64_t t = 0; t < ntiles; ++t) {
    bool all = true;
    for (int64_t c = t * 128; c < std::min(ncols, (t + 1) * 128) && all; ++c) all = m->affine[c / shots] != 0;
    (all ? planar : curved).push_back((int32_t)t);
  }
  if (planar.empty()) return WADG_OK;
  const int64_t Kt = (m->K + 127) / 128;
  planar.insert(planar.end(), curved.begin(), curved.end());
  WADG_CUDA(m, cudaMalloc((void**)&m->d_tlist, planar.size() * sizeof(int32_t)));
  WADG_CUDA(m, cudaMemcpy(m->d_tlist, planar.data(), planar.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  WADG_CUDA(m, cudaMalloc((void**)&m->d_gP, (size_t)Kt * 9 * 128 * sizeof(float)));
  WADG_CUDA(m, cudaMalloc((void**)&m->d_nP, (size_t)Kt * 12 * 128 * sizeof(float)));
  WADG_CUDA(m, launch_geo_planar_pack(m->K, m->ref.Nq, m->ref.Nfq, m->d_G, m->d_nJ, m->d_gP, m->d_nP, 0));
  WADG_CUDA(m, cudaDeviceSynchronize());
  m->n_planar_tiles = (int64_t)planar.size() - (int64_t)curved.size();
  m->n_curved_tiles = (int64_t)curved.size();
  plan_planar_launch(m);
  return WADG_OK;
}

// Stage launch for the mesh's precision: RHS and LSRK stages of
// WADG_FP32_3XBF16 and WADG_FP32_TF32 run on the tensor cores, everything
// else on CUDA cores.
// The strong formulations run the RHS and LSRK stages as their strong modes.
inline int stage_mode(const wadg_mesh* m, int mode) {
  if (m->form == 0) return mode;
  const bool full = m->form == 1;
  if (mode == kRhs) return full ? kRhsStrong : kRhsStrongU;
  if (mode == kLsrk) return full ? kLsrkStrong : kLsrkStrongU;
  return -1;
}

template <typename T>
cudaError_t stage_launch(const wadg_mesh* m, const StageParams<T>& p, int mode, cudaStream_t st) {
  return launch_stage<T>(m->N, p, stage_mode(m, mode), st);
}
template <>
cudaError_t stage_launch<float>(const wadg_mesh* m, const StageParams<float>& p, int mode, cudaStream_t st) {
  if ((m->precision == WADG_FP32_3XBF16 || m->precision == WADG_FP32_TF32) && (mode == 0 || mode == 1)) {
    TcStageParams P;
    P.s = p;
    P.ops = m->d_tcops;
    P.err = m->d_err;
    P.vgeo_il = m->d_vgeo_il;
    P.fgeo_il = m->d_fgeo_il;
    P.meanc = m->d_meanc;
    P.meanc_stride = m->meanc_stride;
    // bulk copies and 16-byte accesses of the field tiles: every field range
    // of a tile starts 16-byte aligned in every field array the stage touches
    auto a16 = [](const void* q) { return ((uintptr_t)q & 15) == 0; };
    P.bulk_q = (p.ncols * m->ref.Np) % 4 == 0 && a16(p.Qin) && a16(p.out) && a16(p.res) && a16(p.Qout);
    if (m->n_planar_launch > 0 && m->N <= 5 && p.ncols == m->K * m->S) {
      // the planar kernel's tiles, then the curved kernel's (disjoint
      // columns; both launches read Q_in only)
      const int64_t total = m->n_planar_tiles + m->n_curved_tiles;
      P.gP = m->d_gP;
      P.nP = m->d_nP;
      P.tiles = m->d_tlist;
      P.ntiles_list = m->n_planar_launch;
      cudaError_t e = m->N == 5 ? launch_stage_tc5_planar(P, mode, m->tc_fmt, m->num_sms, st)
                                : launch_stage_tc_planar(m->N, P, mode, m->tc_fmt, m->num_sms, st);
      if (e != cudaSuccess || m->n_planar_launch == total) return e;
      P.tiles = m->d_tlist + m->n_planar_launch;
      P.ntiles_list = total - m->n_planar_launch;
      return launch_stage_tc(m->N, P, mode, m->tc_fmt, m->num_sms, st);
    }
    return launch_stage_tc(m->N, P, mode, m->tc_fmt, m->num_sms, st);
  }
  return launch_stage<float>(m->N, p, stage_mode(m, mode), st);
}

int check_ready(wadg_mesh* m) {
  if (!m) return WADG_EINVAL;
  if (m->precision < 0) return fail(m, WADG_ESTATE, "wadg_set_operators has not been called");
  if (m->form != 0 && (m->strong_form != m->form || m->strong_precision != m->precision))
    return fail(m, WADG_ESTATE, "the strong-form tables are not built (an earlier call failed)");
  return WADG_OK;
}

template <typename T>
int rhs_t(wadg_mesh* m, const void* Q, void* dQdt, cudaStream_t st) {
  StageParams<T> p = base_params<T>(m);
  p.Qin = (const T*)Q;
  p.out = (T*)dQdt;
  cudaError_t e = stage_launch<T>(m, p, 0, st);
  return e == cudaSuccess ? WADG_OK : cuda_fail(m, e, "stage kernel (rhs)");
}

double ricker(double t, double f0, double t0) {
  const double pi = 3.14159265358979323846;
  double a = pi * f0 * (t - t0);
  a *= a;
  return (1.0 - 2.0 * a) * std::exp(-a);
}

template <typename T>
int step_t(wadg_mesh* m, void* Q, void* res, double t0, double dt, int nsteps, void* traces, cudaStream_t st) {
  StageParams<T> p = base_params<T>(m);
  p.res = (T*)res;
  p.dt = (T)dt;
  if (m->nsrc > 0) {
    p.src_elem = m->d_src_elem;
    p.src_vec = (const T*)m->d_src_vec;
  }
  T* cur = (T*)Q;
  T* other = (T*)m->d_Qtmp;
  const size_t bytes = (size_t)4 * m->K * m->S * m->ref.Np * sizeof(T);
  if (sizeof(T) == 4 && m->compensate && m->d_Qlo) {
    // compensated summation of the state: mode 1 carries the rounding error
    // over this call's stages, mode 2 also from the previous call's
    if (m->compensate == 1) {
      cudaError_t e = cudaMemsetAsync(m->d_Qlo, 0, bytes, st);
      if (e != cudaSuccess) return cuda_fail(m, e, "clearing the compensation");
    }
    p.qlo = (T*)m->d_Qlo;
  }
  for (int n = 0; n < nsteps; ++n) {
    const double t = t0 + n * dt;
    for (int s = 0; s < 5; ++s) {
      p.Qin = cur;
      p.Qout = other;
      p.rk_a = (T)kRkA[s];
      p.rk_b = (T)kRkB[s];
      p.src_amp = (T)(m->nsrc > 0 ? ricker(t + kRkC[s] * dt, m->f0, m->t0) : 0.0);
      cudaError_t e = stage_launch<T>(m, p, 1, st);
      if (e != cudaSuccess) return cuda_fail(m, e, "stage kernel (lsrk)");
      std::swap(cur, other);
    }
    if (traces && m->R > 0) {
      cudaError_t e = launch_receivers<T>(m->K * m->S, m->S, m->R, m->ref.Np, cur, m->d_rec_col,
                                          (const T*)m->d_rec_vec, (T*)traces + (size_t)n * m->S * m->R, st);
      if (e != cudaSuccess) return cuda_fail(m, e, "receiver kernel");
    }
  }
  if (cur != (T*)Q) {
    cudaError_t e = cudaMemcpyAsync(Q, cur, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(m, e, "copy back");
  }
  return WADG_OK;
}

}  // namespace

// The readiness check of the entry points that read the operators, shared
// with the allocation-free energy (csrc/noalloc.cu).
int wadg_mesh_ready(wadg_mesh* m) { return check_ready(m); }

extern "C" {

int wadg_rhs(wadg_mesh* m, const void* Q, void* dQdt, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!Q || !dQdt || Q == dQdt || !aligned16(Q) || !aligned16(dQdt))
    return fail(m, WADG_EINVAL, "Q and dQdt must be distinct 16-byte aligned device pointers");
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  return m->precision == WADG_FP64 ? rhs_t<double>(m, Q, dQdt, s) : rhs_t<float>(m, Q, dQdt, s);
}

int wadg_step(wadg_mesh* m, void* Q, void* res, double t0, double dt, int nsteps, void* traces, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!Q || !res || Q == res || !aligned16(Q) || !aligned16(res))
    return fail(m, WADG_EINVAL, "Q and res must be distinct 16-byte aligned device pointers");
  if (nsteps < 0 || !std::isfinite(dt) || !std::isfinite(t0)) return fail(m, WADG_EINVAL, "nsteps/dt/t0");
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  return m->precision == WADG_FP64 ? step_t<double>(m, Q, res, t0, dt, nsteps, traces, s)
                                   : step_t<float>(m, Q, res, t0, dt, nsteps, traces, s);
}

int wadg_set_formulation(wadg_mesh* m, int form) {
  if (!m) return WADG_EINVAL;
  if (form < 0 || form > 2)
    return fail(m, WADG_EINVAL, "formulation %d (0 strong-weak, 1 strong, 2 strong on the 2N+1 rules)", form);
  if (form != 0 && m->N > 5) return fail(m, WADG_EUNSUPPORTED, "the strong formulation is built for N <= 5");
  if (form != 0 && !collapsed_size(m))
    return fail(m, WADG_EUNSUPPORTED, "the strong formulation is built for the (N+1)^3-point volume rule");
  if (form != 0 && (m->precision == WADG_FP32_3XBF16 || m->precision == WADG_FP32_TF32))
    return fail(m, WADG_EUNSUPPORTED, "the strong formulation runs on the CUDA-core precisions (FP64, FP32)");
  DeviceGuard g(m->device);
  const int prev = m->form;
  m->form = form;
  const int st = prepare_strong(m);
  if (st != WADG_OK) {
    const std::string msg = m->last_error;
    m->form = prev;
    prepare_strong(m);
    m->last_error = msg;
    return st;
  }
  if (form != prev) ++m->generation;  // a captured solve graph holds the other formulation's kernels
  return WADG_OK;
}

int wadg_set_conservation(wadg_mesh* m, int on) {
  if (!m) return WADG_EINVAL;
  if (on != 0 && on != 1) return fail(m, WADG_EINVAL, "conservation %d (0 pointwise weights, 1 conservative)", on);
  DeviceGuard g(m->device);
  const int prev = m->conservative;
  m->conservative = on;
  if (m->precision >= 0 && on != prev) {
    // repack the two weight rows of the geometric factors (all precisions)
    int st = conservative_weights(m);
    const double* Wpu = m->conservative ? m->d_Wpu : nullptr;
    const RefOps& o = m->ref;
    cudaError_t e = cudaSuccess;
    if (st == WADG_OK) {
      e = m->precision == WADG_FP64
              ? launch_geo_pack<double>(m->K, o.Nq, o.Nfq, m->d_J, m->d_G, m->d_c2, Wpu, m->d_nJ,
                                        (double*)m->d_vgeo, (double*)m->d_fgeo, 0)
              : launch_geo_pack<float>(m->K, o.Nq, o.Nfq, m->d_J, m->d_G, m->d_c2, Wpu, m->d_nJ, (float*)m->d_vgeo,
                                       (float*)m->d_fgeo, 0);
      if (e == cudaSuccess && m->d_vgeo_il)
        e = launch_geo_pack_il(m->K, o.Nq, o.Nfq, m->d_J, m->d_G, m->d_c2, Wpu, m->d_nJ, m->d_vgeo_il, m->d_fgeo_il, 0);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e != cudaSuccess) st = cuda_fail(m, e, "repacking the update weights");
      // the tensor-core stage's mean correction carries the update weights
      if (st == WADG_OK && (m->precision == WADG_FP32_3XBF16 || m->precision == WADG_FP32_TF32))
        st = mean_correction(m);
    }
    if (st != WADG_OK) {
      const std::string msg = m->last_error;
      m->conservative = prev;
      dfree(m->d_Wpu);
      m->last_error = msg;
      return st;
    }
  }
  if (on != prev) ++m->generation;
  return WADG_OK;
}

int wadg_set_compensation(wadg_mesh* m, int on) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (on < 0 || on > 2) return fail(m, WADG_EINVAL, "compensation %d (0 off, 1 per call, 2 across calls)", on);
  if (on && m->precision == WADG_FP64) return fail(m, WADG_EUNSUPPORTED, "compensation is for FP32 fields");
  DeviceGuard g(m->device);
  if (on && !m->d_Qlo) WADG_CUDA(m, cudaMalloc(&m->d_Qlo, m->qtmp_bytes));
  if (on) WADG_CUDA(m, cudaMemset(m->d_Qlo, 0, m->qtmp_bytes));  // every call starts a zero carry
  if (!on) dfree(m->d_Qlo);
  if (on != m->compensate) ++m->generation;
  m->compensate = on;
  return WADG_OK;
}

int wadg_compensation_carry(wadg_mesh* m, void* lo, int direction, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!lo || (direction != 0 && direction != 1)) return fail(m, WADG_EINVAL, "carry buffer or direction");
  if (!m->compensate || !m->d_Qlo) return fail(m, WADG_ESTATE, "compensation is off");
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = direction == 0 ? cudaMemcpyAsync(lo, m->d_Qlo, m->qtmp_bytes, cudaMemcpyDefault, s)
                                 : cudaMemcpyAsync(m->d_Qlo, lo, m->qtmp_bytes, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? WADG_OK : cuda_fail(m, e, "copying the compensation carry");
}

int wadg_set_planar_split(wadg_mesh* m, int on) {
  if (!m) return WADG_EINVAL;
  if (on < 0 || on > 2) return fail(m, WADG_EINVAL, "planar split %d (0 off, 1 planned, 2 every affine tile)", on);
  if (on != m->planar_split) ++m->generation;
  m->planar_split = on;
  plan_planar_launch(m);
  return WADG_OK;
}

int wadg_planar_info(const wadg_mesh* m, int64_t info[4]) {
  if (!m || !info) return WADG_EINVAL;
  info[0] = m->n_affine;
  info[1] = m->n_planar_tiles;
  info[2] = m->n_planar_tiles + m->n_curved_tiles;
  info[3] = m->n_planar_launch;
  return WADG_OK;
}

int wadg_step_host(wadg_mesh* m, void* Q, void* res, double t0, double dt, int nsteps, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!Q || Q == res) return fail(m, WADG_EINVAL, "Q and res must be distinct host pointers (res may be NULL)");
  if (nsteps < 0 || !std::isfinite(dt) || !std::isfinite(t0)) return fail(m, WADG_EINVAL, "nsteps/dt/t0");
  if (nsteps == 0) return WADG_OK;
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)4 * m->K * m->S * m->ref.Np * tsize(m->precision);
  if (bytes != m->host_io_bytes) {
    dfree(m->d_hostQ);
    dfree(m->d_hostR);
    m->host_io_bytes = 0;
    WADG_CUDA(m, cudaMalloc(&m->d_hostQ, bytes));
    WADG_CUDA(m, cudaMalloc(&m->d_hostR, bytes));
    m->host_io_bytes = bytes;
  }
  // res is not copied in: the first stage of every step has a_1 = 0 and does
  // not read the incoming residual
  WADG_CUDA(m, cudaMemcpyAsync(m->d_hostQ, Q, bytes, cudaMemcpyHostToDevice, s));
  st = m->precision == WADG_FP64 ? step_t<double>(m, m->d_hostQ, m->d_hostR, t0, dt, nsteps, nullptr, s)
                                 : step_t<float>(m, m->d_hostQ, m->d_hostR, t0, dt, nsteps, nullptr, s);
  if (st != WADG_OK) return st;
  WADG_CUDA(m, cudaMemcpyAsync(Q, m->d_hostQ, bytes, cudaMemcpyDeviceToHost, s));
  if (res) WADG_CUDA(m, cudaMemcpyAsync(res, m->d_hostR, bytes, cudaMemcpyDeviceToHost, s));
  WADG_CUDA(m, cudaStreamSynchronize(s));
  return WADG_OK;
}

int wadg_project(wadg_mesh* m, const double* fq, void* Q, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!fq || !Q) return fail(m, WADG_EINVAL, "null pointer");
  DeviceGuard g(m->device);
  const RefOps& o = m->ref;
  const double* dVq = m->d_ref64;
  const double* dPq = dVq + 4 * (size_t)o.Nq * o.Np;
  cudaError_t e = m->precision == WADG_FP64
                      ? launch_project<double>(m->K * m->S, m->S, o.Np, o.Nq, fq, m->d_J, dVq, dPq, (double*)Q,
                                               (cudaStream_t)stream)
                      : launch_project<float>(m->K * m->S, m->S, o.Np, o.Nq, fq, m->d_J, dVq, dPq, (float*)Q,
                                              (cudaStream_t)stream);
  return e == cudaSuccess ? WADG_OK : cuda_fail(m, e, "projection kernel");
}

static int reduce_common(wadg_mesh* m, int mode, const void* Q, const double* exact, int mask, double* outv,
                         cudaStream_t s) {
  const RefOps& o = m->ref;
  const double* dVq = m->d_ref64;
  const double* dwq = dVq + 4 * (size_t)o.Nq * o.Np + (size_t)o.Nq * o.Np + (size_t)4 * 3 * o.Nfq * o.Np;
  double* partial = m->d_red;
  double* out = m->d_red + m->K * m->S;
  cudaError_t e = m->precision == WADG_FP64
                      ? launch_reduce<double>(mode, m->K * m->S, m->S, o.Np, o.Nq, (const double*)Q, dVq, dwq, m->d_J,
                                              m->d_c2, exact, mask, partial, out, s)
                      : launch_reduce<float>(mode, m->K * m->S, m->S, o.Np, o.Nq, (const float*)Q, dVq, dwq, m->d_J,
                                             m->d_c2, exact, mask, partial, out, s);
  if (e != cudaSuccess) return cuda_fail(m, e, "reduction kernel");
  e = cudaMemcpyAsync(outv, out, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(m, e, "reduction copy");
  return WADG_OK;
}

int wadg_energy(wadg_mesh* m, const void* Q, double* E, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!Q || !E) return fail(m, WADG_EINVAL, "null pointer");
  DeviceGuard g(m->device);
  st = reduce_common(m, 0, Q, nullptr, 0, E, (cudaStream_t)stream);
  if (st != WADG_OK) return st;
  if (!std::isfinite(*E)) return fail(m, WADG_EUNSTABLE, "energy is %g", *E);
  return WADG_OK;
}

int wadg_l2_error(wadg_mesh* m, const void* Q, const double* exact_q, int field_mask, double* err, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!Q || !exact_q || !err || field_mask <= 0 || field_mask > 15) return fail(m, WADG_EINVAL, "bad argument");
  DeviceGuard g(m->device);
  double sq = 0.0;
  st = reduce_common(m, 1, Q, exact_q, field_mask, &sq, (cudaStream_t)stream);
  if (st != WADG_OK) return st;
  *err = std::sqrt(std::max(sq, 0.0));
  return WADG_OK;
}

int wadg_set_sources(wadg_mesh* m, const double* xyz, double f0, double t0) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  DeviceGuard g(m->device);
  dfree(m->d_src_elem);
  dfree(m->d_src_vec);
  m->nsrc = 0;
  if (!xyz) return WADG_OK;
  if (!(f0 > 0) || !std::isfinite(t0)) return fail(m, WADG_EINVAL, "f0 must be > 0");
  const int S = m->S;
  std::vector<int64_t> elem(S);
  std::vector<int32_t> elem32(S);
  const size_t ts = tsize(m->precision);
  std::vector<double> v64;
  std::vector<float> v32;
  st = m->precision == WADG_FP64 ? set_points<double>(m, S, xyz, elem.data(), v64)
                                 : set_points<float>(m, S, xyz, elem.data(), v32);
  if (st != WADG_OK) return st;
  for (int i = 0; i < S; ++i) elem32[i] = (int32_t)elem[i];
  WADG_CUDA(m, cudaMalloc((void**)&m->d_src_elem, S * sizeof(int32_t)));
  WADG_CUDA(m, cudaMalloc(&m->d_src_vec, (size_t)S * m->ref.Np * ts));
  WADG_CUDA(m, cudaMemcpy(m->d_src_elem, elem32.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice));
  WADG_CUDA(m, cudaMemcpy(m->d_src_vec, m->precision == WADG_FP64 ? (void*)v64.data() : (void*)v32.data(),
                          (size_t)S * m->ref.Np * ts, cudaMemcpyHostToDevice));
  m->nsrc = S;
  m->f0 = f0;
  m->t0 = t0;
  ++m->generation;
  return WADG_OK;
}

int wadg_set_receivers(wadg_mesh* m, int R, const double* xyz) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (R < 0 || (R > 0 && !xyz)) return fail(m, WADG_EINVAL, "R=%d", R);
  DeviceGuard g(m->device);
  dfree(m->d_rec_col);
  dfree(m->d_rec_vec);
  m->R = 0;
  if (R == 0) return WADG_OK;
  const int S = m->S, n = S * R;
  std::vector<int64_t> elem(n);
  std::vector<int32_t> col(n);
  const size_t ts = tsize(m->precision);
  std::vector<double> v64;
  std::vector<float> v32;
  st = m->precision == WADG_FP64 ? set_points<double>(m, n, xyz, elem.data(), v64)
                                 : set_points<float>(m, n, xyz, elem.data(), v32);
  if (st != WADG_OK) return st;
  for (int i = 0; i < n; ++i) col[i] = (int32_t)(elem[i] * S + i / R);
  WADG_CUDA(m, cudaMalloc((void**)&m->d_rec_col, n * sizeof(int32_t)));
  WADG_CUDA(m, cudaMalloc(&m->d_rec_vec, (size_t)n * m->ref.Np * ts));
  WADG_CUDA(m, cudaMemcpy(m->d_rec_col, col.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
  WADG_CUDA(m, cudaMemcpy(m->d_rec_vec, m->precision == WADG_FP64 ? (void*)v64.data() : (void*)v32.data(),
                          (size_t)n * m->ref.Np * ts, cudaMemcpyHostToDevice));
  m->R = R;
  ++m->generation;
  return WADG_OK;
}

}  // extern "C"

namespace {

template <typename T>
AdjUpdateParams<T> adj_params(const wadg_mesh* m) {
  AdjUpdateParams<T> a;
  a.vgeo = (const T*)m->d_vgeo;
  a.ops = ops_of(m, T());
  a.ncols = m->K * m->S;
  a.S = m->S;
  return a;
}

template <typename T>
int rhs_adjoint_t(wadg_mesh* m, const void* lam, void* out, cudaStream_t st) {
  AdjUpdateParams<T> a = adj_params<T>(m);
  a.lam = (const T*)lam;
  a.beta = (T*)m->d_Qtmp;
  cudaError_t e = launch_adj_update<T>(m->N, a, 0, st);
  if (e != cudaSuccess) return cuda_fail(m, e, "adjoint update kernel");
  StageParams<T> p = base_params<T>(m);
  p.Qin = (const T*)m->d_Qtmp;
  p.out = (T*)out;
  e = launch_stage<T>(m->N, p, 4, st);
  return e == cudaSuccess ? WADG_OK : cuda_fail(m, e, "stage kernel (adjoint rhs)");
}

template <typename T>
int step_record_t(wadg_mesh* m, void* Q, void* res, double t0, double dt, void* ystore, void* traces,
                  cudaStream_t st) {
  StageParams<T> p = base_params<T>(m);
  p.res = (T*)res;
  p.dt = (T)dt;
  if (m->nsrc > 0) {
    p.src_elem = m->d_src_elem;
    p.src_vec = (const T*)m->d_src_vec;
  }
  T* cur = (T*)Q;
  T* other = (T*)m->d_Qtmp;
  const size_t ny = (size_t)m->K * m->S * m->ref.Nq;
  for (int s = 0; s < 5; ++s) {
    p.Qin = cur;
    p.Qout = other;
    p.rk_a = (T)kRkA[s];
    p.rk_b = (T)kRkB[s];
    p.src_amp = (T)(m->nsrc > 0 ? ricker(t0 + kRkC[s] * dt, m->f0, m->t0) : 0.0);
    p.yrec = ystore ? (T*)ystore + s * ny : nullptr;
    cudaError_t e = ystore ? launch_stage<T>(m->N, p, 2, st) : stage_launch<T>(m, p, 1, st);
    if (e != cudaSuccess) return cuda_fail(m, e, "stage kernel (record)");
    std::swap(cur, other);
  }
  if (traces && m->R > 0) {
    cudaError_t e = launch_receivers<T>(m->K * m->S, m->S, m->R, m->ref.Np, cur, m->d_rec_col,
                                        (const T*)m->d_rec_vec, (T*)traces, st);
    if (e != cudaSuccess) return cuda_fail(m, e, "receiver kernel");
  }
  const size_t bytes = (size_t)4 * m->K * m->S * m->ref.Np * sizeof(T);
  cudaError_t e = cudaMemcpyAsync(Q, cur, bytes, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? WADG_OK : cuda_fail(m, e, "copy back");
}

template <typename T>
int step_adjoint_t(wadg_mesh* m, void* lamQ, void* lamR, double dt, const void* ystore, double* dc2, cudaStream_t st) {
  AdjUpdateParams<T> a = adj_params<T>(m);
  a.lamQ = (T*)lamQ;
  a.lamR = (T*)lamR;
  a.beta = (T*)m->d_Qtmp;
  a.dt = (T)dt;
  a.dc2 = ystore ? dc2 : nullptr;
  StageParams<T> p = base_params<T>(m);
  p.Qin = (const T*)m->d_Qtmp;
  p.Qout = (T*)lamQ;
  p.dt = (T)dt;
  const size_t ny = (size_t)m->K * m->S * m->ref.Nq;
  for (int s = 4; s >= 0; --s) {
    a.rk_a = (T)kRkA[s];
    a.rk_b = (T)kRkB[s];
    a.yrec = ystore ? (const T*)ystore + s * ny : nullptr;
    cudaError_t e = launch_adj_update<T>(m->N, a, 1, st);
    if (e != cudaSuccess) return cuda_fail(m, e, "adjoint update kernel");
    e = launch_stage<T>(m->N, p, 3, st);
    if (e != cudaSuccess) return cuda_fail(m, e, "stage kernel (adjoint)");
  }
  return WADG_OK;
}

// The reverse of a checkpoint segment: the forward recompute that records
// the stage factors (only when they are wanted), then, from the last step to
// the first, the receiver adjoint of the step's trace weights and the reverse
// LSRK step.
template <typename T>
int segment_adjoint_t(wadg_mesh* m, void* Q, void* res, double t0, double dt, int nsteps, const void* weights,
                      void* lamQ, void* lamR, void* ystore, double* dc2, cudaStream_t st) {
  const size_t ny5 = (size_t)5 * m->K * m->S * m->ref.Nq;
  if (ystore)
    for (int n = 0; n < nsteps; ++n) {
      const int r = step_record_t<T>(m, Q, res, t0 + n * dt, dt, (T*)ystore + n * ny5, nullptr, st);
      if (r != WADG_OK) return r;
    }
  for (int n = nsteps - 1; n >= 0; --n) {
    if (weights && m->R > 0) {
      cudaError_t e = launch_receivers_adjoint<T>(m->S, m->R, m->ref.Np, (const T*)weights + (size_t)n * m->S * m->R,
                                                  m->d_rec_col, (const T*)m->d_rec_vec, (T*)lamQ, st);
      if (e != cudaSuccess) return cuda_fail(m, e, "receiver adjoint kernel");
    }
    const int r = step_adjoint_t<T>(m, lamQ, lamR, dt, ystore ? (const T*)ystore + n * ny5 : nullptr, dc2, st);
    if (r != WADG_OK) return r;
  }
  return WADG_OK;
}

}  // namespace

extern "C" {

int wadg_segment_adjoint(wadg_mesh* m, void* Q, void* res, double t0, double dt, int nsteps, const void* weights,
                         void* lamQ, void* lamR, void* ystore, double* dc2, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (m->compensate) return fail(m, WADG_ESTATE, "the adjoint recomputes uncompensated steps: turn compensation off");
  if (m->form != 0) return fail(m, WADG_EUNSUPPORTED, "the adjoint is built for the strong-weak formulation");
  if (!collapsed_size(m)) return fail(m, WADG_EUNSUPPORTED, "the adjoint is built for the (N+1)^3-point volume rule");
  if (nsteps < 0 || !std::isfinite(dt) || !std::isfinite(t0)) return fail(m, WADG_EINVAL, "nsteps/dt/t0");
  if (!lamQ || !lamR || lamQ == lamR || !aligned16(lamQ) || !aligned16(lamR))
    return fail(m, WADG_EINVAL, "lambda_Q and lambda_res must be distinct 16-byte aligned device pointers");
  if ((dc2 != nullptr) != (ystore != nullptr)) return fail(m, WADG_EINVAL, "ystore and dc2 go together");
  if (ystore && (!Q || !res || Q == res || !aligned16(Q) || !aligned16(res) || Q == lamQ || Q == lamR ||
                 res == lamQ || res == lamR))
    return fail(m, WADG_EINVAL, "Q and res must be distinct 16-byte aligned device pointers, apart from the adjoints");
  if (m->conservative && ystore)
    return fail(m, WADG_EUNSUPPORTED, "the c^2 gradient is built for the pointwise update weights");
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  return m->precision == WADG_FP64
             ? segment_adjoint_t<double>(m, Q, res, t0, dt, nsteps, weights, lamQ, lamR, ystore, dc2, s)
             : segment_adjoint_t<float>(m, Q, res, t0, dt, nsteps, weights, lamQ, lamR, ystore, dc2, s);
}

int wadg_rhs_adjoint(wadg_mesh* m, const void* lam, void* out, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (m->form != 0) return fail(m, WADG_EUNSUPPORTED, "the adjoint is built for the strong-weak formulation");
  if (!collapsed_size(m)) return fail(m, WADG_EUNSUPPORTED, "the adjoint is built for the (N+1)^3-point volume rule");
  if (!lam || !out || lam == out || !aligned16(lam) || !aligned16(out))
    return fail(m, WADG_EINVAL, "lambda and out must be distinct 16-byte aligned device pointers");
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  return m->precision == WADG_FP64 ? rhs_adjoint_t<double>(m, lam, out, s) : rhs_adjoint_t<float>(m, lam, out, s);
}

int wadg_step_record(wadg_mesh* m, void* Q, void* res, double t0, double dt, void* ystore, void* traces,
                     wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (m->compensate) return fail(m, WADG_ESTATE, "the adjoint recomputes uncompensated steps: turn compensation off");
  if (m->form != 0) return fail(m, WADG_EUNSUPPORTED, "the adjoint is built for the strong-weak formulation");
  if (!collapsed_size(m)) return fail(m, WADG_EUNSUPPORTED, "the adjoint is built for the (N+1)^3-point volume rule");
  if (m->conservative && ystore)
    return fail(m, WADG_EUNSUPPORTED, "the c^2 gradient is built for the pointwise update weights");
  if (!Q || !res || Q == res || !aligned16(Q) || !aligned16(res))
    return fail(m, WADG_EINVAL, "Q and res must be distinct 16-byte aligned device pointers");
  if (!std::isfinite(dt) || !std::isfinite(t0)) return fail(m, WADG_EINVAL, "dt/t0");
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  return m->precision == WADG_FP64 ? step_record_t<double>(m, Q, res, t0, dt, ystore, traces, s)
                                   : step_record_t<float>(m, Q, res, t0, dt, ystore, traces, s);
}

int wadg_step_adjoint(wadg_mesh* m, void* lamQ, void* lamR, double dt, const void* ystore, double* dc2,
                      wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (m->form != 0) return fail(m, WADG_EUNSUPPORTED, "the adjoint is built for the strong-weak formulation");
  if (!collapsed_size(m)) return fail(m, WADG_EUNSUPPORTED, "the adjoint is built for the (N+1)^3-point volume rule");
  if (!lamQ || !lamR || lamQ == lamR || !aligned16(lamQ) || !aligned16(lamR))
    return fail(m, WADG_EINVAL, "lambda_Q and lambda_res must be distinct 16-byte aligned device pointers");
  if ((dc2 != nullptr) != (ystore != nullptr)) return fail(m, WADG_EINVAL, "ystore and dc2 go together");
  if (m->conservative && ystore)
    return fail(m, WADG_EUNSUPPORTED, "the c^2 gradient is built for the pointwise update weights");
  if (!std::isfinite(dt)) return fail(m, WADG_EINVAL, "dt");
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  return m->precision == WADG_FP64 ? step_adjoint_t<double>(m, lamQ, lamR, dt, ystore, dc2, s)
                                   : step_adjoint_t<float>(m, lamQ, lamR, dt, ystore, dc2, s);
}

int wadg_receivers_adjoint(wadg_mesh* m, const void* weights, void* lamQ, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!weights || !lamQ) return fail(m, WADG_EINVAL, "null pointer");
  if (m->R == 0) return WADG_OK;
  DeviceGuard g(m->device);
  cudaError_t e = m->precision == WADG_FP64
                      ? launch_receivers_adjoint<double>(m->S, m->R, m->ref.Np, (const double*)weights, m->d_rec_col,
                                                         (const double*)m->d_rec_vec, (double*)lamQ,
                                                         (cudaStream_t)stream)
                      : launch_receivers_adjoint<float>(m->S, m->R, m->ref.Np, (const float*)weights, m->d_rec_col,
                                                        (const float*)m->d_rec_vec, (float*)lamQ, (cudaStream_t)stream);
  return e == cudaSuccess ? WADG_OK : cuda_fail(m, e, "receiver adjoint kernel");
}

}  // extern "C"

extern "C" int wadg_solve(wadg_mesh* m, void* Q, void* res, double t0, double T, double dt_max, void* traces,
                          int* nsteps_out, wadg_stream stream) {
  int st = check_ready(m);
  if (st != WADG_OK) return st;
  if (!Q || !res || Q == res || !aligned16(Q) || !aligned16(res))
    return fail(m, WADG_EINVAL, "Q and res must be distinct 16-byte aligned device pointers");
  if (!(T > 0) || !(dt_max > 0) || !std::isfinite(T) || !std::isfinite(t0)) return fail(m, WADG_EINVAL, "T, dt");
  const double ratio = std::ceil(T / dt_max - 1e-12);
  if (ratio > 1e8) return fail(m, WADG_EINVAL, "too many steps");
  const int nsteps = std::max(1, (int)ratio);
  const double dt = T / nsteps;
  if (nsteps_out) *nsteps_out = nsteps;
  DeviceGuard g(m->device);
  if (!m->solve_stream) {
    WADG_CUDA(m, cudaStreamCreateWithFlags(&m->solve_stream, cudaStreamNonBlocking));
    WADG_CUDA(m, cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming));
    WADG_CUDA(m, cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming));
  }
  wadg_mesh::SolveKey key;
  key.Q = Q;
  key.res = res;
  key.traces = traces;
  key.t0 = t0;
  key.dt = dt;
  key.nsteps = nsteps;
  key.precision = m->precision;
  key.S = m->S;
  key.R = m->R;
  key.nsrc = m->nsrc;
  key.generation = m->generation;
  const wadg_mesh::SolveKey& k0 = m->solve_key;
  const bool same = m->solve_exec && k0.Q == key.Q && k0.res == key.res && k0.traces == key.traces &&
                    k0.t0 == key.t0 && k0.dt == key.dt && k0.nsteps == key.nsteps && k0.precision == key.precision &&
                    k0.S == key.S && k0.R == key.R && k0.nsrc == key.nsrc && k0.generation == key.generation;
  if (!same) {
    if (m->solve_exec) {
      WADG_CUDA(m, cudaStreamSynchronize(m->solve_stream));
      cudaGraphExecDestroy(m->solve_exec);
      m->solve_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    WADG_CUDA(m, cudaStreamBeginCapture(m->solve_stream, cudaStreamCaptureModeThreadLocal));
    int rc = m->precision == WADG_FP64 ? step_t<double>(m, Q, res, t0, dt, nsteps, traces, m->solve_stream)
                                       : step_t<float>(m, Q, res, t0, dt, nsteps, traces, m->solve_stream);
    cudaError_t e = cudaStreamEndCapture(m->solve_stream, &graph);
    if (rc != WADG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(m, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&m->solve_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      m->solve_exec = nullptr;
      return cuda_fail(m, e, "cudaGraphInstantiate");
    }
    m->solve_key = key;
  }
  // order the graph after the caller's prior work and the caller's later work after it
  WADG_CUDA(m, cudaEventRecord(m->ev_in, (cudaStream_t)stream));
  WADG_CUDA(m, cudaStreamWaitEvent(m->solve_stream, m->ev_in, 0));
  WADG_CUDA(m, cudaGraphLaunch(m->solve_exec, m->solve_stream));
  WADG_CUDA(m, cudaEventRecord(m->ev_out, m->solve_stream));
  WADG_CUDA(m, cudaStreamWaitEvent((cudaStream_t)stream, m->ev_out, 0));
  return WADG_OK;
}

extern "C" int wadg_device_status(wadg_mesh* m, wadg_stream stream) {
  if (!m) return WADG_EINVAL;
  if (!m->d_err) return WADG_OK;
  DeviceGuard g(m->device);
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "device status");
  if (flag) {
    cudaMemsetAsync(m->d_err, 0, sizeof(int), (cudaStream_t)stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    return fail(m, WADG_ETIMEOUT, "a bounded wait in a tensor-core kernel expired");
  }
  return WADG_OK;
}

extern "C" int wadg_selftest_bounded_wait(wadg_mesh* m, uint32_t max_iters, wadg_stream stream) {
  if (!m) return WADG_EINVAL;
  if (!m->d_err) return fail(m, WADG_ESTATE, "wadg_set_operators has not been called");
  if (max_iters < 1 || max_iters > (1u << 22)) return fail(m, WADG_EINVAL, "max_iters in [1, 2^22]");
  DeviceGuard g(m->device);
  cudaError_t e = launch_bounded_wait_selftest(m->d_err, max_iters, (cudaStream_t)stream);
  return e == cudaSuccess ? WADG_OK : cuda_fail(m, e, "bounded-wait self test");
}
