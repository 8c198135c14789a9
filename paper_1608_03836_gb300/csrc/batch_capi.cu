// C ABI of mesh batches (see include/wadg.h, "Batches").
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "wadg_internal.h"

using namespace wadg;

// Tensor-core batches: the meshes of one class (same degree, volume rule,
// shots and penalties) are stepped as one combined mesh, a library-internal
// wadg_mesh whose elements are the members' in sequence (connectivity offset,
// geometry repacked into one interleaved copy) and which borrows the first
// member's operator tables; every tile of 128 columns of the combined mesh
// may hold columns of several members.  The stage's arithmetic per column is
// that of the member's own stage, so results are bitwise equal to stepping
// the members one by one.
struct TcClass {
  wadg_mesh* cm = nullptr;
  std::vector<int> members;
  std::vector<int64_t> off;  // first element of each member in the combined mesh
  float* dQ = nullptr;       // combined fields and residual [4][K][S][Np]
  float* dR = nullptr;
};

struct wadg_batch {
  std::vector<wadg_mesh*> meshes;
  int device = 0;
  bool tc = false;                 // tensor-core batch (classes) instead of the persistent FP32 launch
  std::vector<TcClass> classes;
  std::vector<int> prec0, S0;      // the members' precision and shots at creation
  // work lists of the tile rules (see batch.cu)
  int rule = 0;
  int nitems_r[kBatchRules] = {};
  int* d_item_mesh_r[kBatchRules] = {};
  int* d_item_blk_r[kBatchRules] = {};
  size_t smem_r[kBatchRules] = {};
  int max_grid_r[kBatchRules] = {};
  int* d_mesh_N = nullptr;
  int grid = 0;
  int nitems() const { return nitems_r[rule]; }
  // parameter tables: slot 2*s + parity for LSRK stage s, slot 10 for the RHS
  StageParams<float>* d_params = nullptr;
  std::vector<StageParams<float>> h_params;
  std::vector<const void*> keyQ, keyR;
  double key_dt = NAN;
  // captured solve
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> gkeyQ, gkeyR;
  double gkey_t0 = NAN, gkey_dt = NAN;
  int gkey_n = -1, gkey_rule = -1, gkey_grid = -1;
  std::string last_error;
};

namespace {

// Runs a body with the batch's device current, restoring the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

int bfail(wadg_batch* b, int status, const std::string& msg) {
  if (b) b->last_error = msg;
  return status;
}

#define BCUDA(b, call)                                                                       \
  do {                                                                                       \
    cudaError_t _e = (call);                                                                 \
    if (_e != cudaSuccess) return bfail((b), WADG_ECUDA, std::string(#call ": ") + cudaGetErrorString(_e)); \
  } while (0)

StageParams<float> mesh_params(const wadg_mesh* m) {
  StageParams<float> p;
  p.vgeo = (const float*)m->d_vgeo;
  p.fgeo = (const float*)m->d_fgeo;
  p.EToE = m->d_EToE;
  p.fcode = m->d_fcode;
  p.ops = m->ops32;
  p.ncols = m->K * m->S;
  p.S = m->S;
  p.tau_p = (float)m->tau_p;
  p.tau_u = (float)m->tau_u;
  return p;
}

// (Re)build the parameter tables for these field buffers and step.
int ensure_tables(wadg_batch* b, void* const* Q, void* const* res, double dt) {
  const size_t nm = b->meshes.size();
  bool same = b->d_params && b->key_dt == dt;
  for (size_t i = 0; same && i < nm; ++i) same = b->keyQ[i] == Q[i] && b->keyR[i] == res[i];
  if (same) return WADG_OK;
  b->h_params.assign(11 * nm, StageParams<float>());
  for (size_t i = 0; i < nm; ++i) {
    const wadg_mesh* m = b->meshes[i];
    for (int s = 0; s < 5; ++s)
      for (int par = 0; par < 2; ++par) {
        StageParams<float> p = mesh_params(m);
        p.Qin = (const float*)(par == 0 ? Q[i] : m->d_Qtmp);
        p.Qout = (float*)(par == 0 ? m->d_Qtmp : Q[i]);
        p.res = (float*)res[i];
        p.rk_a = (float)kRkA[s];
        p.rk_b = (float)kRkB[s];
        p.dt = (float)dt;
        b->h_params[(2 * s + par) * nm + i] = p;
      }
    StageParams<float> r = mesh_params(m);
    r.Qin = (const float*)Q[i];
    r.out = (float*)m->d_Qtmp;
    b->h_params[10 * nm + i] = r;
  }
  BCUDA(b, cudaMemcpy(b->d_params, b->h_params.data(), b->h_params.size() * sizeof(StageParams<float>),
                      cudaMemcpyHostToDevice));
  b->keyQ.assign(Q, Q + nm);
  b->keyR.assign(res, res + nm);
  b->key_dt = dt;
  return WADG_OK;
}

int check_buffers(wadg_batch* b, void* const* Q, void* const* res) {
  if (!Q || !res) return bfail(b, WADG_EINVAL, "null buffer arrays");
  for (size_t i = 0; i < b->meshes.size(); ++i) {
    if (!Q[i] || !res[i] || Q[i] == res[i] || ((uintptr_t)Q[i] & 15u) || ((uintptr_t)res[i] & 15u))
      return bfail(b, WADG_EINVAL, "each Q[i], res[i] must be distinct 16-byte aligned device pointers");
    if (b->meshes[i]->precision != b->prec0[i] || b->meshes[i]->S != b->S0[i])
      return bfail(b, WADG_ESTATE, "a mesh's precision or shots changed since the batch was created");
  }
  return WADG_OK;
}

// Copies between the members' fields and a class's combined fields.
int tc_copy(wadg_batch* b, const TcClass& c, void* const* Q, void* const* res, bool in, cudaStream_t st) {
  const wadg_mesh* cm = c.cm;
  const size_t col = (size_t)cm->S * cm->ref.Np;
  for (size_t j = 0; j < c.members.size(); ++j) {
    const int i = c.members[j];
    const wadg_mesh* m = b->meshes[i];
    const size_t n = (size_t)m->K * col * sizeof(float);
    for (int f = 0; f < 4; ++f) {
      float* gq = c.dQ + ((size_t)f * cm->K + c.off[j]) * col;
      float* gr = c.dR + ((size_t)f * cm->K + c.off[j]) * col;
      float* mq = (float*)Q[i] + (size_t)f * m->K * col;
      float* mr = (float*)res[i] + (size_t)f * m->K * col;
      cudaError_t e = in ? cudaMemcpyAsync(gq, mq, n, cudaMemcpyDeviceToDevice, st)
                         : cudaMemcpyAsync(mq, gq, n, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = in ? cudaMemcpyAsync(gr, mr, n, cudaMemcpyDeviceToDevice, st)
               : cudaMemcpyAsync(mr, gr, n, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return bfail(b, WADG_ECUDA, std::string("batch copy: ") + cudaGetErrorString(e));
    }
  }
  return WADG_OK;
}

// Tensor-core batch: per class, the members' fields into the combined
// buffers, nsteps LSRK steps of the combined mesh, and back.
int enqueue_tc(wadg_batch* b, void* const* Q, void* const* res, double t0, double dt, int nsteps, cudaStream_t st) {
  for (const TcClass& c : b->classes) {
    int r = tc_copy(b, c, Q, res, true, st);
    if (r != WADG_OK) return r;
    r = wadg_step(c.cm, c.dQ, c.dR, t0, dt, nsteps, nullptr, (wadg_stream)st);
    if (r != WADG_OK) return bfail(b, r, std::string("combined step: ") + c.cm->last_error);
    r = tc_copy(b, c, Q, res, false, st);
    if (r != WADG_OK) return r;
  }
  return WADG_OK;
}

void free_class(TcClass& c) {
  if (c.cm) {
    wadg_mesh* m = c.cm;
    cudaFree(m->d_EToE);
    cudaFree(m->d_fcode);
    cudaFree(m->d_vgeo_il);
    cudaFree(m->d_fgeo_il);
    cudaFree(m->d_meanc);
    cudaFree(m->d_err);
    cudaFree(m->d_Qtmp);
    delete m;  // the operator tables are the first member's
  }
  cudaFree(c.dQ);
  cudaFree(c.dR);
  c = TcClass();
}

// The combined mesh of a class.  Interleaved geometry: element k's float4
// (row, group) sits at ((k >> 7) * rows * groups + row * groups + group) * 128
// + (k & 127) (see launch_geo_pack_il), repacked element by element.
int build_class(wadg_batch* b, TcClass& c) {
  const wadg_mesh* m0 = b->meshes[c.members[0]];
  int64_t K = 0;
  for (int i : c.members) {
    c.off.push_back(K);
    K += b->meshes[i]->K;
  }
  const int S = m0->S, Np = m0->ref.Np, Nq = m0->ref.Nq, Nfq = m0->ref.Nfq;
  if (K * S * Np >= ((int64_t)1 << 31)) return bfail(b, WADG_EUNSUPPORTED, "a tensor-core class needs K * S * Np < 2^31");
  wadg_mesh* cm = new (std::nothrow) wadg_mesh();
  if (!cm) return WADG_ENOMEM;
  c.cm = cm;
  cm->device = m0->device;
  cm->N = m0->N;
  cm->K = K;
  cm->ref = m0->ref;
  cm->precision = m0->precision;
  cm->S = S;
  cm->tau_p = m0->tau_p;
  cm->tau_u = m0->tau_u;
  cm->ops32 = m0->ops32;
  cm->d_tcops = m0->d_tcops;
  cm->tc_fmt = m0->tc_fmt;
  cm->num_sms = m0->num_sms;
  std::vector<int32_t> E((size_t)K * 4);
  std::vector<uint8_t> F((size_t)K * 4);
  const int64_t nq4 = (Nq + 3) / 4, nf4 = (Nfq + 3) / 4, Kt = (K + 127) / 128;
  std::vector<float> V((size_t)Kt * 128 * 11 * nq4 * 4, 0.f), G((size_t)Kt * 128 * 12 * nf4 * 4, 0.f);
  for (size_t j = 0; j < c.members.size(); ++j) {
    const wadg_mesh* m = b->meshes[c.members[j]];
    const int64_t o = c.off[j], Km = m->K, Ktm = (Km + 127) / 128;
    for (int64_t k = 0; k < Km * 4; ++k) {
      const int32_t e = m->EToE[k];
      E[o * 4 + k] = e >= 0 ? (int32_t)(e + o) : e;
      F[o * 4 + k] = m->fcode[k];
    }
    std::vector<float> v((size_t)Ktm * 128 * 11 * nq4 * 4), g((size_t)Ktm * 128 * 12 * nf4 * 4);
    BCUDA(b, cudaMemcpy(v.data(), m->d_vgeo_il, v.size() * sizeof(float), cudaMemcpyDeviceToHost));
    BCUDA(b, cudaMemcpy(g.data(), m->d_fgeo_il, g.size() * sizeof(float), cudaMemcpyDeviceToHost));
    auto repack = [&](const std::vector<float>& src, std::vector<float>& dst, int64_t rows_groups) {
      for (int64_t k = 0; k < Km; ++k) {
        const int64_t kc = k + o;
        for (int64_t rg = 0; rg < rows_groups; ++rg) {
          const size_t si = (size_t)(((k >> 7) * rows_groups + rg) * 128 + (k & 127)) * 4;
          const size_t di = (size_t)(((kc >> 7) * rows_groups + rg) * 128 + (kc & 127)) * 4;
          for (int x = 0; x < 4; ++x) dst[di + x] = src[si + x];
        }
      }
    };
    repack(v, V, 11 * nq4);
    repack(g, G, 12 * nf4);
  }
  const size_t qbytes = (size_t)4 * K * S * Np * sizeof(float);
  BCUDA(b, cudaMalloc((void**)&cm->d_EToE, E.size() * sizeof(int32_t)));
  BCUDA(b, cudaMalloc((void**)&cm->d_fcode, F.size()));
  BCUDA(b, cudaMalloc((void**)&cm->d_vgeo_il, V.size() * sizeof(float)));
  BCUDA(b, cudaMalloc((void**)&cm->d_fgeo_il, G.size() * sizeof(float)));
  BCUDA(b, cudaMalloc((void**)&cm->d_err, sizeof(int)));
  BCUDA(b, cudaMalloc(&cm->d_Qtmp, qbytes));
  BCUDA(b, cudaMalloc((void**)&c.dQ, qbytes));
  BCUDA(b, cudaMalloc((void**)&c.dR, qbytes));
  cm->qtmp_bytes = qbytes;
  BCUDA(b, cudaMemset(cm->d_err, 0, sizeof(int)));
  BCUDA(b, cudaMemcpy(cm->d_EToE, E.data(), E.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(cm->d_fcode, F.data(), F.size(), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(cm->d_vgeo_il, V.data(), V.size() * sizeof(float), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(cm->d_fgeo_il, G.data(), G.size() * sizeof(float), cudaMemcpyHostToDevice));
  // the members' mean corrections, element by element in the combined order
  cm->meanc_stride = (K + 3) / 4 * 4 * Np;
  BCUDA(b, cudaMalloc((void**)&cm->d_meanc, (size_t)3 * cm->meanc_stride * sizeof(float)));
  BCUDA(b, cudaMemset(cm->d_meanc, 0, (size_t)3 * cm->meanc_stride * sizeof(float)));
  for (size_t j = 0; j < c.members.size(); ++j) {
    const wadg_mesh* m = b->meshes[c.members[j]];
    if (!m->d_meanc) return bfail(b, WADG_ESTATE, "a tensor-core member has no mean correction");
    for (int i = 0; i < 3; ++i)
      BCUDA(b, cudaMemcpy(cm->d_meanc + i * cm->meanc_stride + c.off[j] * Np, m->d_meanc + i * m->meanc_stride,
                          (size_t)m->K * Np * sizeof(float), cudaMemcpyDeviceToDevice));
  }
  return WADG_OK;
}

int enqueue_steps(wadg_batch* b, void* const* Q, int nsteps, cudaStream_t st) {
  const size_t nm = b->meshes.size();
  for (int n = 0; n < nsteps; ++n)
    for (int s = 0; s < 5; ++s) {
      const int par = (5 * n + s) & 1;
      const int r = b->rule;
      cudaError_t e = launch_batch_stage(1, r, b->d_params + (2 * s + par) * nm, b->d_item_mesh_r[r],
                                         b->d_item_blk_r[r], b->d_mesh_N, b->nitems_r[r], b->grid, b->smem_r[r], st);
      if (e != cudaSuccess) return bfail(b, WADG_ECUDA, std::string("batch stage: ") + cudaGetErrorString(e));
    }
  if ((5 * nsteps) & 1)
    for (size_t i = 0; i < nm; ++i) {
      const wadg_mesh* m = b->meshes[i];
      const size_t bytes = (size_t)4 * m->K * m->S * m->ref.Np * sizeof(float);
      cudaError_t e = cudaMemcpyAsync(Q[i], m->d_Qtmp, bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return bfail(b, WADG_ECUDA, std::string("copy back: ") + cudaGetErrorString(e));
    }
  return WADG_OK;
}

}  // namespace

extern "C" {

void wadg_batch_destroy(wadg_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->stream) cudaStreamDestroy(b->stream);
  for (int r = 0; r < kBatchRules; ++r) {
    cudaFree(b->d_item_mesh_r[r]);
    cudaFree(b->d_item_blk_r[r]);
  }
  for (TcClass& c : b->classes) free_class(c);
  cudaFree(b->d_mesh_N);
  cudaFree(b->d_params);
  delete b;
}

int wadg_batch_create(wadg_mesh* const* meshes, int count, wadg_batch** out) {
  if (!out || !meshes || count < 1) return WADG_EINVAL;
  *out = nullptr;
  wadg_batch* b = new (std::nothrow) wadg_batch();
  if (!b) return WADG_ENOMEM;
  b->meshes.assign(meshes, meshes + count);
  for (int i = 0; i < count; ++i)
    if (!meshes[i]) {
      delete b;
      return WADG_EINVAL;
    }
  for (int i = 0; i < count; ++i) {
    b->prec0.push_back(meshes[i]->precision);
    b->S0.push_back(meshes[i]->S);
    if (meshes[i]->compensate) {  // batches step without compensation
      delete b;
      return WADG_ESTATE;
    }
  }
  const int p0 = meshes[0]->precision;
  if (p0 == WADG_FP32_3XBF16 || p0 == WADG_FP32_TF32) {
    // tensor-core batch: classes of (degree, rule, shots, penalties)
    b->tc = true;
    b->device = meshes[0]->device;
    for (int i = 0; i < count; ++i) {
      const wadg_mesh* m = meshes[i];
      if (m->precision != p0 || m->form != 0 || m->device != b->device || m->nsrc > 0 || m->R > 0) {
        delete b;
        return WADG_ESTATE;
      }
      TcClass* c = nullptr;
      for (TcClass& x : b->classes) {
        const wadg_mesh* a = meshes[x.members[0]];
        if (a->N == m->N && a->ref.Nq == m->ref.Nq && a->S == m->S && a->tau_p == m->tau_p && a->tau_u == m->tau_u)
          c = &x;
      }
      if (!c) {
        b->classes.emplace_back();
        c = &b->classes.back();
      }
      c->members.push_back(i);
    }
    DeviceGuard g(b->device);
    for (TcClass& c : b->classes) {
      const int r = build_class(b, c);
      if (r != WADG_OK) {
        wadg_batch_destroy(b);
        return r;
      }
    }
    *out = b;
    return WADG_OK;
  }
  for (int i = 0; i < count; ++i) {
    const int n1 = meshes[i] ? meshes[i]->N + 1 : 0;
    if (!meshes[i] || meshes[i]->precision != WADG_FP32 || meshes[i]->form != 0 ||
        meshes[i]->ref.Nq != n1 * n1 * n1 || meshes[i]->device != meshes[0]->device) {
      delete b;
      return WADG_ESTATE;
    }
  }
  b->device = meshes[0]->device;
  // work items for each tile rule, heaviest degree first
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return meshes[x]->N > meshes[y]->N; });
  std::vector<int> mn(count);
  for (int i = 0; i < count; ++i) mn[i] = meshes[i]->N;
  const int nsm = meshes[0]->num_sms;
  bool ok = cudaMalloc((void**)&b->d_mesh_N, mn.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc((void**)&b->d_params, 11 * count * sizeof(StageParams<float>)) == cudaSuccess &&
            cudaMemcpy(b->d_mesh_N, mn.data(), mn.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
  for (int r = 0; r < kBatchRules && ok; ++r) {
    std::vector<int> im, ib;
    for (int i = 0; i < count; ++i) b->smem_r[r] = std::max(b->smem_r[r], batch_smem_bytes(meshes[i]->N, r));
    for (int oi : order) {
      const wadg_mesh* m = meshes[oi];
      const int E = batch_cols_per_block(m->N, r);
      const int64_t blocks = (m->K * m->S + E - 1) / E;
      for (int64_t k = 0; k < blocks; ++k) {
        im.push_back(oi);
        ib.push_back((int)k);
      }
    }
    b->nitems_r[r] = (int)im.size();
    b->max_grid_r[r] = batch_max_blocks_per_sm(r, b->smem_r[r]) * nsm;
    ok = cudaMalloc((void**)&b->d_item_mesh_r[r], im.size() * sizeof(int)) == cudaSuccess &&
         cudaMalloc((void**)&b->d_item_blk_r[r], ib.size() * sizeof(int)) == cudaSuccess &&
         cudaMemcpy(b->d_item_mesh_r[r], im.data(), im.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_item_blk_r[r], ib.data(), ib.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    wadg_batch_destroy(b);
    return WADG_ENOMEM;
  }
  b->rule = 0;
  b->grid = std::min(b->max_grid_r[0], std::max(1, b->nitems_r[0]));
  *out = b;
  return WADG_OK;
}

int wadg_batch_info(const wadg_batch* b, int64_t info[5]) {
  if (!b || !info) return WADG_EINVAL;
  if (b->tc) {
    int64_t tiles = 0;
    for (const TcClass& c : b->classes) tiles += (c.cm->K * c.cm->S + 127) / 128;
    info[0] = (int64_t)b->meshes.size();
    info[1] = tiles;
    info[2] = info[3] = b->meshes[0]->num_sms;
    info[4] = -1;
    return WADG_OK;
  }
  info[0] = (int64_t)b->meshes.size();
  info[1] = b->nitems();
  info[2] = b->grid;
  info[3] = b->max_grid_r[b->rule];
  info[4] = b->rule;
  return WADG_OK;
}

int wadg_batch_set_rule(wadg_batch* b, int rule) {
  if (!b || rule < 0 || rule >= kBatchRules) return WADG_EINVAL;
  if (b->tc) return WADG_OK;  // tensor-core batches have one schedule
  b->rule = rule;
  b->grid = std::min(b->grid, std::max(1, b->nitems()));
  return WADG_OK;
}

int wadg_batch_set_grid(wadg_batch* b, int grid) {
  if (!b || grid < 1) return WADG_EINVAL;
  if (b->tc) return WADG_OK;
  b->grid = std::min(grid, std::max(1, b->nitems()));
  return WADG_OK;
}

int wadg_batch_step(wadg_batch* b, void* const* Q, void* const* res, double t0, double dt, int nsteps,
                    wadg_stream stream) {
  if (!b) return WADG_EINVAL;
  int st = check_buffers(b, Q, res);
  if (st != WADG_OK) return st;
  if (nsteps < 0 || !std::isfinite(dt) || !std::isfinite(t0)) return bfail(b, WADG_EINVAL, "nsteps/dt/t0");
  if (b->tc) {
    DeviceGuard g(b->device);
    return enqueue_tc(b, Q, res, t0, dt, nsteps, (cudaStream_t)stream);
  }
  st = ensure_tables(b, Q, res, dt);
  if (st != WADG_OK) return st;
  return enqueue_steps(b, Q, nsteps, (cudaStream_t)stream);
}

// Times each candidate number of persistent blocks on right-hand-side
// launches (the fields are not modified) and keeps the fastest.
int wadg_batch_autotune(wadg_batch* b, void* const* Q, void* const* res, int* grid_out, wadg_stream stream) {
  if (!b) return WADG_EINVAL;
  int st = check_buffers(b, Q, res);
  if (st != WADG_OK) return st;
  if (b->tc) {  // one schedule: a persistent block per SM in every class's launch
    if (grid_out) *grid_out = b->meshes[0]->num_sms;
    return WADG_OK;
  }
  st = ensure_tables(b, Q, res, b->key_dt == b->key_dt ? b->key_dt : 0.0);
  if (st != WADG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nsm = b->meshes[0]->num_sms;
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  const size_t nm = b->meshes.size();
  float best = 1e30f;
  int best_g = b->grid, best_r = b->rule;
  for (int r = 0; r < kBatchRules; ++r) {
    std::vector<int> cands;
    for (int mult : {1, 2, 3, 4, 6, 8})
      if (mult * nsm <= b->max_grid_r[r]) cands.push_back(mult * nsm);
    cands.push_back(std::min(b->nitems_r[r], 1 << 20));
    for (int g : cands) {
      g = std::max(1, std::min(g, b->nitems_r[r]));
      auto run = [&]() {
        return launch_batch_stage(0, r, b->d_params + 10 * nm, b->d_item_mesh_r[r], b->d_item_blk_r[r], b->d_mesh_N,
                                  b->nitems_r[r], g, b->smem_r[r], s);
      };
      run();
      run();
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 5; ++rep) run();
      cudaEventRecord(e1, s);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return bfail(b, WADG_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_g = g;
        best_r = r;
      }
    }
  }
  b->rule = best_r;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->grid = best_g;
  if (grid_out) *grid_out = best_g;
  return WADG_OK;
}

int wadg_batch_solve(wadg_batch* b, void* const* Q, void* const* res, double t0, double T, double dt_max,
                     int* nsteps_out, wadg_stream stream) {
  if (!b) return WADG_EINVAL;
  int st = check_buffers(b, Q, res);
  if (st != WADG_OK) return st;
  if (!(T > 0) || !(dt_max > 0) || !std::isfinite(T) || !std::isfinite(t0)) return bfail(b, WADG_EINVAL, "T, dt");
  const double ratio = std::ceil(T / dt_max - 1e-12);
  if (ratio > 1e8) return bfail(b, WADG_EINVAL, "too many steps");
  const int nsteps = std::max(1, (int)ratio);
  const double dt = T / nsteps;
  if (nsteps_out) *nsteps_out = nsteps;
  if (!b->tc) {
    st = ensure_tables(b, Q, res, dt);
    if (st != WADG_OK) return st;
  }
  DeviceGuard g(b->device);
  if (!b->stream) {
    BCUDA(b, cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    BCUDA(b, cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    BCUDA(b, cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  }
  const size_t nm = b->meshes.size();
  bool same = b->exec && b->gkey_t0 == t0 && b->gkey_dt == dt && b->gkey_n == nsteps &&
              b->gkey_rule == b->rule && b->gkey_grid == b->grid;
  for (size_t i = 0; same && i < nm; ++i) same = b->gkeyQ[i] == Q[i] && b->gkeyR[i] == res[i];
  if (!same) {
    if (b->exec) {
      BCUDA(b, cudaStreamSynchronize(b->stream));
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = b->tc ? enqueue_tc(b, Q, res, t0, dt, nsteps, b->stream) : enqueue_steps(b, Q, nsteps, b->stream);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (rc != WADG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return bfail(b, WADG_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return bfail(b, WADG_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    b->gkeyQ.assign(Q, Q + nm);
    b->gkeyR.assign(res, res + nm);
    b->gkey_t0 = t0;
    b->gkey_dt = dt;
    b->gkey_n = nsteps;
    b->gkey_rule = b->rule;
    b->gkey_grid = b->grid;
  }
  BCUDA(b, cudaEventRecord(b->ev_in, (cudaStream_t)stream));
  BCUDA(b, cudaStreamWaitEvent(b->stream, b->ev_in, 0));
  BCUDA(b, cudaGraphLaunch(b->exec, b->stream));
  BCUDA(b, cudaEventRecord(b->ev_out, b->stream));
  BCUDA(b, cudaStreamWaitEvent((cudaStream_t)stream, b->ev_out, 0));
  return WADG_OK;
}

const char* wadg_batch_last_error(const wadg_batch* b) { return b ? b->last_error.c_str() : ""; }

}  // extern "C"
