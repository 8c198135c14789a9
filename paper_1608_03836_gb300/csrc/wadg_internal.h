// Internal types of the WADG library: the mesh object, device operator
// tables and kernel parameter blocks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "refops.h"
#include "wadg.h"

namespace wadg {

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients
// (the scheme named in Sec. 5.2 of the paper, which does not print them).
inline constexpr double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                   -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
inline constexpr double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                   1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                   2277821191437.0 / 14882151754819.0};
inline constexpr double kRkC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                                   2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

// Device copies of the reference operators in precision T, stored "k-major"
// (A[k][m], consecutive output rows m contiguous, the row count m padded with
// zero rows to a multiple of 4: Nq -> NQP etc.) so that a thread owning 4
// consecutive output rows reads them with one vector load per k.
template <typename T>
struct DevOps {
  const T* VqT = nullptr;     // [Np][NQP]      V_q
  const T* VaT = nullptr;     // [3][Np][NQP]   V_q^a  (d/dr, d/ds, d/dt)
  const T* DwT = nullptr;     // [3][Nq][NPP]   (V_q^a)^T diag(w), one block per a
  const T* VwT = nullptr;     // [Nq][NPP]      V_q^T diag(w)
  const T* VtT = nullptr;     // [Np][NQP]      V_q M^^{-1}
  const T* PqT = nullptr;     // [Nq][NPP]      M^^{-1} V_q^T diag(w)
  const T* VtriT = nullptr;   // [Nfp][NFQP]    face interpolation
  const T* VtriTwT = nullptr; // [Nfq][NFPP]    V_tri^T diag(w_f)
  const T* PqTT = nullptr;    // [Np][NQP]      P_q^T            (adjoint update)
  const T* VtTT = nullptr;    // [Nq][NPP]      (V_q M^^{-1})^T  (adjoint update)
  const int16_t* gidx = nullptr;  // [4][6][Nfp]
  const int16_t* ginv = nullptr;  // [4][6][Np]
  void* base = nullptr;       // single allocation holding all of the above
};

// Stage kernel modes.  kRhsStrong, kLsrkStrong: the strong formulation
// (Sec. 4.1) with its volume and surface terms on the energy-stable rules
// (degree 4N-3 / 4N-2); kRhsStrongU, kLsrkStrongU: the strong formulation on
// the degree 2N+1 rules (under-integrated on curved elements).  N <= 5.
enum StageMode {
  kRhs = 0, kLsrk = 1, kRecord = 2, kAdjLsrk = 3, kAdjRhs = 4,
  kRhsStrong = 5, kLsrkStrong = 6, kRhsStrongU = 7, kLsrkStrongU = 8
};

// Points of the fewer-point symmetric volume rules the stage kernels are
// built for (exact to degree 2N+1): 14 at N = 2, 35 at N = 3, 63 at N = 4,
// 96 at N = 5; 0: none.
constexpr int fewer_point_nq(int N) {
  return N == 2 ? 14 : (N == 3 ? 35 : (N == 4 ? 63 : (N == 5 ? 96 : 0)));
}

// Sizes of the strong-form stage for degree N and formulation FORM (1: the
// energy-stable rules, 2: the degree 2N+1 rules).  The volume terms walk the
// NQS points in NCH chunks of QC points (a multiple of 4; the operator tables
// are padded with zero rows to NQSC = NCH QC); a chunk's 12 derivative values
// per point share the per-column scratch with the face phase (4 jump
// combinations at 4 Nfp face nodes and 4 NFQS face points) and the update
// (4 Nq values).
template <int N, int FORM>
struct StrongDims {
  static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int NFP = (N + 1) * (N + 2) / 2;
  static constexpr int NQ = (N + 1) * (N + 1) * (N + 1);
  static constexpr int NV = FORM == 1 ? (2 * N - 1 > N + 1 ? 2 * N - 1 : N + 1) : N + 1;
  static constexpr int NF = FORM == 1 ? 2 * N : N + 1;
  static constexpr int NQS = NV * NV * NV;
  static constexpr int NFQS = NF * NF;
  static constexpr int NFQSP = (NFQS + 3) / 4 * 4;
  static constexpr int XF = 4 * 4 * NFP + 4 * 4 * NFQS;
  static constexpr int NCH = (12 * NQS + XF - 1) / XF;
  static constexpr int QC = ((NQS + NCH - 1) / NCH + 3) / 4 * 4;
  static constexpr int NQSC = NCH * QC;
  static constexpr int XS0 = XF > 12 * QC ? XF : 12 * QC;
  static constexpr int XS = XS0 > 4 * NQ ? XS0 : 4 * NQ;
  static constexpr int PER_COL = 8 * NP + XS;  // sQ, sR, scratch
};

// Device tables of the strong form's rules, k-major as in DevOps.
template <typename T>
struct StrongOps {
  const T* VaT = nullptr;      // [3][Np][NQSC]  dl_n/dx^_a at the volume points
  const T* VwT = nullptr;      // [NQSC][NPP]    V_q^T diag(w)
  const T* VtriT = nullptr;    // [Nfp][NFQSP]   face interpolation
  const T* VtriTwT = nullptr;  // [NFQS][NFPP]   V_tri^T diag(w_f)
  void* base = nullptr;
};

// Parameters of one fused stage launch (RHS + weight-adjusted update, and in
// LSRK mode the Runge-Kutta update).
template <typename T>
struct StageParams {
  const T* Qin = nullptr;   // [4][ncols][Np]
  T* Qout = nullptr;        // LSRK: Q + b res; may not alias Qin
  T* res = nullptr;         // LSRK: residual, read and written in place
  // LSRK with compensated summation: the rounding error of Q_out carried to
  // the next stage, [4][ncols][Np], read and written in place (nullptr: none)
  T* qlo = nullptr;
  T* out = nullptr;         // RHS mode: dQ/dt
  const T* vgeo = nullptr;  // [K][11][Nq]: G_ai (a-major, 9), c^2/J, 1/J
  const T* fgeo = nullptr;  // [K][3][4 Nfq]: n J^f at the owner face points
  const int32_t* EToE = nullptr;  // [K][4], -1 on the boundary
  const uint8_t* fcode = nullptr; // [K][4]: pi_own + 6 (pi_nbr + 6 f_nbr)
  DevOps<T> ops;
  int64_t ncols = 0;        // K * S
  int S = 1;
  T tau_p = 1, tau_u = 1;
  T rk_a = 0, rk_b = 0, dt = 0;
  // point sources, one per shot (src_elem < 0: none)
  const int32_t* src_elem = nullptr;  // [S]
  const T* src_vec = nullptr;         // [S][Np] l_n(x^_s)
  T src_amp = 0;
  T* yrec = nullptr;                  // record mode: [ncols][Nq]
  int nq = 0;                         // points of the volume rule (selects the kernel)
  // strong form on its own rules (kRhsStrong, kLsrkStrong)
  const T* sgeo = nullptr;   // [K][9][NQS]: G_ai at the strong volume points
  const T* sfgeo = nullptr;  // [K][3][4 NFQS]: n J^f at the strong face points (owner order)
  StrongOps<T> sops;         // tables of the current strong formulation (1 or 2)
};

// Parameters of the adjoint weight-adjusted update beta = U^T mu (local).
template <typename T>
struct AdjUpdateParams {
  const T* lam = nullptr;   // RHS mode: mu = lam
  T* lamQ = nullptr;        // LSRK mode: mu = lamR + b lamQ
  T* lamR = nullptr;        //            lamR <- a mu
  T* beta = nullptr;        // output U^T mu, [4][ncols][Np]
  const T* vgeo = nullptr;
  DevOps<T> ops;
  int64_t ncols = 0;
  int S = 1;
  T rk_a = 0, rk_b = 0, dt = 0;
  const T* yrec = nullptr;  // [ncols][Nq] recorded forward factor (nullable)
  double* dc2 = nullptr;    // [K][Nq] gradient accumulator (nullable)
};

// Tensor-core stage (FP32 fields, split-bf16 products).
struct TcStageParams {
  StageParams<float> s;
  const uint8_t* ops = nullptr;  // packed split operators: NCH volume chunks, then NCH update chunks
  int* err = nullptr;            // set to 1 when a bounded wait expires
  const float* vgeo_il = nullptr;  // column-interleaved geometric factors (see aux_kernels.cu)
  const float* fgeo_il = nullptr;
  int bulk_q = 0;  // fields may be loaded by bulk copies (16-byte aligned tiles, row stride = Np)
  // r_p of the stage for the element-constant velocity e_i (p = 0), [3][stride]
  // with element k's Np values at k * Np: the products run on each column's
  // fields less their element means, and the epilogue adds sum_i ubar_i D_i
  const float* meanc = nullptr;
  int64_t meanc_stride = 0;
  // the tiles to walk (nullptr: all): the list of tiles whose elements are
  // all affine, or of the others; compact geometry of the affine elements,
  // interleaved over 128 elements: G [Kt][9][128], n J^f [Kt][12][128]
  const int32_t* tiles = nullptr;
  int64_t ntiles_list = 0;
  const float* gP = nullptr;
  const float* nP = nullptr;
};
cudaError_t launch_stage_tc(int N, const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream);
// The same over the tiles of P.tiles whose elements are all affine (N <= 4;
// N = 5: launch_stage_tc5_planar).
cudaError_t launch_stage_tc_planar(int N, const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream);
bool pack_tc_ops(int N, const RefOps& o, int fmt, std::vector<uint8_t>& out);
// N = 5 (stage_tc5_kernel.cuh), on the 216-point or the 96-point volume rule.
cudaError_t launch_stage_tc5(const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream);
cudaError_t launch_stage_tc5_planar(const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream);
bool pack_tc5_ops(const RefOps& o, int fmt, std::vector<uint8_t>& out);
cudaError_t launch_bounded_wait_selftest(int* err, uint32_t max_iters, cudaStream_t stream);

// Batches of FP32 meshes (batch.cu).
// Tile rules of mesh batches (batch.cu): 0, 1, 2.
constexpr int kBatchRules = 3;
int batch_cols_per_block(int N, int rule);
size_t batch_smem_bytes(int N, int rule);
int batch_max_blocks_per_sm(int rule, size_t smem);
cudaError_t launch_batch_stage(int mode, int rule, const StageParams<float>* params, const int* item_mesh,
                               const int* item_blk, const int* mesh_N, int nitems, int grid, size_t smem,
                               cudaStream_t st);

// Launchers, one per (precision, degree); modes as in StageMode.
template <typename T>
cudaError_t launch_stage(int N, const StageParams<T>& p, int mode, cudaStream_t stream);
template <typename T>
cudaError_t launch_adj_update(int N, const AdjUpdateParams<T>& p, int lsrk, cudaStream_t stream);

}  // namespace wadg

struct wadg_mesh {
  int device = 0;
  int N = 0;
  int64_t K = 0;
  wadg::RefOps ref;
  // host connectivity
  std::vector<int32_t> EToE;   // [K][4]
  std::vector<int32_t> EToF;   // [K][4]
  std::vector<uint8_t> fcode;  // [K][4]
  std::vector<uint8_t> owner;  // [K][4] 1 if this element owns the face
  std::vector<double> geom;    // [K][Np][3]
  std::vector<uint8_t> affine;  // [K] 1: the element's geometry nodes are its vertices' affine map
  int64_t n_affine = 0;
  int planar_split = 1;          // 0 off, 1 planned (the default), 2 every all-affine tile (wadg_set_planar_split)
  int32_t* d_tlist = nullptr;    // the planar tiles, then the others (tensor-core stage, N <= 5)
  int64_t n_planar_tiles = 0, n_curved_tiles = 0;
  float* d_gP = nullptr;         // compact geometry of the affine elements (see TcStageParams)
  float* d_nP = nullptr;
  int64_t n_planar_launch = 0;   // tiles the planar kernel runs (the head of d_tlist)
  // device geometry (FP64)
  double* d_X = nullptr;       // [K][Np][3]
  double* d_J = nullptr;       // [K][Nq]
  double* d_G = nullptr;       // [K][9][Nq]
  double* d_nJ = nullptr;      // [K][3][4 Nfq]
  double* d_xq = nullptr;      // [K][Nq][3]
  double* d_c2 = nullptr;      // [K][Nq]
  int32_t* d_EToE = nullptr;
  uint8_t* d_fcode = nullptr;
  uint8_t* d_owner = nullptr;
  // FP64 operators (setup kernels, projection, diagnostics)
  double* d_ref64 = nullptr;   // Vq [Nq][Np], Vqa [3][Nq][Np], Pq [Np][Nq], Vfa [4][3][Nfq][Np], wq [Nq]
  // precision-dependent state
  int precision = -1;
  int S = -1;
  double tau_p = 1.0, tau_u = 1.0;
  void* d_vgeo = nullptr;
  void* d_fgeo = nullptr;
  wadg::DevOps<double> ops64;
  wadg::DevOps<float> ops32;
  uint8_t* d_tcops = nullptr;  // operators of the tensor-core stage (split bf16 or tf32)
  int tc_fmt = -1;             // format of d_tcops: 0 split bf16, 1 tf32
  int form = 0;                // 0 strong-weak, 1 strong, 2 strong on the 2N+1 rules (Sec. 4.1)
  // strong-form state for (strong_form, strong_precision): tables, and for
  // form 1 the geometric factors at its rules' points
  int strong_form = 0, strong_precision = -1;
  void* d_sgeo = nullptr;      // [K][9][NQS] in the mesh precision
  void* d_sfgeo = nullptr;     // [K][3][4 NFQS]
  wadg::StrongOps<double> sops64;
  wadg::StrongOps<float> sops32;
  int conservative = 0;        // 1: update weights 1 / Pi_N(J/c^2), 1 / Pi_N(J) (local conservation)
  double* d_Wpu = nullptr;     // [K][2][Nq] those weights (FP64), while conservative
  void* d_hostQ = nullptr;     // device copies for wadg_step_host
  void* d_hostR = nullptr;
  size_t host_io_bytes = 0;
  float* d_vgeo_il = nullptr;  // column-interleaved geometry for the tensor-core stage
  float* d_fgeo_il = nullptr;
  float* d_meanc = nullptr;     // the tensor-core stage's mean correction [3][Kp][Np], Kp = K rounded up to 4
  int64_t meanc_stride = 0;
  int* d_err = nullptr;        // device error flag (bounded waits)
  int num_sms = 0;
  void* d_Qtmp = nullptr;      // ping-pong buffer for LSRK stages
  int compensate = 0;          // 1: LSRK steps with compensated summation of the state (FP32 fields)
  void* d_Qlo = nullptr;       // the carried rounding error of the state, like Q
  size_t qtmp_bytes = 0;
  double* d_red = nullptr;     // reduction scratch
  // sources and receivers
  int nsrc = 0;
  double f0 = 5.0, t0 = 0.24;
  int32_t* d_src_elem = nullptr;
  void* d_src_vec = nullptr;
  int R = 0;
  int32_t* d_rec_col = nullptr;   // [S][R] column index k*S+s
  void* d_rec_vec = nullptr;      // [S][R][Np]
  // wadg_solve: captured graph of the last solve and its key
  cudaStream_t solve_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t solve_exec = nullptr;
  struct SolveKey {
    void* Q = nullptr;
    void* res = nullptr;
    void* traces = nullptr;
    double t0 = 0, dt = 0;
    int nsteps = -1, precision = -1, S = -1, R = -1, nsrc = -1;
    uint64_t generation = 0;
  } solve_key;
  uint64_t generation = 0;  // bumped by every call that changes operators, sources or receivers
  std::string last_error;
};

// WADG_OK when the entry points that read the operators may run (operators
// uploaded; strong-form tables built when a strong form is selected), else
// the status those entry points return, with last_error set.
int wadg_mesh_ready(wadg_mesh* m);
