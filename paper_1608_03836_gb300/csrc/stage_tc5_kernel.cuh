// Fused WADG stage on the tensor cores at N = 5 (Np = 56), for the FP32-field
// precisions with split-bf16 or tf32 products, FP32 accumulation in TMEM.
//
// The N <= 4 kernel (stage_tc_kernel.cuh) keeps all four fields' split operands, an
// FP32 field tile, seven face interpolants and three pressure accumulators
// live at once; at N = 5 that needs about 720 TMEM columns and 322 KB of
// shared memory.  This kernel keeps the same persistent 128-column tiles,
// thread layout (four threads per column, warps w, w + 4, w + 8, w + 12 on the
// TMEM lanes of quarter w) and operand formats, and fits the budgets
// (512 TMEM columns, 214 KB of shared memory) by:
//   - the four b accumulators in TMEM columns 256..511 for the whole tile;
//   - faces in two passes sharing the TMEM columns 0..255: pass A interpolates
//     [p] and {u} to the face points, forms the pressure flux and lifts it;
//     pass B interpolates [u] into the columns {u} held, forms the velocity
//     fluxes (with [p] from pass A) and lifts them into the columns the
//     interpolants held (Sec. 4.1, Sec. 6.4);
//   - no FP32 field tile: the face gathers read their own column's values
//     from global memory (L2) like the neighbour's, and the split field
//     operands are written from global memory after the faces;
//   - the three pressure test products chained into one accumulator, and
//     single-buffered operator slots for the volume chunks (16 points);
//   - the weight-adjusted update (Sec. 6.2, Eq. (matfree); Sec. 7) in chunks of
//     16 points, its operators double-buffered.
// The epilogue (dQ/dt or the LSRK update, Sec. 5.2) is the N <= 4 kernel's.
// Waits are bounded as there; on expiry the CTA records an error, issues no
// further copies or products, drains (bounded) and returns.
#pragma once
#include "tc_stage_common.cuh"

namespace wadg {

template <int NQX = 216>
struct TcDims5 {
  static constexpr int N = 5;
  using D = Dims<5, NQX>;
  static constexpr int NP = D::NP, NQ = D::NQ, NFP = D::NFP, NFQ = D::NFQ;
  static constexpr int KP = 64, QC = 16, NCH = (NQ + QC - 1) / QC, TILE = 128;
  static constexpr int A_FIELD = TILE * KP * 2, SZ_AQ = 4 * 2 * A_FIELD;  // split field tiles (128 KB)
  static constexpr int A_CH = TILE * QC * 2, SZ_AX = 6 * 2 * A_CH;        // U^a, g_i of a chunk (48 KB)
  static constexpr int B_V = QC * KP * 2, B_P = KP * QC * 2;
  static constexpr int UQC = 16, UNCH = (NQ + UQC - 1) / UQC;
  static constexpr int A_UCH = TILE * UQC * 2, B_UV = UQC * KP * 2, B_UP = KP * UQC * 2;
  // the update operators in three bf16 parts (the fourth product of mma4_chain)
  static constexpr int SZ_VA = 8 * B_V, SZ_VB = 8 * B_P, SZ_UA = 3 * B_UV, SZ_UB = 3 * B_UP;
  static constexpr int SZ_OPV = SZ_VA + SZ_VB, SZ_OPU = SZ_UA + SZ_UB;
  static constexpr int SZ_OPS = NCH * SZ_OPV + UNCH * SZ_OPU;
  static constexpr int NFP16 = 32, NFQ16 = 48;
  static constexpr int A_FN = TILE * NFP16 * 2, A_FQ = TILE * NFQ16 * 2;
  static constexpr int B_TRI = NFQ16 * NFP16 * 2, SZ_FOPS = 4 * B_TRI;
  // shared memory: region 0 (the split fields / b; during the faces the
  // combinations, fluxes and lifted values; the output tile at the end), the
  // two operator slots, region X (chunk arrays; the face operators during
  // the faces), tables
  static constexpr int OFF_FB = 4 * 2 * A_FN;           // pass-B combinations after pass A's four
  static constexpr int SZ_SLOT = 16384;
  static constexpr int OFF_SA = SZ_AQ, OFF_SB = OFF_SA + SZ_SLOT, OFF_X = OFF_SB + SZ_SLOT;
  static constexpr int SZ_X = SZ_AX;
  static constexpr int OFF_GI = OFF_X + SZ_X, SZ_GI = (4 * 6 * NP * 2 + 15) / 16 * 16;
  static constexpr int OFF_GX = OFF_GI + SZ_GI, SZ_GX = (4 * 6 * NFP * 2 + 15) / 16 * 16;
  static constexpr int OFF_NB = OFF_GX + SZ_GX, OFF_MEAN = OFF_NB + TILE * 20;  // element means [4][128]
  static constexpr int OFF_BAR = OFF_MEAN + 4 * TILE * 4, SMEM = OFF_BAR + 128;
  // TMEM columns
  static constexpr int TB = 256;        // b accumulators of the four fields, 64 each; then r
  static constexpr int T1 = 96;         // volume chunk outputs (u_i: 3 x 16, dp/dx^_a: 48), buffers at 0, 96
  static constexpr int T1U = 64;        // update chunk outputs (4 x 16), buffers at 0, 64
  static constexpr int TI = 0;          // interpolants: [p] at 0, {u} then [u] at 48..191
  static constexpr int TLP = 192;       // lifted pressure flux (32)
  static constexpr int TLU = 0;         // lifted velocity fluxes (3 x 32) over [p] and [u]_1
  static_assert(NP == 56 && NFP == 21 && NFQ == 36, "N = 5");
  static_assert(2 * T1 <= TB && 2 * T1U <= TB && TI + 4 * NFQ16 <= TLP && TLP + NFP16 <= TB &&
                    TLU + 3 * NFP16 <= TI + 4 * NFQ16 && TB + 4 * KP <= 512,
                "TMEM plan");
  static_assert(SZ_VA <= SZ_SLOT && SZ_VB <= SZ_SLOT && 2 * SZ_UA <= SZ_SLOT && 2 * SZ_UB <= SZ_SLOT, "slots");
  static_assert(OFF_FB + 3 * 2 * A_FN <= SZ_AQ && 3 * 2 * A_FQ <= SZ_AQ && 4 * NFP16 * TILE * 4 <= SZ_AQ &&
                    4 * TILE * NP * 4 <= SZ_AQ && 4 * 2 * A_UCH <= SZ_X && SZ_FOPS <= SZ_X,
                "region plan");
  static_assert(SMEM <= 232448, "shared memory");
};

namespace {

// PLANAR: every element of the tiles this launch walks is affine (constant
// geometric factors and face normals, read once per element from compact
// tables); the others run with PLANAR = false.
template <int MODE, int FMT, int NQX, bool PLANAR = false>
__global__ void __launch_bounds__(kThreads, 1) stage_tc5_kernel(const TcStageParams P) {
  using OF = OpFmt<FMT>;
  using T = TcDims5<NQX>;
  constexpr int N = 5, NP = T::NP, NQ = T::NQ, NFP = T::NFP, NFQ = T::NFQ, KP = T::KP, QC = T::QC;
  constexpr int TILE = T::TILE, NFP16 = T::NFP16, NFQ16 = T::NFQ16, NCH = T::NCH;
  constexpr int NQ4 = (NQ + 3) / 4, NF4 = (NFQ + 3) / 4;
  const StageParams<float>& p = P.s;
  const DevOps<float>& ops = p.ops;

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAQ = smem;                                     // split fields, then b
  uint8_t* sFA = smem;                                     // face combinations (pass A), then the fluxes
  uint8_t* sFB = smem + T::OFF_FB;                         // face combinations (pass B)
  float* sLS = reinterpret_cast<float*>(smem);             // lifted face values [4][NFP16][128]
  float* sTT = reinterpret_cast<float*>(smem);             // output tile [4][128][NP], global row stride
  uint8_t* sAX = smem + T::OFF_X;                          // chunk arrays; the face operators during faces
  uint8_t* sFT = smem + T::OFF_X;
  int16_t* sGI = reinterpret_cast<int16_t*>(smem + T::OFF_GI);
  int16_t* sGX = reinterpret_cast<int16_t*>(smem + T::OFF_GX);
  uint4* sNB = reinterpret_cast<uint4*>(smem + T::OFF_NB);
  uint32_t* sC4 = reinterpret_cast<uint32_t*>(smem + T::OFF_NB + TILE * 16);
  float* sMean = reinterpret_cast<float*>(smem + T::OFF_MEAN);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + T::OFF_BAR);
  // bars: 0-3 operator slots, 4-5 first products of a chunk, 6 second products, 7 faces, 8 drain
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + T::OFF_BAR + 80);
  int* sflag = reinterpret_cast<int*>(smem + T::OFF_BAR + 84);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, grp = warp >> 2;
  const bool issuer = lane == 0;
  const int mrow = quarter * 32 + lane;
  const int64_t ncols = p.ncols;
  const int64_t fs = ncols * NP;
  const int S = p.S;
  const int64_t ntiles = (ncols + TILE - 1) / TILE;
  // the tiles this launch walks: all, or those of the list P.tiles
  const int64_t nwalk = P.tiles ? P.ntiles_list : ntiles;
  auto tile_at = [&](int64_t i) -> int64_t { return P.tiles ? (int64_t)P.tiles[i] : i; };

  if (tid == 0) {
    for (int i = 0; i < 9; ++i) tc::mbar_init(tc::smem_addr(bars + i), i < 4 ? 1 : kIssuers);
    *sflag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), 512);
  for (int i = tid; i < 4 * 6 * NP; i += kThreads) sGI[i] = ops.ginv[i];
  for (int i = tid; i < 4 * 6 * NFP; i += kThreads) sGX[i] = ops.gidx[i];
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
  const uint32_t bar0 = tc::smem_addr(bars);
  auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  uint32_t par_t1 = 0, par_m2 = 0, par_f = 0;
  uint32_t par_ld = 0, pend = 0;
  bool failed = false;

  const uint32_t aq = tc::smem_addr(sAQ), ax = tc::smem_addr(sAX), fa = tc::smem_addr(sFA), fb = tc::smem_addr(sFB);
  const uint32_t ft = tc::smem_addr(sFT);
  // slots: 0 = A part (16 KB), 1 = B part (16 KB); the update's second
  // buffers 2, 3 are the upper halves of 0, 1
  auto slot_addr = [&](int s) {
    return tc::smem_addr(smem + (s & 1 ? T::OFF_SB : T::OFF_SA) + (s >= 2 ? T::SZ_SLOT / 2 : 0));
  };
  const uint32_t sbo_KP = OF::sbo(KP), sbo_16 = OF::sbo(16);
  const uint8_t* vol_ops = P.ops;
  const uint8_t* upd_ops = P.ops + (size_t)NCH * T::SZ_OPV;

  auto live = [&]() { return *(volatile int*)sflag == 0; };
  auto load_slot = [&](int s, const uint8_t* src, int bytes) {  // thread 0
    if (!live()) return;
    tc::mbar_expect_tx(bar(s), (uint32_t)bytes);
    tc::bulk_g2s(slot_addr(s), src, (uint32_t)bytes, bar(s));
    pend |= 1u << s;
  };
  auto wait_slot = [&](int s) {
    if (issuer && !tc::mbar_wait(bar(s), (par_ld >> s) & 1u, kWaitIters)) atomicExch(sflag, 1);
    par_ld ^= 1u << s;
    pend &= ~(1u << s);
  };
  auto wait_all = [&](int b, uint32_t parity) {
    if (!tc::mbar_wait(bar(b), parity, kWaitIters)) atomicExch(sflag, 1);
    tc::fence_after();
  };
  auto sync_check = [&]() {
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    failed = *(volatile int*)sflag != 0;
  };
  // the first volume chunk's operators, loaded while the faces run
  auto prefetch_volume = [&]() {
    load_slot(0, vol_ops, T::SZ_VA);
    load_slot(1, vol_ops + T::SZ_VA, T::SZ_VB);
  };
  // volume products of chunk c: u_i = V_q u_i (warps 8-10, N = 16),
  // dp/dx^_a = V_q^a p (warp 11, N = 48)
  auto issue_V = [&](int c, int w) {
    if (!live()) return;
    const uint32_t sl = slot_addr(0), d = tmem + (uint32_t)((c & 1) * T::T1);
    const int i = w - 8;
    if (i >= 0 && i < 3)
      OF::template chain<KP>(mk_mma3(d + 16 * i, aq + (2 * (1 + i)) * T::A_FIELD, aq + (2 * (1 + i) + 1) * T::A_FIELD,
                                     sbo_KP, sl, sl + T::B_V, sbo_KP, OF::idesc(128, 16), false));
    else if (i == 3)
      OF::template chain<KP>(mk_mma3(d + 48, aq, aq + T::A_FIELD, sbo_KP, sl + 2 * T::B_V, sl + 5 * T::B_V, sbo_KP,
                                     OF::idesc(128, 48), false));
  };
  // test products of chunk c onto the surface terms: b_p += sum_a Dw_a U^a
  // (one accumulator, warp 0), b_ui += Vw g_i (warps 1-3)
  auto issue_DW = [&](int w) {
    if (!live()) return;
    const uint32_t sl = slot_addr(1), bvw = sl + 6 * T::B_P;
    if (w == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
        OF::template chain<16>(mk_mma3(tmem + T::TB, ax + (2 * a) * T::A_CH, ax + (2 * a + 1) * T::A_CH, sbo_16,
                                       sl + 2 * a * T::B_P, sl + (2 * a + 1) * T::B_P, sbo_16, OF::idesc(128, KP),
                                       true));
    } else if (w < 4) {
      OF::template chain<16>(mk_mma3(tmem + T::TB + KP * w, ax + (2 * (2 + w)) * T::A_CH,
                                     ax + (2 * (2 + w) + 1) * T::A_CH, sbo_16, bvw, bvw + T::B_P, sbo_16,
                                     OF::idesc(128, KP), true));
    }
  };
  auto ua_slot = [](int c) { return c & 1 ? 2 : 0; };
  auto ub_slot = [](int c) { return c & 1 ? 3 : 1; };
  auto issue_U1 = [&](int c, int w) {  // (V_q M^^{-1}) b per field (N = 16), warps 8-11
    if (!live()) return;
    const uint32_t sl = slot_addr(ua_slot(c)), d = tmem + (uint32_t)((c & 1) * T::T1U);
    const int f = w - 8;
    if (f >= 0 && f < 4)
      OF::template chain4<KP>(mk_mma4(d + T::UQC * f, aq + (2 * f) * T::A_FIELD, aq + (2 * f + 1) * T::A_FIELD, sbo_KP,
                                      sl, sl + T::B_UV, sl + 2 * T::B_UV, sbo_KP, OF::idesc(128, T::UQC), false));
  };
  auto issue_U2 = [&](int c, int f) {  // r += P_q (W ...) per field (N = 64, K = 16), warps 0-3
    if (!live()) return;
    const uint32_t sl = slot_addr(ub_slot(c));
    if (f < 4)
      OF::template chain4<T::UQC>(mk_mma4(tmem + T::TB + KP * f, ax + (2 * f) * T::A_UCH, ax + (2 * f + 1) * T::A_UCH,
                                          sbo_16, sl, sl + T::B_UP, sl + 2 * T::B_UP, sbo_16, OF::idesc(128, KP), c > 0));
  };
  // the tile's field ranges are 16-byte aligned (L2 prefetch of the epilogue's reads)
  const bool aligned = P.bulk_q != 0;

  if (tid == 0 && (int64_t)blockIdx.x < nwalk) prefetch_volume();

  for (int64_t iw = blockIdx.x; iw < nwalk && !failed; iw += gridDim.x) {
    const int64_t tile = tile_at(iw);
    const int64_t col0 = tile * TILE;
    const int ncol_t = (int)(ncols - col0 < TILE ? ncols - col0 : TILE);
    int64_t cm = col0 + mrow;
    cm = cm < ncols ? cm : ncols - 1;
    const int64_t km = cm / S;
    const int sh = (int)(cm - km * S);
    const uint32_t code4 = __ldg(reinterpret_cast<const unsigned int*>(p.fcode) + km);
    if (grp == 0) {
      const int4 e4 = __ldg(reinterpret_cast<const int4*>(p.EToE) + km);
      auto nbo = [&](int kn) {
        return kn >= 0 ? (uint32_t)(((int64_t)kn * S + sh) * NP) : ((uint32_t)(cm * NP) | 0x80000000u);
      };
      sNB[mrow] = make_uint4(nbo(e4.x), nbo(e4.y), nbo(e4.z), nbo(e4.w));
      sC4[mrow] = code4;
    }
    // face operators into region X (the previous tile's chunk arrays are free)
    stage_copy(sFT, P.ops + (size_t)T::SZ_OPS, T::SZ_FOPS);
    {  // the element mean of this thread's field and column (from global memory)
      float a = 0.f;
      const float* q = p.Qin + grp * fs + cm * NP;
      if (aligned) {
#pragma unroll
        for (int n4 = 0; n4 < NP / 4; ++n4) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(q) + n4);
          a += (v.x + v.y) + (v.z + v.w);
        }
      } else {
#pragma unroll 8
        for (int n = 0; n < NP; ++n) a += __ldg(q + n);
      }
      sMean[grp * TILE + mrow] = P.meanc ? a * (1.f / NP) : 0.f;
    }
    __syncthreads();

    // ---- surface terms (Sec. 4.1, Sec. 6.4), face by face, two passes ----
    float nv[3][12];  // n J^f at this thread's 12 face points (groups of four) of the current face
    auto load_nv = [&](int f) {
      if constexpr (PLANAR) {  // one n J^f per face
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
          const float v = __ldg(P.nP + ((km >> 7) * 12 + dd * 4 + f) * 128 + (km & 127));
#pragma unroll
          for (int j = 0; j < 12; ++j) nv[dd][j] = v;
        }
        return;
      }
      const float4* nfg = reinterpret_cast<const float4*>(P.fgeo_il) + (km >> 7) * 12 * NF4 * 128 + (km & 127);
#pragma unroll
      for (int dd = 0; dd < 3; ++dd)
#pragma unroll
        for (int h = 0; h < 3; ++h) {
          const int g = 3 * grp + h;
          const float4 v = g < NF4 ? __ldg(nfg + (size_t)((dd * 4 + f) * NF4 + g) * 128) : make_float4(0.f, 0.f, 0.f, 0.f);
          nv[dd][4 * h] = v.x;
          nv[dd][4 * h + 1] = v.y;
          nv[dd][4 * h + 2] = v.z;
          nv[dd][4 * h + 3] = v.w;
        }
    };
    // interpolant values of combination column block `col` (48 columns from
    // TMEM column base + col) at this thread's points q0 + 4 b4 + j
    auto ld_face4 = [&](uint32_t base, uint32_t (&v)[4]) { tc::tmem_ld4_nw(lane_base + base, v); };
    const int q0 = 12 * grp;

    for (int f = 0; f < 4 && !failed; ++f) {
      load_nv(f);
      // (i) [p], {u}, [u] at the face nodes in the owner's node order, own and
      // neighbour values from global memory; a warp takes the 32 (padded)
      // face nodes of one column
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        float qp[4][4], qm[4][4];
        bool bnd[4];
#pragma unroll
        for (int it = 0; it < 4; ++it) {
          const int r = (half * 4 + it) * 16 + (tid >> 5), j = lane;
          const uint32_t cd = (sC4[r] >> (8 * f)) & 0xffu;
          const int po = (int)(cd % 6), pn = (int)((cd / 6) % 6), fnb = (int)(cd / 36);
          const uint4 o4 = sNB[r];
          const uint32_t nbo = f == 0 ? o4.x : f == 1 ? o4.y : f == 2 ? o4.z : o4.w;
          const int jj = j < NFP ? j : 0;
          int64_t cr = col0 + r;
          cr = cr < ncols ? cr : ncols - 1;
          const int64_t b = (int64_t)(nbo & 0x7fffffffu) + sGX[(fnb * 6 + pn) * NFP + jj];
          const int64_t o = cr * NP + sGX[(f * 6 + po) * NFP + jj];
          bnd[it] = (nbo & 0x80000000u) != 0;
#pragma unroll
          for (int fl = 0; fl < 4; ++fl) {
            qp[it][fl] = __ldg(p.Qin + fl * fs + b);
            qm[it][fl] = __ldg(p.Qin + fl * fs + o);
          }
        }
#pragma unroll
        for (int it = 0; it < 4; ++it) {
          const int r = (half * 4 + it) * 16 + (tid >> 5), j = lane;
          const bool on = j < NFP;
          // Dirichlet ghost state on the boundary (Sec. 4.1): p+ = -p-, u+ = u-
          const float pp = bnd[it] ? -qm[it][0] : qp[it][0];
          OF::st1(sFA, T::A_FN, r, j, NFP16, on ? pp - qm[it][0] : 0.f);
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float up = bnd[it] ? qm[it][1 + i] : qp[it][1 + i];
            // {u} less the element mean
            OF::st1(sFA + (2 * (1 + i)) * T::A_FN, T::A_FN, r, j, NFP16,
                    on ? 0.5f * (up + qm[it][1 + i]) - sMean[(1 + i) * TILE + r] : 0.f);
            OF::st1(sFB + (2 * i) * T::A_FN, T::A_FN, r, j, NFP16, on ? up - qm[it][1 + i] : 0.f);
          }
        }
      }
      sync_check();
      if (failed) break;
      // (ii) pass A: [p], {u}_1..3 -> face points (warps 0-3, N = 48)
      if (issuer) {
        if (warp < 4 && live())
          OF::template chain<NFP16>(mk_mma3(tmem + T::TI + warp * NFQ16, fa + (2 * warp) * T::A_FN,
                                            fa + (2 * warp + 1) * T::A_FN, OF::sbo(NFP16), ft, ft + T::B_TRI,
                                            OF::sbo(NFP16), OF::idesc(128, NFQ16), false));
        tc::commit(bar(7));
      }
      wait_all(7, par_f);
      par_f ^= 1u;
      // pressure flux F_p = -{u}.n J^f + 1/2 tau_p [p] J^f at this thread's points
#pragma unroll
      for (int b4 = 0; b4 < 12; b4 += 4) {
        uint32_t v[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) ld_face4(T::TI + c * NFQ16 + q0 + b4, v[c]);
        tc::wait_ld();
#pragma unroll
        for (int c = 0; c < 4; ++c) tc::pin4(v[c]);
        float F[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float nx = nv[0][b4 + j], ny = nv[1][b4 + j], nz = nv[2][b4 + j];
          F[j] = 0.f;
          if (q0 + b4 + j < NFQ) {
            const float Jf = sqrtf(nx * nx + ny * ny + nz * nz);
            const float aun =
                __uint_as_float(v[1][j]) * nx + __uint_as_float(v[2][j]) * ny + __uint_as_float(v[3][j]) * nz;
            F[j] = -aun + 0.5f * p.tau_p * __uint_as_float(v[0][j]) * Jf;
          }
        }
        OF::st4(sFA, T::A_FQ, mrow, q0 + b4, NFQ16, F);
      }
      sync_check();
      if (failed) break;
      // lift of F_p (warp 8, N = 32) and pass B: [u]_1..3 -> face points into
      // the columns {u} held (warps 4-6)
      if (issuer) {
        if (warp == 8 && live())
          OF::template chain<NFQ16>(mk_mma3(tmem + T::TLP, fa, fa + T::A_FQ, OF::sbo(NFQ16), ft + 2 * T::B_TRI,
                                            ft + 3 * T::B_TRI, OF::sbo(NFQ16), OF::idesc(128, NFP16), false));
        if (warp >= 4 && warp < 7 && live())
          OF::template chain<NFP16>(mk_mma3(tmem + T::TI + (warp - 3) * NFQ16, fb + (2 * (warp - 4)) * T::A_FN,
                                            fb + (2 * (warp - 4) + 1) * T::A_FN, OF::sbo(NFP16), ft, ft + T::B_TRI,
                                            OF::sbo(NFP16), OF::idesc(128, NFQ16), false));
        tc::commit(bar(7));
      }
      wait_all(7, par_f);
      par_f ^= 1u;
      // velocity fluxes F_ui = -1/2 ([p] - tau_u [u].n) n_i J^f
#pragma unroll
      for (int b4 = 0; b4 < 12; b4 += 4) {
        uint32_t v[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) ld_face4(T::TI + c * NFQ16 + q0 + b4, v[c]);
        tc::wait_ld();
#pragma unroll
        for (int c = 0; c < 4; ++c) tc::pin4(v[c]);
        float F[3][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float nx = nv[0][b4 + j], ny = nv[1][b4 + j], nz = nv[2][b4 + j];
          F[0][j] = F[1][j] = F[2][j] = 0.f;
          if (q0 + b4 + j < NFQ) {
            const float nn = nx * nx + ny * ny + nz * nz;
            const float rJ = rsqrtf(nn);  // 1 / J^f (|n J^f| = J^f)
            const float jun =
                (__uint_as_float(v[1][j]) * nx + __uint_as_float(v[2][j]) * ny + __uint_as_float(v[3][j]) * nz) * rJ;
            const float sc = -0.5f * (__uint_as_float(v[0][j]) - p.tau_u * jun);
            F[0][j] = sc * nx;
            F[1][j] = sc * ny;
            F[2][j] = sc * nz;
          }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) OF::st4(sFA + (2 * i) * T::A_FQ, T::A_FQ, mrow, q0 + b4, NFQ16, F[i]);
      }
      sync_check();
      if (failed) break;
      // lifts of F_u1..3 (warps 8-10, N = 32) into the columns [p] and [u]_1 held
      if (issuer) {
        const int i = warp - 8;
        if (i >= 0 && i < 3 && live())
          OF::template chain<NFQ16>(mk_mma3(tmem + T::TLU + i * NFP16, fa + (2 * i) * T::A_FQ,
                                            fa + (2 * i + 1) * T::A_FQ, OF::sbo(NFQ16), ft + 2 * T::B_TRI,
                                            ft + 3 * T::B_TRI, OF::sbo(NFQ16), OF::idesc(128, NFP16), false));
        tc::commit(bar(7));
      }
      wait_all(7, par_f);
      par_f ^= 1u;
      // (iii) lifted values of field grp (owner's node order) -> this thread's
      // scratch -> the face's volume nodes, summed in the b accumulator
      {
        const int pio = (int)((code4 >> (8 * f)) & 0xffu) % 6;
        const uint32_t tl = grp == 0 ? T::TLP : T::TLU + (grp - 1) * NFP16;
        uint32_t L[NFP16 / 8][8];
#pragma unroll
        for (int j8 = 0; j8 < NFP16 / 8; ++j8) tc::tmem_ld8_nw(lane_base + tl + 8 * j8, L[j8]);
        tc::wait_ld();
#pragma unroll
        for (int j8 = 0; j8 < NFP16 / 8; ++j8) tc::pin8(L[j8]);
#pragma unroll
        for (int j = 0; j < NFP; ++j) sLS[(grp * NFP16 + j) * TILE + mrow] = __uint_as_float(L[j >> 3][j & 7]);
        const int16_t* gi = sGI + (f * 6 + pio) * NP;
        const uint32_t tb = lane_base + T::TB + KP * grp;
        auto add_face = [&](auto fc) {
          constexpr int F = decltype(fc)::value;
          constexpr FaceNodeList<N> FN = make_face_nodes<N>();
          constexpr uint32_t gm = F == 0 ? (1u << (KP / 8)) - 1u : face_group_mask<N, F>();
          uint32_t acc[KP / 8][8];
          if (F > 0) {
#pragma unroll
            for (int n8 = 0; n8 < KP / 8; ++n8)
              if (gm & (1u << n8)) tc::tmem_ld8_nw(tb + 8 * n8, acc[n8]);
            tc::wait_ld();
#pragma unroll
            for (int n8 = 0; n8 < KP / 8; ++n8)
              if (gm & (1u << n8)) tc::pin8(acc[n8]);
          } else {
#pragma unroll
            for (int n8 = 0; n8 < KP / 8; ++n8)
#pragma unroll
              for (int j = 0; j < 8; ++j) acc[n8][j] = 0u;
          }
#pragma unroll
          for (int t = 0; t < NFP; ++t) {
            const int n = FN.v[F][t];
            const int jj = gi[n];
            acc[n >> 3][n & 7] =
                __float_as_uint(__uint_as_float(acc[n >> 3][n & 7]) + sLS[(grp * NFP16 + jj) * TILE + mrow]);
          }
#pragma unroll
          for (int n8 = 0; n8 < KP / 8; ++n8)
            if (gm & (1u << n8)) {
              float v[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(acc[n8][j]);
              tc::tmem_st8(tb + 8 * n8, v);
            }
          tc::wait_st();
        };
        switch (f) {
          case 0: add_face(std::integral_constant<int, 0>()); break;
          case 1: add_face(std::integral_constant<int, 1>()); break;
          case 2: add_face(std::integral_constant<int, 2>()); break;
          default: add_face(std::integral_constant<int, 3>()); break;
        }
      }
      sync_check();  // the scratch is read before the next face's combinations overwrite it
      if (failed) break;
    }
    if (failed) break;

    // ---- field grp of this thread's column less its element mean -> split A
    // operand (from global memory) ----
    {
      const float4* q4 = reinterpret_cast<const float4*>(p.Qin + grp * fs + cm * NP);
      const float mu = sMean[grp * TILE + mrow];
#pragma unroll
      for (int n0 = 0; n0 < KP; n0 += 8) {
        float x[8];
        if (n0 + 8 <= NP) {
          const float4 a = __ldg(q4 + n0 / 4), b = __ldg(q4 + n0 / 4 + 1);
          x[0] = a.x - mu; x[1] = a.y - mu; x[2] = a.z - mu; x[3] = a.w - mu;
          x[4] = b.x - mu; x[5] = b.y - mu; x[6] = b.z - mu; x[7] = b.w - mu;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) x[j] = 0.f;
        }
        OF::st8(sAQ + (2 * grp) * T::A_FIELD, T::A_FIELD, mrow, n0, KP, x);
      }
    }
    sync_check();
    if (failed) break;

    // ---- volume terms (Sec. 6.4), chunks of 16 points: V(c + 1) runs on the
    // tensor cores while the CUDA cores form U^a, g_i of chunk c; one operator
    // slot of each kind ----
    float G[9][4];
    auto load_G = [&](int c) {
      if constexpr (PLANAR) {  // one G per element
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const float v = __ldg(P.gP + ((km >> 7) * 9 + k) * 128 + (km & 127));
          G[k][0] = G[k][1] = G[k][2] = G[k][3] = v;
        }
        return;
      }
      const float4* gk = reinterpret_cast<const float4*>(P.vgeo_il) + (km >> 7) * 11 * NQ4 * 128 + (km & 127);
      const int g = c * (QC / 4) + grp;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float4 v = g < NQ4 ? __ldg(gk + (size_t)(k * NQ4 + g) * 128) : make_float4(0.f, 0.f, 0.f, 0.f);
        G[k][0] = v.x;
        G[k][1] = v.y;
        G[k][2] = v.z;
        G[k][3] = v.w;
      }
    };
    load_G(0);
    wait_slot(0);
    if (issuer) {
      issue_V(0, warp);
      tc::commit(bar(4));
    }
    for (int c = 0; c < NCH; ++c) {
      wait_all(4 + (c & 1), (par_t1 >> (c & 1)) & 1u);
      par_t1 ^= 1u << (c & 1);
      // the A slot is free once V(c) has completed
      if (tid == 0 && c + 1 < NCH) load_slot(0, vol_ops + (size_t)(c + 1) * T::SZ_OPV, T::SZ_VA);
      float U[3][4], g[3][4];
      {
        const uint32_t t = lane_base + (uint32_t)((c & 1) * T::T1) + 4 * grp;
        uint32_t u[3][4], d[3][4];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          tc::tmem_ld4_nw(t + 16 * i, u[i]);
          tc::tmem_ld4_nw(t + 48 + 16 * i, d[i]);
        }
        tc::wait_ld();
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          tc::pin4(u[i]);
          tc::pin4(d[i]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float u0 = __uint_as_float(u[0][j]), u1 = __uint_as_float(u[1][j]), u2 = __uint_as_float(u[2][j]);
          const float d0 = __uint_as_float(d[0][j]), d1 = __uint_as_float(d[1][j]), d2 = __uint_as_float(d[2][j]);
#pragma unroll
          for (int a = 0; a < 3; ++a) U[a][j] = G[a * 3][j] * u0 + G[a * 3 + 1][j] * u1 + G[a * 3 + 2][j] * u2;
#pragma unroll
          for (int i = 0; i < 3; ++i) g[i][j] = -(G[i][j] * d0 + G[3 + i][j] * d1 + G[6 + i][j] * d2);
        }
      }
      if (c > 0) {  // the chunk arrays and the B slot are free once DW(c - 1) has completed
        wait_all(6, par_m2);
        par_m2 ^= 1u;
        if (tid == 0) load_slot(1, vol_ops + (size_t)c * T::SZ_OPV + T::SZ_VA, T::SZ_VB);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        OF::st4(sAX + (2 * a) * T::A_CH, T::A_CH, mrow, 4 * grp, QC, U[a]);
        OF::st4(sAX + (2 * (3 + a)) * T::A_CH, T::A_CH, mrow, 4 * grp, QC, g[a]);
      }
      sync_check();
      if (failed) break;
      if (c + 1 < NCH) load_G(c + 1);
      wait_slot(1);
      if (issuer) {
        issue_DW(warp);
        tc::commit(bar(6));
      }
      if (c + 1 < NCH) {
        wait_slot(0);
        if (issuer) {
          issue_V(c + 1, warp);
          tc::commit(bar(4 + ((c + 1) & 1)));
        }
      }
    }
    if (failed) break;
    wait_all(6, par_m2);
    par_m2 ^= 1u;
    if (tid == 0) {  // update operators of chunks 0 and 1
      if (aligned) {
        // the epilogue's reads of Q_in and res (and of the mean correction
        // when a column is one element) for this tile, into L2 while the update runs
        const uint32_t bytes = (uint32_t)(ncol_t * NP * 4);
        if (MODE == kLsrk)
          for (int f = 0; f < 4; ++f) {
            tc::bulk_prefetch_l2(p.Qin + f * fs + col0 * NP, bytes);
            if (p.rk_a != 0.f) tc::bulk_prefetch_l2(p.res + f * fs + col0 * NP, bytes);
          }
        if (P.meanc && S == 1)
          for (int i = 0; i < 3; ++i) tc::bulk_prefetch_l2(P.meanc + i * P.meanc_stride + col0 * NP, bytes);
      }
      load_slot(ua_slot(0), upd_ops, T::SZ_UA);
      load_slot(ub_slot(0), upd_ops + T::SZ_UA, T::SZ_UB);
      if (T::UNCH > 1) {
        load_slot(ua_slot(1), upd_ops + T::SZ_OPU, T::SZ_UA);
        load_slot(ub_slot(1), upd_ops + T::SZ_OPU + T::SZ_UA, T::SZ_UB);
      }
    }

    // ---- b of field grp (+ point source, Sec. 4.1 load vector) -> split A operand ----
    {
      const bool src = grp == 0 && p.src_elem != nullptr && p.src_elem[sh] == (int32_t)km;
#pragma unroll
      for (int n0 = 0; n0 < KP; n0 += 8) {
        uint32_t v[8];
        tc::tmem_ld8_nw(lane_base + T::TB + KP * grp + n0, v);
        tc::wait_ld();
        tc::pin8(v);
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float b = __uint_as_float(v[j]) + (src && n0 + j < NP ? p.src_amp * p.src_vec[sh * NP + n0 + j] : 0.f);
          x[j] = n0 + j < NP ? b : 0.f;
        }
        OF::st8(sAQ + (2 * grp) * T::A_FIELD, T::A_FIELD, mrow, n0, KP, x);
      }
    }
    sync_check();
    if (failed) break;

    // ---- weight-adjusted update (Sec. 6.2, Eq. (matfree); Sec. 7), chunks of 16 points ----
    constexpr int UQC = T::UQC, UNCH = T::UNCH;
    float wt[UQC];
    auto load_W = [&](int c) {
      const float4* w =
          reinterpret_cast<const float4*>(P.vgeo_il) + ((km >> 7) * 11 + (grp == 0 ? 9 : 10)) * NQ4 * 128 + (km & 127);
#pragma unroll
      for (int h = 0; h < UQC / 4; ++h) {
        const int g = c * (UQC / 4) + h;
        const float4 v = g < NQ4 ? __ldg(w + (size_t)g * 128) : make_float4(0.f, 0.f, 0.f, 0.f);
        wt[4 * h] = v.x;
        wt[4 * h + 1] = v.y;
        wt[4 * h + 2] = v.z;
        wt[4 * h + 3] = v.w;
      }
    };
    load_W(0);
    wait_slot(ua_slot(0));
    if (issuer) {
      issue_U1(0, warp);
      tc::commit(bar(4));
    }
    if (UNCH > 1) {
      wait_slot(ua_slot(1));
      if (issuer) {
        issue_U1(1, warp);
        tc::commit(bar(5));
      }
    }
    for (int c = 0; c < UNCH; ++c) {
      wait_all(4 + (c & 1), (par_t1 >> (c & 1)) & 1u);
      par_t1 ^= 1u << (c & 1);
      if (tid == 0 && c + 2 < UNCH) load_slot(ua_slot(c), upd_ops + (size_t)(c + 2) * T::SZ_OPU, T::SZ_UA);
      float x[UQC / 8][8];
      {
        const uint32_t t = lane_base + (uint32_t)((c & 1) * T::T1U) + UQC * grp;
        uint32_t v[UQC / 8][8];
#pragma unroll
        for (int h8 = 0; h8 < UQC / 8; ++h8) tc::tmem_ld8_nw(t + 8 * h8, v[h8]);
        tc::wait_ld();
#pragma unroll
        for (int h8 = 0; h8 < UQC / 8; ++h8) {
          tc::pin8(v[h8]);
#pragma unroll
          for (int j = 0; j < 8; ++j) x[h8][j] = __uint_as_float(v[h8][j]) * wt[8 * h8 + j];
        }
      }
      if (c > 0) {
        wait_all(6, par_m2);
        par_m2 ^= 1u;
        if (tid == 0 && c + 1 < UNCH)
          load_slot(ub_slot(c + 1), upd_ops + (size_t)(c + 1) * T::SZ_OPU + T::SZ_UA, T::SZ_UB);
      }
#pragma unroll
      for (int h8 = 0; h8 < UQC / 8; ++h8) OF::st8(sAX + (2 * grp) * T::A_UCH, T::A_UCH, mrow, 8 * h8, UQC, x[h8]);
      sync_check();
      if (failed) break;
      if (c + 1 < UNCH) load_W(c + 1);
      wait_slot(ub_slot(c));
      if (issuer) {
        issue_U2(c, warp);
        tc::commit(bar(6));
      }
      if (c + 2 < UNCH) {
        wait_slot(ua_slot(c));
        if (issuer) {
          issue_U1(c + 2, warp);
          tc::commit(bar(4 + (c & 1)));
        }
      }
    }
    if (failed) break;
    wait_all(6, par_m2);
    par_m2 ^= 1u;
    if (tid == 0 && iw + gridDim.x < nwalk) prefetch_volume();  // the slots are free

    // ---- epilogue: r -> FP32 tile -> coalesced dQ/dt, or the LSRK update (Sec. 5.2) ----
    // The tile has the global row stride (NP = 56, a multiple of 8): each
    // thread writes its row as float4s (two-way bank conflicts at stride 224 B)
#pragma unroll
    for (int n0 = 0; n0 < NP; n0 += 8) {
      uint32_t v[8];
      tc::tmem_ld8_nw(lane_base + T::TB + KP * grp + n0, v);
      tc::wait_ld();
      tc::pin8(v);
      float4* d = reinterpret_cast<float4*>(sTT + (grp * TILE + mrow) * NP + n0);
      d[0] = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]), __uint_as_float(v[3]));
      d[1] = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]), __uint_as_float(v[6]), __uint_as_float(v[7]));
    }
    sync_check();
    // r_p += sum_i ubar_i D_i (the element-constant velocity's term, in FP32)
    // at entry r = c NP + n of the tile's p field
    const int64_t mst = P.meanc_stride;
    auto corr1 = [&](int r) -> float {
      if (!P.meanc) return 0.f;
      const int c = r / NP, n = r - c * NP;
      const float* d = P.meanc + ((col0 + c) / S) * NP + n;
      return sMean[TILE + c] * __ldg(d) + sMean[2 * TILE + c] * __ldg(d + mst) +
             sMean[3 * TILE + c] * __ldg(d + 2 * mst);
    };
    // four entries of one column (NP is a multiple of 4)
    auto corr4 = [&](int r4) -> float4 {
      if (!P.meanc) return make_float4(0.f, 0.f, 0.f, 0.f);
      const int c = 4 * r4 / NP, n = 4 * r4 - c * NP;
      const float4* d = reinterpret_cast<const float4*>(P.meanc + ((col0 + c) / S) * NP + n);
      const float4 a = __ldg(d), b = __ldg(d + mst / 4), e = __ldg(d + mst / 2);
      const float m1 = sMean[TILE + c], m2 = sMean[2 * TILE + c], m3 = sMean[3 * TILE + c];
      return make_float4(m1 * a.x + m2 * b.x + m3 * e.x, m1 * a.y + m2 * b.y + m3 * e.y,
                         m1 * a.z + m2 * b.z + m3 * e.z, m1 * a.w + m2 * b.w + m3 * e.w);
    };
    if (aligned) {
      // 16-byte global accesses: every field range of the tile starts 16-byte aligned
      constexpr int F4 = TILE * NP / 4, NIT4 = (4 * F4 + kThreads - 1) / kThreads;
      const int nval4 = ncol_t * NP / 4;
      const float4* sT4 = reinterpret_cast<const float4*>(sTT);
      if (MODE == kRhs) {
#pragma unroll 7
        for (int it = 0; it < NIT4; ++it) {
          const int i = tid + it * kThreads, f = i / F4, r4 = i - f * F4;
          if (i < 4 * F4 && r4 < nval4) {
            float4 v = sT4[f * F4 + r4];
            if (f == 0) {
              const float4 c = corr4(r4);
              v.x += c.x;
              v.y += c.y;
              v.z += c.z;
              v.w += c.w;
            }
            reinterpret_cast<float4*>(p.out + f * fs + col0 * NP)[r4] = v;
          }
        }
      } else {
        // LSRK: res = a res + dt r, Q_out = Q_in + b res; the loads of EB4
        // iterations are issued before their stores
        constexpr int EB4 = 7;
        const bool rd = p.rk_a != 0.f;
        for (int i0 = 0; i0 < NIT4; i0 += EB4) {
          float4 vv[EB4], rs[EB4], qi[EB4];
          int64_t ix[EB4];
#pragma unroll
          for (int e = 0; e < EB4; ++e) {
            const int i = tid + (i0 + e) * kThreads, f = i / F4, r4 = i - f * F4;
            const bool ok = i0 + e < NIT4 && i < 4 * F4 && r4 < nval4;
            ix[e] = ok ? (f * fs + col0 * NP) / 4 + r4 : -1;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            vv[e] = ok ? sT4[f * F4 + r4] : z;
            if (ok && f == 0) {
              const float4 c = corr4(r4);
              vv[e].x += c.x;
              vv[e].y += c.y;
              vv[e].z += c.z;
              vv[e].w += c.w;
            }
            rs[e] = ok && rd ? __ldg(reinterpret_cast<const float4*>(p.res) + ix[e]) : z;
            qi[e] = ok ? __ldg(reinterpret_cast<const float4*>(p.Qin) + ix[e]) : z;
          }
#pragma unroll
          for (int e = 0; e < EB4; ++e) {
            if (ix[e] < 0) continue;
            float4 rr;
            rr.x = rd ? p.rk_a * rs[e].x + p.dt * vv[e].x : p.dt * vv[e].x;
            rr.y = rd ? p.rk_a * rs[e].y + p.dt * vv[e].y : p.dt * vv[e].y;
            rr.z = rd ? p.rk_a * rs[e].z + p.dt * vv[e].z : p.dt * vv[e].z;
            rr.w = rd ? p.rk_a * rs[e].w + p.dt * vv[e].w : p.dt * vv[e].w;
            reinterpret_cast<float4*>(p.res)[ix[e]] = rr;
            if (p.qlo) {
              float4 l = reinterpret_cast<const float4*>(p.qlo)[ix[e]];
              reinterpret_cast<float4*>(p.Qout)[ix[e]] =
                  make_float4(lsrk_comp(qi[e].x, p.rk_b, rr.x, l.x), lsrk_comp(qi[e].y, p.rk_b, rr.y, l.y),
                              lsrk_comp(qi[e].z, p.rk_b, rr.z, l.z), lsrk_comp(qi[e].w, p.rk_b, rr.w, l.w));
              reinterpret_cast<float4*>(p.qlo)[ix[e]] = l;
            } else {
              reinterpret_cast<float4*>(p.Qout)[ix[e]] =
                  make_float4(qi[e].x + p.rk_b * rr.x, qi[e].y + p.rk_b * rr.y, qi[e].z + p.rk_b * rr.z,
                              qi[e].w + p.rk_b * rr.w);
            }
          }
        }
      }
    } else {
      const int nval = ncol_t * NP;
      if (MODE == kRhs) {
#pragma unroll 4
        for (int i = tid; i < 4 * TILE * NP; i += kThreads) {
          const int f = i / (TILE * NP), r = i - f * (TILE * NP);
          if (r < nval) p.out[f * fs + col0 * NP + r] = sTT[i] + (f == 0 ? corr1(r) : 0.f);
        }
      } else {
        constexpr int NIT = (4 * TILE * NP + kThreads - 1) / kThreads, EB = 7;
        const bool rd = p.rk_a != 0.f;
        for (int i0 = 0; i0 < NIT; i0 += EB) {
          float vv[EB], rs[EB], qi[EB];
          int64_t ix[EB];
#pragma unroll
          for (int e = 0; e < EB; ++e) {
            const int i = tid + (i0 + e) * kThreads;
            const int f = i / (TILE * NP), r = i - f * (TILE * NP);
            const bool ok = i0 + e < NIT && i < 4 * TILE * NP && r < nval;
            ix[e] = ok ? f * fs + col0 * NP + r : -1;
            vv[e] = ok ? sTT[i] + (f == 0 ? corr1(r) : 0.f) : 0.f;
            rs[e] = ok && rd ? __ldg(p.res + ix[e]) : 0.f;
            qi[e] = ok ? __ldg(p.Qin + ix[e]) : 0.f;
          }
#pragma unroll
          for (int e = 0; e < EB; ++e) {
            if (ix[e] < 0) continue;
            const float rr = rd ? p.rk_a * rs[e] + p.dt * vv[e] : p.dt * vv[e];
            p.res[ix[e]] = rr;
            if (p.qlo) {
              float l = p.qlo[ix[e]];
              p.Qout[ix[e]] = lsrk_comp(qi[e], p.rk_b, rr, l);
              p.qlo[ix[e]] = l;
            } else {
              p.Qout[ix[e]] = qi[e] + p.rk_b * rr;
            }
          }
        }
      }
    }
    __syncthreads();
  }

  // drain: operator copies still in flight and every issued product
  if (tid == 0) {
    for (int s = 0; s < 4; ++s)
      if (pend & (1u << s)) tc::mbar_wait(bar(s), (par_ld >> s) & 1u, kWaitIters);
  }
  if (issuer) {
    tc::commit(bar(8));
    tc::mbar_wait(bar(8), 0, kWaitIters);
  }
  __syncthreads();
  if (tid == 0 && *(volatile int*)sflag != 0) atomicExch(P.err, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

template <int MODE, int FMT, int NQX, bool PLANAR>
cudaError_t launch5(const TcStageParams& P, int grid, cudaStream_t stream) {
  using T = TcDims5<NQX>;
  auto kern = stage_tc5_kernel<MODE, FMT, NQX, PLANAR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, T::SMEM, stream>>>(P);
  return cudaGetLastError();
}

}  // namespace

template <int NQX, bool PLANAR>
cudaError_t launch_stage_tc5_q(const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream) {
  using T = TcDims5<NQX>;
  const int64_t ntiles = P.tiles ? P.ntiles_list : (P.s.ncols + T::TILE - 1) / T::TILE;
  if (ntiles == 0) return cudaSuccess;
  const int g = (int)(ntiles < grid ? ntiles : grid);
  if (mode == kRhs)
    return fmt == 0 ? launch5<kRhs, 0, NQX, PLANAR>(P, g, stream) : launch5<kRhs, 1, NQX, PLANAR>(P, g, stream);
  return fmt == 0 ? launch5<kLsrk, 0, NQX, PLANAR>(P, g, stream) : launch5<kLsrk, 1, NQX, PLANAR>(P, g, stream);
}

// N = 5 on the collapsed (N+1)^3 = 216-point volume rule or on the
// fewer-point symmetric rule exact to degree 11.
template <bool PLANAR>
cudaError_t launch_stage_tc5_n(const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream) {
  if (P.s.nq == 216) return launch_stage_tc5_q<216, PLANAR>(P, mode, fmt, grid, stream);
  if (P.s.nq == fewer_point_nq(5)) return launch_stage_tc5_q<fewer_point_nq(5), PLANAR>(P, mode, fmt, grid, stream);
  return cudaErrorInvalidValue;
}

}  // namespace wadg
