// Fused WADG stage on the 5th-generation tensor cores: FP32 fields, the dense
// products as tcgen05.mma with FP32 accumulation in TMEM, operands either split
// bf16 (x = hi + lo, a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi) or tf32.
//
// A persistent CTA (512 threads, one per SM) walks tiles of 128 columns
// (element, shot).  A column is one MMA row (M = 128) and one TMEM lane; four
// threads share it (warps w, w + 4, w + 8, w + 12 own the lanes of quarter w),
// each taking one field or a quarter of the points.  The reference operators
// are the B operands (N = operator rows), packed on the host in the K-major
// no-swizzle core-matrix layout (see tc_ops.cuh) and streamed from L2 into
// four shared-memory slots by bulk asynchronous copies ahead of use.  Per tile:
//   fields -> an FP32 tile (bulk copies issued during the previous tile);
//   surface (Sec. 4.1, Sec. 6.4), face by face: 16 lanes gather the face nodes
//     of one column ([p], {u}, [u] in the owner's node order), V_tri products
//     to the face points, the strong-weak flux with n J^f on the CUDA cores,
//     lift products, and the lifted values scattered to the face's volume
//     nodes (lists fixed at compile time) and summed in the b accumulators in
//     TMEM;
//   volume (Sec. 6.4), chunks of 16 points, software-pipelined: V_q u_i and
//     V_q^a p of chunk c + 2 and the test products of chunk c run on the tensor
//     cores while the CUDA cores form U^a = sum_i G_ai u_i and
//     g_i = -sum_a G_ai dp/dx^_a of chunk c + 1;
//   update (Sec. 6.2, Eq. (matfree); Sec. 7), chunks of 32 points: b -> V_q
//     M^^{-1} b, times W = c^2/J or 1/J, P_q (...) accumulated in TMEM;
//   epilogue: dQ/dt, or the LSRK update (Sec. 5.2), written coalesced; in
//     LSRK mode the tile's Q_in and res are prefetched into L2 during the
//     update and read several iterations ahead of the stores.
// The volume rule has NQ points (the collapsed (N+1)^3 rule or a fewer-point
// symmetric rule), a template parameter.
// Geometric factors come from copies interleaved over 128 elements in groups
// of four points (one 16-byte load per four points).  Every tcgen05.mma holds
// its issuing thread for 100-200 cycles, so lane 0 of every warp issues at
// most one accumulator chain per step.  Waits on the tensor cores and the bulk
// copies are bounded; on expiry the CTA records an error in P.err, issues no
// further copies or products, waits (again bounded) for those already issued,
// frees its TMEM and returns.  The report is best effort: work still in flight
// when the drain's own bound runs out is not waited for.
#pragma once

#include "tc_stage_common.cuh"

namespace wadg {

template <int N, int NQX = (N + 1) * (N + 1) * (N + 1)>
struct TcDims {
  using D = Dims<N, NQX>;
  static constexpr int NP = D::NP, NQ = D::NQ, NFP = D::NFP, NFQ = D::NFQ;
  static constexpr int KP = (NP + 15) / 16 * 16;  // node count padded to the MMA K / N granule
  static constexpr int NPS = NP | 1;              // odd row stride of FP32 tiles in shared memory
  static constexpr int QC = 16;                   // quadrature points per chunk
  static constexpr int NCH = (NQ + QC - 1) / QC;
  static constexpr int TILE = 128;
  static constexpr int A_FIELD = TILE * KP * 2;   // bytes of one bf16 part of one [128 x KP] field tile
  static constexpr int SZ_AQ = 4 * 2 * A_FIELD;
  static constexpr int A_CH = TILE * QC * 2;      // one part of a [128 x 16] chunk array
  static constexpr int SZ_AX = 6 * 2 * A_CH;
  static constexpr int B_V = QC * KP * 2;         // one part of a [16 x KP] operator chunk
  static constexpr int B_P = KP * QC * 2;         // one part of a [KP x 16] operator chunk
  // packed operators per chunk: volume A part (V_q, V_q^a), volume B part
  // ((V_q^a)^T diag(w), V_q^T diag(w)), update A part (V_q M^^{-1}), update B part (P_q)
  // the update runs in chunks of 32 points (its four outputs per point fit
  // twice in TMEM beside the r accumulators)
  static constexpr int UQC = 32;
  static constexpr int UNCH = (NQ + UQC - 1) / UQC;
  static constexpr int A_UCH = TILE * UQC * 2;    // one part of a [128 x 32] update chunk array
  static constexpr int B_UV = UQC * KP * 2;       // one part of a [32 x KP] operator chunk
  static constexpr int B_UP = KP * UQC * 2;       // one part of a [KP x 32] operator chunk
  // the update operators in three bf16 parts (the fourth product of mma4_chain)
  static constexpr int SZ_VA = 8 * B_V, SZ_VB = 8 * B_P, SZ_UA = 3 * B_UV, SZ_UB = 3 * B_UP;
  static constexpr int SZ_OPV = SZ_VA + SZ_VB, SZ_OPU = SZ_UA + SZ_UB;
  static constexpr int SZ_OPS = NCH * SZ_OPV + UNCH * SZ_OPU;  // packed chunks before the face operators
  static constexpr int SZ_SLOT = SZ_VA > SZ_VB ? (SZ_VA > SZ_UA ? SZ_VA : SZ_UA) : (SZ_VB > SZ_UA ? SZ_VB : SZ_UA);
  static constexpr int NFP16 = (NFP + 15) / 16 * 16, NFQ16 = (NFQ + 15) / 16 * 16;
  static constexpr int A_FN = TILE * NFP16 * 2;    // one part of a [128 x NFP16] face-node tile
  static constexpr int A_FQ = TILE * NFQ16 * 2;    // one part of a [128 x NFQ16] face-point tile
  static constexpr int SZ_FA = (7 * 2 * A_FN > 4 * 2 * A_FQ ? 7 * 2 * A_FN : 4 * 2 * A_FQ);
  static constexpr int SZ_LS = 4 * NFP16 * TILE * 4;  // lifted face values, [4][NFP16][128] FP32
  static constexpr int SZ_T32 = 4 * TILE * NPS * 4;   // FP32 field tile [4][128][NPS]
  static constexpr int R0A = SZ_AQ > SZ_FA + SZ_LS ? SZ_AQ : SZ_FA + SZ_LS;
  static constexpr int SZ_R0 = ((R0A > SZ_T32 ? R0A : SZ_T32) + 127) / 128 * 128;
  static constexpr int OFF_SLOT = SZ_R0;
  static constexpr int OFF_AX = OFF_SLOT + 4 * SZ_SLOT;
  static constexpr int OFF_QS = OFF_AX;  // FP32 input tile: from the load to the split (before the volume)
  static constexpr int END_AX = OFF_AX + SZ_AX, END_QS = OFF_QS + SZ_T32, END_UX = OFF_AX + 8 * A_UCH;
  static constexpr int END_X = END_AX > END_QS ? (END_AX > END_UX ? END_AX : END_UX) : (END_QS > END_UX ? END_QS : END_UX);
  static constexpr int OFF_FT = (END_X + 127) / 128 * 128;
  static constexpr int B_TRI = NFQ16 * NFP16 * 2;  // one part of V_tri [NFQ16 x NFP16] or of its lift
  static constexpr int SZ_FOPS = 4 * B_TRI;
  static constexpr int OFF_GI = OFF_FT + SZ_FOPS;
  static constexpr int SZ_GI = (4 * 6 * NP * 2 + 15) / 16 * 16;
  static constexpr int OFF_GX = OFF_GI + SZ_GI;
  static constexpr int SZ_GX = (4 * 6 * NFP * 2 + 15) / 16 * 16;
  // per tile column: offset of each face's neighbour column (4 x uint32, top bit: boundary), face codes,
  // the neighbour's row in the tile (4 x uint8, 0xff: outside the tile)
  static constexpr int OFF_NB = OFF_GX + SZ_GX;
  static constexpr int OFF_MEAN = OFF_NB + TILE * 24;  // element means of the tile's columns [4][128]
  static constexpr int OFF_BAR = OFF_MEAN + 4 * TILE * 4;
  static constexpr int SMEM = OFF_BAR + 128;
  // TMEM columns
  static constexpr int T1 = 96;                    // volume chunk outputs, two buffers at 0 and T1
  static constexpr int T1U = 128;                  // update chunk outputs (4 x 32), two buffers at 0 and T1U
  static constexpr int TB = 320;                   // b accumulators b_p (a = r), b_u1..3 (4 x KP), then r
  static constexpr int TBX = 224;                  // b_p for a = s, t (2 x KP), summed into b_p
  static constexpr int TI = 0, TL = 7 * NFQ16;     // face interpolants (7 x NFQ16), lifted faces (4 x NFP16)
  static_assert(2 * T1 <= TBX && TBX + 2 * KP <= TB && TB + 4 * KP <= 512 && TL + 4 * NFP16 <= TB, "TMEM plan");
  static_assert(2 * T1U <= TB && SZ_UA <= SZ_SLOT && SZ_UB <= SZ_SLOT, "update plan");
  static_assert(SMEM <= 232448, "shared memory");
};


// PLANAR: every element of the tiles this launch walks is affine (constant
// geometric factors and face normals, read once per element from compact
// tables); the others run with PLANAR = false.
template <int N, int MODE, int FMT, int NQX, bool PLANAR = false>
__global__ void __launch_bounds__(kThreads, 1) stage_tc_kernel(const TcStageParams P) {
  using OF = OpFmt<FMT>;
  using T = TcDims<N, NQX>;
  constexpr int NP = T::NP, NQ = T::NQ, NFP = T::NFP, NFQ = T::NFQ, KP = T::KP, QC = T::QC, NPS = T::NPS;
  constexpr int TILE = T::TILE, NFP16 = T::NFP16, NFQ16 = T::NFQ16, NCH = T::NCH;
  constexpr int NQ4 = (NQ + 3) / 4, NF4 = (NFQ + 3) / 4;  // groups of four points in the interleaved geometry
  static_assert(NFP16 == 16, "the face gather maps 8 lanes x 2 nodes to the 16 padded face nodes");
  const StageParams<float>& p = P.s;
  const DevOps<float>& ops = p.ops;

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAQ = smem;                                        // A operand: fields, then b
  uint8_t* sFA = smem;                                        // per face: combinations, then fluxes
  float* sLS = reinterpret_cast<float*>(smem + T::SZ_FA);     // per face: lifted values [4][NFP16][128]
  float* sTT = reinterpret_cast<float*>(smem);                // output tile [4][128][NPS]
  uint8_t* sAX = smem + T::OFF_AX;                            // A operand: chunk arrays
  float* sQS = reinterpret_cast<float*>(smem + T::OFF_QS);    // input tile [4][128][NPS]
  uint8_t* sFT = smem + T::OFF_FT;                            // face B operands
  int16_t* sGI = reinterpret_cast<int16_t*>(smem + T::OFF_GI);  // ginv [4][6][NP]
  int16_t* sGX = reinterpret_cast<int16_t*>(smem + T::OFF_GX);  // gidx [4][6][NFP]
  uint4* sNB = reinterpret_cast<uint4*>(smem + T::OFF_NB);                     // [128] neighbour offsets
  uint32_t* sC4 = reinterpret_cast<uint32_t*>(smem + T::OFF_NB + TILE * 16);   // [128] face codes
  uint32_t* sIT = reinterpret_cast<uint32_t*>(smem + T::OFF_NB + TILE * 20);   // [128] neighbour rows in the tile
  float* sMean = reinterpret_cast<float*>(smem + T::OFF_MEAN);                  // [4][128] element means
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + T::OFF_BAR);
  // bars: 0-3 operator slots, 4-5 first products of a chunk, 6 second products, 7 faces, 8 drain, 9 fields
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + T::OFF_BAR + 80);
  int* sflag = reinterpret_cast<int*>(smem + T::OFF_BAR + 84);

  // Four threads per column: warps w, w + 4, w + 8, w + 12 share the TMEM lanes
  // of quarter w; the group g = w / 4 takes field g, or a quarter of the points.
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, grp = warp >> 2;
  const bool issuer = lane == 0;  // lane 0 of every warp issues at most one accumulator chain per step
  const int mrow = quarter * 32 + lane;  // this thread's column within the tile (TMEM lane)
  const int64_t ncols = p.ncols;
  const int64_t fs = ncols * NP;
  const int S = p.S;
  const int64_t ntiles = (ncols + TILE - 1) / TILE;
  // the tiles this launch walks: all of them, or the entries of a tile list
  const int64_t nwalk = P.tiles ? P.ntiles_list : ntiles;
  auto tile_at = [&](int64_t i) -> int64_t { return P.tiles ? (int64_t)P.tiles[i] : i; };

  if (tid == 0) {
    for (int i = 0; i < 10; ++i) tc::mbar_init(tc::smem_addr(bars + i), i < 4 || i == 9 ? 1 : kIssuers);
    *sflag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), 512);
  stage_copy(sFT, P.ops + (size_t)T::SZ_OPS, T::SZ_FOPS);
  for (int i = tid; i < 4 * 6 * NP; i += kThreads) sGI[i] = ops.ginv[i];
  for (int i = tid; i < 4 * 6 * NFP; i += kThreads) sGX[i] = ops.gidx[i];
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
  const uint32_t bar0 = tc::smem_addr(bars);
  auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  uint32_t par_t1 = 0, par_m2 = 0, par_f = 0;  // phase parities (uniform)
  uint32_t par_ld = 0, pend = 0;               // operator slots (loads by thread 0)
  bool failed = false;

  const uint32_t aq = tc::smem_addr(sAQ), ax = tc::smem_addr(sAX), fa = tc::smem_addr(sFA);
  const uint32_t ft = tc::smem_addr(sFT), slots = tc::smem_addr(smem + T::OFF_SLOT);
  auto slot_addr = [&](int s) { return slots + (uint32_t)(s * T::SZ_SLOT); };
  const uint32_t sbo_KP = OF::sbo(KP), sbo_16 = OF::sbo(16);
  const uint8_t* vol_ops = P.ops;
  const uint8_t* upd_ops = P.ops + (size_t)NCH * T::SZ_OPV;

  // once a wait has expired (sflag set) no further copy or product is issued,
  // so the drain at the end only waits for work issued before the failure
  auto live = [&]() { return *(volatile int*)sflag == 0; };
  // thread 0: operator slots (bulk copies completing on bars[s])
  auto load_slot = [&](int s, const uint8_t* src, int bytes) {
    if (!live()) return;
    tc::mbar_expect_tx(bar(s), (uint32_t)bytes);
    tc::bulk_g2s(slot_addr(s), src, (uint32_t)bytes, bar(s));
    pend |= 1u << s;
  };
  // every thread: the issuers wait for a slot's copy before reading it
  auto wait_slot = [&](int s) {
    if (issuer && !tc::mbar_wait(bar(s), (par_ld >> s) & 1u, kWaitIters)) atomicExch(sflag, 1);
    par_ld ^= 1u << s;
    pend &= ~(1u << s);
  };
  auto prefetch_volume = [&]() {
    load_slot(0, vol_ops, T::SZ_VA);
    load_slot(2, vol_ops + T::SZ_VA, T::SZ_VB);
    if (NCH > 1) {
      load_slot(1, vol_ops + T::SZ_OPV, T::SZ_VA);
      load_slot(3, vol_ops + T::SZ_OPV + T::SZ_VA, T::SZ_VB);
    }
  };
  // every thread: bounded wait on an mbarrier phase
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
  // Products of chunk c, one accumulator chain per issuing warp w: the V and
  // U1 chains (9 instructions each at N = 4) on warps 8-11, the DW and U2
  // chains (3 each) on warps 0-5.
  auto issue_V = [&](int c, int w) {  // u_i = V_q u_i (N = 16 each), dp/dx^_a = V_q^a p (N = 48)
    if (!live()) return;
    const uint32_t sl = slot_addr(c & 1), d = tmem + (uint32_t)((c & 1) * T::T1);
    const int i = w - 8;
    if (i >= 0 && i < 3)
      OF::template chain<KP>(mk_mma3(d + 16 * i, aq + (2 * (1 + i)) * T::A_FIELD, aq + (2 * (1 + i) + 1) * T::A_FIELD,
                                  sbo_KP, sl, sl + T::B_V, sbo_KP, OF::idesc(128, 16), false));
    else if (i == 3)
      OF::template chain<KP>(mk_mma3(d + 48, aq, aq + T::A_FIELD, sbo_KP, sl + 2 * T::B_V, sl + 5 * T::B_V, sbo_KP,
                                  OF::idesc(128, 48), false));
  };
  // b_p += sum_a Dw_a U^a (one accumulator per a; a = r holds the surface
  // term), b_ui += Vw g_i (onto the surface terms)
  auto issue_DW = [&](int c, int i) {
    if (!live()) return;
    const uint32_t sl = slot_addr(2 + (c & 1)), bvw = sl + 6 * T::B_P;
    if (i < 3)
      OF::template chain<16>(mk_mma3(tmem + (i == 0 ? T::TB : T::TBX + KP * (i - 1)), ax + (2 * i) * T::A_CH,
                            ax + (2 * i + 1) * T::A_CH, sbo_16, sl + 2 * i * T::B_P, sl + (2 * i + 1) * T::B_P, sbo_16,
                            OF::idesc(128, KP), i == 0 || c > 0));
    else if (i < 6)
      OF::template chain<16>(mk_mma3(tmem + T::TB + KP * (i - 2), ax + (2 * i) * T::A_CH, ax + (2 * i + 1) * T::A_CH, sbo_16,
                            bvw, bvw + T::B_P, sbo_16, OF::idesc(128, KP), true));
  };
  auto issue_U1 = [&](int c, int w) {  // (V_q M^^{-1}) b per field (N = 32)
    if (!live()) return;
    const uint32_t sl = slot_addr(c & 1), d = tmem + (uint32_t)((c & 1) * T::T1U);
    const int f = w - 8;
    if (f >= 0 && f < 4)
      OF::template chain4<KP>(mk_mma4(d + T::UQC * f, aq + (2 * f) * T::A_FIELD, aq + (2 * f + 1) * T::A_FIELD, sbo_KP,
                                      sl, sl + T::B_UV, sl + 2 * T::B_UV, sbo_KP, OF::idesc(128, T::UQC), false));
  };
  auto issue_U2 = [&](int c, int f) {  // r += P_q (W ...) per field (N = KP, K = 32)
    if (!live()) return;
    const uint32_t sl = slot_addr(2 + (c & 1)), sbo_32 = OF::sbo(T::UQC);
    if (f < 4)
      OF::template chain4<T::UQC>(mk_mma4(tmem + T::TB + KP * f, ax + (2 * f) * T::A_UCH, ax + (2 * f + 1) * T::A_UCH,
                                          sbo_32, sl, sl + T::B_UP, sl + 2 * T::B_UP, sbo_32, OF::idesc(128, KP), c > 0));
  };

  // fields of a tile by bulk copies (when the FP32 tile has the global row
  // stride and the copies are 16-byte aligned), issued one tile ahead
  const bool bulkq = NPS == NP && P.bulk_q != 0;
  uint32_t par_q = 0;
  auto load_q = [&](int64_t t) {  // thread 0
    if (!live()) return;
    const int64_t c0 = t * TILE;
    const uint32_t bytes = (uint32_t)((ncols - c0 < TILE ? ncols - c0 : TILE) * NP * 4);
    tc::mbar_expect_tx(bar(9), 4 * bytes);
    for (int f = 0; f < 4; ++f)
      tc::bulk_g2s(tc::smem_addr(sQS + f * TILE * NPS), p.Qin + f * fs + c0 * NP, bytes, bar(9));
    pend |= 16u;
  };

  if (tid == 0 && (int64_t)blockIdx.x < nwalk) {
    prefetch_volume();
    if (bulkq) load_q(tile_at(blockIdx.x));
  }

  for (int64_t iw = blockIdx.x; iw < nwalk && !failed; iw += gridDim.x) {
    const int64_t tile = tile_at(iw);
    const int64_t col0 = tile * TILE;
    const int ncol_t = (int)(ncols - col0 < TILE ? ncols - col0 : TILE);
    int64_t cm = col0 + mrow;
    cm = cm < ncols ? cm : ncols - 1;
    const int64_t km = cm / S;
    const int sh = (int)(cm - km * S);
    const uint32_t code4 = __ldg(reinterpret_cast<const unsigned int*>(p.fcode) + km);
    if (grp == 0) {  // per column: the face codes and each face's neighbour column
      const int4 e4 = __ldg(reinterpret_cast<const int4*>(p.EToE) + km);
      auto nbo = [&](int kn) {  // element offset of the neighbour column; own column (top bit set) on the boundary
        return kn >= 0 ? (uint32_t)(((int64_t)kn * S + sh) * NP) : ((uint32_t)(cm * NP) | 0x80000000u);
      };
      sNB[mrow] = make_uint4(nbo(e4.x), nbo(e4.y), nbo(e4.z), nbo(e4.w));
      sC4[mrow] = code4;
      auto row = [&](int kn) {  // the neighbour column's row when this tile holds it (its values are in sQS)
        const int64_t c = (int64_t)kn * S + sh - col0;
        return kn >= 0 && c >= 0 && c < ncol_t ? (uint32_t)c : 0xffu;
      };
      sIT[mrow] = row(e4.x) | row(e4.y) << 8 | row(e4.z) << 16 | row(e4.w) << 24;
    }

    // ---- fields -> FP32 tile in shared memory (coalesced; or the bulk copies issued one tile ahead) ----
    // the element mean of this thread's field and column
    auto field_mean = [&]() {
      float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int n = 0; n < NP; ++n) a[n % 5] += sQS[(grp * TILE + mrow) * NPS + n];
      sMean[grp * TILE + mrow] = P.meanc ? ((a[0] + a[1]) + (a[2] + a[3]) + a[4]) * (1.f / NP) : 0.f;
    };
    if (bulkq) {
      wait_all(9, par_q);  // the copied tile is visible to every waiting thread
      par_q ^= 1u;
      pend &= ~16u;
      field_mean();
      __syncthreads();
    } else {
      const int nval = ncol_t * NP;
#pragma unroll 5
      for (int i = tid; i < 4 * TILE * NP; i += kThreads) {
        const int f = i / (TILE * NP), r = i - f * (TILE * NP);
        const int c = r / NP, n = r - c * NP;
        sQS[(f * TILE + c) * NPS + n] = r < nval ? __ldg(p.Qin + f * fs + col0 * NP + r) : 0.f;
      }
      __syncthreads();
      field_mean();
      __syncthreads();
    }

    // ---- surface terms (Sec. 4.1, Sec. 6.4), face by face; the lifted terms
    // are gathered at this thread's volume nodes and summed in the b
    // accumulators in TMEM ----
    // normals x surface Jacobian at this thread's face points of face f (8 per
    // group, two 16-byte loads per component), loaded one face ahead
    float nv[3][8];
    auto load_nv = [&](int f) {
      if constexpr (PLANAR) {  // one n J^f per face
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
          const float v = __ldg(P.nP + ((km >> 7) * 12 + dd * 4 + f) * 128 + (km & 127));
#pragma unroll
          for (int j = 0; j < 8; ++j) nv[dd][j] = v;
        }
        return;
      }
      const float4* nfg = reinterpret_cast<const float4*>(P.fgeo_il) + (km >> 7) * 12 * NF4 * 128 + (km & 127);
#pragma unroll
      for (int dd = 0; dd < 3; ++dd)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int g = 2 * grp + h;
          const float4 v = g < NF4 ? __ldg(nfg + (size_t)((dd * 4 + f) * NF4 + g) * 128) : make_float4(0.f, 0.f, 0.f, 0.f);
          nv[dd][4 * h] = v.x;
          nv[dd][4 * h + 1] = v.y;
          nv[dd][4 * h + 2] = v.z;
          nv[dd][4 * h + 3] = v.w;
        }
    };
    // (iii) lifted values of field grp of face f (owner's node order) -> this
    // thread's scratch -> volume nodes; run while the next face's first
    // products execute (the lift outputs, the interpolants and the b
    // accumulators occupy disjoint TMEM columns)
    auto scatter = [&](int f) {
      const int pio = (int)((code4 >> (8 * f)) & 0xffu) % 6;
      {
        uint32_t L[NFP16 / 8][8];
#pragma unroll
        for (int j8 = 0; j8 < NFP16 / 8; ++j8) tc::tmem_ld8_nw(lane_base + T::TL + grp * NFP16 + 8 * j8, L[j8]);
        tc::wait_ld();
#pragma unroll
        for (int j8 = 0; j8 < NFP16 / 8; ++j8) tc::pin8(L[j8]);
#pragma unroll
        for (int j = 0; j < NFP; ++j) sLS[(grp * NFP16 + j) * TILE + mrow] = __uint_as_float(L[j >> 3][j & 7]);
        // add to this field's b accumulator (the first face initialises it):
        // only the face's nodes change, and f is uniform across the CTA
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
    };
    load_nv(0);
    for (int f = 0; f < 4 && !failed; ++f) {
      const int q0 = 8 * grp;
      // (i) [p], {u}, [u] at the face nodes, owner's node order -> split A
      // operands.  Eight lanes take the face nodes of one column, two
      // adjacent nodes each (one packed store per part and combination), so
      // that the neighbour's values come from a few sectors of its row.
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int r = it * 64 + (tid >> 3), j0 = 2 * (tid & 7);
        const uint32_t cd = (sC4[r] >> (8 * f)) & 0xffu;
        const int po = (int)(cd % 6), pn = (int)((cd / 6) % 6), fnb = (int)(cd / 36);
        const uint4 o4 = sNB[r];
        const uint32_t nbo = f == 0 ? o4.x : f == 1 ? o4.y : f == 2 ? o4.z : o4.w;
        const bool bnd = (nbo & 0x80000000u) != 0;
        // a neighbour inside this tile (most neighbours within the same hexahedron or row) is read
        // from the FP32 tile, the others from global memory (L2)
        const uint32_t nrow = (sIT[r] >> (8 * f)) & 0xffu;
        float qp[2][4], qm[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int jj = j0 + h < NFP ? j0 + h : 0;
          const int nn = sGX[(fnb * 6 + pn) * NFP + jj];
          const int64_t b = (int64_t)(nbo & 0x7fffffffu) + nn;
          const int o = sGX[(f * 6 + po) * NFP + jj];
#pragma unroll
          for (int fl = 0; fl < 4; ++fl) {
            qp[h][fl] = nrow != 0xffu ? sQS[(fl * TILE + nrow) * NPS + nn] : __ldg(p.Qin + fl * fs + b);
            qm[h][fl] = sQS[(fl * TILE + r) * NPS + o];
          }
        }
        float cv[7][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const bool on = j0 + h < NFP;
          // Dirichlet ghost state on the boundary (Sec. 4.1): p+ = -p-, u+ = u-
          const float pp = bnd ? -qm[h][0] : qp[h][0];
          cv[0][h] = on ? pp - qm[h][0] : 0.f;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float up = bnd ? qm[h][1 + i] : qp[h][1 + i];
            cv[1 + i][h] = on ? 0.5f * (up + qm[h][1 + i]) - sMean[(1 + i) * TILE + r] : 0.f;  // {u} less the element mean
            cv[4 + i][h] = on ? up - qm[h][1 + i] : 0.f;
          }
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) OF::st2(sFA + (2 * c) * T::A_FN, T::A_FN, r, j0, NFP16, cv[c][0], cv[c][1]);
      }
      sync_check();
      if (failed) break;
      if (issuer) {
        if (warp < 7 && live())
          OF::template chain<NFP16>(mk_mma3(tmem + T::TI + warp * NFQ16, fa + (2 * warp) * T::A_FN,
                                         fa + (2 * warp + 1) * T::A_FN, OF::sbo(NFP16), ft, ft + T::B_TRI,
                                         OF::sbo(NFP16), OF::idesc(128, NFQ16), false));
        tc::commit(bar(7));
      }
      if (f > 0) scatter(f - 1);
      wait_all(7, par_f);
      par_f ^= 1u;
      // (ii) strong-weak flux (Sec. 4.1) at this thread's face points -> split A operands
      if (q0 < NFQ16) {
#pragma unroll
        for (int b4 = 0; b4 < 8; b4 += 4) {
          uint32_t v[7][4];
#pragma unroll
          for (int c = 0; c < 7; ++c) tc::tmem_ld4_nw(lane_base + T::TI + c * NFQ16 + q0 + b4, v[c]);
          tc::wait_ld();
#pragma unroll
          for (int c = 0; c < 7; ++c) tc::pin4(v[c]);
          float F[4][4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float nx = nv[0][b4 + j], ny = nv[1][b4 + j], nz = nv[2][b4 + j];
            const float jp = __uint_as_float(v[0][j]);
            F[0][j] = F[1][j] = F[2][j] = F[3][j] = 0.f;
            if (q0 + b4 + j < NFQ) {
              const float nn = nx * nx + ny * ny + nz * nz;
              const float rJ = rsqrtf(nn);  // 1 / J^f (|n J^f| = J^f)
              const float Jf = nn * rJ;
              const float aun = __uint_as_float(v[1][j]) * nx + __uint_as_float(v[2][j]) * ny +
                                __uint_as_float(v[3][j]) * nz;
              const float jun = (__uint_as_float(v[4][j]) * nx + __uint_as_float(v[5][j]) * ny +
                                 __uint_as_float(v[6][j]) * nz) *
                                rJ;
              F[0][j] = -aun + 0.5f * p.tau_p * jp * Jf;
              const float sc = -0.5f * (jp - p.tau_u * jun);
              F[1][j] = sc * nx;
              F[2][j] = sc * ny;
              F[3][j] = sc * nz;
            }
          }
#pragma unroll
          for (int fld = 0; fld < 4; ++fld) OF::st4(sFA + (2 * fld) * T::A_FQ, T::A_FQ, mrow, q0 + b4, NFQ16, F[fld]);
        }
      }
      sync_check();
      if (failed) break;
      if (f < 3) load_nv(f + 1);
      if (issuer) {
        const uint32_t bl = ft + 2 * T::B_TRI;
        const int fld = warp - 8;
        if (fld >= 0 && fld < 4 && live())
          OF::template chain<NFQ16>(mk_mma3(tmem + T::TL + fld * NFP16, fa + (2 * fld) * T::A_FQ,
                                         fa + (2 * fld + 1) * T::A_FQ, OF::sbo(NFQ16), bl, bl + T::B_TRI,
                                         OF::sbo(NFQ16), OF::idesc(128, NFP16), false));
        tc::commit(bar(7));
      }
      wait_all(7, par_f);
      par_f ^= 1u;
    }
    if (failed) break;
    scatter(3);

    // ---- field grp less its element mean -> split A operand (over the
    // lifted-value scratch: every thread has finished with it) ----
    __syncthreads();
    const float fmean = sMean[grp * TILE + mrow];
#pragma unroll
    for (int n0 = 0; n0 < KP; n0 += 8) {
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = n0 + j < NP ? sQS[(grp * TILE + mrow) * NPS + n0 + j] - fmean : 0.f;
      OF::st8(sAQ + (2 * grp) * T::A_FIELD, T::A_FIELD, mrow, n0, KP, x);
    }
    sync_check();
    if (failed) break;

    // ---- volume terms (Sec. 6.4), chunks of 16 quadrature points, pipelined:
    // the products of chunk c + 2 and of chunk c run while the CUDA cores
    // work on chunk c + 1 ----
    // geometric factors at this thread's 4 quadrature points of chunk c (one
    // 16-byte load each), loaded before the products of the previous step are
    // issued so that the issue time hides their latency
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
    if (NCH > 1) {
      wait_slot(1);
      if (issuer) {
        issue_V(1, warp);
        tc::commit(bar(5));
      }
    }
    for (int c = 0; c < NCH; ++c) {
      wait_all(4 + (c & 1), (par_t1 >> (c & 1)) & 1u);
      par_t1 ^= 1u << (c & 1);
      if (tid == 0 && c + 2 < NCH) load_slot(c & 1, vol_ops + (size_t)(c + 2) * T::SZ_OPV, T::SZ_VA);
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
      if (c > 0) {  // the chunk arrays and the B slot of chunk c - 1 are free once its products complete
        wait_all(6, par_m2);
        par_m2 ^= 1u;
        if (tid == 0 && c + 1 < NCH)
          load_slot(2 + ((c + 1) & 1), vol_ops + (size_t)(c + 1) * T::SZ_OPV + T::SZ_VA, T::SZ_VB);
      }
      {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          OF::st4(sAX + (2 * a) * T::A_CH, T::A_CH, mrow, 4 * grp, QC, U[a]);
          OF::st4(sAX + (2 * (3 + a)) * T::A_CH, T::A_CH, mrow, 4 * grp, QC, g[a]);
        }
      }
      sync_check();
      if (failed) break;
      if (c + 1 < NCH) load_G(c + 1);
      wait_slot(2 + (c & 1));
      if (issuer) {
        issue_DW(c, warp);
        tc::commit(bar(6));
      }
      if (c + 2 < NCH) {
        wait_slot(c & 1);
        if (issuer) {
          issue_V(c + 2, warp);
          tc::commit(bar(4 + (c & 1)));
        }
      }
    }
    if (failed) break;
    wait_all(6, par_m2);
    par_m2 ^= 1u;
    if (tid == 0) {  // update operators of chunks 0 and 1
      if (bulkq) {
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
      load_slot(0, upd_ops, T::SZ_UA);
      load_slot(2, upd_ops + T::SZ_UA, T::SZ_UB);
      if (T::UNCH > 1) {
        load_slot(1, upd_ops + T::SZ_OPU, T::SZ_UA);
        load_slot(3, upd_ops + T::SZ_OPU + T::SZ_UA, T::SZ_UB);
      }
    }

    // ---- b of field grp (+ point source, Sec. 4.1 load vector) -> split A operand ----
    {
      const bool src = grp == 0 && p.src_elem != nullptr && p.src_elem[sh] == (int32_t)km;
#pragma unroll
      for (int n0 = 0; n0 < KP; n0 += 8) {
        uint32_t v[8], v1[8], v2[8];
        tc::tmem_ld8_nw(lane_base + T::TB + KP * grp + n0, v);
        tc::tmem_ld8_nw(lane_base + T::TBX + n0, v1);
        tc::tmem_ld8_nw(lane_base + T::TBX + KP + n0, v2);
        tc::wait_ld();
        tc::pin8(v);
        tc::pin8(v1);
        tc::pin8(v2);
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          // b_p = sum over the three derivative directions
          float b = __uint_as_float(v[j]);
          if (grp == 0) b += __uint_as_float(v1[j]) + __uint_as_float(v2[j]) + (src ? p.src_amp * p.src_vec[sh * NP + n0 + j] : 0.f);
          x[j] = n0 + j < NP ? b : 0.f;
        }
        OF::st8(sAQ + (2 * grp) * T::A_FIELD, T::A_FIELD, mrow, n0, KP, x);
      }
    }
    sync_check();
    if (failed) break;

    // ---- weight-adjusted update (Sec. 6.2, Eq. (matfree); Sec. 7), pipelined
    // like the volume, in chunks of 32 points ----
    constexpr int UQC = T::UQC, UNCH = T::UNCH;
    // weights of field grp (c^2/J for p, 1/J for u) at the 32 points of chunk c,
    // loaded ahead like the geometric factors of the volume
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
    wait_slot(0);
    if (issuer) {
      issue_U1(0, warp);
      tc::commit(bar(4));
    }
    if (UNCH > 1) {
      wait_slot(1);
      if (issuer) {
        issue_U1(1, warp);
        tc::commit(bar(5));
      }
    }
    for (int c = 0; c < UNCH; ++c) {
      wait_all(4 + (c & 1), (par_t1 >> (c & 1)) & 1u);
      par_t1 ^= 1u << (c & 1);
      if (tid == 0 && c + 2 < UNCH) load_slot(c & 1, upd_ops + (size_t)(c + 2) * T::SZ_OPU, T::SZ_UA);
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
          load_slot(2 + ((c + 1) & 1), upd_ops + (size_t)(c + 1) * T::SZ_OPU + T::SZ_UA, T::SZ_UB);
      }
#pragma unroll
      for (int h8 = 0; h8 < UQC / 8; ++h8) OF::st8(sAX + (2 * grp) * T::A_UCH, T::A_UCH, mrow, 8 * h8, UQC, x[h8]);
      sync_check();
      if (failed) break;
      if (c + 1 < UNCH) load_W(c + 1);
      wait_slot(2 + (c & 1));
      if (issuer) {
        issue_U2(c, warp);
        tc::commit(bar(6));
      }
      if (c + 2 < UNCH) {
        wait_slot(c & 1);
        if (issuer) {
          issue_U1(c + 2, warp);
          tc::commit(bar(4 + (c & 1)));
        }
      }
    }
    if (failed) break;
    wait_all(6, par_m2);
    par_m2 ^= 1u;
    if (tid == 0 && iw + gridDim.x < nwalk) {
      prefetch_volume();
      if (bulkq) load_q(tile_at(iw + gridDim.x));  // the FP32 tile area is free: the update's products are complete
    }

    // ---- epilogue: r -> FP32 tile -> coalesced dQ/dt, or the LSRK update (Sec. 5.2) ----
    // With 16-byte accesses and one element per column, the mean correction
    // of the p-field float4 entries r4 = tid + e kThreads that this thread
    // takes below is loaded before the TMEM reads (its latency overlaps them)
    // and added to the FP32 tile by the same thread.
    constexpr int F4P = TILE * NP / 4, NEP = (F4P + kThreads - 1) / kThreads;
    const bool dpre = bulkq && S == 1 && P.meanc != nullptr;
    const int nvalp4 = ncol_t * NP / 4;
    float4 dA[NEP], dB[NEP], dC[NEP];
    if constexpr (NPS == NP) {
#pragma unroll
      for (int e = 0; e < NEP; ++e) {
        const int r4 = tid + e * kThreads;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool ok = dpre && r4 < nvalp4;
        const float4* d = reinterpret_cast<const float4*>(P.meanc + col0 * NP) + r4;
        dA[e] = ok ? __ldg(d) : z;
        dB[e] = ok ? __ldg(d + P.meanc_stride / 4) : z;
        dC[e] = ok ? __ldg(d + P.meanc_stride / 2) : z;
      }
    }
#pragma unroll
    for (int n0 = 0; n0 < KP; n0 += 8) {
      uint32_t v[8];
      tc::tmem_ld8_nw(lane_base + T::TB + KP * grp + n0, v);
      tc::wait_ld();
      tc::pin8(v);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (n0 + j < NP) sTT[(grp * TILE + mrow) * NPS + n0 + j] = __uint_as_float(v[j]);
    }
    sync_check();
    if constexpr (NPS == NP) {
      if (dpre) {
        float4* sT4w = reinterpret_cast<float4*>(sTT);
#pragma unroll
        for (int e = 0; e < NEP; ++e) {
          const int r4 = tid + e * kThreads;
          if (r4 >= nvalp4) continue;
          const float da[4] = {dA[e].x, dA[e].y, dA[e].z, dA[e].w}, db[4] = {dB[e].x, dB[e].y, dB[e].z, dB[e].w},
                      dc[4] = {dC[e].x, dC[e].y, dC[e].z, dC[e].w};
          const int c0 = 4 * r4 / NP, n0 = 4 * r4 - c0 * NP;
          float o[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int c = c0 + (n0 + t >= NP ? 1 : 0);
            o[t] = sMean[TILE + c] * da[t] + sMean[2 * TILE + c] * db[t] + sMean[3 * TILE + c] * dc[t];
          }
          float4 v = sT4w[r4];
          v.x += o[0];
          v.y += o[1];
          v.z += o[2];
          v.w += o[3];
          sT4w[r4] = v;
        }
      }
    }
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
    if (bulkq) {
      // 16-byte accesses: the FP32 tile has the global row stride (NPS = NP)
      // and every field range of the tile starts 16-byte aligned
      constexpr int F4 = TILE * NP / 4, NIT4 = (4 * F4 + kThreads - 1) / kThreads;
      const int nval4 = ncol_t * NP / 4;
      const float4* sT4 = reinterpret_cast<const float4*>(sTT);
      auto corr4 = [&](int r4) -> float4 {
        float o[4];
        if (P.meanc && S == 1) {  // one element per column: D has the field's layout
          const float4* d = reinterpret_cast<const float4*>(P.meanc + col0 * NP) + r4;
          const float4 a = __ldg(d), b = __ldg(d + mst / 4), c = __ldg(d + mst / 2);
          const float da[4] = {a.x, a.y, a.z, a.w}, db[4] = {b.x, b.y, b.z, b.w}, dc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int cc = (4 * r4 + t) / NP;
            o[t] = sMean[TILE + cc] * da[t] + sMean[2 * TILE + cc] * db[t] + sMean[3 * TILE + cc] * dc[t];
          }
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) o[t] = corr1(4 * r4 + t);
        }
        return make_float4(o[0], o[1], o[2], o[3]);
      };
      if (MODE == kRhs) {
#pragma unroll 3
        for (int it = 0; it < NIT4; ++it) {
          const int i = tid + it * kThreads, f = i / F4, r4 = i - f * F4;
          if (i < 4 * F4 && r4 < nval4) {
            float4 v = sT4[f * F4 + r4];
            if (f == 0 && !dpre) {
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
        // LSRK (Sec. 5.2) as below, EB4 float4 loads of res and Q_in issued
        // before their stores
        constexpr int EB4 = 3;
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
            if (ok && f == 0 && !dpre) {
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
          if (r >= nval) continue;
          const int c = r / NP, n = r - c * NP;
          p.out[f * fs + col0 * NP + r] = sTT[(f * TILE + c) * NPS + n] + (f == 0 ? corr1(r) : 0.f);
        }
      } else {
        // LSRK (Sec. 5.2): res = a res + dt r, Q_out = Q_in + b res.  The loads of
        // EB iterations are issued before their stores, so that EB round trips
        // to L2 overlap.  The first stage (a_1 = 0) does not read res.
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
            const int c = r / NP, n = r - c * NP;
            ix[e] = ok ? f * fs + col0 * NP + r : -1;
            vv[e] = ok ? sTT[(f * TILE + c) * NPS + n] + (f == 0 ? corr1(r) : 0.f) : 0.f;
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
    if (pend & 16u) tc::mbar_wait(bar(9), par_q, kWaitIters);
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

template <int N, int MODE, int FMT, int NQX, bool PLANAR>
cudaError_t launch_one(const TcStageParams& P, int grid, cudaStream_t stream) {
  using T = TcDims<N, NQX>;
  auto kern = stage_tc_kernel<N, MODE, FMT, NQX, PLANAR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, T::SMEM, stream>>>(P);
  return cudaGetLastError();
}

template <int N, int NQX, bool PLANAR>
cudaError_t launch_stage_tc_q(const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream) {
  using T = TcDims<N, NQX>;
  const int64_t ntiles = P.tiles ? P.ntiles_list : (P.s.ncols + T::TILE - 1) / T::TILE;
  if (ntiles == 0) return cudaSuccess;
  const int g = (int)(ntiles < grid ? ntiles : grid);
  if (mode == kRhs)
    return fmt == 0 ? launch_one<N, kRhs, 0, NQX, PLANAR>(P, g, stream) : launch_one<N, kRhs, 1, NQX, PLANAR>(P, g, stream);
  return fmt == 0 ? launch_one<N, kLsrk, 0, NQX, PLANAR>(P, g, stream) : launch_one<N, kLsrk, 1, NQX, PLANAR>(P, g, stream);
}

// The volume rule: the collapsed (N+1)^3 rule or the fewer-point rule.
template <int N, bool PLANAR>
cudaError_t launch_stage_tc_n(const TcStageParams& P, int mode, int fmt, int grid, cudaStream_t stream) {
  if (P.s.nq == Dims<N>::NQ) return launch_stage_tc_q<N, Dims<N>::NQ, PLANAR>(P, mode, fmt, grid, stream);
  if constexpr (fewer_point_nq(N) > 0)
    if (P.s.nq == fewer_point_nq(N)) return launch_stage_tc_q<N, fewer_point_nq(N), PLANAR>(P, mode, fmt, grid, stream);
  return cudaErrorInvalidValue;
}

}  // namespace wadg
