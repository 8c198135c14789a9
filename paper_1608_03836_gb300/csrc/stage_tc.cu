// Fused WADG stage on the 5th-generation tensor cores (FP32 fields, products
// in split bf16: x = hi + lo, a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32
// accumulation in TMEM).
//
// A persistent CTA (256 threads, one per SM) walks tiles of 128 columns
// (element, shot).  A column is one MMA row (M = 128) and one TMEM lane; the
// reference operators are the B operands (N = operator rows), streamed from
// L2 in chunks of 16 volume quadrature points, pre-split and pre-laid-out in
// the K-major no-swizzle core-matrix layout (see tc_ops.cuh).  Per tile:
//   volume (Sec. 6.4): per chunk, u_i = V_q u_i and dp/dx^_a = V_q^a p (MMA),
//     U^a = sum_i G_ai u_i and -(J grad p)_i (epilogue, one thread per column),
//     b_p += sum_a (V_q^a)^T diag(w) U^a, b_ui -= V_q^T diag(w) (J grad p)_i
//     (MMA, accumulated in TMEM over the chunks);
//   surface (Sec. 6.4): on CUDA cores, 16 columns at a time, exactly as the
//     CUDA-core stage kernel (gather in the owner's node order, V_tri, flux,
//     V_tri^T diag(w_f), scatter), into a shared-memory accumulator;
//   update (Sec. 6.2, Eq. (matfree); Sec. 7): b is split into an A operand;
//     per chunk, (V_q M^^{-1}) b (MMA), times W = c^2/J or 1/J (epilogue),
//     P_q (...) accumulated in TMEM (MMA);
//   epilogue: dQ/dt = r, or the LSRK update (Sec. 5.2).
// Waits on the tensor cores are bounded; on expiry the CTA records an error
// in p.err, frees its TMEM and returns.
#include <cstring>
#include <vector>

#include "stage_simt.cuh"
#include "tc_ops.cuh"

namespace wadg {

template <int N>
struct TcDims {
  using D = Dims<N>;
  static constexpr int NP = D::NP, NQ = D::NQ, NFP = D::NFP, NFQ = D::NFQ;
  static constexpr int KP = (NP + 15) / 16 * 16;  // node count padded to the MMA K / N granule
  static constexpr int QC = 16;                   // quadrature points per chunk
  static constexpr int NCH = (NQ + QC - 1) / QC;
  static constexpr int TILE = 128;
  static constexpr int A_FIELD = TILE * KP * 2;   // bytes of one bf16 part of one field tile
  static constexpr int SZ_AQ = 4 * 2 * A_FIELD;
  static constexpr int A_CH = TILE * QC * 2;      // one part of a [128 x 16] array
  static constexpr int SZ_AX = 6 * 2 * A_CH;
  static constexpr int B_V = QC * KP * 2;         // one part of a [16 x KP] operator chunk
  static constexpr int B_P = KP * QC * 2;         // one part of a [KP x 16] operator chunk
  static constexpr int SZ_OPV = 2 * B_V + 2 * 3 * B_V + 2 * 3 * B_P + 2 * B_P;
  static constexpr int SZ_OPU = 2 * B_V + 2 * B_P;
  static constexpr int SZ_OP = SZ_OPV > SZ_OPU ? SZ_OPV : SZ_OPU;
  static constexpr int FE = 16, FLD = 20;         // face sub-tile columns and row stride
  static constexpr int SZ_FACE = (7 * 4 * NFP + 7 * 4 * NFQ) * FLD * 4;
  static constexpr int SZ_BF = 4 * NP * TILE * 4;
  static constexpr int OFF_AX = SZ_AQ;
  static constexpr int OFF_OP = SZ_AQ + SZ_AX;
  static constexpr int OFF_BF = ((SZ_AQ > SZ_FACE ? SZ_AQ : SZ_FACE) + 127) / 128 * 128;
  static constexpr int END1 = OFF_OP + SZ_OP, END2 = OFF_BF + SZ_BF;
  static constexpr int MAIN = END1 > END2 ? END1 : END2;
  static constexpr int SMEM = MAIN + 128;         // + mbarrier and TMEM slot
  // TMEM columns
  static constexpr int TV = 0;                    // chunk outputs: u1 u2 u3 (16 each), dp (48)
  static constexpr int TB = 128;                  // b accumulators, 4 x KP
  static constexpr int TU = 0;                    // update chunk: 4 x 16
  static constexpr int TR = 320;                  // r accumulators, 4 x KP
  static_assert(TB + 4 * KP <= 512 && TR + 4 * KP <= 512 && TV + 96 <= TB, "TMEM plan");
};

namespace {

constexpr uint32_t kWaitIters = 1u << 22;

// Cooperative copy of `bytes` (multiple of 16) from global to shared memory.
__device__ __forceinline__ void stage_copy(uint8_t* dst, const uint8_t* __restrict__ src, int bytes) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

__device__ __forceinline__ void put_split(uint8_t* base_hi, uint8_t* base_lo, uint32_t off, float x) {
  __nv_bfloat16 h, l;
  tc::split_bf16(x, h, l);
  *reinterpret_cast<__nv_bfloat16*>(base_hi + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(base_lo + off) = l;
}

// D (+)= A B^T with split operators: hi*hi + hi*lo + lo*hi, K in steps of 16.
__device__ __forceinline__ void mma3(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t a_sbo, uint32_t b_hi,
                                     uint32_t b_lo, uint32_t b_sbo, int ksteps, uint32_t idesc, bool accumulate) {
  for (int ks = 0; ks < ksteps; ++ks) {
    const uint32_t o = (uint32_t)ks * 256u;
    const uint64_t ah = tc::smem_desc(a_hi + o, 128, a_sbo), al = tc::smem_desc(a_lo + o, 128, a_sbo);
    const uint64_t bh = tc::smem_desc(b_hi + o, 128, b_sbo), bl = tc::smem_desc(b_lo + o, 128, b_sbo);
    tc::mma_bf16(d, ah, bh, idesc, (accumulate || ks > 0) ? 1u : 0u);
    tc::mma_bf16(d, ah, bl, idesc, 1u);
    tc::mma_bf16(d, al, bh, idesc, 1u);
  }
}

}  // namespace

template <int N, int MODE>
__global__ void __launch_bounds__(256, 1) stage_tc_kernel(const TcStageParams P) {
  using T = TcDims<N>;
  constexpr int NP = T::NP, NQ = T::NQ, NFP = T::NFP, NFQ = T::NFQ, KP = T::KP, QC = T::QC;
  constexpr int FE = T::FE, FLD = T::FLD, TILE = T::TILE;
  const StageParams<float>& p = P.s;
  const DevOps<float>& ops = p.ops;

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAQ = smem;                 // A operand: fields (volume), then b (update)
  uint8_t* sAX = smem + T::OFF_AX;     // A operand: chunk arrays
  uint8_t* sOP = smem + T::OFF_OP;     // B operand staging
  float* sBF = reinterpret_cast<float*>(smem + T::OFF_BF);  // [4][NP][128] surface terms
  float* sFN = reinterpret_cast<float*>(smem);              // face sub-tile arrays
  float* sFQ = sFN + 7 * 4 * NFP * FLD;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + T::MAIN);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + T::MAIN + 8);
  int* sflag = reinterpret_cast<int*>(smem + T::MAIN + 16);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int mrow = quarter * 32 + lane;  // this thread's column within the tile (TMEM lane)
  const int64_t ncols = p.ncols;
  const int64_t fs = ncols * NP;
  const int S = p.S;
  const int64_t ntiles = (ncols + TILE - 1) / TILE;

  if (tid == 0) {
    tc::mbar_init(tc::smem_addr(mbar), 1);
    *sflag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
  const uint32_t mb = tc::smem_addr(mbar);
  uint32_t phase = 0;
  bool failed = false;

  auto wait_mma = [&]() {
    if (!tc::mbar_wait(mb, phase, kWaitIters)) atomicExch(sflag, 1);
    phase ^= 1u;
    tc::fence_after();
    __syncthreads();
    failed = *(volatile int*)sflag != 0;
  };

  const uint32_t aq = tc::smem_addr(sAQ), ax = tc::smem_addr(sAX), op = tc::smem_addr(sOP);
  const uint32_t sbo_KP = (KP / 8) * 128, sbo_16 = 2 * 128;

  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t col0 = tile * TILE;
    int64_t cm = col0 + mrow;
    const bool valid = cm < ncols;
    cm = valid ? cm : ncols - 1;
    const int64_t km = cm / S;

    // ---- fields -> split A operand (each half loads two fields of its column) ----
    for (int f = 2 * half; f < 2 * half + 2; ++f) {
      uint8_t* hi = sAQ + (2 * f) * T::A_FIELD;
      uint8_t* lo = hi + T::A_FIELD;
      const float* q = p.Qin + f * fs + cm * NP;
      for (int n = 0; n < KP; ++n) put_split(hi, lo, tc::kmajor_offset(mrow, n, KP), n < NP ? __ldg(q + n) : 0.f);
    }

    // ---- volume terms, chunk by chunk ----
    for (int ch = 0; ch < T::NCH && !failed; ++ch) {
      stage_copy(sOP, P.ops + (size_t)ch * T::SZ_OPV, T::SZ_OPV);
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        // u_i = A(u_i) B(V_q chunk)^T, N = 16
        const uint32_t bvq = op, bva = op + 2 * T::B_V;
        for (int i = 0; i < 3; ++i)
          mma3(tmem + T::TV + 16 * i, aq + (2 * (1 + i)) * T::A_FIELD, aq + (2 * (1 + i) + 1) * T::A_FIELD, sbo_KP,
               bvq, bvq + T::B_V, sbo_KP, KP / 16, tc::idesc_bf16(128, 16), false);
        // dp/dx^_a = A(p) B(V_q^a chunk)^T, N = 48 (rows a*16 + q)
        mma3(tmem + T::TV + 48, aq, aq + T::A_FIELD, sbo_KP, bva, bva + 3 * T::B_V, sbo_KP, KP / 16,
             tc::idesc_bf16(128, 48), false);
        tc::commit(mb);
      }
      wait_mma();
      if (failed) break;
      // epilogue: U^a and -(J grad p)_i at this thread's 8 quadrature points
      {
        float u[3][8], d[3][8];
        for (int i = 0; i < 3; ++i) tc::tmem_ld8(lane_base + T::TV + 16 * i + 8 * half, u[i]);
        for (int a = 0; a < 3; ++a) tc::tmem_ld8(lane_base + T::TV + 48 + 16 * a + 8 * half, d[a]);
        const float* gk = p.vgeo + km * 11 * NQ;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int ql = 8 * half + j, q = ch * QC + ql;
          float G[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) G[c] = q < NQ ? __ldg(gk + c * NQ + q) : 0.f;
          const uint32_t off = tc::kmajor_offset(mrow, ql, QC);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float U = G[a * 3] * u[0][j] + G[a * 3 + 1] * u[1][j] + G[a * 3 + 2] * u[2][j];
            put_split(sAX + (2 * a) * T::A_CH, sAX + (2 * a + 1) * T::A_CH, off, U);
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float g = -(G[i] * d[0][j] + G[3 + i] * d[1][j] + G[6 + i] * d[2][j]);
            put_split(sAX + (2 * (3 + i)) * T::A_CH, sAX + (2 * (3 + i) + 1) * T::A_CH, off, g);
          }
        }
      }
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        const uint32_t bdw = op + 8 * T::B_V, bvw = bdw + 6 * T::B_P;
        for (int a = 0; a < 3; ++a)
          mma3(tmem + T::TB, ax + (2 * a) * T::A_CH, ax + (2 * a + 1) * T::A_CH, sbo_16, bdw + 2 * a * T::B_P,
               bdw + (2 * a + 1) * T::B_P, sbo_16, 1, tc::idesc_bf16(128, KP), ch > 0 || a > 0);
        for (int i = 0; i < 3; ++i)
          mma3(tmem + T::TB + KP * (1 + i), ax + (2 * (3 + i)) * T::A_CH, ax + (2 * (3 + i) + 1) * T::A_CH, sbo_16,
               bvw, bvw + T::B_P, sbo_16, 1, tc::idesc_bf16(128, KP), ch > 0);
        tc::commit(mb);
      }
      wait_mma();
    }
    if (failed) break;

    // ---- surface terms on CUDA cores, FE columns at a time, into sBF ----
    for (int sub = 0; sub < TILE / FE; ++sub) {
      const int64_t s0 = col0 + sub * FE;
      // face nodes: [p], {u}, [u] in the owner's node order
      for (int it = tid; it < 4 * NFP * FE; it += 256) {
        const int j = it % NFP, f = (it / NFP) % 4, e = it / (4 * NFP);
        int64_t c = s0 + e;
        c = c < ncols ? c : ncols - 1;
        const int64_t k = c / S;
        const int sh = (int)(c - k * S);
        const int code = p.fcode[k * 4 + f];
        const int pio = code % 6, pin = (code / 6) % 6, fn = code / 36;
        const int64_t bo = c * NP + ops.gidx[(f * 6 + pio) * NFP + j];
        const float pm = __ldg(p.Qin + bo), u1m = __ldg(p.Qin + fs + bo), u2m = __ldg(p.Qin + 2 * fs + bo),
                    u3m = __ldg(p.Qin + 3 * fs + bo);
        const int64_t kn = p.EToE[k * 4 + f];
        float pp, u1p, u2p, u3p;
        if (kn >= 0) {
          const int64_t b = (kn * S + sh) * NP + ops.gidx[(fn * 6 + pin) * NFP + j];
          pp = __ldg(p.Qin + b);
          u1p = __ldg(p.Qin + fs + b);
          u2p = __ldg(p.Qin + 2 * fs + b);
          u3p = __ldg(p.Qin + 3 * fs + b);
        } else {
          pp = -pm;
          u1p = u1m;
          u2p = u2m;
          u3p = u3m;
        }
        const int row = f * NFP + j;
        sFN[(0 * 4 * NFP + row) * FLD + e] = pp - pm;
        sFN[(1 * 4 * NFP + row) * FLD + e] = 0.5f * (u1p + u1m);
        sFN[(2 * 4 * NFP + row) * FLD + e] = 0.5f * (u2p + u2m);
        sFN[(3 * 4 * NFP + row) * FLD + e] = 0.5f * (u3p + u3m);
        sFN[(4 * 4 * NFP + row) * FLD + e] = u1p - u1m;
        sFN[(5 * 4 * NFP + row) * FLD + e] = u2p - u2m;
        sFN[(6 * 4 * NFP + row) * FLD + e] = u3p - u3m;
      }
      __syncthreads();
      {
        constexpr int RG = Dims<N>::NFQP / 4, NG = FE / 4;
        for (int it = tid; it < 28 * RG * NG; it += 256) {
          const int g = it % NG, m0 = ((it / NG) % RG) * 4, job = it / (RG * NG);
          float acc[4][4];
          tile_dot<float, FLD, 4, Dims<N>::NFQP, NFP>(ops.VtriT, sFN + job * NFP * FLD + g * 4, m0, acc);
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (m0 + r < NFQ) sts_cols(sFQ + (job * NFQ + m0 + r) * FLD + g * 4, acc[r]);
        }
      }
      __syncthreads();
      for (int it = tid; it < 4 * NFQ * FE; it += 256) {
        const int qf = it % (4 * NFQ), e = it / (4 * NFQ);
        int64_t c = s0 + e;
        c = c < ncols ? c : ncols - 1;
        const float* fg = p.fgeo + (c / S) * 3 * 4 * NFQ + qf;
        const float nx = __ldg(fg), ny = __ldg(fg + 4 * NFQ), nz = __ldg(fg + 8 * NFQ);
        const float Jf = sqrtf(nx * nx + ny * ny + nz * nz);
        const float jp = sFQ[(0 * 4 * NFQ + qf) * FLD + e];
        const float a1 = sFQ[(1 * 4 * NFQ + qf) * FLD + e], a2 = sFQ[(2 * 4 * NFQ + qf) * FLD + e],
                    a3 = sFQ[(3 * 4 * NFQ + qf) * FLD + e];
        const float j1 = sFQ[(4 * 4 * NFQ + qf) * FLD + e], j2 = sFQ[(5 * 4 * NFQ + qf) * FLD + e],
                    j3 = sFQ[(6 * 4 * NFQ + qf) * FLD + e];
        const float aun = a1 * nx + a2 * ny + a3 * nz;
        const float jun = (j1 * nx + j2 * ny + j3 * nz) / Jf;
        const float Fp = -aun + 0.5f * p.tau_p * jp * Jf;
        const float sc = -0.5f * (jp - p.tau_u * jun);
        sFQ[(0 * 4 * NFQ + qf) * FLD + e] = Fp;
        sFQ[(1 * 4 * NFQ + qf) * FLD + e] = sc * nx;
        sFQ[(2 * 4 * NFQ + qf) * FLD + e] = sc * ny;
        sFQ[(3 * 4 * NFQ + qf) * FLD + e] = sc * nz;
      }
      __syncthreads();
      {
        constexpr int RG = Dims<N>::NFPP / 2, NG = FE / 4;
        for (int it = tid; it < 16 * RG * NG; it += 256) {
          const int g = it % NG, m0 = ((it / NG) % RG) * 2, job = it / (RG * NG);
          float acc[2][4];
          tile_dot<float, FLD, 2, Dims<N>::NFPP, NFQ>(ops.VtriTwT, sFQ + job * NFQ * FLD + g * 4, m0, acc);
#pragma unroll
          for (int r = 0; r < 2; ++r)
            if (m0 + r < NFP) sts_cols(sFN + (job * NFP + m0 + r) * FLD + g * 4, acc[r]);
        }
      }
      __syncthreads();
      for (int it = tid; it < 4 * NP * FE; it += 256) {
        const int e = it % FE, n = (it / FE) % NP, fld = it / (FE * NP);
        int64_t c = s0 + e;
        c = c < ncols ? c : ncols - 1;
        const int64_t k = c / S;
        float acc = 0.f;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int pio = p.fcode[k * 4 + f] % 6;
          const int jo = ops.ginv[(f * 6 + pio) * NP + n];
          if (jo >= 0) acc += sFN[((fld * 4 + f) * NFP + jo) * FLD + e];
        }
        sBF[(fld * NP + n) * TILE + sub * FE + e] = acc;
      }
      __syncthreads();
    }

    // ---- b = volume (TMEM) + surface (smem) + source -> split A operand ----
    {
      const int sh = (int)(cm - km * S);
      const bool src = p.src_elem != nullptr && p.src_elem[sh] == (int32_t)km;
      for (int f = 2 * half; f < 2 * half + 2; ++f) {
        uint8_t* hi = sAQ + (2 * f) * T::A_FIELD;
        uint8_t* lo = hi + T::A_FIELD;
        for (int n0 = 0; n0 < KP; n0 += 8) {
          float v[8];
          tc::tmem_ld8(lane_base + T::TB + KP * f + n0, v);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = n0 + j;
            float b = 0.f;
            if (n < NP) {
              b = v[j] + sBF[(f * NP + n) * TILE + mrow];
              if (f == 0 && src) b += p.src_amp * p.src_vec[sh * NP + n];
            }
            put_split(hi, lo, tc::kmajor_offset(mrow, n, KP), b);
          }
        }
      }
    }

    // ---- weight-adjusted update, chunk by chunk ----
    for (int ch = 0; ch < T::NCH && !failed; ++ch) {
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      stage_copy(sOP, P.ops + (size_t)T::NCH * T::SZ_OPV + (size_t)ch * T::SZ_OPU, T::SZ_OPU);
      tc::fence_async_smem();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        for (int f = 0; f < 4; ++f)
          mma3(tmem + T::TU + 16 * f, aq + (2 * f) * T::A_FIELD, aq + (2 * f + 1) * T::A_FIELD, sbo_KP, op,
               op + T::B_V, sbo_KP, KP / 16, tc::idesc_bf16(128, 16), false);
        tc::commit(mb);
      }
      wait_mma();
      if (failed) break;
      for (int f = 2 * half; f < 2 * half + 2; ++f) {
        const float* w = p.vgeo + (km * 11 + (f == 0 ? 9 : 10)) * NQ;
        for (int h8 = 0; h8 < 2; ++h8) {
          float v[8];
          tc::tmem_ld8(lane_base + T::TU + 16 * f + 8 * h8, v);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int ql = 8 * h8 + j, q = ch * QC + ql;
            const float x = q < NQ ? v[j] * __ldg(w + q) : 0.f;
            put_split(sAX + (2 * f) * T::A_CH, sAX + (2 * f + 1) * T::A_CH, tc::kmajor_offset(mrow, ql, QC), x);
          }
        }
      }
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        const uint32_t bpq = op + 2 * T::B_V;
        for (int f = 0; f < 4; ++f)
          mma3(tmem + T::TR + KP * f, ax + (2 * f) * T::A_CH, ax + (2 * f + 1) * T::A_CH, sbo_16, bpq, bpq + T::B_P,
               sbo_16, 1, tc::idesc_bf16(128, KP), ch > 0);
        tc::commit(mb);
      }
      wait_mma();
    }
    if (failed) break;

    // ---- epilogue: RHS or LSRK ----
    for (int f = 2 * half; f < 2 * half + 2; ++f) {
      for (int n0 = 0; n0 < KP; n0 += 8) {
        float v[8];
        tc::tmem_ld8(lane_base + T::TR + KP * f + n0, v);
        if (!valid) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + j;
          if (n >= NP) continue;
          const int64_t idx = f * fs + cm * NP + n;
          if (MODE == kRhs) {
            p.out[idx] = v[j];
          } else {
            const float r = p.rk_a * p.res[idx] + p.dt * v[j];
            p.res[idx] = r;
            p.Qout[idx] = __ldg(p.Qin + idx) + p.rk_b * r;
          }
        }
      }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }

  if (failed && tid == 0) atomicExch(P.err, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

template <int N>
cudaError_t launch_stage_tc_n(const TcStageParams& P, int mode, int grid, cudaStream_t stream) {
  using T = TcDims<N>;
  const int64_t ntiles = (P.s.ncols + T::TILE - 1) / T::TILE;
  if (ntiles == 0) return cudaSuccess;
  const int g = (int)(ntiles < grid ? ntiles : grid);
  if (mode == kRhs) {
    auto kern = stage_tc_kernel<N, kRhs>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<g, 256, T::SMEM, stream>>>(P);
  } else {
    auto kern = stage_tc_kernel<N, kLsrk>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<g, 256, T::SMEM, stream>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t launch_stage_tc(int N, const TcStageParams& P, int mode, int grid, cudaStream_t stream) {
  switch (N) {
    case 1: return launch_stage_tc_n<1>(P, mode, grid, stream);
    case 2: return launch_stage_tc_n<2>(P, mode, grid, stream);
    case 3: return launch_stage_tc_n<3>(P, mode, grid, stream);
    case 4: return launch_stage_tc_n<4>(P, mode, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

size_t tc_ops_bytes(int N) {
  switch (N) {
    case 1: return (size_t)TcDims<1>::NCH * (TcDims<1>::SZ_OPV + TcDims<1>::SZ_OPU);
    case 2: return (size_t)TcDims<2>::NCH * (TcDims<2>::SZ_OPV + TcDims<2>::SZ_OPU);
    case 3: return (size_t)TcDims<3>::NCH * (TcDims<3>::SZ_OPV + TcDims<3>::SZ_OPU);
    case 4: return (size_t)TcDims<4>::NCH * (TcDims<4>::SZ_OPV + TcDims<4>::SZ_OPU);
    default: return 0;
  }
}

// ---------------------------------------------------------------------------
// Host: pack the operators of the tensor-core stage, split into bf16 hi + lo,
// in the K-major no-swizzle layout, chunk by chunk in the order the kernel
// stages them.
// ---------------------------------------------------------------------------
namespace {

uint16_t bf16_bits_rne(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
  const uint32_t bias = 0x7fffu + ((u >> 16) & 1u);  // round half to even on the dropped 16 bits
  return (uint16_t)((u + bias) >> 16);
}

float bf16_bits_to_float(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}

size_t host_kmajor_offset(int row, int k, int K) {
  return (size_t)(((row >> 3) * (K >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Writes a [R x K] split tile: hi part at dst, lo part at dst + part_bytes.
template <typename F>
void put_tile(uint8_t* dst, size_t part_bytes, int R, int K, F value) {
  for (int r = 0; r < R; ++r)
    for (int k = 0; k < K; ++k) {
      const double x = value(r, k);
      const uint16_t h = bf16_bits_rne((float)x);
      const uint16_t l = bf16_bits_rne((float)(x - (double)bf16_bits_to_float(h)));
      const size_t off = host_kmajor_offset(r, k, K);
      std::memcpy(dst + off, &h, 2);
      std::memcpy(dst + part_bytes + off, &l, 2);
    }
}

template <int N>
void pack_n(const RefOps& o, std::vector<uint8_t>& out) {
  using T = TcDims<N>;
  const int Np = o.Np, Nq = o.Nq, KP = T::KP, QC = T::QC;
  out.assign((size_t)T::NCH * (T::SZ_OPV + T::SZ_OPU), 0);
  for (int ch = 0; ch < T::NCH; ++ch) {
    uint8_t* v = out.data() + (size_t)ch * T::SZ_OPV;
    auto qn = [&](int r) { return ch * QC + r; };
    put_tile(v, T::B_V, QC, KP, [&](int r, int n) {
      const int q = qn(r);
      return (q < Nq && n < Np) ? o.Vq[q * Np + n] : 0.0;
    });
    put_tile(v + 2 * T::B_V, 3 * T::B_V, 3 * QC, KP, [&](int r, int n) {
      const int a = r / QC, q = qn(r % QC);
      return (q < Nq && n < Np) ? o.Vqa[(a * Nq + q) * Np + n] : 0.0;
    });
    for (int a = 0; a < 3; ++a)
      put_tile(v + 8 * T::B_V + 2 * a * T::B_P, T::B_P, KP, QC, [&](int n, int k) {
        const int q = qn(k);
        return (q < Nq && n < Np) ? o.Dw[(a * Np + n) * Nq + q] : 0.0;
      });
    put_tile(v + 8 * T::B_V + 6 * T::B_P, T::B_P, KP, QC, [&](int n, int k) {
      const int q = qn(k);
      return (q < Nq && n < Np) ? o.Vw[n * Nq + q] : 0.0;
    });
    uint8_t* u = out.data() + (size_t)T::NCH * T::SZ_OPV + (size_t)ch * T::SZ_OPU;
    put_tile(u, T::B_V, QC, KP, [&](int r, int n) {
      const int q = qn(r);
      return (q < Nq && n < Np) ? o.Vtilde[q * Np + n] : 0.0;
    });
    put_tile(u + 2 * T::B_V, T::B_P, KP, QC, [&](int n, int k) {
      const int q = qn(k);
      return (q < Nq && n < Np) ? o.Pq[n * Nq + q] : 0.0;
    });
  }
}

}  // namespace

bool pack_tc_ops(int N, const RefOps& o, std::vector<uint8_t>& out) {
  switch (N) {
    case 1: pack_n<1>(o, out); return true;
    case 2: pack_n<2>(o, out); return true;
    case 3: pack_n<3>(o, out); return true;
    case 4: pack_n<4>(o, out); return true;
    default: return false;
  }
}

}  // namespace wadg
