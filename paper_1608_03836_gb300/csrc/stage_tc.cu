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
//   surface (Sec. 6.4), face by face: the face-node combinations [p], {u},
//     [u] are gathered in the owner's node order (CUDA cores), interpolated
//     to the face points by V_tri (MMA), turned into the strong-weak flux with
//     n J^f (epilogue), lifted by V_tri^T diag(w_f) (MMA) and added to a
//     shared-memory accumulator at the volume nodes (epilogue);
//   geometric factors are read from column-interleaved copies, so that the 32
//   lanes of a warp (32 consecutive elements) read 128 contiguous bytes;
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
  static constexpr int SZ_BF = 4 * NP * TILE * 4;  // surface terms, FP32 [4][NP][128]
  // surface products on the tensor cores: face nodes padded to NFP16 (K of the
  // interpolation, N of the lift), face points to NFQ16 (N, then K)
  static constexpr int NFP16 = (NFP + 15) / 16 * 16, NFQ16 = (NFQ + 15) / 16 * 16;
  static constexpr int A_FN = TILE * NFP16 * 2;    // one part of a [128 x NFP16] combination tile
  static constexpr int A_FQ = TILE * NFQ16 * 2;    // one part of a [128 x NFQ16] flux tile
  static constexpr int SZ_FACE = (7 * 2 * A_FN > 4 * 2 * A_FQ ? 7 * 2 * A_FN : 4 * 2 * A_FQ);
  static constexpr int B_TRI = NFQ16 * NFP16 * 2;  // one part of V_tri [NFQ16 x NFP16] or its lift
  static constexpr int OFF_AX = SZ_AQ;
  static constexpr int OFF_OP = SZ_AQ + SZ_AX;
  static constexpr int OFF_BF = ((SZ_FACE > SZ_AQ ? SZ_FACE : SZ_AQ) + 127) / 128 * 128;
  static constexpr int END1 = OFF_OP + SZ_OP, END2 = OFF_BF + SZ_BF;
  static constexpr int MAIN = END1 > END2 ? END1 : END2;
  static constexpr int OFF_FT = MAIN + 128;       // face B operands: V_tri (hi, lo), lift (hi, lo)
  static constexpr int SMEM = OFF_FT + 4 * B_TRI;
  static constexpr int SZ_FOPS = 4 * B_TRI;       // packed after the volume and update chunks
  // TMEM columns
  static constexpr int TV = 0;                    // chunk outputs: u1 u2 u3 (16 each), dp (48)
  static constexpr int TB = 128;                  // b accumulators, 4 x KP
  static constexpr int TU = 0;                    // update chunk: 4 x 16
  static constexpr int TR = 320;                  // r accumulators, 4 x KP
  static_assert(TB + 4 * KP <= 512 && TR + 4 * KP <= 512 && TV + 96 <= TB, "TMEM plan");
  // TMEM for the surface products: combinations 0-3 in [0, 4 NFQ16), 4-6 at
  // [TR, TR + 3 NFQ16), lifted fluxes after them
  static constexpr int TI_LO = 0, TI_HI = TR, TL = TR + 3 * NFQ16;
  static_assert(4 * NFQ16 <= TB && TL + 4 * NFP16 <= 512, "TMEM plan (surface)");

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
  constexpr int TILE = T::TILE, NFP16 = T::NFP16, NFQ16 = T::NFQ16;
  const StageParams<float>& p = P.s;
  const DevOps<float>& ops = p.ops;

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAQ = smem;                 // A operand: fields (volume), then b (update)
  uint8_t* sAX = smem + T::OFF_AX;     // A operand: chunk arrays
  uint8_t* sOP = smem + T::OFF_OP;     // B operand staging
  float* sBF = reinterpret_cast<float*>(smem + T::OFF_BF);  // [4][NP][128] surface terms
  uint8_t* sFA = smem;                                       // per face: A operands (combinations, then fluxes)
  uint8_t* sFT = smem + T::OFF_FT;                           // face B operands
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
  stage_copy(sFT, P.ops + (size_t)T::NCH * (T::SZ_OPV + T::SZ_OPU), T::SZ_FOPS);
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
  const uint32_t fa = tc::smem_addr(sFA), ft = tc::smem_addr(sFT);
  const uint32_t sbo_KP = (KP / 8) * 128, sbo_16 = 2 * 128;

  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t col0 = tile * TILE;
    int64_t cm = col0 + mrow;
    const bool valid = cm < ncols;
    cm = valid ? cm : ncols - 1;
    const int64_t km = cm / S;

    // ---- fields -> split A operand: coalesced FP32 tile in the (free) A_X/B
    // staging area, then each half splits two fields of its column ----
    {
      float* stg = reinterpret_cast<float*>(sAX);  // [4][TILE * NP]
      const int64_t nval = (ncols - col0 < TILE ? ncols - col0 : TILE) * NP;
      for (int f = 0; f < 4; ++f) {
        const float* src = p.Qin + f * fs + col0 * NP;
        for (int i = tid; i < TILE * NP; i += 256) stg[f * TILE * NP + i] = i < nval ? __ldg(src + i) : 0.f;
      }
      __syncthreads();
      for (int f = 2 * half; f < 2 * half + 2; ++f) {
        uint8_t* hi = sAQ + (2 * f) * T::A_FIELD;
        uint8_t* lo = hi + T::A_FIELD;
        const float* q = stg + f * TILE * NP + mrow * NP;
        for (int n = 0; n < KP; ++n) put_split(hi, lo, tc::kmajor_offset(mrow, n, KP), n < NP ? q[n] : 0.f);
      }
      __syncthreads();  // the staging area is reused by the operator chunks
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
      // geometric factors of this thread's 8 quadrature points, loaded while the MMA runs
      float G[9][8];
      {
        const float* gk = P.vgeo_il + (km >> 7) * 11 * NQ * 128 + (km & 127);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int q = ch * QC + 8 * half + j;
#pragma unroll
          for (int c = 0; c < 9; ++c) G[c][j] = q < NQ ? __ldg(gk + (size_t)(c * NQ + q) * 128) : 0.f;
        }
      }
      wait_mma();
      if (failed) break;
      // epilogue: U^a and -(J grad p)_i at this thread's 8 quadrature points
      {
        float u[3][8], d[3][8];
        tc::tmem_ld24(lane_base + T::TV + 8 * half, lane_base + T::TV + 16 + 8 * half, lane_base + T::TV + 32 + 8 * half,
                      u[0], u[1], u[2]);
        tc::tmem_ld24(lane_base + T::TV + 48 + 8 * half, lane_base + T::TV + 64 + 8 * half,
                      lane_base + T::TV + 80 + 8 * half, d[0], d[1], d[2]);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int ql = 8 * half + j;
          const uint32_t off = tc::kmajor_offset(mrow, ql, QC);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float U = G[a * 3][j] * u[0][j] + G[a * 3 + 1][j] * u[1][j] + G[a * 3 + 2][j] * u[2][j];
            put_split(sAX + (2 * a) * T::A_CH, sAX + (2 * a + 1) * T::A_CH, off, U);
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float g = -(G[i][j] * d[0][j] + G[3 + i][j] * d[1][j] + G[6 + i][j] * d[2][j]);
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

    // ---- surface terms (Sec. 6.4), face by face: gather on CUDA cores, V_tri
    // and the lift V_tri^T diag(w_f) on the tensor cores, flux in between ----
    for (int i = tid; i < 4 * NP * TILE; i += 256) sBF[i] = 0.f;
    for (int f = 0; f < 4 && !failed; ++f) {
      const int col = mrow;
      int pio_f;
      // (i) [p], {u}, [u] at the face nodes, owner's node order -> split A operands
      {
        constexpr int JH = NFP16 / 2;
        const int code = p.fcode[km * 4 + f];
        const int pio = code % 6, pin = (code / 6) % 6, fn = code / 36;
        pio_f = pio;
        const int sh = (int)(cm - km * S);
        const int64_t kn = p.EToE[km * 4 + f];
        const int16_t* go = ops.gidx + (f * 6 + pio) * NFP;
        const int16_t* gn = ops.gidx + (fn * 6 + pin) * NFP;
        const int64_t nb = kn >= 0 ? (kn * S + sh) * NP : 0;
#pragma unroll
        for (int jj = 0; jj < JH; ++jj) {
          const int j = half * JH + jj;
          float cv[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          if (j < NFP) {
            const int64_t bo = cm * NP + go[j];
            const float pm = __ldg(p.Qin + bo), u1m = __ldg(p.Qin + fs + bo), u2m = __ldg(p.Qin + 2 * fs + bo),
                        u3m = __ldg(p.Qin + 3 * fs + bo);
            float pp, u1p, u2p, u3p;
            if (kn >= 0) {
              const int64_t b = nb + gn[j];
              pp = __ldg(p.Qin + b);
              u1p = __ldg(p.Qin + fs + b);
              u2p = __ldg(p.Qin + 2 * fs + b);
              u3p = __ldg(p.Qin + 3 * fs + b);
            } else {  // Dirichlet ghost state (Sec. 4.1)
              pp = -pm;
              u1p = u1m;
              u2p = u2m;
              u3p = u3m;
            }
            cv[0] = pp - pm;
            cv[1] = 0.5f * (u1p + u1m);
            cv[2] = 0.5f * (u2p + u2m);
            cv[3] = 0.5f * (u3p + u3m);
            cv[4] = u1p - u1m;
            cv[5] = u2p - u2m;
            cv[6] = u3p - u3m;
          }
          const uint32_t off = tc::kmajor_offset(col, j, NFP16);
#pragma unroll
          for (int c = 0; c < 7; ++c) put_split(sFA + (2 * c) * T::A_FN, sFA + (2 * c + 1) * T::A_FN, off, cv[c]);
        }
      }
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        for (int c = 0; c < 7; ++c) {
          const uint32_t d = tmem + (c < 4 ? T::TI_LO + c * NFQ16 : T::TI_HI + (c - 4) * NFQ16);
          mma3(d, fa + (2 * c) * T::A_FN, fa + (2 * c + 1) * T::A_FN, (NFP16 / 8) * 128, ft, ft + T::B_TRI,
               (NFP16 / 8) * 128, NFP16 / 16, tc::idesc_bf16(128, NFQ16), false);
        }
        tc::commit(mb);
      }
      // normals x surface Jacobian at this thread's face points, loaded while the MMA runs
      constexpr int QH = NFQ16 / 2;
      float nv[3][QH];
      {
        const float* nfg = P.fgeo_il + ((km >> 7) * 12 * NFQ + f * NFQ) * 128 + (km & 127);
#pragma unroll
        for (int qq = 0; qq < QH; ++qq) {
          const int q = half * QH + qq;
#pragma unroll
          for (int dd = 0; dd < 3; ++dd) nv[dd][qq] = q < NFQ ? __ldg(nfg + (size_t)(dd * 4 * NFQ + q) * 128) : 0.f;
        }
      }
      wait_mma();
      if (failed) break;
      // (ii) strong-weak flux (Sec. 4.1) at this thread's face points -> split A operands
      {
        float v[7][QH];
#pragma unroll
        for (int c = 0; c < 7; ++c) {
          const uint32_t base = lane_base + (c < 4 ? T::TI_LO + c * NFQ16 : T::TI_HI + (c - 4) * NFQ16) + half * QH;
#pragma unroll
          for (int q8 = 0; q8 < QH; q8 += 8) {
            float x[8];
            tc::tmem_ld8(base + q8, x);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[c][q8 + j] = x[j];
          }
        }
#pragma unroll
        for (int qq = 0; qq < QH; ++qq) {
          const int q = half * QH + qq;
          const float nx = nv[0][qq], ny = nv[1][qq], nz = nv[2][qq];
          float F[4] = {0.f, 0.f, 0.f, 0.f};
          if (q < NFQ) {
            const float Jf = sqrtf(nx * nx + ny * ny + nz * nz);
            const float aun = v[1][qq] * nx + v[2][qq] * ny + v[3][qq] * nz;
            const float jun = (v[4][qq] * nx + v[5][qq] * ny + v[6][qq] * nz) / Jf;
            F[0] = -aun + 0.5f * p.tau_p * v[0][qq] * Jf;
            const float sc = -0.5f * (v[0][qq] - p.tau_u * jun);
            F[1] = sc * nx;
            F[2] = sc * ny;
            F[3] = sc * nz;
          }
          const uint32_t off = tc::kmajor_offset(col, q, NFQ16);
#pragma unroll
          for (int fld = 0; fld < 4; ++fld)
            put_split(sFA + (2 * fld) * T::A_FQ, sFA + (2 * fld + 1) * T::A_FQ, off, F[fld]);
        }
      }
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        const uint32_t bl = ft + 2 * T::B_TRI;
        for (int fld = 0; fld < 4; ++fld)
          mma3(tmem + T::TL + fld * NFP16, fa + (2 * fld) * T::A_FQ, fa + (2 * fld + 1) * T::A_FQ, (NFQ16 / 8) * 128, bl,
               bl + T::B_TRI, (NFQ16 / 8) * 128, NFQ16 / 16, tc::idesc_bf16(128, NFP16), false);
        tc::commit(mb);
      }
      wait_mma();
      if (failed) break;
      // (iii) add the lifted face terms to the volume nodes of this thread's two fields
#pragma unroll
      for (int fi = 0; fi < 2; ++fi) {
        const int fld = 2 * half + fi;
        const int16_t* go = ops.gidx + (f * 6 + pio_f) * NFP;
#pragma unroll
        for (int j8 = 0; j8 < NFP16; j8 += 8) {
          float x[8];
          tc::tmem_ld8(lane_base + T::TL + fld * NFP16 + j8, x);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j8 + j < NFP) sBF[(fld * NP + go[j8 + j]) * TILE + col] += x[j];
        }
      }
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
    }
    if (failed) break;

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
      // weights of this thread's two fields at the 16 points of the chunk, loaded while the MMA runs
      float wt[2][16];
#pragma unroll
      for (int fi = 0; fi < 2; ++fi) {
        const int f = 2 * half + fi;
        const float* w = P.vgeo_il + ((km >> 7) * 11 + (f == 0 ? 9 : 10)) * NQ * 128 + (km & 127);
#pragma unroll
        for (int ql = 0; ql < 16; ++ql) {
          const int q = ch * QC + ql;
          wt[fi][ql] = q < NQ ? __ldg(w + (size_t)q * 128) : 0.f;
        }
      }
      wait_mma();
      if (failed) break;
#pragma unroll
      for (int fi = 0; fi < 2; ++fi) {
        const int f = 2 * half + fi;
        float v0[8], v1[8], vdummy[8];
        tc::tmem_ld24(lane_base + T::TU + 16 * f, lane_base + T::TU + 16 * f + 8, lane_base + T::TU + 16 * f, v0, v1,
                      vdummy);
#pragma unroll
        for (int ql = 0; ql < 16; ++ql) {
          const float x = (ql < 8 ? v0[ql] : v1[ql - 8]) * wt[fi][ql];
          put_split(sAX + (2 * f) * T::A_CH, sAX + (2 * f + 1) * T::A_CH, tc::kmajor_offset(mrow, ql, QC), x);
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
    case 1: return (size_t)TcDims<1>::NCH * (TcDims<1>::SZ_OPV + TcDims<1>::SZ_OPU) + TcDims<1>::SZ_FOPS;
    case 2: return (size_t)TcDims<2>::NCH * (TcDims<2>::SZ_OPV + TcDims<2>::SZ_OPU) + TcDims<2>::SZ_FOPS;
    case 3: return (size_t)TcDims<3>::NCH * (TcDims<3>::SZ_OPV + TcDims<3>::SZ_OPU) + TcDims<3>::SZ_FOPS;
    case 4: return (size_t)TcDims<4>::NCH * (TcDims<4>::SZ_OPV + TcDims<4>::SZ_OPU) + TcDims<4>::SZ_FOPS;
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
  out.assign((size_t)T::NCH * (T::SZ_OPV + T::SZ_OPU) + T::SZ_FOPS, 0);
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
  // face operators: V_tri as [NFQ16 rows (q) x NFP16 (j)], the lift
  // V_tri^T diag(w_f) as [NFP16 rows (j) x NFQ16 (q)]
  const int Nfp = o.Nfp, Nfq = o.Nfq;
  uint8_t* fo = out.data() + (size_t)T::NCH * (T::SZ_OPV + T::SZ_OPU);
  put_tile(fo, T::B_TRI, T::NFQ16, T::NFP16, [&](int q, int j) {
    return (q < Nfq && j < Nfp) ? o.Vtri[q * Nfp + j] : 0.0;
  });
  put_tile(fo + 2 * T::B_TRI, T::B_TRI, T::NFP16, T::NFQ16, [&](int j, int q) {
    return (q < Nfq && j < Nfp) ? o.VtriTw[j * Nfq + q] : 0.0;
  });
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
