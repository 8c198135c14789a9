// Shared pieces of the tensor-core stage kernels (stage_tc.cu for N <= 4,
// stage_tc5.cu for N = 5): the face-node lists of the reference faces, the
// launch constants, the split-bf16 and tf32 operand formats and their
// accumulator chains, and the host-side packing of operator tiles into the
// K-major no-swizzle core-matrix layout of tcgen05 (see tc_ops.cuh).
#pragma once

#include <cstring>
#include <type_traits>
#include <vector>

#include "stage_simt.cuh"
#include "tc_ops.cuh"

namespace wadg {

// Volume nodes of each reference face (t = -1, s = -1, r + s + t = -1,
// r = -1) on the equispaced lattice, node (i, j, k) at index
// sum_{k' < k} (N-k'+1)(N-k'+2)/2 + j (N-k+1) - j (j-1)/2 + i.  Fixed by N and
// the face alone; the host checks them against the runtime face tables.
template <int N>
struct FaceNodeList {
  static constexpr int NFP = (N + 1) * (N + 2) / 2;
  int v[4][NFP];
};
template <int N>
constexpr int lattice_index(int i, int j, int k) {
  int base = 0;
  for (int kk = 0; kk < k; ++kk) base += (N - kk + 1) * (N - kk + 2) / 2;
  return base + j * (N - k + 1) - j * (j - 1) / 2 + i;
}
template <int N>
constexpr FaceNodeList<N> make_face_nodes() {
  FaceNodeList<N> r{};
  for (int f = 0; f < 4; ++f) {
    int t = 0;
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j <= N - k; ++j)
        for (int i = 0; i <= N - j - k; ++i) {
          const bool on = f == 0 ? k == 0 : f == 1 ? j == 0 : f == 2 ? i + j + k == N : i == 0;
          if (on) r.v[f][t++] = lattice_index<N>(i, j, k);
        }
  }
  return r;
}
// 8-column TMEM groups of the b accumulators that face F's nodes fall in.
template <int N, int F>
constexpr uint32_t face_group_mask() {
  constexpr FaceNodeList<N> L = make_face_nodes<N>();
  uint32_t m = 0;
  for (int t = 0; t < FaceNodeList<N>::NFP; ++t) m |= 1u << (L.v[F][t] >> 3);
  return m;
}

namespace {

constexpr uint32_t kWaitIters = 1u << 22;
constexpr int kThreads = 512;      // four threads per column of a 128-column tile
constexpr uint32_t kIssuers = 16;  // threads issuing tensor-core products (lane 0 of each warp)

// LSRK state update with compensated summation: q = qi + (b rr + lo) and
// the new lo = the rounding error of that sum (Fast2Sum, exact for
// |qi| >= |b rr + lo|, which holds for a stage increment).
__device__ __forceinline__ float lsrk_comp(float qi, float b, float rr, float& lo) {
  const float y = fmaf(b, rr, lo);
  const float q = qi + y;
  lo = (qi - q) + y;
  return q;
}

// Cooperative copy of `bytes` (multiple of 16) from global to shared memory.
__device__ __forceinline__ void stage_copy(uint8_t* dst, const uint8_t* __restrict__ src, int bytes) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

// One product D (+)= A B^T with split operators (hi*hi + hi*lo + lo*hi).
struct Mma3 {
  uint32_t d, idesc;
  uint64_t ah, al, bh, bl;  // descriptors of the first K step
  bool acc;                 // accumulate onto D from the first instruction on
};

__device__ __forceinline__ Mma3 mk_mma3(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t a_sbo, uint32_t b_hi,
                                        uint32_t b_lo, uint32_t b_sbo, uint32_t idesc, bool acc) {
  return Mma3{d, idesc, tc::smem_desc(a_hi, 128, a_sbo), tc::smem_desc(a_lo, 128, a_sbo),
              tc::smem_desc(b_hi, 128, b_sbo), tc::smem_desc(b_lo, 128, b_sbo), acc};
}

// One accumulator chain over KS steps of K = 16 (a K step moves the
// descriptors' start address by 256 bytes, 16 in the address field).  A
// thread blocks for about 100-200 cycles per tcgen05.mma it issues, so the
// stage spreads its independent chains over eight issuing threads.
template <int KS>
__device__ __forceinline__ void mma3_chain(const Mma3& g) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const uint64_t o = (uint64_t)(16 * ks);
    tc::mma_bf16(g.d, g.ah + o, g.bh + o, g.idesc, (g.acc || ks > 0) ? 1u : 0u);
    tc::mma_bf16(g.d, g.ah + o, g.bl + o, g.idesc, 1u);
    tc::mma_bf16(g.d, g.al + o, g.bh + o, g.idesc, 1u);
  }
}

// The same with the B operand in three bf16 parts b = bh + bl + b3 (the
// residual of the two-part split in a third part) and a fourth product
// ah*b3 per K step: the operator's rounding drops from 2^-18 to 2^-27 of its
// entries, and what remains of the product's rounding (the A operand's
// split, the dropped al*bl) changes with the data instead of being the same
// perturbation of the operator at every stage.
struct Mma4 {
  Mma3 g;
  uint64_t b3;
};

__device__ __forceinline__ Mma4 mk_mma4(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t a_sbo, uint32_t b_hi,
                                        uint32_t b_lo, uint32_t b_3, uint32_t b_sbo, uint32_t idesc, bool acc) {
  return Mma4{mk_mma3(d, a_hi, a_lo, a_sbo, b_hi, b_lo, b_sbo, idesc, acc), tc::smem_desc(b_3, 128, b_sbo)};
}

template <int KS>
__device__ __forceinline__ void mma4_chain(const Mma4& m) {
  const Mma3& g = m.g;
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const uint64_t o = (uint64_t)(16 * ks);
    tc::mma_bf16(g.d, g.ah + o, g.bh + o, g.idesc, (g.acc || ks > 0) ? 1u : 0u);
    tc::mma_bf16(g.d, g.ah + o, g.bl + o, g.idesc, 1u);
    tc::mma_bf16(g.d, g.al + o, g.bh + o, g.idesc, 1u);
    tc::mma_bf16(g.d, g.ah + o, m.b3 + o, g.idesc, 1u);
  }
}

// Operand formats.  A tile of R rows by K values takes R K 4 bytes in both:
// format 0 holds the bf16 hi part at the tile base and the lo part `part`
// bytes after it (three products per K step of 16); format 1 holds tf32
// values (one product per K step of 8).  Both use the K-major no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix), and one
// instruction's K step is 256 bytes (16 in the descriptor address) in both.
template <int FMT>
struct OpFmt;

template <>
struct OpFmt<0> {
  __host__ __device__ static constexpr uint32_t sbo(int K) { return (uint32_t)(K / 8) * 128u; }
  __host__ __device__ static constexpr uint32_t idesc(int M, int Nn) { return tc::idesc_bf16(M, Nn); }
  __device__ static void st8(uint8_t* base, int part, int row, int k0, int K, const float (&x)[8]) {
    const uint32_t o = tc::kmajor_offset(row, k0, K);
    tc::split_store8(base + o, base + part + o, x);
  }
  __device__ static void st4(uint8_t* base, int part, int row, int k0, int K, const float (&x)[4]) {
    const uint32_t o = tc::kmajor_offset(row, k0, K);
    tc::split_store4(base + o, base + part + o, x);
  }
  __device__ static void st1(uint8_t* base, int part, int row, int k, int K, float x) {
    const uint32_t o = tc::kmajor_offset(row, k, K);
    __nv_bfloat16 h, l;
    tc::split_bf16(x, h, l);
    *reinterpret_cast<__nv_bfloat16*>(base + o) = h;
    *reinterpret_cast<__nv_bfloat16*>(base + part + o) = l;
  }
  // values at k0, k0 + 1 (k0 even): one 4-byte store per part
  __device__ static void st2(uint8_t* base, int part, int row, int k0, int K, float x0, float x1) {
    const uint32_t o = tc::kmajor_offset(row, k0, K);
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    *reinterpret_cast<__nv_bfloat162*>(base + o) = hb;
    *reinterpret_cast<__nv_bfloat162*>(base + part + o) = lb;
  }
  template <int KE>
  __device__ static void chain4(const Mma4& m) {
    mma4_chain<KE / 16>(m);
  }
  template <int KE>
  __device__ static void chain(const Mma3& g) {
    mma3_chain<KE / 16>(g);
  }
};

template <>
struct OpFmt<1> {
  __host__ __device__ static constexpr uint32_t sbo(int K) { return (uint32_t)(K / 4) * 128u; }
  __host__ __device__ static constexpr uint32_t idesc(int M, int Nn) { return tc::idesc_tf32(M, Nn); }
  __device__ static void st8(uint8_t* base, int, int row, int k0, int K, const float (&x)[8]) {
    uint8_t* d = base + tc::kmajor_offset4(row, k0, K);
    *reinterpret_cast<uint4*>(d) = make_uint4(tc::to_tf32(x[0]), tc::to_tf32(x[1]), tc::to_tf32(x[2]), tc::to_tf32(x[3]));
    *reinterpret_cast<uint4*>(d + 128) =
        make_uint4(tc::to_tf32(x[4]), tc::to_tf32(x[5]), tc::to_tf32(x[6]), tc::to_tf32(x[7]));
  }
  __device__ static void st4(uint8_t* base, int, int row, int k0, int K, const float (&x)[4]) {
    *reinterpret_cast<uint4*>(base + tc::kmajor_offset4(row, k0, K)) =
        make_uint4(tc::to_tf32(x[0]), tc::to_tf32(x[1]), tc::to_tf32(x[2]), tc::to_tf32(x[3]));
  }
  __device__ static void st1(uint8_t* base, int, int row, int k, int K, float x) {
    *reinterpret_cast<uint32_t*>(base + tc::kmajor_offset4(row, k, K)) = tc::to_tf32(x);
  }
  // values at k0, k0 + 1 (k0 even): one 8-byte store
  __device__ static void st2(uint8_t* base, int, int row, int k0, int K, float x0, float x1) {
    *reinterpret_cast<uint2*>(base + tc::kmajor_offset4(row, k0, K)) = make_uint2(tc::to_tf32(x0), tc::to_tf32(x1));
  }
  template <int KE>
  __device__ static void chain(const Mma3& g) {
#pragma unroll
    for (int ks = 0; ks < KE / 8; ++ks) {
      const uint64_t o = (uint64_t)(16 * ks);
      tc::mma_tf32(g.d, g.ah + o, g.bh + o, g.idesc, (g.acc || ks > 0) ? 1u : 0u);
    }
  }
  // tf32 operators are one part
  template <int KE>
  __device__ static void chain4(const Mma4& m) {
    chain<KE>(m.g);
  }
};

}  // namespace

// Host side: operator tiles in the operand formats.
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

// tf32 bits of x: round to nearest, ties away from zero, at bit 13.
uint32_t tf32_bits_rna(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return u & 0xffffe000u;
  return (u + 0x1000u) & 0xffffe000u;
}

// Writes a [R x K] operand tile of the given format: format 0, the split bf16
// parts (hi at dst, lo at dst + part_bytes); format 1, tf32 values in the
// 4-byte K-major layout (the same R K 4 bytes).
template <typename F>
void put_tile(int fmt, uint8_t* dst, size_t part_bytes, int R, int K, F value) {
  for (int r = 0; r < R; ++r)
    for (int k = 0; k < K; ++k) {
      const double x = value(r, k);
      if (fmt == 0) {
        const uint16_t h = bf16_bits_rne((float)x);
        const uint16_t l = bf16_bits_rne((float)(x - (double)bf16_bits_to_float(h)));
        const size_t off = host_kmajor_offset(r, k, K);
        std::memcpy(dst + off, &h, 2);
        std::memcpy(dst + part_bytes + off, &l, 2);
      } else {
        const uint32_t t = tf32_bits_rna((float)x);
        const size_t off = (size_t)(((r >> 3) * (K >> 2) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
        std::memcpy(dst + off, &t, 4);
      }
    }
}

// As put_tile, with the residual of the two-part bf16 split in a third part
// at dst + 2 part_bytes (format 0); format 1 as put_tile.
template <typename F>
void put_tile3(int fmt, uint8_t* dst, size_t part_bytes, int R, int K, F value) {
  put_tile(fmt, dst, part_bytes, R, K, value);
  if (fmt != 0) return;
  for (int r = 0; r < R; ++r)
    for (int k = 0; k < K; ++k) {
      const double x = value(r, k);
      const uint16_t h = bf16_bits_rne((float)x);
      const double rh = x - (double)bf16_bits_to_float(h);
      const uint16_t l = bf16_bits_rne((float)rh);
      const uint16_t t = bf16_bits_rne((float)(rh - (double)bf16_bits_to_float(l)));
      std::memcpy(dst + 2 * part_bytes + host_kmajor_offset(r, k, K), &t, 2);
    }
}

// The packed operators of a tensor-core stage with dimensions T, chunk by
// chunk in the order the kernel stages them: per volume chunk of QC points
// the A part (V_q, V_q^a) and the B part ((V_q^a)^T diag(w), V_q^T diag(w)),
// per update chunk of UQC points V_q M^^{-1} and P_q, then the face operators.
template <typename T>
void pack_dims(const RefOps& o, int fmt, std::vector<uint8_t>& out) {
  const int Np = o.Np, Nq = o.Nq, KP = T::KP, QC = T::QC;
  out.assign((size_t)T::SZ_OPS + T::SZ_FOPS, 0);
  for (int ch = 0; ch < T::NCH; ++ch) {
    uint8_t* v = out.data() + (size_t)ch * T::SZ_OPV;
    auto qn = [&](int r) { return ch * QC + r; };
    put_tile(fmt, v, T::B_V, QC, KP, [&](int r, int n) {
      const int q = qn(r);
      return (q < Nq && n < Np) ? o.Vq[q * Np + n] : 0.0;
    });
    put_tile(fmt, v + 2 * T::B_V, 3 * T::B_V, 3 * QC, KP, [&](int r, int n) {
      const int a = r / QC, q = qn(r % QC);
      return (q < Nq && n < Np) ? o.Vqa[(a * Nq + q) * Np + n] : 0.0;
    });
    for (int a = 0; a < 3; ++a)
      put_tile(fmt, v + 8 * T::B_V + 2 * a * T::B_P, T::B_P, KP, QC, [&](int n, int k) {
        const int q = qn(k);
        return (q < Nq && n < Np) ? o.Dw[(a * Np + n) * Nq + q] : 0.0;
      });
    put_tile(fmt, v + 8 * T::B_V + 6 * T::B_P, T::B_P, KP, QC, [&](int n, int k) {
      const int q = qn(k);
      return (q < Nq && n < Np) ? o.Vw[n * Nq + q] : 0.0;
    });
  }
  for (int ch = 0; ch < T::UNCH; ++ch) {
    auto qn = [&](int r) { return ch * T::UQC + r; };
    uint8_t* u = out.data() + (size_t)T::NCH * T::SZ_OPV + (size_t)ch * T::SZ_OPU;
    put_tile3(fmt, u, T::B_UV, T::UQC, KP, [&](int r, int n) {
      const int q = qn(r);
      return (q < Nq && n < Np) ? o.Vtilde[q * Np + n] : 0.0;
    });
    put_tile3(fmt, u + T::SZ_UA, T::B_UP, KP, T::UQC, [&](int n, int k) {
      const int q = qn(k);
      return (q < Nq && n < Np) ? o.Pq[n * Nq + q] : 0.0;
    });
  }
  // face operators: V_tri as [NFQ16 rows (q) x NFP16 (j)], the lift
  // V_tri^T diag(w_f) as [NFP16 rows (j) x NFQ16 (q)]
  const int Nfp = o.Nfp, Nfq = o.Nfq;
  uint8_t* fo = out.data() + (size_t)T::SZ_OPS;
  put_tile(fmt, fo, T::B_TRI, T::NFQ16, T::NFP16, [&](int q, int j) {
    return (q < Nfq && j < Nfp) ? o.Vtri[q * Nfp + j] : 0.0;
  });
  put_tile(fmt, fo + 2 * T::B_TRI, T::B_TRI, T::NFP16, T::NFQ16, [&](int j, int q) {
    return (q < Nfq && j < Nfp) ? o.VtriTw[j * Nfq + q] : 0.0;
  });
}

}  // namespace

// The kernel's compile-time face node lists equal the runtime face tables:
// node n lies on face f exactly when ginv[f][pi][n] >= 0, for every pi.
template <int N>
bool face_nodes_match(const RefOps& o) {
  constexpr FaceNodeList<N> FN = make_face_nodes<N>();
  for (int f = 0; f < 4; ++f)
    for (int pi = 0; pi < 6; ++pi) {
      std::vector<int> on(o.Np, 0);
      for (int t = 0; t < FaceNodeList<N>::NFP; ++t) on[FN.v[f][t]] = 1;
      for (int n = 0; n < o.Np; ++n)
        if ((o.ginv[(f * 6 + pi) * o.Np + n] >= 0) != (on[n] != 0)) return false;
    }
  return true;
}

}  // namespace wadg
