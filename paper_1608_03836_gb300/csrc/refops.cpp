// Reference-element operators (host, FP64).  See refops.h.
//
// Basis: orthonormal collapsed-coordinate polynomials on the reference
// tetrahedron and triangle, turned into the Lagrange basis of the equispaced
// lattice by inverting the generalised Vandermonde matrix.  Quadrature:
// collapsed Gauss-Jacobi rules, nodes by Newton iteration with deflation on
// the classical Jacobi polynomial, weights by the Christoffel function
// w_k = 1 / sum_{m<n} p_m(x_k)^2 of the orthonormal polynomials.
#include "refops.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace wadg {

const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
const double kFaceNormal[4][3] = {{0, 0, -1}, {0, -1, 0}, {1, 1, 1}, {-1, 0, 0}};

static const double kRefV[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
static const int kFaceV[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

// ---------------------------------------------------------------------------
// Jacobi polynomials.  Classical P_n^{(a,b)} by the three-term recurrence
//   2n(n+a+b)(2n+a+b-2) P_n = (2n+a+b-1)((2n+a+b)(2n+a+b-2) x + a^2-b^2) P_{n-1}
//                             - 2(n+a-1)(n+b-1)(2n+a+b) P_{n-2},
// normalised by h_n = 2^{a+b+1}/(2n+a+b+1) G(n+a+1)G(n+b+1)/(G(n+a+b+1) n!).
// ---------------------------------------------------------------------------
static double jacobi_classical(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int m = 2; m <= n; ++m) {
    double c = 2.0 * m + a + b;
    double A = 2.0 * m * (m + a + b) * (c - 2.0);
    double B = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b);
    double C = 2.0 * (m + a - 1.0) * (m + b - 1.0) * c;
    double p2 = (B * p1 - C * p0) / A;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

static double jacobi_lognorm(int n, double a, double b) {
  // log h_n
  return (a + b + 1.0) * std::log(2.0) - std::log(2.0 * n + a + b + 1.0) + std::lgamma(n + a + 1.0) +
         std::lgamma(n + b + 1.0) - std::lgamma(n + a + b + 1.0) - std::lgamma(n + 1.0);
}

// Orthonormal p_n and its derivative.
static double jac(int n, double a, double b, double x) {
  return jacobi_classical(n, a, b, x) * std::exp(-0.5 * jacobi_lognorm(n, a, b));
}
static double djac(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  // d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}
  double dP = 0.5 * (n + a + b + 1.0) * jacobi_classical(n - 1, a + 1.0, b + 1.0, x);
  return dP * std::exp(-0.5 * jacobi_lognorm(n, a, b));
}

void gauss_jacobi(int n, double alpha, double beta, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    double xk = -std::cos((2.0 * k + 1.0) * pi / (2.0 * n));
    if (k > 0) xk = 0.5 * (xk + x[k - 1]);
    for (int it = 0; it < 100; ++it) {
      double p = jacobi_classical(n, alpha, beta, xk);
      double dp = 0.5 * (n + alpha + beta + 1.0) * jacobi_classical(n - 1, alpha + 1.0, beta + 1.0, xk);
      double defl = 0.0;
      for (int j = 0; j < k; ++j) defl += 1.0 / (xk - x[j]);
      double delta = -p / (dp - defl * p);
      xk += delta;
      if (std::fabs(delta) < 1e-16) break;
    }
    x[k] = xk;
  }
  std::sort(x, x + n);
  for (int k = 0; k < n; ++k) {
    double sum = 0.0;
    for (int m = 0; m < n; ++m) {
      double p = jac(m, alpha, beta, x[k]);
      sum += p * p;
    }
    w[k] = 1.0 / sum;
  }
}

// ---------------------------------------------------------------------------
// Orthonormal simplex bases.  Collapsed coordinates of the tetrahedron:
//   a = 2(1+r)/(-s-t) - 1, b = 2(1+s)/(1-t) - 1, c = t.
//   psi_ijk = 2 sqrt2 p_i(a) p_j^{(2i+1,0)}(b) (1-b)^i p_k^{(2i+2j+2,0)}(c) (1-c)^{i+j}
// ---------------------------------------------------------------------------
static void collapse(double r, double s, double t, double& a, double& b, double& c) {
  double d = -s - t;
  a = (std::fabs(d) > 1e-14) ? 2.0 * (1.0 + r) / d - 1.0 : -1.0;
  b = (std::fabs(1.0 - t) > 1e-14) ? 2.0 * (1.0 + s) / (1.0 - t) - 1.0 : -1.0;
  c = t;
}

static double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// values [Np], grads [3][Np] (nullable) at one point
static void tet_modal(int N, double r, double s, double t, double* v, double* g, int Np) {
  double a, b, c;
  collapse(r, s, t, a, b, c);
  const double k2 = 2.0 * std::sqrt(2.0);
  int m = 0;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j)
      for (int k = 0; k <= N - i - j; ++k, ++m) {
        double fa = jac(i, 0, 0, a), ga = jac(j, 2 * i + 1, 0, b), ha = jac(k, 2 * i + 2 * j + 2, 0, c);
        v[m] = k2 * fa * ga * ipow(1 - b, i) * ha * ipow(1 - c, i + j);
        if (!g) continue;
        double dfa = djac(i, 0, 0, a), dga = djac(j, 2 * i + 1, 0, b), dha = djac(k, 2 * i + 2 * j + 2, 0, c);
        // dpsi/da / ((1-b)(1-c))
        double A = (i >= 1) ? k2 * dfa * ga * ipow(1 - b, i - 1) * ha * ipow(1 - c, i + j - 1) : 0.0;
        // dpsi/db / (1-c)
        double gb = dga * ipow(1 - b, i) - (i >= 1 ? i * ga * ipow(1 - b, i - 1) : 0.0);
        double B = (i + j >= 1) ? k2 * fa * gb * ha * ipow(1 - c, i + j - 1) : 0.0;
        // dpsi/dc
        double hc = dha * ipow(1 - c, i + j) - (i + j >= 1 ? (i + j) * ha * ipow(1 - c, i + j - 1) : 0.0);
        double C = k2 * fa * ga * ipow(1 - b, i) * hc;
        g[0 * Np + m] = 4.0 * A;
        g[1 * Np + m] = 2.0 * (1.0 + a) * A + 2.0 * B;
        g[2 * Np + m] = 2.0 * (1.0 + a) * A + (1.0 + b) * B + C;
      }
}

static void tri_modal(int N, double r, double s, double* v) {
  double a = (std::fabs(1.0 - s) > 1e-14) ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
  double b = s;
  int m = 0;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j, ++m) v[m] = std::sqrt(2.0) * jac(i, 0, 0, a) * jac(j, 2 * i + 1, 0, b) * ipow(1 - b, i);
}

// Gauss-Jordan inverse with partial pivoting, n x n row-major.
static bool invert(int n, const std::vector<double>& A, std::vector<double>& Ainv) {
  std::vector<double> M(A);
  Ainv.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Ainv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(M[r * n + col]) > std::fabs(M[piv * n + col])) piv = r;
    if (std::fabs(M[piv * n + col]) < 1e-300) return false;
    if (piv != col)
      for (int c = 0; c < n; ++c) {
        std::swap(M[piv * n + c], M[col * n + c]);
        std::swap(Ainv[piv * n + c], Ainv[col * n + c]);
      }
    double d = 1.0 / M[col * n + col];
    for (int c = 0; c < n; ++c) {
      M[col * n + c] *= d;
      Ainv[col * n + c] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = M[r * n + col];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        M[r * n + c] -= f * M[col * n + c];
        Ainv[r * n + c] -= f * Ainv[col * n + c];
      }
    }
  }
  return true;
}

int tet_lattice_index(int N, int i, int j, int k) {
  int idx = 0;
  for (int kk = 0; kk < k; ++kk) idx += (N - kk + 1) * (N - kk + 2) / 2;
  return idx + tri_lattice_index(N - k, i, j);
}

static void eval_nodal(int N, int Np, const std::vector<double>& VnInv, int npts, const double* r, const double* s,
                       const double* t, double* vals, double* grads) {
  std::vector<double> v(Np), g(3 * Np);
  for (int p = 0; p < npts; ++p) {
    tet_modal(N, r[p], s[p], t[p], v.data(), grads ? g.data() : nullptr, Np);
    // l_n(x) = sum_m psi_m(x) VnInv[m][n]
    for (int n = 0; n < Np; ++n) {
      double acc = 0.0;
      for (int m = 0; m < Np; ++m) acc += v[m] * VnInv[m * Np + n];
      vals[p * Np + n] = acc;
      if (grads)
        for (int a = 0; a < 3; ++a) {
          double ga = 0.0;
          for (int m = 0; m < Np; ++m) ga += g[a * Np + m] * VnInv[m * Np + n];
          grads[(size_t)a * npts * Np + p * Np + n] = ga;
        }
    }
  }
}

void lattice_basis(const RefOps& ops, int npts, const double* r, const double* s, const double* t, double* vals,
                   double* grads) {
  eval_nodal(ops.N, ops.Np, ops.VnInv, npts, r, s, t, vals, grads);
}

// Collapsed Gauss-Jacobi rule with n points per direction on the reference
// tetrahedron (exact to degree 2n-1); point (ia, ib, ic) at ia + n (ib + n ic).
static void tet_rule(int n, std::vector<double>& r, std::vector<double>& s, std::vector<double>& t,
                     std::vector<double>& w) {
  std::vector<double> xa(n), wa(n), xb(n), wb(n), xc(n), wc(n);
  gauss_jacobi(n, 0.0, 0.0, xa.data(), wa.data());
  gauss_jacobi(n, 1.0, 0.0, xb.data(), wb.data());
  gauss_jacobi(n, 2.0, 0.0, xc.data(), wc.data());
  const int nq = n * n * n;
  r.resize(nq);
  s.resize(nq);
  t.resize(nq);
  w.resize(nq);
  for (int ic = 0; ic < n; ++ic)
    for (int ib = 0; ib < n; ++ib)
      for (int ia = 0; ia < n; ++ia) {
        int q = ia + n * (ib + n * ic);
        double a = xa[ia], b = xb[ib], c = xc[ic];
        r[q] = 0.25 * (1 + a) * (1 - b) * (1 - c) - 1.0;
        s[q] = 0.5 * (1 + b) * (1 - c) - 1.0;
        t[q] = c;
        w[q] = wa[ia] * wb[ib] * wc[ic] / 8.0;
      }
}

// Collapsed rule with n points per direction on the reference triangle.
static void tri_rule(int n, std::vector<double>& r, std::vector<double>& s, std::vector<double>& w) {
  std::vector<double> xa(n), wa(n), xb(n), wb(n);
  gauss_jacobi(n, 0.0, 0.0, xa.data(), wa.data());
  gauss_jacobi(n, 1.0, 0.0, xb.data(), wb.data());
  r.resize(n * n);
  s.resize(n * n);
  w.resize(n * n);
  for (int ib = 0; ib < n; ++ib)
    for (int ia = 0; ia < n; ++ia) {
      int q = ia + n * ib;
      r[q] = 0.5 * (1 + xa[ia]) * (1 - xb[ib]) - 1.0;
      s[q] = xb[ib];
      w[q] = wa[ia] * wb[ib] / 2.0;
    }
}

// Triangle Lagrange basis of the degree-N lattice at npts points: out [npts][Nfp].
static void tri_lagrange(int N, int Nfp, const std::vector<double>& VtInv, int npts, const double* r, const double* s,
                         double* out) {
  std::vector<double> vt(Nfp);
  for (int q = 0; q < npts; ++q) {
    tri_modal(N, r[q], s[q], vt.data());
    for (int j = 0; j < Nfp; ++j) {
      double acc = 0.0;
      for (int m = 0; m < Nfp; ++m) acc += vt[m] * VtInv[m * Nfp + j];
      out[q * Nfp + j] = acc;
    }
  }
}

// Basis values Vf [4][npts][Np] (nullable) and derivatives Vfa [4][3][npts][Np]
// at the images of the triangle points (rf, sf) on each face.
static void face_ops(int N, int Np, const std::vector<double>& VnInv, int npts, const double* rf, const double* sf,
                     double* Vf, double* Vfa) {
  std::vector<double> fr(npts), fs(npts), ft(npts), vals((size_t)npts * Np);
  for (int f = 0; f < 4; ++f) {
    const double* A = kRefV[kFaceV[f][0]];
    const double* B = kRefV[kFaceV[f][1]];
    const double* C = kRefV[kFaceV[f][2]];
    for (int q = 0; q < npts; ++q) {
      double la = -0.5 * (rf[q] + sf[q]), lb = 0.5 * (1 + rf[q]), lc = 0.5 * (1 + sf[q]);
      fr[q] = la * A[0] + lb * B[0] + lc * C[0];
      fs[q] = la * A[1] + lb * B[1] + lc * C[1];
      ft[q] = la * A[2] + lb * B[2] + lc * C[2];
    }
    eval_nodal(N, Np, VnInv, npts, fr.data(), fs.data(), ft.data(), Vf ? &Vf[(size_t)f * npts * Np] : vals.data(),
               &Vfa[(size_t)f * 3 * npts * Np]);
  }
}

void strong_rule_points(int N, int form, int* nv, int* nf) {
  if (form == 1) {
    *nv = std::max(N + 1, 2 * N - 1);
    *nf = 2 * N;
  } else {
    *nv = N + 1;
    *nf = N + 1;
  }
}

bool build_rule_ops(const RefOps& o, int nv, int nf, RuleOps& out, char* err, int errlen) {
  if (o.N < 1 || nv < 1 || nf < 1 || nv > 16 || nf > 16 || (int)o.VtInv.size() != o.Nfp * o.Nfp) {
    std::snprintf(err, errlen, "rules (%d, %d) for N=%d", nv, nf, o.N);
    return false;
  }
  const int N = o.N, Np = o.Np, Nfp = o.Nfp;
  out.nv = nv;
  out.nf = nf;
  tet_rule(nv, out.rq, out.sq, out.tq, out.wq);
  tri_rule(nf, out.rf, out.sf, out.wf);
  out.Nq = nv * nv * nv;
  out.Nfq = nf * nf;
  out.Vq.assign((size_t)out.Nq * Np, 0.0);
  out.Vqa.assign((size_t)3 * out.Nq * Np, 0.0);
  eval_nodal(N, Np, o.VnInv, out.Nq, out.rq.data(), out.sq.data(), out.tq.data(), out.Vq.data(), out.Vqa.data());
  out.Vtri.assign((size_t)out.Nfq * Nfp, 0.0);
  tri_lagrange(N, Nfp, o.VtInv, out.Nfq, out.rf.data(), out.sf.data(), out.Vtri.data());
  out.VtriTw.assign((size_t)Nfp * out.Nfq, 0.0);
  for (int j = 0; j < Nfp; ++j)
    for (int q = 0; q < out.Nfq; ++q) out.VtriTw[j * out.Nfq + q] = out.Vtri[q * Nfp + j] * out.wf[q];
  out.Vfa.assign((size_t)4 * 3 * out.Nfq * Np, 0.0);
  face_ops(N, Np, o.VnInv, out.Nfq, out.rf.data(), out.sf.data(), nullptr, out.Vfa.data());
  return true;
}

bool build_refops(int N, RefOps& o, char* err, int errlen, int nq, const double* rule) {
  if (N < 1 || N > 6) {
    std::snprintf(err, errlen, "degree N=%d outside 1..6", N);
    return false;
  }
  o.N = N;
  o.Np = (N + 1) * (N + 2) * (N + 3) / 6;
  o.Nfp = (N + 1) * (N + 2) / 2;
  o.Nq = rule ? nq : (N + 1) * (N + 1) * (N + 1);
  o.Nfq = (N + 1) * (N + 1);
  const int Np = o.Np, Nq = o.Nq, Nfp = o.Nfp, Nfq = o.Nfq, n1 = N + 1;

  // lattice
  o.r.resize(Np);
  o.s.resize(Np);
  o.t.resize(Np);
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j <= N - k; ++j)
      for (int i = 0; i <= N - j - k; ++i) {
        int id = tet_lattice_index(N, i, j, k);
        o.r[id] = -1.0 + 2.0 * i / N;
        o.s[id] = -1.0 + 2.0 * j / N;
        o.t[id] = -1.0 + 2.0 * k / N;
      }

  // rules
  if (rule) {
    if (nq < 1) {
      std::snprintf(err, errlen, "volume rule with %d points", nq);
      return false;
    }
    o.rq.resize(nq);
    o.sq.resize(nq);
    o.tq.resize(nq);
    o.wq.resize(nq);
    for (int q = 0; q < nq; ++q) {
      o.rq[q] = rule[4 * q];
      o.sq[q] = rule[4 * q + 1];
      o.tq[q] = rule[4 * q + 2];
      o.wq[q] = rule[4 * q + 3];
      const double l0 = -(1.0 + o.rq[q] + o.sq[q] + o.tq[q]) / 2;
      const bool inside = std::isfinite(l0) && l0 >= -1e-12 && o.rq[q] >= -1 - 1e-12 && o.sq[q] >= -1 - 1e-12 &&
                          o.tq[q] >= -1 - 1e-12;
      if (!inside || !(o.wq[q] > 0)) {
        std::snprintf(err, errlen, "volume rule point %d is outside the tetrahedron or has weight <= 0", q);
        return false;
      }
    }
  } else {
    tet_rule(n1, o.rq, o.sq, o.tq, o.wq);
  }
  tri_rule(n1, o.rf, o.sf, o.wf);

  // Vandermonde at the lattice and its inverse
  std::vector<double> Vn(Np * Np), VnInv, tmp(3 * Np);
  for (int p = 0; p < Np; ++p) tet_modal(N, o.r[p], o.s[p], o.t[p], &Vn[p * Np], nullptr, Np);
  if (!invert(Np, Vn, VnInv)) {
    std::snprintf(err, errlen, "singular lattice Vandermonde (N=%d)", N);
    return false;
  }
  o.VnInv = VnInv;

  // volume operators
  o.Vq.assign(Nq * Np, 0.0);
  o.Vqa.assign(3 * Nq * Np, 0.0);
  eval_nodal(N, Np, VnInv, Nq, o.rq.data(), o.sq.data(), o.tq.data(), o.Vq.data(), o.Vqa.data());
  // M^^{-1} = Vn Vn^T
  o.Minv.assign(Np * Np, 0.0);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double acc = 0.0;
      for (int m = 0; m < Np; ++m) acc += Vn[i * Np + m] * Vn[j * Np + m];
      o.Minv[i * Np + j] = acc;
    }
  o.Vtilde.assign(Nq * Np, 0.0);
  for (int q = 0; q < Nq; ++q)
    for (int j = 0; j < Np; ++j) {
      double acc = 0.0;
      for (int m = 0; m < Np; ++m) acc += o.Vq[q * Np + m] * o.Minv[m * Np + j];
      o.Vtilde[q * Np + j] = acc;
    }
  o.Vw.assign(Np * Nq, 0.0);
  o.Dw.assign(3 * Np * Nq, 0.0);
  for (int n = 0; n < Np; ++n)
    for (int q = 0; q < Nq; ++q) {
      o.Vw[n * Nq + q] = o.Vq[q * Np + n] * o.wq[q];
      for (int a = 0; a < 3; ++a) o.Dw[(a * Np + n) * Nq + q] = o.Vqa[(a * Nq + q) * Np + n] * o.wq[q];
    }
  o.Pq.assign(Np * Nq, 0.0);
  for (int i = 0; i < Np; ++i)
    for (int q = 0; q < Nq; ++q) {
      double acc = 0.0;
      for (int m = 0; m < Np; ++m) acc += o.Minv[i * Np + m] * o.Vw[m * Nq + q];
      o.Pq[i * Nq + q] = acc;
    }
  // self-check P_q V_q = I (exactness of the rule to degree 2N)
  double maxdev = 0.0;
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double acc = 0.0;
      for (int q = 0; q < Nq; ++q) acc += o.Pq[i * Nq + q] * o.Vq[q * Np + j];
      maxdev = std::max(maxdev, std::fabs(acc - (i == j ? 1.0 : 0.0)));
    }
  if (maxdev > 1e-10) {
    std::snprintf(err, errlen, "P_q V_q != I (dev %.3e) for N=%d", maxdev, N);
    return false;
  }

  // face operators: triangle Lagrange basis of the face lattice at face points
  std::vector<double> Vt(Nfp * Nfp), VtInv;
  for (int j = 0; j <= N; ++j)
    for (int i = 0; i <= N - j; ++i) {
      int id = tri_lattice_index(N, i, j);
      tri_modal(N, -1.0 + 2.0 * i / N, -1.0 + 2.0 * j / N, &Vt[id * Nfp]);
    }
  if (!invert(Nfp, Vt, VtInv)) {
    std::snprintf(err, errlen, "singular triangle Vandermonde (N=%d)", N);
    return false;
  }
  o.VtInv = VtInv;
  o.Vtri.assign(Nfq * Nfp, 0.0);
  tri_lagrange(N, Nfp, VtInv, Nfq, o.rf.data(), o.sf.data(), o.Vtri.data());
  o.VtriTw.assign(Nfp * Nfq, 0.0);
  for (int j = 0; j < Nfp; ++j)
    for (int q = 0; q < Nfq; ++q) o.VtriTw[j * Nfq + q] = o.Vtri[q * Nfp + j] * o.wf[q];

  // face points, basis and derivatives there
  o.Vf.assign(4 * Nfq * Np, 0.0);
  o.Vfa.assign(4 * 3 * Nfq * Np, 0.0);
  face_ops(N, Np, VnInv, Nfq, o.rf.data(), o.sf.data(), o.Vf.data(), o.Vfa.data());

  // Fmask: face-lattice node (i,j) of face f -> volume node
  o.Fmask.assign(4 * Nfp, -1);
  for (int f = 0; f < 4; ++f)
    for (int j = 0; j <= N; ++j)
      for (int i = 0; i <= N - j; ++i) {
        double la = double(N - i - j) / N, lb = double(i) / N, lc = double(j) / N;
        double x[3];
        for (int d = 0; d < 3; ++d)
          x[d] = la * kRefV[kFaceV[f][0]][d] + lb * kRefV[kFaceV[f][1]][d] + lc * kRefV[kFaceV[f][2]][d];
        int I = (int)std::lround((x[0] + 1.0) * N / 2.0);
        int J = (int)std::lround((x[1] + 1.0) * N / 2.0);
        int K = (int)std::lround((x[2] + 1.0) * N / 2.0);
        o.Fmask[f * Nfp + tri_lattice_index(N, i, j)] = tet_lattice_index(N, I, J, K);
      }
  // gidx[f][pi][j]: volume node of my face holding the owner-order node j.
  // Owner node j = (i,j) has owner barycentrics beta = (N-i-j, i, j); mine are
  // beta'[m] = beta[sigma(m)].
  o.gidx.assign(4 * 6 * Nfp, -1);
  o.ginv.assign(4 * 6 * Np, -1);
  for (int f = 0; f < 4; ++f)
    for (int pi = 0; pi < 6; ++pi)
      for (int j = 0; j <= N; ++j)
        for (int i = 0; i <= N - j; ++i) {
          int beta[3] = {N - i - j, i, j};
          int mine[3] = {beta[kPerm[pi][0]], beta[kPerm[pi][1]], beta[kPerm[pi][2]]};
          int jo = tri_lattice_index(N, i, j);
          int vol = o.Fmask[f * Nfp + tri_lattice_index(N, mine[1], mine[2])];
          o.gidx[(f * 6 + pi) * Nfp + jo] = vol;
          o.ginv[(f * 6 + pi) * Np + vol] = jo;
        }
  return true;
}

}  // namespace wadg
