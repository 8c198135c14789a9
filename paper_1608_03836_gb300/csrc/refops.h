// Reference-element operators for the WADG library (host, FP64).
//
// Everything here depends only on the degree N: quadrature rules, the nodal
// basis at the equispaced lattice, and the reference matrices of the volume,
// surface and update kernels (Chan, Hewett & Warburton, Sec. 6.2-6.4).
#pragma once

#include <vector>

namespace wadg {

struct RefOps {
  int N = 0, Np = 0, Nq = 0, Nfp = 0, Nfq = 0;
  // equispaced lattice, [Np] each
  std::vector<double> r, s, t;
  // volume rule (degree 2N+1), [Nq]
  std::vector<double> rq, sq, tq, wq;
  // face rule on the reference triangle (degree 2N+1), [Nfq]
  std::vector<double> rf, sf, wf;
  // Nodal (Lagrange at the lattice) operators, row-major:
  std::vector<double> Vq;      // [Nq][Np]     l_n(x_q)
  std::vector<double> Vqa;     // [3][Nq][Np]  dl_n/dx^_a (x_q)
  std::vector<double> Minv;    // [Np][Np]     M^^{-1}
  std::vector<double> Vtilde;  // [Nq][Np]     V_q M^^{-1}
  std::vector<double> Pq;      // [Np][Nq]     M^^{-1} V_q^T diag(w)
  std::vector<double> Dw;      // [3][Np][Nq]  (V_q^a)^T diag(w)
  std::vector<double> Vw;      // [Np][Nq]     V_q^T diag(w)
  std::vector<double> Vtri;    // [Nfq][Nfp]   triangle Lagrange basis at face points
  std::vector<double> VtriTw;  // [Nfp][Nfq]   V_tri^T diag(w_f)
  std::vector<double> Vf;      // [4][Nfq][Np] l_n at face-f points
  std::vector<double> Vfa;     // [4][3][Nfq][Np] dl_n/dx^_a at face-f points
  std::vector<int> Fmask;      // [4][Nfp] volume node of face-lattice node j
  std::vector<int> gidx;       // [4][6][Nfp] volume node at owner-order position j
  std::vector<int> ginv;       // [4][6][Np] owner-order position of node n (-1: not on face)
  std::vector<double> VnInv;   // [Np][Np] modal coefficients of the Lagrange basis
  std::vector<double> VtInv;   // [Nfp][Nfp] same for the triangle lattice
};

// A second pair of rules on the same element: collapsed rules with nv points
// per direction on the volume (exact to degree 2 nv - 1) and nf on each face,
// with the operators that the strong form's volume and surface terms use.
struct RuleOps {
  int nv = 0, nf = 0, Nq = 0, Nfq = 0;
  std::vector<double> rq, sq, tq, wq;  // [Nq]
  std::vector<double> rf, sf, wf;      // [Nfq] on the reference triangle
  std::vector<double> Vqa;     // [3][Nq][Np]  dl_n/dx^_a (x_q)
  std::vector<double> Vq;      // [Nq][Np]     l_n(x_q)
  std::vector<double> Vtri;    // [Nfq][Nfp]   triangle Lagrange basis at the face points
  std::vector<double> VtriTw;  // [Nfp][Nfq]   V_tri^T diag(w_f)
  std::vector<double> Vfa;     // [4][3][Nfq][Np] dl_n/dx^_a at face-f points
};

// Points per direction of the strong form's rules (Sec. 4.1).  form 1: the
// energy-stable rules, exact for the degree 4N-3 volume and 4N-2 surface
// integrands of an isoparametric map (max(N+1, 2N-1) and 2N points); form 2:
// the degree 2N+1 rules of the strong-weak form (N+1 and N+1 points).
void strong_rule_points(int N, int form, int* nv, int* nf);

// Builds the operators of the rules (nv, nf) for the element of o.
bool build_rule_ops(const RefOps& o, int nv, int nf, RuleOps& out, char* err, int errlen);

// The six vertex permutations sigma of a triangle, lexicographic.
extern const int kPerm[6][3];
// Reference outward normal times reference face area scale, per face.
extern const double kFaceNormal[4][3];

// Builds the operators; returns false (and a message) on failure.  The volume
// rule is the collapsed (N+1)^3 rule, or, when rule is given, its nq points
// rule[q] = (r, s, t, w) on the reference tetrahedron (weights positive,
// points inside; the operators are checked for P_q V_q = I).
bool build_refops(int N, RefOps& ops, char* err, int errlen, int nq = 0, const double* rule = nullptr);

// Gauss-Jacobi rule for the weight (1-x)^alpha (1+x)^beta, ascending nodes.
void gauss_jacobi(int n, double alpha, double beta, double* x, double* w);

// Lagrange basis at the lattice evaluated at arbitrary points (host).
// vals [npts][Np]; grads (nullable) [3][npts][Np].
void lattice_basis(const RefOps& ops, int npts, const double* r, const double* s, const double* t,
                   double* vals, double* grads);

inline int tri_lattice_index(int N, int i, int j) {
  // node (i,j), i fastest: rows j' < j hold N+1-j' nodes each
  return j * (N + 1) - j * (j - 1) / 2 + i;
}
int tet_lattice_index(int N, int i, int j, int k);

}  // namespace wadg
