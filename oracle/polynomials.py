"""Orthonormal Jacobi polynomials, Gauss-Jacobi rules and simplex bases (FP64).

Test infrastructure (see the package header).  The paper leaves the basis
free (Sec. 6: "any basis can be used with WADG") and integrates with rules
exact to degree 2N+1 (Sec. 4, Sec. 6.2); this oracle uses the orthonormal
collapsed-coordinate (Dubiner) basis, whose mass matrix on the reference
element is the identity, and collapsed Gauss-Jacobi rules built by the
Golub-Welsch eigenvalue method.
"""
from __future__ import annotations

import math

import numpy as np


def _recurrence(n: int, alpha: float, beta: float):
    """Jacobi-matrix entries (a_0..a_{n-1}, b_0..b_{n-1}) of the orthonormal
    Jacobi polynomials for the weight (1-x)^alpha (1+x)^beta on [-1, 1]:
        x p_m = b_m p_{m+1} + a_m p_m + b_{m-1} p_{m-1}.
    """
    m = np.arange(n, dtype=np.float64)
    s = 2.0 * m + alpha + beta
    a = np.empty(n)
    b = np.empty(n)
    for i in range(n):
        si = s[i]
        if i == 0:
            a[i] = (beta - alpha) / (alpha + beta + 2.0)
        else:
            a[i] = (beta * beta - alpha * alpha) / (si * (si + 2.0))
        num = 4.0 * (i + 1) * (i + alpha + 1) * (i + beta + 1) * (i + alpha + beta + 1)
        den = (si + 1.0) * (si + 2.0) ** 2 * (si + 3.0)
        b[i] = math.sqrt(num / den)
    return a, b


def _mu0(alpha: float, beta: float) -> float:
    """Integral of the weight (1-x)^alpha (1+x)^beta over [-1, 1]."""
    return 2.0 ** (alpha + beta + 1) * math.gamma(alpha + 1) * math.gamma(beta + 1) / math.gamma(alpha + beta + 2)


def jacobi(x, n: int, alpha: float, beta: float = 0.0) -> np.ndarray:
    """Orthonormal Jacobi polynomial p_n^{(alpha,beta)} evaluated at x."""
    x = np.asarray(x, dtype=np.float64)
    a, b = _recurrence(n + 1, alpha, beta)
    p_prev = np.zeros_like(x)
    p = np.full_like(x, 1.0 / math.sqrt(_mu0(alpha, beta)))
    for m in range(n):
        p_next = ((x - a[m]) * p - (b[m - 1] if m > 0 else 0.0) * p_prev) / b[m]
        p_prev, p = p, p_next
    return p


def djacobi(x, n: int, alpha: float, beta: float = 0.0) -> np.ndarray:
    """d/dx p_n^{(alpha,beta)} = sqrt(n (n+alpha+beta+1)) p_{n-1}^{(alpha+1,beta+1)}."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return math.sqrt(n * (n + alpha + beta + 1.0)) * jacobi(x, n - 1, alpha + 1.0, beta + 1.0)


def gauss_jacobi(npts: int, alpha: float, beta: float = 0.0):
    """Gauss-Jacobi nodes (ascending) and weights by Golub-Welsch.

    The nodes are the eigenvalues of the symmetric tridiagonal Jacobi matrix;
    each weight is mu0 times the squared first component of the normalised
    eigenvector.  Exact for polynomials of degree 2 npts - 1 against the
    weight (1-x)^alpha (1+x)^beta.
    """
    a, b = _recurrence(npts, alpha, beta)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    x, V = np.linalg.eigh(T)
    w = _mu0(alpha, beta) * V[0, :] ** 2
    return x, w


# ----------------------------------------------------------------------------
# Reference simplices.  Tetrahedron {r,s,t >= -1, r+s+t <= -1}; triangle
# {r,s >= -1, r+s <= 0}.  Collapsed coordinates (a,b,c) in [-1,1]^3:
#   r = (1+a)(1-b)(1-c)/4 - 1,  s = (1+b)(1-c)/2 - 1,  t = c.
# ----------------------------------------------------------------------------

def tet_index(N: int):
    """Modal index list (i,j,k), i+j+k <= N."""
    return [(i, j, k) for i in range(N + 1) for j in range(N + 1 - i) for k in range(N + 1 - i - j)]


def tri_index(N: int):
    return [(i, j) for i in range(N + 1) for j in range(N + 1 - i)]


def rst_to_abc(r, s, t):
    r, s, t = (np.asarray(v, dtype=np.float64) for v in (r, s, t))
    st = -s - t
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(np.abs(st) > 1e-14, 2.0 * (1.0 + r) / np.where(np.abs(st) > 1e-14, st, 1.0) - 1.0, -1.0)
        b = np.where(np.abs(1.0 - t) > 1e-14, 2.0 * (1.0 + s) / np.where(np.abs(1.0 - t) > 1e-14, 1.0 - t, 1.0) - 1.0, -1.0)
    return a, b, t.copy()


def dubiner_tet(N: int, r, s, t) -> np.ndarray:
    """Orthonormal tetrahedral basis values, shape (npts, Np).

    psi_ijk = 2 sqrt(2) p_i^{(0,0)}(a) p_j^{(2i+1,0)}(b) (1-b)^i
                        p_k^{(2i+2j+2,0)}(c) (1-c)^{i+j}.
    """
    a, b, c = rst_to_abc(r, s, t)
    cols = []
    for (i, j, k) in tet_index(N):
        cols.append(2.0 * math.sqrt(2.0) * jacobi(a, i, 0.0) * jacobi(b, j, 2 * i + 1.0) * (1 - b) ** i
                    * jacobi(c, k, 2 * i + 2 * j + 2.0) * (1 - c) ** (i + j))
    return np.stack(cols, axis=-1)


def dubiner_tet_grad(N: int, r, s, t):
    """(d/dr, d/ds, d/dt) of the tetrahedral basis, each (npts, Np).

    Chain rule through the collapsed coordinates with
      da/dr = 4/((1-b)(1-c)),  da/ds = da/dt = 2(1+a)/((1-b)(1-c)),
      db/ds = 2/(1-c),  db/dt = (1+b)/(1-c),  dc/dt = 1,
    where the factors (1-b)^{-1}(1-c)^{-1} are cancelled against the basis'
    own (1-b)^i (1-c)^{i+j} before evaluation.  Valid away from the collapsed
    vertex and edge (b = 1 or c = 1), i.e. at every quadrature point used.
    """
    a, b, c = rst_to_abc(r, s, t)
    cr, cs, ct = [], [], []
    k2 = 2.0 * math.sqrt(2.0)
    for (i, j, k) in tet_index(N):
        fa, dfa = jacobi(a, i, 0.0), djacobi(a, i, 0.0)
        gb, dgb = jacobi(b, j, 2 * i + 1.0), djacobi(b, j, 2 * i + 1.0)
        hc, dhc = jacobi(c, k, 2 * i + 2 * j + 2.0), djacobi(c, k, 2 * i + 2 * j + 2.0)
        # dpsi/da divided by (1-b)(1-c)
        if i >= 1:
            da_red = k2 * dfa * gb * (1 - b) ** (i - 1) * hc * (1 - c) ** (i + j - 1)
        else:
            da_red = np.zeros_like(a)
        # dpsi/db divided by (1-c)
        db_val = dgb * (1 - b) ** i - (i * gb * (1 - b) ** (i - 1) if i >= 1 else 0.0)
        if i + j >= 1:
            db_red = k2 * fa * db_val * hc * (1 - c) ** (i + j - 1)
        else:
            db_red = np.zeros_like(a)
        # dpsi/dc
        dc_val = dhc * (1 - c) ** (i + j) - ((i + j) * hc * (1 - c) ** (i + j - 1) if i + j >= 1 else 0.0)
        dpsi_dc = k2 * fa * gb * (1 - b) ** i * dc_val
        dr = 4.0 * da_red
        ds = 2.0 * (1 + a) * da_red + 2.0 * db_red
        dt = 2.0 * (1 + a) * da_red + (1 + b) * db_red + dpsi_dc
        cr.append(dr)
        cs.append(ds)
        ct.append(dt)
    return np.stack(cr, -1), np.stack(cs, -1), np.stack(ct, -1)


def dubiner_tri(N: int, r, s) -> np.ndarray:
    """Orthonormal triangle basis sqrt(2) p_i(a) p_j^{(2i+1,0)}(b)(1-b)^i, (npts, Nfp)."""
    r, s = np.asarray(r, dtype=np.float64), np.asarray(s, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(np.abs(1 - s) > 1e-14, 2.0 * (1 + r) / np.where(np.abs(1 - s) > 1e-14, 1 - s, 1.0) - 1.0, -1.0)
    b = s
    cols = [math.sqrt(2.0) * jacobi(a, i, 0.0) * jacobi(b, j, 2 * i + 1.0) * (1 - b) ** i for (i, j) in tri_index(N)]
    return np.stack(cols, -1)


def tet_rule(n: int):
    """Collapsed Gauss-Jacobi rule with n points per direction on the tetrahedron.

    Exact for total degree 2n-1.  Point (ia, ib, ic) has index
    ia + n (ib + n ic).  Returns (rst (n^3, 3), w (n^3,)).
    """
    xa, wa = gauss_jacobi(n, 0.0)
    xb, wb = gauss_jacobi(n, 1.0)
    xc, wc = gauss_jacobi(n, 2.0)
    C, B, A = np.meshgrid(xc, xb, xa, indexing="ij")
    WC, WB, WA = np.meshgrid(wc, wb, wa, indexing="ij")
    A, B, C = A.ravel(), B.ravel(), C.ravel()
    r = (1 + A) * (1 - B) * (1 - C) / 4.0 - 1.0
    s = (1 + B) * (1 - C) / 2.0 - 1.0
    t = C
    w = (WA * WB * WC).ravel() / 8.0
    return np.stack([r, s, t], axis=1), w


def tri_rule(n: int):
    """Collapsed Gauss-Jacobi rule with n points per direction on the triangle.

    Exact for total degree 2n-1.  Point (ia, ib) has index ia + n ib.
    """
    xa, wa = gauss_jacobi(n, 0.0)
    xb, wb = gauss_jacobi(n, 1.0)
    B, A = np.meshgrid(xb, xa, indexing="ij")
    WB, WA = np.meshgrid(wb, wa, indexing="ij")
    A, B = A.ravel(), B.ravel()
    r = (1 + A) * (1 - B) / 2.0 - 1.0
    s = B
    w = (WA * WB).ravel() / 2.0
    return np.stack([r, s], axis=1), w
