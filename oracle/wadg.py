"""Strong-weak DG for acoustics with exact or weight-adjusted mass inverse (FP64).

Test infrastructure (see the package header).  All arrays of coefficients are
modal (orthonormal basis, reference mass matrix M^ = I); the nodal interface
format is reached through RefTet.to_modal / to_nodal.

Passages followed (Chan, Hewett & Warburton, arXiv:1608.03836):
  * Sec. 4.1, strong-weak formulation: for test functions (v, tau) on D^k
        int (1/c^2) p_t v   =  int u . grad v
                               - int_{dD} 1/2 (2 {u}.n - tau_p [p]) v
        int u_t . tau       = -int grad p . tau
                               - int_{dD} 1/2 ([p] - tau_u [u].n) tau . n
    with [q] = q+ - q-, {q} = (q+ + q-)/2; on the boundary p+ = -p-,
    u+ = u- (homogeneous Dirichlet, Sec. 4.1).
  * Sec. 4: dQ/dt = -M^{-1} A_h Q, M block diagonal with (M_J)_ij = int phi_i
    phi_j J; WADG replaces M_J^{-1} by M^^{-1} M_{1/J} M^^{-1}.
  * Sec. 6.2, Eq. (matfree): M~^{-1} A_h Q = P_q diag(1/J_q) V_q M^^{-1} A_h Q.
  * Sec. 7: with variable c^2 the pressure row uses diag(c^2_q/J_q).
  * Sec. 3, Theorem (pseudo-projection): P_N u = Pi_N(J^{-1} Pi_N(u J)).
  * Sec. 5.2: low-storage five-stage fourth-order Runge-Kutta of Carpenter and
    Kennedy (1994).  The paper does not print the coefficients; the published
    rational set is used and pinned by its order conditions in the tests.
"""
from __future__ import annotations

import numpy as np

from . import polynomials as P
from .discretization import Mesh, RefTet


# ---------------------------------------------------------------------------
# Strong-weak right-hand side a_h(Q) (the functional tested against the
# basis, before any mass inverse).  Q: (4, K, Np) modal -> (4, K, Np) modal.
# ---------------------------------------------------------------------------

def traces(mesh: Mesh, c: np.ndarray):
    """Own and neighbour traces at each face's owner quadrature points.

    Returns (minus, plus), each (4, K, 4, Nfq).  Boundary faces get the ghost
    state p+ = -p-, u+ = u-.
    """
    K = mesh.K
    Nfq = mesh.ref.Nfq
    minus = np.zeros((4, K, 4, Nfq))
    for (f, sig), ks in mesh.face_groups.items():
        V = mesh.face_V[(f, sig)]
        minus[:, ks, f, :] = np.einsum("fkm,pm->fkp", c[:, ks], V)
    # The neighbour's trace at the same physical points: both faces enumerate
    # the owner's point set in the owner's order.
    k2, f2 = mesh.EToE, mesh.EToF
    interior = k2 >= 0
    plus = minus[:, np.where(interior, k2, 0), np.where(interior, f2, 0)]
    bd = ~interior
    plus[0][bd] = -minus[0][bd]
    plus[1:, bd] = minus[1:, bd]
    return minus, plus


def fluxes(mesh: Mesh, minus, plus, tau_p=1.0, tau_u=1.0):
    """Surface integrands F_p, F_u (4, K, 4, Nfq) including n J^f (Sec. 4.1).

    F_p   = -1/2 (2 {u}.nJ - tau_p [p] J^f)
    F_u_i = -1/2 ([p] - tau_u [u].n) nJ_i
    """
    nJ = np.moveaxis(mesh.nJ, -1, 0)                          # (3, K, 4, Nfq)
    Jf = mesh.Jf
    jp = plus[0] - minus[0]
    ju = plus[1:] - minus[1:]
    au = 0.5 * (plus[1:] + minus[1:])
    au_n = np.sum(au * nJ, axis=0)
    ju_n = np.sum(ju * nJ, axis=0) / Jf                       # [u].n J^f / J^f ... = [u].n
    F = np.empty_like(minus)
    F[0] = -0.5 * (2.0 * au_n - tau_p * jp * Jf)
    F[1:] = -0.5 * (jp - tau_u * ju_n) * nJ
    return F


def a_h(mesh: Mesh, c: np.ndarray, tau_p=1.0, tau_u=1.0) -> np.ndarray:
    """Strong-weak right-hand side functional, modal (4, K, Np)."""
    ref = mesh.ref
    w = ref.w_q
    p, u = c[0], c[1:]
    uq = np.einsum("qm,ikm->ikq", ref.Vq, u)                  # (3, K, Nq)
    dpq = np.einsum("aqm,km->akq", ref.Vq_a, p)                # (3, K, Nq): d p / d x^_a
    G = mesh.G                                                 # (K, Nq, a, i)
    U = np.einsum("kqai,ikq->akq", G, uq)                      # U^a = sum_i G_ai u_i
    gp = np.einsum("kqai,akq->ikq", G, dpq)                    # sum_a G_ai dp/dx^_a = J dp/dx_i
    out = np.zeros_like(c)
    # volume: int u . grad v  = sum_a (V_q^a)^T diag(w) U^a
    out[0] = np.einsum("aqm,akq->km", ref.Vq_a, w * U)
    # volume: -int grad p . tau = -V_q^T diag(w) J grad p
    out[1:] = -np.einsum("qm,ikq->ikm", ref.Vq, w * gp)
    # surface
    minus, plus = traces(mesh, c)
    F = fluxes(mesh, minus, plus, tau_p, tau_u)
    for (f, sig), ks in mesh.face_groups.items():
        V = mesh.face_V[(f, sig)]
        out[:, ks] += np.einsum("fkp,pm->fkm", F[:, ks, f] * ref.w_f, V)
    return out


def strong_rule_points(N: int) -> tuple[int, int]:
    """Points per direction of the collapsed volume and face rules of the
    energy-stable strong form (Sec. 4.1): the volume integrands (J div u) v
    have degree 2(N-1) + (N-1) + N = 4N-3 and the surface integrands
    [u].nJ^f v degree (2N-2) + 2N = 4N-2 for an isoparametric map; an n-point
    collapsed rule is exact to degree 2n-1.  The volume count never drops
    below the N+1 of the degree 2N+1 rule."""
    return max(N + 1, 2 * N - 1), 2 * N


def strong_mesh(mesh: Mesh) -> Mesh:
    """The same mesh and geometry with the strong form's rules (cached)."""
    sm = getattr(mesh, "_strong_mesh", None)
    if sm is None:
        nv, nf = strong_rule_points(mesh.ref.N)
        sm = Mesh(RefTet(mesh.ref.N, nv, nf), mesh.VXYZ, mesh.EToV, mesh.geom_xyz)
        mesh._strong_mesh = sm
    return sm


def a_h_strong(mesh: Mesh, c: np.ndarray, tau_p=1.0, tau_u=1.0) -> np.ndarray:
    """Strong right-hand side functional (Sec. 4.1, the strong DG form), modal
    (4, K, Np): both equations integrated by parts twice,

        p:  -int (div u) v - int_dD 1/2 ([u].n - tau_p [p]) v,
        u:  -int grad p . tau - int_dD 1/2 ([p] - tau_u [u].n) tau.n,

    with J div u = sum_{a,i} G_ai du_i/dx^_a at the volume points.  With rules
    exact for the volume (degree 4N-3) and surface (4N-2) integrands it equals
    the strong-weak functional a_h (discrete integration by parts)."""
    ref = mesh.ref
    w = ref.w_q
    p, u = c[0], c[1:]
    du = np.einsum("aqm,ikm->aikq", ref.Vq_a, u)               # (3 a, 3 i, K, Nq): du_i/dx^_a
    dpq = np.einsum("aqm,km->akq", ref.Vq_a, p)
    G = mesh.G                                                 # (K, Nq, a, i)
    jdiv = np.einsum("kqai,aikq->kq", G, du)                   # J div u
    gp = np.einsum("kqai,akq->ikq", G, dpq)                    # J grad p
    out = np.zeros_like(c)
    out[0] = -np.einsum("qm,kq->km", ref.Vq, w * jdiv)
    out[1:] = -np.einsum("qm,ikq->ikm", ref.Vq, w * gp)
    minus, plus = traces(mesh, c)
    nJ = np.moveaxis(mesh.nJ, -1, 0)
    jp = plus[0] - minus[0]
    ju_nJ = np.sum((plus[1:] - minus[1:]) * nJ, axis=0)        # [u].n J^f
    F = np.empty_like(minus)
    F[0] = -0.5 * (ju_nJ - tau_p * jp * mesh.Jf)
    F[1:] = -0.5 * (jp - tau_u * ju_nJ / mesh.Jf) * nJ
    for (f, sig), ks in mesh.face_groups.items():
        V = mesh.face_V[(f, sig)]
        out[:, ks] += np.einsum("fkp,pm->fkm", F[:, ks, f] * ref.w_f, V)
    return out


# ---------------------------------------------------------------------------
# Mass inverses.
# ---------------------------------------------------------------------------

def wadg_weights(mesh: Mesh, c2q=None, conservative: bool = False):
    """Weights (W_p, W_u) at the volume points of the weight-adjusted update.

    Default (Sec. 6.2, Sec. 7): W_p = c^2_q / J_q, W_u = 1 / J_q, i.e. the
    reciprocals of the mass weights w_p = J/c^2 and w_u = J.
    conservative=True (Sec. 3, after the moment estimate): local conservation
    is restored by replacing each mass weight w by its projection Pi_N w onto
    P^N within the weight-adjusted inner product: W = 1 / (Pi_N w)(x_q), the
    projection taken with the volume rule (Pi_N w = V_q P_q w_q).  Then for a
    load b the update r = P_q diag(W) V_q b has zeroth moment
    sum_q w_q (w r)_q = b(1) exactly (mass weight w at the points).
    """
    ref = mesh.ref
    wu = mesh.J
    wp = wu if c2q is None else mesh.J / c2q
    if conservative:
        def proj(f):
            coef = np.einsum("qm,kq->km", ref.Vq, f * ref.w_q)      # modal, M^ = I
            return np.einsum("qm,km->kq", ref.Vq, coef)
        wu, wp = proj(wu), proj(wp)
        if np.any(wu <= 0) or np.any(wp <= 0):
            raise ValueError("projected mass weight is not positive at a volume point")
    return 1.0 / wp, 1.0 / wu


def wadg_apply(mesh: Mesh, r: np.ndarray, c2q=None, conservative: bool = False) -> np.ndarray:
    """Weight-adjusted inverse, matrix free: P_q diag(W_q) V_q r (Sec. 6.2, Sec. 7).

    W_q = c^2_q / J_q for the pressure row, 1 / J_q for the velocity rows
    (or their locally conservative variants, see wadg_weights).
    In the orthonormal basis P_q = V_q^T diag(w_q).
    """
    ref = mesh.ref
    Wp, Wu = wadg_weights(mesh, c2q, conservative)
    rq = np.einsum("qm,fkm->fkq", ref.Vq, r)
    rq[0] *= Wp
    rq[1:] *= Wu
    return np.einsum("qm,fkq->fkm", ref.Vq, rq * ref.w_q)


def wadg_dense_nodal(mesh: Mesh, b_nodal: np.ndarray, c2q=None) -> np.ndarray:
    """Weight-adjusted inverse assembled explicitly in the nodal (lattice) basis,
    M^^{-1} M_W M^^{-1} b (Sec. 4), with (M_W)_ij = sum_q w_q l_i l_j W_q and
    M^_ij = sum_q w_q l_i l_j.  b_nodal (4, K, Np) is the nodal load vector
    b_i = a_h(q, l_i); W = c^2/J (pressure) or 1/J (velocity).
    """
    ref = mesh.ref
    L = ref.Vq @ ref.Vn_inv                                    # Lagrange basis at quad points
    Mhat = L.T @ (ref.w_q[:, None] * L)
    Wu = 1.0 / mesh.J
    Wp = Wu if c2q is None else c2q / mesh.J
    out = np.empty_like(b_nodal)
    for k in range(mesh.K):
        for fld in range(4):
            W = Wp[k] if fld == 0 else Wu[k]
            MW = L.T @ ((ref.w_q * W)[:, None] * L)
            y = np.linalg.solve(Mhat, b_nodal[fld, k])
            out[fld, k] = np.linalg.solve(Mhat, MW @ y)
    return out


def exact_mass_inverse(mesh: Mesh, r: np.ndarray, c2fun=None, qpts=None) -> np.ndarray:
    """Exact curvilinear DG: solve M_{J/c^2} x = r (pressure), M_J x = r (velocity)
    per element by Cholesky, M assembled with a high-degree rule (Sec. 4).

    The mass integrand phi_i phi_j J is of degree 2N + 3(N-1) = 5N-3; the rule
    uses ceil((5N-2)/2) points per direction.
    """
    ref = mesh.ref
    N = ref.N
    n = qpts if qpts is not None else (5 * N - 2 + 1) // 2 + 1
    rst, w = P.tet_rule(n)
    V = P.dubiner_tet(N, *rst.T)
    Jm = mesh.jacobian_matrix(np.arange(mesh.K), rst)
    J = np.linalg.det(Jm)
    if c2fun is not None:
        x = np.einsum("pm,kmd->kpd", V, mesh.Xmodal)
        c2 = c2fun(x)
    out = np.empty_like(r)
    for k in range(mesh.K):
        MJ = V.T @ ((w * J[k])[:, None] * V)
        Lc = np.linalg.cholesky(MJ)
        for fld in range(1, 4):
            out[fld, k] = np.linalg.solve(Lc.T, np.linalg.solve(Lc, r[fld, k]))
        Mp = MJ if c2fun is None else V.T @ ((w * J[k] / c2[k])[:, None] * V)
        Lp = np.linalg.cholesky(Mp)
        out[0, k] = np.linalg.solve(Lp.T, np.linalg.solve(Lp, r[0, k]))
    return out


def rhs(mesh: Mesh, c: np.ndarray, variant: str = "wadg", tau_p=1.0, tau_u=1.0,
        c2q=None, c2fun=None, form: str = "strong_weak", conservative: bool = False) -> np.ndarray:
    """dQ/dt = -M^{-1} A_h Q in modal coefficients (sign folded into a_h).

    form: "strong_weak" (default, the mesh's degree 2N+1 rules); "strong",
    the strong form with its volume and surface terms on the degree 4N-3 /
    4N-2 rules of strong_mesh (Sec. 4.1, energy stable); or
    "strong_underintegrated", the strong form on the mesh's degree 2N+1 rules
    (Sec. 6.5: faster, stability not guaranteed).  The mass inverse always
    uses the mesh's degree 2N+1 volume rule (Sec. 6.2); conservative selects
    the locally conservative weights of wadg_weights (variant "wadg")."""
    if form == "strong_weak":
        r = a_h(mesh, c, tau_p, tau_u)
    elif form == "strong":
        r = a_h_strong(strong_mesh(mesh), c, tau_p, tau_u)
    elif form == "strong_underintegrated":
        r = a_h_strong(mesh, c, tau_p, tau_u)
    else:
        raise ValueError(form)
    if variant == "wadg":
        return wadg_apply(mesh, r, c2q, conservative)
    if variant == "exact":
        return exact_mass_inverse(mesh, r, c2fun)
    raise ValueError(variant)


def rhs_nodal(mesh: Mesh, Qn: np.ndarray, **kw) -> np.ndarray:
    """Same as rhs() with nodal (lattice) input and output, (4, K, Np)."""
    ref = mesh.ref
    return ref.to_nodal(rhs(mesh, ref.to_modal(Qn), **kw))


# ---------------------------------------------------------------------------
# Time integration: 2N-storage LSRK(5,4) of Carpenter & Kennedy (1994).
# ---------------------------------------------------------------------------

LSRK_A = np.array([0.0,
                   -567301805773.0 / 1357537059087.0,
                   -2404267990393.0 / 2016746695238.0,
                   -3550918686646.0 / 2091501179385.0,
                   -1275806237668.0 / 842570457699.0])
LSRK_B = np.array([1432997174477.0 / 9575080441755.0,
                   5161836677717.0 / 13612068292357.0,
                   1720146321549.0 / 2090206949498.0,
                   3134564353537.0 / 4481467310338.0,
                   2277821191437.0 / 14882151754819.0])
LSRK_C = np.array([0.0,
                   1432997174477.0 / 9575080441755.0,
                   2526269341429.0 / 6820363962896.0,
                   2006345519317.0 / 3224310063776.0,
                   2802321613138.0 / 2924317926251.0])


def lsrk_step(L, q, res, t, dt):
    """One step: for each stage s, res = a_s res + dt L(q, t + c_s dt);
    q = q + b_s res.  Returns (q, res)."""
    for s in range(5):
        res = LSRK_A[s] * res + dt * L(q, t + LSRK_C[s] * dt)
        q = q + LSRK_B[s] * res
    return q, res


# ---------------------------------------------------------------------------
# Projection, norms, energy.
# ---------------------------------------------------------------------------

def wadg_projection(mesh: Mesh, fq: np.ndarray) -> np.ndarray:
    """Pseudo-projection P_N u = Pi_N(J^{-1} Pi_N(u J)) of values fq (F, K, Nq)
    at the volume quadrature points, returned modal (F, K, Np)."""
    ref = mesh.ref
    c1 = np.einsum("qm,fkq->fkm", ref.Vq, fq * mesh.J * ref.w_q)      # Pi_N(u J)
    v = np.einsum("qm,fkm->fkq", ref.Vq, c1) / mesh.J
    return np.einsum("qm,fkq->fkm", ref.Vq, v * ref.w_q)               # Pi_N(J^-1 .)


def l2_projection(mesh: Mesh, fun, npts: int | None = None) -> np.ndarray:
    """Exact (curvilinear) L2 projection of fun(x) -> (F, ...) by a high-degree rule."""
    ref = mesh.ref
    n = npts if npts is not None else ref.N + 5
    rst, w = P.tet_rule(n)
    V = P.dubiner_tet(ref.N, *rst.T)
    J = np.linalg.det(mesh.jacobian_matrix(np.arange(mesh.K), rst))
    x = np.einsum("pm,kmd->kpd", V, mesh.Xmodal)
    fv = fun(x)                                                         # (F, K, npts)
    b = np.einsum("pm,fkp->fkm", V, fv * J * w)
    out = np.empty_like(b)
    for k in range(mesh.K):
        MJ = V.T @ ((w * J[k])[:, None] * V)
        out[:, k] = np.linalg.solve(MJ, b[:, k].T).T
    return out


def l2_error(mesh: Mesh, c: np.ndarray, fun, fields=(0,), npts: int | None = None) -> float:
    """|| q_h - q ||_{L2(Omega)} over the listed fields with a rule exact to 2N+6."""
    ref = mesh.ref
    n = npts if npts is not None else ref.N + 4
    rst, w = P.tet_rule(n)
    V = P.dubiner_tet(ref.N, *rst.T)
    J = np.linalg.det(mesh.jacobian_matrix(np.arange(mesh.K), rst))
    x = np.einsum("pm,kmd->kpd", V, mesh.Xmodal)
    ex = fun(x)
    err = 0.0
    for f in fields:
        d = np.einsum("pm,km->kp", V, c[f]) - ex[f]
        err += float(np.sum(w * J * d * d))
    return float(np.sqrt(err))


def wadg_energy(mesh: Mesh, c: np.ndarray, c2q=None) -> float:
    """1/2 Q^T M~ Q with M~ = M^ M_W^{-1} M^ (M^ = I): 1/2 sum_k c^T M_W^{-1} c,
    W = c^2/J (pressure) or 1/J (velocity), M_W by the 2N+1 rule (Sec. 4)."""
    ref = mesh.ref
    Wu = 1.0 / mesh.J
    Wp = Wu if c2q is None else c2q / mesh.J
    E = 0.0
    for k in range(mesh.K):
        for fld in range(4):
            W = Wp[k] if fld == 0 else Wu[k]
            MW = ref.Vq.T @ ((ref.w_q * W)[:, None] * ref.Vq)
            E += 0.5 * float(c[fld, k] @ np.linalg.solve(MW, c[fld, k]))
    return E


def quadrature_energy(mesh: Mesh, c: np.ndarray, c2q=None) -> float:
    """1/2 int (p^2/c^2 + |u|^2) by the 2N+1 rule."""
    ref = mesh.ref
    vals = np.einsum("qm,fkm->fkq", ref.Vq, c)
    inv_c2 = 1.0 if c2q is None else 1.0 / c2q
    dens = vals[0] ** 2 * inv_c2 + np.sum(vals[1:] ** 2, axis=0)
    return 0.5 * float(np.sum(ref.w_q * mesh.J * dens))


def dissipation(mesh: Mesh, c: np.ndarray, tau_p=1.0, tau_u=1.0) -> float:
    """Right side of the discrete energy identity (Sec. 4.1):
    -1/2 sum_{interior f} int (tau_p [p]^2 + tau_u ([u].n)^2) - tau_p sum_{bdry} int p^2,
    each face counted once, at the owner's quadrature points."""
    minus, plus = traces(mesh, c)
    w = mesh.ref.w_f
    total = 0.0
    for k in range(mesh.K):
        for f in range(4):
            k2 = mesh.EToE[k, f]
            Jf = mesh.Jf[k, f]
            if k2 < 0:
                total -= tau_p * float(np.sum(w * Jf * minus[0, k, f] ** 2))
            elif k2 > k:
                n = mesh.nJ[k, f] / Jf[:, None]
                jp = plus[0, k, f] - minus[0, k, f]
                jun = np.sum((plus[1:, k, f] - minus[1:, k, f]).T * n, axis=1)
                total -= 0.5 * float(np.sum(w * Jf * (tau_p * jp ** 2 + tau_u * jun ** 2)))
    return total


def build(n: int, N: int, amplitude: float = 0.1, VXYZ=None, EToV=None, geom=None):
    """Reference element and warped-cube mesh for (n, N)."""
    from synthetic import warped_cube
    ref = RefTet(N)
    if VXYZ is None:
        VXYZ, EToV, geom = warped_cube(n, N, amplitude)
    return ref, Mesh(ref, VXYZ, EToV, geom)
