"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle part to something other than itself: closed forms,
library routines for special cases, brute force, invariants of the discrete
scheme, and the convergence / stability claims of the paper
(Chan, Hewett & Warburton, arXiv:1608.03836).
"""
import math

import numpy as np
import pytest

from oracle import polynomials as P
from oracle import wadg as W
from oracle.discretization import Mesh, RefTet, FACE_VERTS, REF_VERTS
from synthetic import kuhn_cube, geometry_nodes, warped_cube, lattice_tet, standing_wave, OMEGA


def _mesh(n, N, amp=0.1):
    VXYZ, EToV, geom = warped_cube(n, N, amp)
    ref = RefTet(N)
    return ref, Mesh(ref, VXYZ, EToV, geom)


# ----------------------------------------------------------------------------
# Quadrature (Sec. 4 / Sec. 6.2: rules exact to degree 2N+1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_gauss_legendre_matches_library(n):
    """alpha = beta = 0 reduces to Gauss-Legendre (numpy's leggauss)."""
    x, w = P.gauss_jacobi(n, 0.0)
    xl, wl = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xl, atol=1e-14, rtol=0)
    assert np.allclose(w, wl, atol=1e-14, rtol=0)


@pytest.mark.parametrize("alpha", [1.0, 2.0, 5.0])
def test_gauss_jacobi_brute_force_moments(alpha):
    """n-point rule integrates (1-x)^alpha x^m exactly for m <= 2n-1 (closed-form
    moments from the Beta function)."""
    n = 4
    x, w = P.gauss_jacobi(n, alpha)
    for m in range(2 * n):
        # int_{-1}^{1} (1-x)^alpha (1+x)^m dx = 2^{alpha+m+1} B(alpha+1, m+1)
        exact = 2.0 ** (alpha + m + 1) * math.gamma(alpha + 1) * math.gamma(m + 1) / math.gamma(alpha + m + 2)
        assert abs(np.sum(w * (1 + x) ** m) - exact) <= 1e-13 * exact


def _tet_monomial(a, b, c):
    # int over the bi-unit tet of (1+r)^a (1+s)^b (1+t)^c: unit simplex Dirichlet integral
    return 8.0 * 2.0 ** (a + b + c) * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)


def _tri_monomial(a, b):
    return 4.0 * 2.0 ** (a + b) * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_volume_and_face_rules_exact_to_2N_plus_1(N):
    rst, w = P.tet_rule(N + 1)
    assert abs(w.sum() - 4.0 / 3.0) < 1e-14
    for a in range(2 * N + 2):
        for b in range(2 * N + 2 - a):
            for c in range(2 * N + 2 - a - b):
                v = np.sum(w * (1 + rst[:, 0]) ** a * (1 + rst[:, 1]) ** b * (1 + rst[:, 2]) ** c)
                ex = _tet_monomial(a, b, c)
                assert abs(v - ex) <= 1e-13 * ex
    rs, wf = P.tri_rule(N + 1)
    assert abs(wf.sum() - 2.0) < 1e-14
    for a in range(2 * N + 2):
        for b in range(2 * N + 2 - a):
            ex = _tri_monomial(a, b)
            assert abs(np.sum(wf * (1 + rs[:, 0]) ** a * (1 + rs[:, 1]) ** b) - ex) <= 1e-13 * ex


# ----------------------------------------------------------------------------
# Basis and reference operators
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 3, 6])
def test_basis_orthonormal_and_PqVq_identity(N):
    ref = RefTet(N)
    M = ref.Vq.T @ (ref.w_q[:, None] * ref.Vq)
    assert np.abs(M - np.eye(ref.Np)).max() < 1e-13
    Pq = ref.Vq.T * ref.w_q                       # M^^{-1} V_q^T diag(w), M^ = I
    assert np.abs(Pq @ ref.Vq - np.eye(ref.Np)).max() < 1e-13
    rs, w = P.tri_rule(N + 1)
    Vt = P.dubiner_tri(N, *rs.T)
    assert np.abs(Vt.T @ (w[:, None] * Vt) - np.eye(Vt.shape[1])).max() < 1e-13


@pytest.mark.parametrize("N", [2, 5])
def test_basis_gradient_matches_finite_differences(N):
    rng = np.random.default_rng(3)
    lam = rng.dirichlet(np.ones(4), size=6)
    pts = lam @ REF_VERTS
    g = P.dubiner_tet_grad(N, *pts.T)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (P.dubiner_tet(N, *(pts + e).T) - P.dubiner_tet(N, *(pts - e).T)) / (2 * h)
        assert np.abs(g[d] - fd).max() < 1e-7


def test_basis_spans_PN():
    """Every monomial of degree <= N is reproduced by its L2 projection."""
    N = 3
    ref = RefTet(N)
    x = ref.rst_q
    for (a, b, c) in [(0, 0, 0), (3, 0, 0), (1, 1, 1), (0, 2, 1)]:
        f = x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c
        coef = ref.Vq.T @ (ref.w_q * f)
        assert np.abs(ref.Vq @ coef - f).max() < 1e-13


def test_lattice_is_the_interface_node_set():
    for N in range(1, 7):
        assert np.array_equal(RefTet(N).lattice, lattice_tet(N))


# ----------------------------------------------------------------------------
# Geometry (Sec. 2, Sec. 4.1)
# ----------------------------------------------------------------------------

def test_affine_geometry_constant_factors():
    VXYZ, EToV = kuhn_cube(2)
    N = 3
    ref = RefTet(N)
    mesh = Mesh(ref, VXYZ, EToV, geometry_nodes(VXYZ, EToV, N, 0.0))
    h = 1.0
    # Kuhn tet of a cube with side h has volume h^3/6 = (4/3) J
    assert np.allclose(mesh.J, h ** 3 / 8.0, atol=1e-14)
    assert np.abs(mesh.G - mesh.G[:, :1]).max() < 1e-13
    assert np.abs(mesh.nJ - mesh.nJ[:, :, :1]).max() < 1e-13


def test_closed_surface_and_divergence_theorem():
    """sum_f int n dS = 0, and int div F = int F.n for F = (x^2, y z, z) on
    curved elements (checked with a rule rich enough to be exact)."""
    ref, mesh = _mesh(2, 3)
    closed = np.einsum("kfqd,q->kd", mesh.nJ, ref.w_f)
    assert np.abs(closed).max() < 1e-14
    VXYZ, EToV, geom = warped_cube(2, 3, 0.1)
    rich = RefTet(3, qdeg_pts=11)            # exact to degree 21 >= 5N-3 and 4N-2
    mesh2 = Mesh(rich, VXYZ, EToV, geom)
    x = mesh2.xq
    div = 2 * x[..., 0] + x[..., 2] + 1.0
    vol = np.einsum("kq,q->k", mesh2.J * div, rich.w_q)
    xf = np.stack([_face_x(mesh2, f) for f in range(4)], 1)
    F = np.stack([xf[..., 0] ** 2, xf[..., 1] * xf[..., 2], xf[..., 2]], -1)
    surf = np.einsum("kfqd,kfqd,q->k", F, mesh2.nJ, rich.w_f)
    assert np.abs(vol - surf).max() < 1e-12


def _face_x(mesh, f):
    """Physical coordinates of each element's face-f points, (K, Nfq, 3)."""
    out = np.empty((mesh.K, mesh.ref.Nfq, 3))
    for (ff, sig), ks in mesh.face_groups.items():
        if ff == f:
            out[ks] = np.einsum("pm,kmd->kpd", mesh.face_V[(ff, sig)], mesh.Xmodal[ks])
    return out


def test_shared_faces_match_and_boundary_is_planar():
    ref, mesh = _mesh(2, 4)
    for k in range(mesh.K):
        for f in range(4):
            k2, f2 = mesh.EToE[k, f], mesh.EToF[k, f]
            if k2 >= 0:
                # same physical points, opposite normals, equal surface Jacobians
                assert np.abs(_face_x(mesh, f)[k] - _face_x(mesh, f2)[k2]).max() < 1e-14
                assert np.abs(mesh.nJ[k, f] + mesh.nJ[k2, f2]).max() < 1e-13
            else:
                n = mesh.nJ[k, f] / mesh.Jf[k, f][:, None]
                axis = np.argmax(np.abs(n[0]))
                assert np.abs(np.abs(n[:, axis]) - 1).max() < 1e-13
                assert np.abs(np.abs(_face_x(mesh, f)[k][:, axis]) - 1).max() < 1e-14


# ----------------------------------------------------------------------------
# Weight-adjusted mass inverse (Sec. 4, Sec. 6.2, Sec. 7)
# ----------------------------------------------------------------------------

def test_wadg_equals_exact_inverse_on_affine_elements():
    VXYZ, EToV = kuhn_cube(2)
    N = 3
    ref = RefTet(N)
    mesh = Mesh(ref, VXYZ, EToV, geometry_nodes(VXYZ, EToV, N, 0.0))
    rng = np.random.default_rng(5)
    r = rng.standard_normal((4, mesh.K, ref.Np))
    a = W.wadg_apply(mesh, r)
    b = W.exact_mass_inverse(mesh, r)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_wadg_differs_from_exact_inverse_on_curved_elements():
    """Guard against a degenerate pin: on curved elements the two must differ."""
    ref, mesh = _mesh(2, 3)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((4, mesh.K, ref.Np))
    a = W.wadg_apply(mesh, r)
    b = W.exact_mass_inverse(mesh, r)
    assert np.abs(a - b).max() > 1e-6 * np.abs(b).max()


def test_matrix_free_equals_dense_nodal_assembly():
    ref, mesh = _mesh(2, 3)
    rng = np.random.default_rng(6)
    c = rng.standard_normal((4, mesh.K, ref.Np))
    c2q = 1.0 + 0.5 * rng.uniform(size=mesh.J.shape)
    b_modal = W.a_h(mesh, c)
    b_nodal = np.einsum("mn,fkm->fkn", ref.Vn_inv, b_modal)        # b_i = a_h(q, l_i)
    dense = W.wadg_dense_nodal(mesh, b_nodal, c2q)
    mf = ref.to_nodal(W.wadg_apply(mesh, b_modal, c2q))
    assert np.abs(dense - mf).max() < 1e-12 * np.abs(dense).max()


def test_pseudo_projection_reproduces_polynomials_on_affine_elements():
    VXYZ, EToV = kuhn_cube(2)
    N = 3
    ref = RefTet(N)
    mesh = Mesh(ref, VXYZ, EToV, geometry_nodes(VXYZ, EToV, N, 0.0))
    x = mesh.xq
    f = np.stack([x[..., 0] ** 3 - x[..., 1] * x[..., 2], x[..., 2] ** 2, 1 + 0 * x[..., 0], x[..., 0] * x[..., 1]])
    c = W.wadg_projection(mesh, f)
    assert np.abs(np.einsum("qm,fkm->fkq", ref.Vq, c) - f).max() < 1e-12


def test_pseudo_projection_formula_theorem():
    """Sec. 3 Theorem: P_N u solves (T_{1/J}^{-1} P_N u, v) = (uJ, v), i.e.
    M_{1/J}^{-1} c = Pi_N(uJ) with M_{1/J} by the same rule."""
    ref, mesh = _mesh(2, 2)
    rng = np.random.default_rng(9)
    f = rng.standard_normal((1, mesh.K, ref.Nq))
    c = W.wadg_projection(mesh, f)
    b = np.einsum("qm,fkq->fkm", ref.Vq, f * mesh.J * ref.w_q)
    for k in range(mesh.K):
        M = ref.Vq.T @ ((ref.w_q / mesh.J[k])[:, None] * ref.Vq)
        assert np.abs(np.linalg.solve(M, c[0, k]) - b[0, k]).max() < 1e-12 * np.abs(b[0, k]).max()


# ----------------------------------------------------------------------------
# Strong-weak RHS (Sec. 4.1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 2, 3])
def test_affine_linear_velocity_gives_unit_divergence(N):
    """p = 0, u = (x, 0, 0): p_t = -div u = -1, u_t = -grad p = 0, exactly for
    affine elements (both fields are in P^N and the flux terms vanish in the
    interior and cancel on the boundary)."""
    VXYZ, EToV = kuhn_cube(2)
    geom = geometry_nodes(VXYZ, EToV, N, 0.0)
    ref = RefTet(N)
    mesh = Mesh(ref, VXYZ, EToV, geom)
    Qn = np.zeros((4, mesh.K, ref.Np))
    Qn[1] = geom[..., 0]
    r = W.rhs_nodal(mesh, Qn)
    assert np.abs(r[0] + 1.0).max() < 1e-12
    assert np.abs(r[1:]).max() < 1e-12


def test_gradient_of_linear_pressure_interior():
    """p = z on an affine mesh: u_t = -grad p = (0,0,-1) on elements away from the
    boundary (the Dirichlet ghost state perturbs boundary elements)."""
    VXYZ, EToV = kuhn_cube(3)
    N = 2
    geom = geometry_nodes(VXYZ, EToV, N, 0.0)
    ref = RefTet(N)
    mesh = Mesh(ref, VXYZ, EToV, geom)
    Qn = np.zeros((4, mesh.K, ref.Np))
    Qn[0] = geom[..., 2]
    r = W.rhs_nodal(mesh, Qn)
    interior = np.all(mesh.EToE >= 0, axis=1) & np.all(mesh.EToE[mesh.EToE] >= 0, axis=(1, 2))
    assert interior.sum() > 0
    assert np.abs(r[3, interior] + 1.0).max() < 1e-12
    assert np.abs(r[1:3, interior]).max() < 1e-12
    assert np.abs(r[0, interior]).max() < 1e-12


@pytest.mark.parametrize("N", [2, 3])
def test_discrete_energy_identity(N):
    """Q^T a_h(Q) = -1/2 sum_int (tau_p[p]^2 + tau_u([u].n)^2) - tau_p sum_bdry p^2
    for any Q (Sec. 4.1); with tau = 0 it vanishes."""
    ref, mesh = _mesh(2, N)
    rng = np.random.default_rng(1)
    c = rng.standard_normal((4, mesh.K, ref.Np))
    for tau in (0.0, 1.0, 0.3):
        lhs = float(np.sum(W.a_h(mesh, c, tau, tau) * c))
        rhs = W.dissipation(mesh, c, tau, tau)
        scale = float(np.sum(c * c))
        assert abs(lhs - rhs) < 1e-12 * scale
    assert abs(float(np.sum(W.a_h(mesh, c, 0.0, 0.0) * c))) < 1e-12 * float(np.sum(c * c))


def test_spectrum_central_imaginary_upwind_dissipative():
    """Sec. 5.2 (eigenspectra): tau = 0 gives a purely imaginary spectrum,
    tau = 1 a spectrum in the closed left half plane; WADG and DG agree closely
    for the large eigenvalues."""
    ref, mesh = _mesh(1, 2)
    n = 4 * mesh.K * ref.Np
    for tau in (0.0, 1.0):
        for variant in ("wadg", "exact"):
            A = np.empty((n, n))
            for j in range(n):
                e = np.zeros(n)
                e[j] = 1.0
                A[:, j] = W.rhs(mesh, e.reshape(4, mesh.K, ref.Np), variant=variant, tau_p=tau, tau_u=tau).ravel()
            lam = np.linalg.eigvals(A)
            scale = np.abs(lam).max()
            if tau == 0.0:
                assert np.abs(lam.real).max() < 1e-10 * scale
            else:
                assert lam.real.max() < 1e-10 * scale
                assert lam.real.min() < -1e-3 * scale
            if variant == "wadg":
                lw = np.sort(np.abs(lam))
            else:
                le = np.sort(np.abs(lam))
        assert abs(lw[-1] - le[-1]) < 0.02 * le[-1]


# ----------------------------------------------------------------------------
# Time integration (Sec. 5.2, Carpenter & Kennedy LSRK(5,4))
# ----------------------------------------------------------------------------

def test_lsrk_stability_polynomial():
    from numpy.polynomial import Polynomial
    q, res = W.lsrk_step(lambda y, t: y * Polynomial([0.0, 1.0]), Polynomial([1.0]), Polynomial([0.0]), 0.0, 1.0)
    coef = q.coef
    assert np.allclose(coef[:5], [1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0], atol=1e-10, rtol=0)
    assert len(coef) == 6


def test_lsrk_fourth_order_nonautonomous():
    """y' = -y + cos(3t): observed order 4 (exercises the stage times c_s)."""
    def exact(t):
        # y(0) = 1; particular solution (cos 3t + 3 sin 3t)/10
        return (1 - 0.1) * np.exp(-t) + (np.cos(3 * t) + 3 * np.sin(3 * t)) / 10.0

    errs = []
    for nsteps in (20, 40, 80):
        dt = 2.0 / nsteps
        y, r = 1.0, 0.0
        for s in range(nsteps):
            y, r = W.lsrk_step(lambda q, t: -q + np.cos(3 * t), y, r, s * dt, dt)
        errs.append(abs(y - exact(2.0)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 3.8


# ----------------------------------------------------------------------------
# Full solve: energy, convergence, WADG vs exact DG (Sec. 4, Sec. 5.3)
# ----------------------------------------------------------------------------

def _cfl_dt(mesh, N, cfl=0.5):
    h = mesh.J.min(1) / mesh.Jf.reshape(mesh.K, -1).max(1)
    return cfl * h.min() / (N + 1) ** 2


def _solve(mesh, T, variant="wadg"):
    ref = mesh.ref
    dt = _cfl_dt(mesh, ref.N)
    ns = int(math.ceil(T / dt))
    dt = T / ns
    if variant == "wadg":
        c = W.wadg_projection(mesh, standing_wave(mesh.xq, 0.0))
    else:
        c = W.l2_projection(mesh, lambda x: standing_wave(x, 0.0))
    res = np.zeros_like(c)
    energies = [W.wadg_energy(mesh, c)]
    for s in range(ns):
        c, res = W.lsrk_step(lambda q, t: W.rhs(mesh, q, variant=variant), c, res, s * dt, dt)
        energies.append(W.wadg_energy(mesh, c))
    return c, np.array(energies)


def test_standing_wave_solves_the_pde():
    """The analytic solution satisfies p_t + div u = 0, u_t + grad p = 0 (FD check)."""
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, size=(10, 3))
    h, t = 1e-5, 0.3
    d = lambda f, i: (f(x + h * np.eye(3)[i], t) - f(x - h * np.eye(3)[i], t)) / (2 * h)
    sw = lambda y, tt: standing_wave(y, tt)
    dt_ = (standing_wave(x, t + h) - standing_wave(x, t - h)) / (2 * h)
    div_u = sum(d(sw, i)[1 + i] for i in range(3))
    assert np.abs(dt_[0] + div_u).max() < 1e-8
    for i in range(3):
        assert np.abs(dt_[1 + i] + d(sw, i)[0]).max() < 1e-8
    assert abs(OMEGA - math.sqrt(3) * math.pi / 2) < 1e-15


@pytest.mark.slow
def test_convergence_energy_and_dg_agreement():
    """N = 1, 2 on n = 2, 4: observed rate >= N + 1/2 - 0.15 on these coarse meshes,
    M~-energy non-increasing every step, WADG and exact-DG errors within 5 %."""
    T = 0.25
    for N in (1, 2):
        errs = []
        for n in (2, 4):
            ref, mesh = _mesh(n, N)
            c, E = _solve(mesh, T)
            assert np.all(np.diff(E) <= 1e-13 * E[0])
            errs.append(W.l2_error(mesh, c, lambda x: standing_wave(x, T)))
            if n == 2:
                ce, _ = _solve(mesh, T, "exact")
                ee = W.l2_error(mesh, ce, lambda x: standing_wave(x, T))
                assert abs(errs[-1] / ee - 1) < 0.05
        rate = math.log2(errs[0] / errs[1])
        assert rate > N + 0.5 - 0.15, (N, errs, rate)


@pytest.mark.slow
def test_convergence_rates_on_three_meshes():
    """Sec. 5.3: the strong-weak WADG error to the analytic standing wave falls
    at least like h^(N+1/2).  N = 2..4 on n = 2, 4, 8 hexes per side (48 to
    3,072 tets, warped): the slope over the whole range and over the finest
    pair must both reach N + 1/2 (a dropped or mis-signed term in the volume,
    flux, lift or update costs at least one order).  T = 0.05 at CFL 1; the
    time error (fourth order) is far below the spatial one."""
    T = 0.05
    for N in (2, 3, 4):
        errs = []
        for n in (2, 4, 8):
            ref, mesh = _mesh(n, N)
            dt = _cfl_dt(mesh, N, cfl=1.0)
            ns = int(math.ceil(T / dt))
            dt = T / ns
            c = W.wadg_projection(mesh, standing_wave(mesh.xq, 0.0))
            res = np.zeros_like(c)
            for s in range(ns):
                c, res = W.lsrk_step(lambda q, t: W.rhs(mesh, q), c, res, s * dt, dt)
            errs.append(W.l2_error(mesh, c, lambda x: standing_wave(x, T)))
        overall = math.log2(errs[0] / errs[2]) / 2
        finest = math.log2(errs[1] / errs[2])
        assert overall >= N + 0.5 and finest >= N + 0.5, (N, errs, overall, finest)


def test_quadrature_energy_weights_pressure_by_inverse_wave_speed():
    """The energy 1/2 int (p^2/c^2 + |u|^2) in closed form on the warped cube
    (N = 3: J has degree 6 <= 2N+1, so the rule integrates J exactly and the
    curved elements fill the volume 8 of [-1,1]^3): p = 1, u = 0 with c^2 = 4
    gives 1/2 * 8/4 = 1 (a missing 1/c^2 gives 4, an inverted one 16);
    p = 0, u = (1, 1, 1) gives 12 whatever c^2 is; c^2 = 1 + x^2 sampled at
    the points gives 1/2 int 1/(1 + x^2) = 1/2 * 4 * 2 arctan(1) = pi up to
    the rule's error for a non-polynomial integrand."""
    ref, mesh = _mesh(2, 3)
    ones = np.ones((mesh.K, ref.Np))
    zero = np.zeros_like(ones)
    cp = ref.to_modal(np.stack([ones, zero, zero, zero]))
    cu = ref.to_modal(np.stack([zero, ones, ones, ones]))
    c2 = np.full(mesh.J.shape, 4.0)
    assert abs(W.quadrature_energy(mesh, cp, c2q=c2) - 1.0) < 1e-13
    assert abs(W.quadrature_energy(mesh, cp) - 4.0) < 1e-13
    assert abs(W.quadrature_energy(mesh, cu, c2q=c2) - 12.0) < 1e-13
    c2x = 1.0 + mesh.xq[..., 0] ** 2
    assert abs(W.quadrature_energy(mesh, cp, c2q=c2x) - math.pi) < 2e-5


def test_wave_speed_enters_the_pressure_row():
    """Sec. 7: with constant c^2 = 4 the standing wave oscillates at 2 omega.
    p = C cos(2 omega t), u = -grad C sin(2 omega t) / (2 omega).  A weight on
    the wrong row (or a missing c^2) leaves the error O(1)."""
    ref, mesh = _mesh(2, 3)
    c2 = 4.0
    csp = 2.0

    def exact(x, t):
        q = standing_wave(x, csp * t)
        q[1:] /= csp
        return q

    T = 0.2
    dt = _cfl_dt(mesh, ref.N) / csp
    ns = int(math.ceil(T / dt))
    dt = T / ns
    c2q = np.full(mesh.J.shape, c2)
    c = W.wadg_projection(mesh, exact(mesh.xq, 0.0))
    res = np.zeros_like(c)
    for s in range(ns):
        c, res = W.lsrk_step(lambda q, t: W.rhs(mesh, q, c2q=c2q), c, res, s * dt, dt)
    e_right = W.l2_error(mesh, c, lambda x: exact(x, T), fields=(0, 1, 2, 3))
    e_wrong = W.l2_error(mesh, c, lambda x: standing_wave(x, T), fields=(0, 1, 2, 3))
    assert e_right < 0.1 * e_wrong
    assert e_right < 0.03


# ----------------------------------------------------------------------------
# Point sources and receivers
# ----------------------------------------------------------------------------

def test_point_source_zeroth_moment():
    """With u = p = 0 and c^2 = 1 the only right-hand side is the point source:
    int_Omega p_t = f(t) * 1(x_s) = f(t) for the exact inverse, and for WADG on
    affine elements (where it equals the exact inverse)."""
    from oracle import sources as OS
    VXYZ, EToV = kuhn_cube(2)
    N = 3
    ref = RefTet(N)
    mesh = Mesh(ref, VXYZ, EToV, geometry_nodes(VXYZ, EToV, N, 0.0))
    src = OS.PointSet(mesh, [[0.13, -0.41, 0.27]])
    amp = 0.7
    b = OS.source_load(mesh, src, amp, 0)
    for dq in (W.wadg_apply(mesh, b), W.exact_mass_inverse(mesh, b)):
        vals = np.einsum("qm,km->kq", ref.Vq, dq[0])
        total = float(np.sum(ref.w_q * mesh.J * vals))
        assert abs(total - amp) < 1e-12


def test_receivers_sample_a_linear_field_on_curved_elements():
    """locate + sample reproduce p = x + 2y - z at arbitrary points: the field's
    L2 projection is exact in every element because x_h is the identity map of
    the warped elements' own coordinates only for the geometry, so the check
    uses the isoparametric field p = x_h(x^) . (1, 2, -1), which is in P^N."""
    from oracle import sources as OS
    ref, mesh = _mesh(2, 4)
    c = np.einsum("kmd,d->km", mesh.Xmodal, np.array([1.0, 2.0, -1.0]))
    pts = np.array([[0.1, 0.2, -0.3], [-0.77, 0.5, 0.61], [0.9, -0.9, 0.05]])
    rec = OS.PointSet(mesh, pts)
    got = OS.sample(c, rec, np.arange(3))
    assert np.abs(got - pts @ np.array([1.0, 2.0, -1.0])).max() < 1e-12


# ----------------------------------------------------------------------------
# Discrete adjoint (O12): finite differences in FP64
# ----------------------------------------------------------------------------

def _misfit_problem():
    from oracle import adjoint as OA
    from synthetic import c2_perturbed_samples
    ref, mesh = _mesh(1, 2)
    c2q = c2_perturbed_samples(mesh.J.shape)
    prob = OA.MisfitProblem(mesh, c2q, [0.1, -0.2, 0.15], np.array([[0.3, 0.1, -0.4], [-0.5, 0.2, 0.3]]),
                            f0=5.0, t0=0.02, dt=4e-3, nsteps=6)
    return ref, mesh, prob


@pytest.mark.slow
def test_adjoint_gradients_match_central_differences():
    """8 seeded directions each for p0 and c^2: <grad, d> vs central differences.
    J is quadratic in p0 (central differences exact up to rounding) and smooth
    in c^2 (step 1e-5: truncation ~1e-10)."""
    ref, mesh, prob = _misfit_problem()
    rng = np.random.default_rng(2024)
    p0 = rng.standard_normal((mesh.K, ref.Np))
    J, gp, gc = prob.gradients(p0)
    for _ in range(8):
        d = rng.standard_normal(p0.shape)
        eps = 1e-3
        fd = (prob.misfit(p0 + eps * d) - prob.misfit(p0 - eps * d)) / (2 * eps)
        assert abs(fd - np.sum(gp * d)) < 1e-8 * abs(fd)
        dc = rng.standard_normal(gc.shape)
        eps = 1e-5
        fd = (prob.misfit(p0, prob.c2q + eps * dc) - prob.misfit(p0, prob.c2q - eps * dc)) / (2 * eps)
        assert abs(fd - np.sum(gc * dc)) < 1e-6 * abs(fd)


def _strong_case(n, N, amp, nq=None):
    from oracle.discretization import Mesh, RefTet
    from synthetic import warped_cube
    VXYZ, EToV, geom = warped_cube(n, N, amp)
    return Mesh(RefTet(N, nq), VXYZ, EToV, geom)


def test_strong_equals_strong_weak_with_exact_rules():
    """Sec. 4.1: the strong and strong-weak forms agree at the discrete level
    when the quadrature integrates the volume (degree 4N-3) and surface
    (4N-2) integrands exactly; collapsed rules with 2N points per direction
    (exact to 4N-1) on a curved mesh, random data, tau = (1, 0.5)."""
    from oracle import wadg as OW
    from synthetic import random_fields
    N = 3
    m = _strong_case(2, N, 0.1, nq=2 * N)
    c = random_fields((4, m.K, m.ref.Np), 17)
    a = OW.a_h(m, c, 1.0, 0.5)
    b = OW.a_h_strong(m, c, 1.0, 0.5)
    assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(a)


def test_strong_equals_strong_weak_on_affine_elements():
    """Affine elements: constant G and n J^f make the integrands of degree 2N - 1
    (volume) and 2N (faces), which the degree 2N+1 rules integrate exactly."""
    from oracle import wadg as OW
    from synthetic import random_fields
    m = _strong_case(2, 3, 0.0)
    c = random_fields((4, m.K, m.ref.Np), 18)
    a, b = OW.a_h(m, c), OW.a_h_strong(m, c)
    assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(a)


def test_strong_differs_from_strong_weak_when_under_integrated():
    """On curved elements with the degree 2N+1 rules the two forms differ (the
    under-integrated strong form is a different discretisation), so the
    exact-rule pin above is not trivially satisfied."""
    from oracle import wadg as OW
    from synthetic import random_fields
    m = _strong_case(2, 3, 0.1)
    c = random_fields((4, m.K, m.ref.Np), 19)
    a, b = OW.a_h(m, c), OW.a_h_strong(m, c)
    assert np.linalg.norm(a - b) > 1e-6 * np.linalg.norm(a)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_strong_rules_are_exact_and_minimal(N):
    """Sec. 4.1: the strong form equals the strong-weak form (on the same face
    rule, so that the non-polynomial penalty terms coincide) once the rules
    integrate the degree 4N-3 volume and 4N-2 surface integrands exactly; the
    strong form's rules (2N-1 volume, 2N face points per direction) do, and one
    point fewer in either direction does not (curved mesh, tau = (1, 0.5))."""
    from oracle import wadg as OW
    from oracle.discretization import Mesh, RefTet
    from synthetic import random_fields, warped_cube
    nv, nf = OW.strong_rule_points(N)
    assert (nv, nf) == (max(N + 1, 2 * N - 1), 2 * N)
    VXYZ, EToV, geom = warped_cube(2, N, 0.1)
    c = random_fields((4, len(EToV), (N + 1) * (N + 2) * (N + 3) // 6), 40 + N)

    def gap(v, f):
        m = Mesh(RefTet(N, v, f), VXYZ, EToV, geom)
        a, b = OW.a_h(m, c, 1.0, 0.5), OW.a_h_strong(m, c, 1.0, 0.5)
        return np.linalg.norm(a - b) / np.linalg.norm(a)

    assert gap(nv, nf) < 1e-12
    assert gap(nv - 1, nf) > 1e-7
    assert gap(nv, nf - 1) > 1e-7


@pytest.mark.parametrize("N", [2, 3])
def test_strong_form_energy_identity(N):
    """The strong form on its exact rules satisfies the strong-weak discrete
    energy identity Q^T a_h(Q) = dissipation (Sec. 4.1: energy stable), for
    tau = 0 (conservative) and tau > 0; the same form on the degree 2N+1
    rules does not (curved mesh)."""
    from oracle.discretization import Mesh, RefTet
    from synthetic import warped_cube
    VXYZ, EToV, geom = warped_cube(2, N, 0.1)
    mesh = Mesh(RefTet(N), VXYZ, EToV, geom)
    sm = W.strong_mesh(mesh)
    assert sm.ref.Nq == W.strong_rule_points(N)[0] ** 3 and sm.ref.Nfq == (2 * N) ** 2
    rng = np.random.default_rng(7 + N)
    c = rng.standard_normal((4, mesh.K, mesh.ref.Np))
    scale = float(np.sum(c * c))
    for tau in (0.0, 1.0):
        lhs = float(np.sum(W.a_h_strong(sm, c, tau, tau) * c))
        assert abs(lhs - W.dissipation(sm, c, tau, tau)) < 1e-12 * scale
    under = float(np.sum(W.a_h_strong(mesh, c, 0.0, 0.0) * c))
    assert abs(under) > 1e-8 * scale


def test_strong_rhs_forms_select_rules():
    """rhs(form=...) routes the strong form to the strong rules and the
    under-integrated variant to the mesh's own rules; the mass inverse uses
    the degree 2N+1 rule in both (the results equal the direct compositions)."""
    from oracle.discretization import Mesh, RefTet
    from synthetic import warped_cube
    VXYZ, EToV, geom = warped_cube(2, 3, 0.1)
    mesh = Mesh(RefTet(3), VXYZ, EToV, geom)
    c = np.random.default_rng(3).standard_normal((4, mesh.K, mesh.ref.Np))
    full = W.rhs(mesh, c, form="strong")
    under = W.rhs(mesh, c, form="strong_underintegrated")
    assert np.allclose(full, W.wadg_apply(mesh, W.a_h_strong(W.strong_mesh(mesh), c)), rtol=0, atol=1e-12)
    assert np.allclose(under, W.wadg_apply(mesh, W.a_h_strong(mesh, c)), rtol=0, atol=1e-12)
    assert np.linalg.norm(full - under) > 1e-6 * np.linalg.norm(full)
    with pytest.raises(ValueError):
        W.rhs(mesh, c, form="weak")


# ----------------------------------------------------------------------------
# Local conservation (Sec. 3, after the moment estimate)
# ----------------------------------------------------------------------------

def _moments(mesh, r, c2q):
    """Per element and field, sum_q w_q w(x_q) r(x_q) with the mass weights
    w = J/c^2 (pressure) and J (velocity) at the volume points."""
    ref = mesh.ref
    vals = np.einsum("qm,fkm->fkq", ref.Vq, r)
    w = np.broadcast_to(mesh.J, vals.shape).copy()
    w[0] = mesh.J / c2q
    return np.einsum("q,fkq->fk", ref.w_q, w * vals)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_conservative_weights_restore_local_conservation(N):
    """With the mass weights projected onto P^N the update conserves every
    element's zeroth moment exactly: sum_q w_q w_q r_q = b(1) for any load b
    (curved mesh, heterogeneous c^2); with the pointwise weights it does not
    (the moment error of the weight-adjusted inner product)."""
    from synthetic import c2_heterogeneous
    ref, mesh = _mesh(2, N)
    c2q = c2_heterogeneous(mesh.xq)
    b = np.random.default_rng(50 + N).standard_normal((4, mesh.K, ref.Np))
    one = np.einsum("qm,q->m", ref.Vq, ref.w_q)           # modal coefficients of 1
    want = np.einsum("fkm,m->fk", b, one)                  # b(1)
    scale = np.abs(want).max()
    got = _moments(mesh, W.wadg_apply(mesh, b, c2q, conservative=True), c2q)
    assert np.abs(got - want).max() < 1e-12 * scale
    plain = _moments(mesh, W.wadg_apply(mesh, b, c2q), c2q)
    assert np.abs(plain - want).max() > 1e-8 * scale


def test_conservative_weights_equal_pointwise_for_polynomial_jacobian():
    """A global quadratic map has J of degree 3, in P^N for N = 3, so its
    projection is J itself (the degree 7 rule integrates J phi exactly) and
    the two weight sets coincide (c^2 = 1); a curved warp separates them."""
    N = 3
    VXYZ, EToV = kuhn_cube(2)
    X = geometry_nodes(VXYZ, EToV, N, 0.0)
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    Xq = np.stack([x + 0.05 * y * y, y + 0.04 * z * z, z + 0.03 * x * x], -1)
    mesh = Mesh(RefTet(N), VXYZ, EToV, Xq)
    a, b = W.wadg_weights(mesh), W.wadg_weights(mesh, conservative=True)
    assert np.abs(a[1] - b[1]).max() < 1e-12 * np.abs(a[1]).max()
    assert np.abs(a[0] - b[0]).max() < 1e-12 * np.abs(a[0]).max()
    _, curved = _mesh(2, N)
    a, b = W.wadg_weights(curved), W.wadg_weights(curved, conservative=True)
    assert np.abs(a[1] - b[1]).max() > 1e-6 * np.abs(a[1]).max()


def test_point_source_zeroth_moment_on_curved_elements_with_conservative_weights():
    """int J p_t = f(t) for a point source on curved elements holds to round-off
    with the conservative weights, and only to the moment error otherwise."""
    from oracle import sources as OS
    ref, mesh = _mesh(2, 3)
    src = OS.PointSet(mesh, [[0.13, -0.41, 0.27]])
    amp = 0.7
    b = OS.source_load(mesh, src, amp, 0)

    def total(dq):
        vals = np.einsum("qm,km->kq", ref.Vq, dq[0])
        return float(np.sum(ref.w_q * mesh.J * vals))

    assert abs(total(W.wadg_apply(mesh, b, conservative=True)) - amp) < 1e-13
    assert abs(total(W.wadg_apply(mesh, b)) - amp) > 1e-9


def test_rhs_conservative_flag_reaches_the_update():
    """rhs(conservative=True) equals the conservative update of the same
    functional, for both formulations it is offered with."""
    ref, mesh = _mesh(2, 3)
    c = np.random.default_rng(4).standard_normal((4, mesh.K, ref.Np))
    for form, a_h in (("strong_weak", W.a_h), ("strong", lambda m, q, tp, tu: W.a_h_strong(W.strong_mesh(m), q, tp, tu))):
        got = W.rhs(mesh, c, form=form, conservative=True)
        want = W.wadg_apply(mesh, a_h(mesh, c, 1.0, 1.0), conservative=True)
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


# ----------------------------------------------------------------------------
# Fewer-point symmetric volume rules (tabulated inputs)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("N,npts", [(2, 14), (3, 35), (4, 63), (5, 96)])
def test_fewer_point_rules_exact_to_2N_plus_1_and_not_beyond(N, npts):
    """Every monomial of degree <= 2N+1 integrates exactly (closed form), some
    of degree 2N+2 do not; positive weights, interior points."""
    from synthetic import fewer_point_rule
    rst, w = fewer_point_rule(N)
    assert len(w) == npts and w.min() > 0
    lam = np.column_stack([-(1 + rst.sum(1)) / 2, (1 + rst) / 2])
    assert lam.min() > 0
    worst, beyond = 0.0, 0.0
    for a in range(2 * N + 3):
        for b in range(2 * N + 3 - a):
            for c in range(2 * N + 3 - a - b):
                v = np.sum(w * (1 + rst[:, 0]) ** a * (1 + rst[:, 1]) ** b * (1 + rst[:, 2]) ** c)
                e = abs(v - _tet_monomial(a, b, c)) / _tet_monomial(a, b, c)
                if a + b + c <= 2 * N + 1:
                    worst = max(worst, e)
                else:
                    beyond = max(beyond, e)
    assert worst < 1e-12 and beyond > 1e-9


@pytest.mark.parametrize("degree", [5, 7, 9, 11])
def test_fewer_point_rules_are_symmetric(degree):
    """The point set with its weights is invariant under the 24 vertex
    permutations of the tetrahedron."""
    from synthetic import symmetric_rule
    rst, w = symmetric_rule(degree)
    lam = np.column_stack([-(1 + rst.sum(1)) / 2, (1 + rst) / 2])
    key = {tuple(np.round(l, 12)): wi for l, wi in zip(lam, w)}
    assert len(key) == len(w)
    for perm in __import__("itertools").permutations(range(4)):
        for l, wi in zip(lam, w):
            assert abs(key[tuple(np.round(l[list(perm)], 12))] - wi) < 1e-15


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_fewer_point_rule_rhs_equals_collapsed_rule_on_affine_elements(N):
    """On affine elements with c^2 = 1 every integrand of the right-hand side
    and of the update is a polynomial of degree <= 2N, which both rules
    integrate exactly: the two discretisations coincide."""
    from synthetic import fewer_point_rule
    VXYZ, EToV, geom = warped_cube(2, N, 0.0)
    a = Mesh(RefTet(N), VXYZ, EToV, geom)
    b = Mesh(RefTet(N, volume_rule=fewer_point_rule(N)), VXYZ, EToV, geom)
    assert b.ref.Nq < a.ref.Nq
    c = np.random.default_rng(6).standard_normal((4, a.K, a.ref.Np))
    ra, rb = W.rhs(a, c), W.rhs(b, c)
    assert np.abs(ra - rb).max() < 1e-11 * np.abs(ra).max()
    _, curved = _mesh(2, N)
    cb = Mesh(RefTet(N, volume_rule=fewer_point_rule(N)), curved.VXYZ, curved.EToV, curved.geom_xyz)
    d = np.abs(W.rhs(curved, c) - W.rhs(cb, c)).max() / np.abs(W.rhs(curved, c)).max()
    assert 1e-10 < d < 1e-1     # curved: both rules under-integrate the rational integrands, differently


@pytest.mark.parametrize("N", [2, 3])
def test_fewer_point_rule_has_the_collapsed_rule_accuracy(N):
    """Standing wave on the curved 48-tet mesh, N = 2 and 3, to T = 0.1 (same
    dt): the L2 errors against the analytic solution with the collapsed and
    the symmetric rule of the same degree 2N+1 agree within 5 %."""
    from synthetic import fewer_point_rule
    T = 0.1
    VXYZ, EToV, geom = warped_cube(2, N, 0.1)
    errs = []
    for rule in (None, fewer_point_rule(N)):
        mesh = Mesh(RefTet(N, volume_rule=rule), VXYZ, EToV, geom)
        c = W.wadg_projection(mesh, standing_wave(mesh.xq, 0.0))
        res = np.zeros_like(c)
        nst = 8
        dt = T / nst
        for k in range(nst):
            c, res = W.lsrk_step(lambda q, t: W.rhs(mesh, q), c, res, k * dt, dt)
        errs.append(W.l2_error(mesh, c, lambda x: standing_wave(x, T)))
    assert abs(errs[1] - errs[0]) < 0.05 * errs[0], errs
