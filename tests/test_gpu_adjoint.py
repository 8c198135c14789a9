"""The discrete adjoint on the GPU: transpose identities, parity with the
oracle's brute-force adjoint, and finite differences of the misfit."""
import numpy as np
import pytest

from gpu_util import TOL, library_mesh, make_mesh_inputs, oracle_case, rel_errors, to_torch
from synthetic import c2_perturbed_samples, random_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.0, 0.0), (1.0, 0.3)])
def test_dot_product_identity(W, tau):
    """<L x, y> = <x, L^T y> for the FP64 operators, curved mesh, c^2 varying,
    two shots."""
    import torch
    VXYZ, EToV, geom = make_mesh_inputs(2, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, "fp64", shots=2, c2="heterogeneous", tau=tau)
    x = to_torch(random_fields((4, m.K, 2, m.Np), 1), torch.float64)
    y = to_torch(random_fields((4, m.K, 2, m.Np), 2), torch.float64)
    Lx, LTy = torch.empty_like(x), torch.empty_like(y)
    W.wadg_rhs(m, x, Lx)
    W.wadg_rhs_adjoint(m, y, LTy)
    a, b = float((Lx * y).sum()), float((x * LTy).sum())
    assert abs(a - b) < 1e-12 * float(Lx.norm() * y.norm())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rhs_adjoint_matches_oracle_transpose(W, precision):
    from oracle import adjoint as OA
    N = 2
    VXYZ, EToV, geom = make_mesh_inputs(1, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    c2q = c2_perturbed_samples((om.K, om.ref.Nq), seed=5)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2=c2q)
    L = OA.dense_operator(om, c2q)
    lam = random_fields((4, om.K, om.ref.Np), 9)
    # nodal transpose: L_nodal^T = Vn^-T L_modal^T Vn^T
    Vn, Vi = om.ref.Vn, om.ref.Vn_inv
    lam_m = np.einsum("nm,fkn->fkm", Vn, lam)
    want = np.einsum("mn,fkm->fkn", Vi, (L.T @ lam_m.ravel()).reshape(lam.shape))
    import torch
    out = torch.empty((4, om.K, 1, om.ref.Np), dtype=m.dtype, device="cuda")
    W.wadg_rhs_adjoint(m, to_torch(lam[:, :, None, :], m.dtype), out)
    l2, mx = rel_errors(out.double().cpu().numpy()[:, :, 0], want)
    assert l2 < TOL[precision] and mx < 10 * TOL[precision], (l2, mx)


def _gpu_problem(W, precision, prob, om, c2q):
    VXYZ, EToV, geom = om._inputs
    m = library_mesh(VXYZ, EToV, geom, om.ref.N, precision, c2=c2q)
    W.wadg_set_sources(m, np.array([[0.1, -0.2, 0.15]]), 5.0, 0.02)
    W.wadg_set_receivers(m, np.array([[[0.3, 0.1, -0.4], [-0.5, 0.2, 0.3]]]))
    return m


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_misfit_gradients_match_oracle_adjoint(W, precision):
    """J = sum of squared receiver pressures over 6 steps; gradients w.r.t. the
    nodal initial pressure and c^2 at the volume points, with checkpoints every
    4 steps (one full and one ragged segment)."""
    import torch
    from oracle import adjoint as OA
    from paper_1608_03836_gb300.adjoint import receiver_traces
    N = 2
    VXYZ, EToV, geom = make_mesh_inputs(1, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    om._inputs = (VXYZ, EToV, geom)
    c2q = c2_perturbed_samples((om.K, om.ref.Nq))
    prob = OA.MisfitProblem(om, c2q, [0.1, -0.2, 0.15], np.array([[0.3, 0.1, -0.4], [-0.5, 0.2, 0.3]]),
                            f0=5.0, t0=0.02, dt=4e-3, nsteps=6)
    p0_nodal = random_fields((om.K, om.ref.Np), 77)
    p0_modal = om.ref.to_modal(p0_nodal)
    J, gp_modal, gc = prob.gradients(p0_modal)
    gp_nodal = np.einsum("mn,km->kn", om.ref.Vn_inv, gp_modal)     # chain rule through c = Vn^-1 q

    m = _gpu_problem(W, precision, prob, om, c2q)
    p0 = to_torch(p0_nodal[:, None, :], m.dtype).requires_grad_(True)
    c2 = torch.tensor(c2q, dtype=torch.float64, device="cuda", requires_grad=True)
    tr = receiver_traces(m, p0, c2, 4e-3, 6, checkpoint=4)
    Jg = (tr.double() ** 2).sum()
    Jg.backward()
    tol = {"fp64": 1e-9, "fp32": 1e-4}[precision]
    assert abs(float(Jg) - J) < tol * J
    l2p, _ = rel_errors(p0.grad.double().cpu().numpy()[:, 0], gp_nodal)
    l2c, _ = rel_errors(c2.grad.cpu().numpy(), gc)
    print(f"{precision}: J rel {abs(float(Jg) - J) / J:.2e}, grad p0 {l2p:.2e}, grad c2 {l2c:.2e}")
    assert l2p < tol and l2c < tol, (l2p, l2c)


def test_misfit_gradients_match_finite_differences_on_gpu(W):
    """FP64 GPU: <grad, d> against central differences of the GPU misfit along
    8 seeded directions for each parameter, to 1e-6 relative."""
    import torch
    from paper_1608_03836_gb300.adjoint import receiver_traces
    N = 3
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    om._inputs = (VXYZ, EToV, geom)
    c2q = c2_perturbed_samples((om.K, om.ref.Nq))
    m = _gpu_problem(W, "fp64", None, om, c2q)
    dt, ns = 3e-3, 12

    def misfit(p0, c2):
        with torch.no_grad():
            return float((receiver_traces(m, p0, c2, dt, ns, checkpoint=5) ** 2).sum())

    p0 = to_torch(random_fields((m.K, 1, m.Np), 5), torch.float64).requires_grad_(True)
    c2 = torch.tensor(c2q, dtype=torch.float64, device="cuda", requires_grad=True)
    (receiver_traces(m, p0, c2, dt, ns, checkpoint=5) ** 2).sum().backward()
    gp, gc = p0.grad.clone(), c2.grad.clone()
    rng = np.random.default_rng(8)
    for _ in range(8):
        d = to_torch(rng.standard_normal(p0.shape), torch.float64)
        eps = 1e-3
        fd = (misfit(p0.detach() + eps * d, c2.detach()) - misfit(p0.detach() - eps * d, c2.detach())) / (2 * eps)
        assert abs(fd - float((gp * d).sum())) < 1e-6 * abs(fd)
        dc = to_torch(rng.standard_normal(c2.shape), torch.float64)
        eps = 1e-5
        fd = (misfit(p0.detach(), c2.detach() + eps * dc) - misfit(p0.detach(), c2.detach() - eps * dc)) / (2 * eps)
        assert abs(fd - float((gc * dc).sum())) < 1e-6 * abs(fd)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_segment_adjoint_equals_the_step_by_step_calls(W, precision):
    """wadg_segment_adjoint (recompute with recording, then receiver adjoints
    and reverse steps, one call) gives bit for bit what the per-step calls
    give, with and without the c^2 record; without it the state is not read."""
    import torch
    N, ns, dt, t0 = 3, 5, 3e-3, 0.01
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    om._inputs = (VXYZ, EToV, geom)
    m = _gpu_problem(W, precision, None, om, c2_perturbed_samples((om.K, om.ref.Nq)))
    Q0 = to_torch(random_fields((4, m.K, 1, m.Np), 21), m.dtype)
    g = to_torch(random_fields((ns, 1, 2), 22), m.dtype)
    lq0 = to_torch(random_fields((4, m.K, 1, m.Np), 23), m.dtype)
    lr0 = to_torch(random_fields((4, m.K, 1, m.Np), 24), m.dtype)
    for record in (True, False):
        # per-step reference
        Q, R = Q0.clone(), torch.zeros_like(Q0)
        ys = torch.empty((ns, 5, m.K, 1, m.Nq), dtype=m.dtype, device="cuda") if record else None
        lq, lr = lq0.clone(), lr0.clone()
        dc = torch.zeros((m.K, m.Nq), dtype=torch.float64, device="cuda") if record else None
        if record:
            for n in range(ns):
                W.wadg_step_record(m, Q, R, t0 + n * dt, dt, ys[n])
        for n in reversed(range(ns)):
            W.wadg_receivers_adjoint(m, g[n], lq)
            W.wadg_step_adjoint(m, lq, lr, dt, None if ys is None else ys[n], dc)
        # one call
        Q2, R2 = Q0.clone(), torch.zeros_like(Q0)
        ys2 = torch.empty_like(ys) if record else None
        lq2, lr2 = lq0.clone(), lr0.clone()
        dc2 = torch.zeros_like(dc) if record else None
        W.wadg_segment_adjoint(m, Q2 if record else None, R2 if record else None, t0, dt, ns, g, lq2, lr2, ys2, dc2)
        torch.cuda.synchronize()
        assert torch.equal(lq, lq2) and torch.equal(lr, lr2)
        if record:
            assert torch.equal(Q, Q2) and torch.equal(R, R2) and torch.equal(ys, ys2)
            assert float((dc - dc2).abs().max()) <= 1e-14 * float(dc.abs().max())
