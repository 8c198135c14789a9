"""The strong formulation (Sec. 4.1) on the CUDA-core path against the
oracle's strong form: form "strong" with its volume and surface terms on the
energy-stable rules (degree 4N-3 / 4N-2), form "strong_underintegrated" on the
degree 2N+1 rules; the weight-adjusted update uses the degree 2N+1 rule in
both."""
import numpy as np
import pytest

from gpu_util import TOL, library_mesh, make_mesh_inputs, oracle_c2, oracle_case, random_Q, rel_errors, to_torch

pytestmark = pytest.mark.gpu
FORMS = ["strong", "strong_underintegrated"]


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


def _rhs(W, m, Q):
    import torch
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,n", [(1, 3), (2, 2), (3, 2), (4, 2), (4, 3), (5, 2)])
def test_strong_rhs_matches_oracle(W, form, precision, N, n):
    """Element by element against the oracle at N = 1..5; the n = 3 meshes
    (162 tets) span several blocks with a ragged last block."""
    from oracle import wadg as OW
    VXYZ, EToV, geom = make_mesh_inputs(n, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous")
    W.wadg_set_formulation(m, form)
    Q = random_Q(m.K, 1, m.Np, seed=200 + N)
    got = _rhs(W, m, Q).double().cpu().numpy()[:, :, 0]
    c2o = oracle_c2(om, "heterogeneous")
    want = OW.rhs_nodal(om, Q[:, :, 0], c2q=c2o, form=form)
    l2, mx = rel_errors(got, want)
    # each form is a different discretisation on curved elements (for N >= 2):
    # the test would see any of the other two as a failure
    others = [rel_errors(OW.rhs_nodal(om, Q[:, :, 0], c2q=c2o, form=f), want)[0]
              for f in ("strong_weak", "strong", "strong_underintegrated") if f != form]
    print(f"{form} N={N} K={m.K} {precision}: rel L2 {l2:.3e} (max {mx:.3e}); other forms differ by "
          + ", ".join(f"{d:.2e}" for d in others))
    assert l2 < TOL[precision] and mx < 10 * TOL[precision]
    if N >= 2:
        assert min(others) > 3 * TOL[precision]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_strong_lsrk_steps_match_oracle(W, form, precision):
    """Three LSRK steps with 3 shots and penalties (1, 0.5); wadg_solve's graph
    replays the same steps."""
    import torch
    from oracle import wadg as OW
    N, S, tau = 3, 3, (1.0, 0.5)
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous", tau=tau)
    W.wadg_set_formulation(m, form)
    c2o = oracle_c2(om, "heterogeneous")
    Q0 = random_Q(m.K, S, m.Np, seed=23)
    dt, nsteps = 2e-3, 3
    Qt = to_torch(Q0, m.dtype)
    Rt = torch.zeros_like(Qt)
    W.wadg_step(m, Qt, Rt, 0.0, dt, nsteps)
    Qg, Rg = to_torch(Q0, m.dtype), torch.zeros_like(Qt)
    assert W.wadg_solve(m, Qg, Rg, 0.0, nsteps * dt, dt) == nsteps
    torch.cuda.synchronize()
    assert torch.equal(Qg, Qt) and torch.equal(Rg, Rt)
    ref = om.ref
    for s in range(S):
        c = ref.to_modal(Q0[:, :, s])
        res = np.zeros_like(c)
        for k in range(nsteps):
            c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o, tau_p=tau[0], tau_u=tau[1], form=form),
                                  c, res, k * dt, dt)
        l2, _ = rel_errors(Qt.double().cpu().numpy()[:, :, s], ref.to_nodal(c))
        l2r, _ = rel_errors(Rt.double().cpu().numpy()[:, :, s], ref.to_nodal(res))
        assert l2 < TOL[precision] and l2r < 10 * TOL[precision], (s, l2, l2r)


def test_formulation_switches_and_call_order(W):
    """Switching the formulation back and forth rebuilds the same state
    (bitwise equal results); set_operators after set_formulation (a precision
    change) rebuilds the strong tables in the new precision."""
    from oracle import wadg as OW
    N = 3
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    m = library_mesh(VXYZ, EToV, geom, N, "fp64", c2="heterogeneous")
    Q = random_Q(m.K, 1, m.Np, seed=5)
    sw = _rhs(W, m, Q)
    W.wadg_set_formulation(m, "strong")
    st1 = _rhs(W, m, Q)
    W.wadg_set_formulation(m, "strong_underintegrated")
    su = _rhs(W, m, Q)
    W.wadg_set_formulation(m, "strong_weak")
    assert (_rhs(W, m, Q) == sw).all()
    W.wadg_set_formulation(m, "strong")
    assert (_rhs(W, m, Q) == st1).all()
    assert not (st1 == su).all() and not (st1 == sw).all()
    om = oracle_case(VXYZ, EToV, geom, N)
    c2o = oracle_c2(om, "heterogeneous")
    W.wadg_set_operators(m, "fp32", 1, 1.0, 1.0, c2o)
    got = _rhs(W, m, Q).double().cpu().numpy()[:, :, 0]
    assert rel_errors(got, OW.rhs_nodal(om, Q[:, :, 0], c2q=c2o, form="strong"))[0] < TOL["fp32"]


def test_strong_formulation_is_refused_where_not_built(W):
    """Tensor-core precisions, N = 6, the adjoint and batches are built for the
    strong-weak form: WADG_EUNSUPPORTED (-8) before any launch; an unknown
    formulation is WADG_EINVAL (-1) and leaves the current one in effect."""
    import torch
    VXYZ, EToV, geom = make_mesh_inputs(1, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, "fp32_3xbf16")
    for form in FORMS:
        with pytest.raises(W.WadgError) as e:
            W.wadg_set_formulation(m, form)
        assert e.value.status == -8
    m6 = library_mesh(*make_mesh_inputs(1, 6), 6, "fp32")
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_formulation(m6, "strong")
    assert e.value.status == -8
    m3 = library_mesh(VXYZ, EToV, geom, 3, "fp32")
    W.wadg_set_formulation(m3, "strong")
    Q = random_Q(m3.K, 1, m3.Np, seed=8)
    before = _rhs(W, m3, Q)
    assert W.load().wadg_set_formulation(m3.handle, 3) == -1
    assert (_rhs(W, m3, Q) == before).all()
    lam = torch.zeros((4, m3.K, 1, m3.Np), dtype=torch.float32, device="cuda")
    with pytest.raises(W.WadgError) as e:
        W.wadg_rhs_adjoint(m3, lam, torch.empty_like(lam))
    assert e.value.status == -8
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_operators(m3, "fp32_3xbf16", 1, 1.0, 1.0, None)
    assert e.value.status == -8
    with pytest.raises(W.WadgError):
        W.wadg_batch_create([m3])
