"""The strong formulation (Sec. 4.1) on the CUDA-core path against the
oracle's strong form, with the same degree 2N+1 rules."""
import numpy as np
import pytest

from gpu_util import TOL, library_mesh, make_mesh_inputs, oracle_c2, oracle_case, random_Q, rel_errors, to_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,n", [(1, 3), (2, 2), (3, 2), (4, 2), (5, 2)])
def test_strong_rhs_matches_oracle(W, precision, N, n):
    import torch
    from oracle import wadg as OW
    VXYZ, EToV, geom = make_mesh_inputs(n, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous")
    W.wadg_set_formulation(m, "strong")
    Q = random_Q(m.K, 1, m.Np, seed=200 + N)
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()[:, :, 0]
    want = OW.rhs_nodal(om, Q[:, :, 0], c2q=oracle_c2(om, "heterogeneous"), form="strong")
    l2, mx = rel_errors(got, want)
    # the under-integrated strong form is a different discretisation: make sure
    # the test would see the strong-weak result as a failure
    other = OW.rhs_nodal(om, Q[:, :, 0], c2q=oracle_c2(om, "heterogeneous"))
    print(f"strong N={N} {precision}: rel L2 {l2:.3e}, strong-weak differs by {rel_errors(other, want)[0]:.3e}")
    assert l2 < TOL[precision] and mx < 10 * TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_strong_lsrk_steps_match_oracle(W, precision):
    """Three LSRK steps with 3 shots and penalties (1, 0.5); wadg_solve's graph
    replays the same steps."""
    import torch
    from oracle import wadg as OW
    N, S, tau = 3, 3, (1.0, 0.5)
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous", tau=tau)
    W.wadg_set_formulation(m, "strong")
    c2o = oracle_c2(om, "heterogeneous")
    Q0 = random_Q(m.K, S, m.Np, seed=23)
    dt, nsteps = 2e-3, 3
    Qt, Rt = to_torch(Q0, m.dtype), None
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
            c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o, tau_p=tau[0], tau_u=tau[1], form="strong"),
                                  c, res, k * dt, dt)
        l2, _ = rel_errors(Qt.double().cpu().numpy()[:, :, s], ref.to_nodal(c))
        l2r, _ = rel_errors(Rt.double().cpu().numpy()[:, :, s], ref.to_nodal(res))
        assert l2 < TOL[precision] and l2r < 10 * TOL[precision], (s, l2, l2r)


def test_strong_formulation_is_refused_where_not_built(W):
    """Tensor-core precisions, N = 6, the adjoint and batches are built for the
    strong-weak form: WADG_EUNSUPPORTED (-8) before any launch."""
    import torch
    VXYZ, EToV, geom = make_mesh_inputs(1, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, "fp32_3xbf16")
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_formulation(m, "strong")
    assert e.value.status == -8
    m6 = library_mesh(*make_mesh_inputs(1, 6), 6, "fp32")
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_formulation(m6, "strong")
    assert e.value.status == -8
    m3 = library_mesh(VXYZ, EToV, geom, 3, "fp32")
    W.wadg_set_formulation(m3, "strong")
    lam = torch.zeros((4, m3.K, 1, m3.Np), dtype=torch.float32, device="cuda")
    with pytest.raises(W.WadgError) as e:
        W.wadg_rhs_adjoint(m3, lam, torch.empty_like(lam))
    assert e.value.status == -8
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_operators(m3, "fp32_3xbf16", 1, 1.0, 1.0, None)
    assert e.value.status == -8
    with pytest.raises(W.WadgError):
        W.wadg_batch_create([m3])
